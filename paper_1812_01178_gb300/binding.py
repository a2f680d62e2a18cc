"""Thin ctypes binding of the C ABI in include/ns.h (argument marshalling only).

Every computation runs in the CUDA library libns_gb300.so built from csrc/ (see build.py).
There is no CPU or PyTorch fallback: if the library is missing or fails to load, importing
this module's `lib()` raises.  PyTorch is used only to own device memory and streams.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libns_gb300.so")

NS_OK, NS_ERR_ARG, NS_ERR_SIZE, NS_ERR_CUDA, NS_ERR_TIMEOUT, NS_ERR_STATE, NS_ERR_UNSUPPORTED = range(7)
NS_FP64, NS_MIXED = 0, 1
NS_PART_AUTO, NS_PART_PPT, NS_PART_PDD = 0, 1, 2
NS_PRESSURE_DELTA, NS_PRESSURE_KIM_MOIN = 0, 1
NS_BUF_RU, NS_BUF_RV, NS_BUF_RW, NS_BUF_NU, NS_BUF_NV, NS_BUF_NW, NS_BUF_PHI, NS_BUF_SPEC, NS_BUF_POIS_MODE = range(9)

STATUS_NAMES = {0: "NS_OK", 1: "NS_ERR_ARG", 2: "NS_ERR_SIZE", 3: "NS_ERR_CUDA", 4: "NS_ERR_TIMEOUT",
                5: "NS_ERR_STATE", 6: "NS_ERR_UNSUPPORTED"}

# Every symbol declared in include/ns.h.
EXPORTS = ["ns_workspace_bytes", "ns_init", "ns_rhs", "ns_adi_sweep", "ns_poisson_solve", "ns_project",
           "ns_substep", "ns_step", "ns_launches_per_step", "ns_convective_rate", "ns_set_dt", "ns_step_cfl", "ns_step_profiled", "ns_kernel_count", "ns_kernel_name", "ns_step_host", "ns_make_divergence_free", "ns_set_partition",
           "ns_get_partition", "ns_autotune", "ns_get_buffer", "ns_poisson_solve_static", "ns_fp64_fma_probe", "ns_sync",
           "ns_last_error", "ns_destroy", "ns_batch_workspace_bytes", "ns_batch_init", "ns_batch_step",
           "ns_batch_launches_per_step", "ns_batch_autotune", "ns_batch_set_partition", "ns_batch_instance",
           "ns_batch_sync", "ns_batch_last_error", "ns_batch_destroy",
           "ns_slab_rows", "ns_slab_slot_bytes", "ns_slab_slots", "ns_slab_workspace_bytes", "ns_slab_init",
           "ns_slab_phase", "ns_slab_buffers", "ns_slab_mode", "ns_slab_context", "ns_slab_sync",
           "ns_slab_last_error", "ns_slab_destroy", "ns_slab_solve_line_host"]
NS_STATIC_SCRATCH_BYTES = 48 * 1024 * 1024


class ns_config(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("lx", C.c_double), ("lz", C.c_double),
                ("yf", C.POINTER(C.c_double)),
                ("bc_x", C.c_int), ("bc_ytop", C.c_int),
                ("re", C.c_double), ("fx", C.c_double), ("dt", C.c_double),
                ("precision", C.c_int), ("u_conv", C.c_double), ("pressure_update", C.c_int),
                ("recycle_i", C.c_int), ("delta_in", C.c_double)]


class ns_fields(C.Structure):
    _fields_ = [("u", C.c_void_p), ("v", C.c_void_p), ("w", C.c_void_p), ("p", C.c_void_p),
                ("u_out", C.c_void_p), ("v_in", C.c_void_p), ("v_out", C.c_void_p),
                ("w_in", C.c_void_p), ("w_out", C.c_void_p)]


class NSError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


_LIB = None


def lib(path: str = LIB_PATH):
    """Load the CUDA library (raises if it is missing: there is no fallback)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise RuntimeError("CUDA library %s is missing: run paper_1812_01178_gb300/build.py "
                           "(or __graft_entry__.build())" % path)
    L = C.CDLL(path)
    vp, i, d, sz = C.c_void_p, C.c_int, C.c_double, C.c_size_t
    P = C.POINTER
    L.ns_workspace_bytes.argtypes = [P(ns_config)]
    L.ns_workspace_bytes.restype = sz
    L.ns_init.argtypes = [P(vp), P(ns_config), P(ns_fields), vp, sz, vp]
    for name in ("ns_rhs", "ns_poisson_solve", "ns_project", "ns_substep", "ns_step"):
        getattr(L, name).argtypes = [vp, i]
    L.ns_adi_sweep.argtypes = [vp, i, i]
    L.ns_convective_rate.argtypes = [vp, P(d)]
    L.ns_set_dt.argtypes = [vp, d]
    L.ns_step_cfl.argtypes = [vp, i, d, P(d)]
    L.ns_step_host.argtypes = [vp, vp, vp, vp, vp, i]
    L.ns_step_profiled.argtypes = [vp, i, P(C.c_float), i]
    L.ns_kernel_count.argtypes = []
    L.ns_kernel_name.argtypes = [i]
    L.ns_kernel_name.restype = C.c_char_p
    L.ns_make_divergence_free.argtypes = [vp]
    L.ns_set_partition.argtypes = [vp, i, i, i]
    L.ns_get_partition.argtypes = [vp, i, P(i), P(i), P(d)]
    L.ns_autotune.argtypes = [vp]
    L.ns_get_buffer.argtypes = [vp, i, P(vp), P(sz)]
    L.ns_poisson_solve_static.argtypes = [P(ns_config), vp, vp, vp, vp, i, vp]
    L.ns_fp64_fma_probe.argtypes = [vp, i, i, vp]
    L.ns_slab_rows.argtypes = [i, i, i, P(i), P(i)]
    L.ns_slab_slot_bytes.argtypes = [P(ns_config), i, i]
    L.ns_slab_slot_bytes.restype = sz
    L.ns_slab_slots.argtypes = [i, i, i, i, P(i), P(i)]
    L.ns_slab_workspace_bytes.argtypes = [P(ns_config), i, i]
    L.ns_slab_workspace_bytes.restype = sz
    L.ns_slab_init.argtypes = [P(vp), P(ns_config), i, i, i, P(ns_fields), vp, sz, vp]
    L.ns_slab_phase.argtypes = [vp, i, i]
    L.ns_slab_buffers.argtypes = [vp, i, P(vp), P(vp), P(sz)]
    L.ns_slab_mode.argtypes = [vp, P(i), P(d)]
    L.ns_slab_context.argtypes = [vp]
    L.ns_slab_context.restype = vp
    L.ns_slab_sync.argtypes = [vp]
    L.ns_slab_last_error.argtypes = [vp]
    L.ns_slab_last_error.restype = C.c_char_p
    L.ns_slab_destroy.argtypes = [vp]
    L.ns_slab_destroy.restype = None
    L.ns_slab_solve_line_host.argtypes = [i, P(d), P(d), P(d), P(d), i, i, P(d), P(d)]
    L.ns_sync.argtypes = [vp]
    L.ns_last_error.argtypes = [vp]
    L.ns_last_error.restype = C.c_char_p
    L.ns_destroy.argtypes = [vp]
    L.ns_destroy.restype = None
    L.ns_batch_workspace_bytes.argtypes = [P(ns_config), i]
    L.ns_batch_workspace_bytes.restype = sz
    L.ns_batch_init.argtypes = [P(vp), P(ns_config), P(ns_fields), i, vp, sz, vp]
    L.ns_batch_step.argtypes = [vp, i]
    L.ns_batch_launches_per_step.argtypes = [vp]
    L.ns_launches_per_step.argtypes = [vp]
    L.ns_batch_autotune.argtypes = [vp]
    L.ns_batch_set_partition.argtypes = [vp, i, i, i]
    L.ns_batch_instance.argtypes = [vp, i]
    L.ns_batch_instance.restype = vp
    L.ns_batch_sync.argtypes = [vp]
    L.ns_batch_last_error.argtypes = [vp]
    L.ns_batch_last_error.restype = C.c_char_p
    L.ns_batch_destroy.argtypes = [vp]
    L.ns_batch_destroy.restype = None
    for name in EXPORTS:
        if name not in ("ns_workspace_bytes", "ns_last_error", "ns_destroy", "ns_kernel_name",
                        "ns_batch_workspace_bytes", "ns_batch_instance", "ns_batch_last_error", "ns_batch_destroy"):
            getattr(L, name).restype = i
    _LIB = L
    return L


def make_config(case, precision=None):
    """ns_config from an inputs.Case (keeps the yf array alive on the returned object)."""
    yf = np.ascontiguousarray(case.yf, dtype=np.float64)
    cfg = ns_config(case.nx, case.ny, case.nz, case.lx, case.lz,
                    yf.ctypes.data_as(C.POINTER(C.c_double)), case.bc_x, case.bc_ytop,
                    case.re, case.fx, case.dt, case.precision if precision is None else precision,
                    getattr(case, "u_conv", 1.0), getattr(case, "pressure_update", NS_PRESSURE_DELTA),
                    getattr(case, "recycle_i", 0), getattr(case, "delta_in", 0.0))
    cfg._yf_keep = yf
    return cfg


# ---------------------------------------------------------------------- C-ABI names
def ns_workspace_bytes(cfg):
    return lib().ns_workspace_bytes(C.byref(cfg))


def _check(ctx, status):
    if status != NS_OK:
        raise NSError(status, lib().ns_last_error(ctx).decode())


def ns_init(cfg, fields, workspace_ptr, ws_bytes, stream_ptr):
    ctx = C.c_void_p()
    s = lib().ns_init(C.byref(ctx), C.byref(cfg), C.byref(fields), workspace_ptr, ws_bytes, stream_ptr)
    if s != NS_OK:
        raise NSError(s, lib().ns_last_error(None).decode())
    return ctx


def ns_rhs(ctx, k):
    _check(ctx, lib().ns_rhs(ctx, k))


def ns_adi_sweep(ctx, direction, k):
    _check(ctx, lib().ns_adi_sweep(ctx, direction, k))


def ns_poisson_solve(ctx, k):
    _check(ctx, lib().ns_poisson_solve(ctx, k))


def ns_project(ctx, k):
    _check(ctx, lib().ns_project(ctx, k))


def ns_substep(ctx, k):
    _check(ctx, lib().ns_substep(ctx, k))


def ns_step(ctx, nsteps):
    _check(ctx, lib().ns_step(ctx, nsteps))


def ns_convective_rate(ctx):
    r = C.c_double()
    _check(ctx, lib().ns_convective_rate(ctx, C.byref(r)))
    return r.value


def ns_set_dt(ctx, dt):
    _check(ctx, lib().ns_set_dt(ctx, dt))


def ns_step_cfl(ctx, nsteps, cfl):
    dts = (C.c_double * max(nsteps, 1))()
    _check(ctx, lib().ns_step_cfl(ctx, nsteps, cfl, dts))
    return list(dts)[:nsteps]


def ns_step_profiled(ctx, nsteps):
    """Returns {kernel name: summed ms} over nsteps steps (3 launches of each kernel per step)."""
    n = lib().ns_kernel_count()
    buf = (C.c_float * n)()
    _check(ctx, lib().ns_step_profiled(ctx, nsteps, buf, n))
    return {ns_kernel_name(q): float(buf[q]) for q in range(n)}


def ns_kernel_count():
    return lib().ns_kernel_count()


def ns_kernel_name(idx):
    return lib().ns_kernel_name(idx).decode()


def ns_step_host(ctx, u, v, w, p, nsteps):
    """u, v, w, p: C-contiguous float64 host arrays (pinned recommended), updated in place."""
    _check(ctx, lib().ns_step_host(ctx, u.ctypes.data, v.ctypes.data, w.ctypes.data, p.ctypes.data, nsteps))


def ns_make_divergence_free(ctx):
    _check(ctx, lib().ns_make_divergence_free(ctx))


def ns_set_partition(ctx, direction, P, mode):
    _check(ctx, lib().ns_set_partition(ctx, direction, P, mode))


def ns_get_partition(ctx, direction=0):
    P, mode, drop = C.c_int(), C.c_int(), C.c_double()
    _check(ctx, lib().ns_get_partition(ctx, direction, C.byref(P), C.byref(mode), C.byref(drop)))
    return P.value, mode.value, drop.value


def ns_autotune(ctx):
    _check(ctx, lib().ns_autotune(ctx))


def ns_get_buffer(ctx, which):
    ptr, n = C.c_void_p(), C.c_size_t()
    _check(ctx, lib().ns_get_buffer(ctx, which, C.byref(ptr), C.byref(n)))
    return ptr.value, n.value


def ns_poisson_solve_static(cfg, u_ptr, v_ptr, w_ptr, phi_ptr, substep, stream_ptr):
    """Context-free Poisson solve with no device allocation (scratch in a static device array)."""
    s = lib().ns_poisson_solve_static(C.byref(cfg), u_ptr, v_ptr, w_ptr, phi_ptr, substep, stream_ptr)
    if s != NS_OK:
        raise NSError(s, lib().ns_last_error(None).decode())


def ns_fp64_fma_probe(out_ptr, n_blocks, n_iter, stream_ptr):
    """Enqueue the FP64 FMA throughput kernel: 16 * n_iter flops for each of n_blocks * 256 threads."""
    s = lib().ns_fp64_fma_probe(out_ptr, n_blocks, n_iter, stream_ptr)
    if s != NS_OK:
        raise NSError(s, lib().ns_last_error(None).decode())


def ns_sync(ctx):
    _check(ctx, lib().ns_sync(ctx))


def ns_last_error(ctx):
    return lib().ns_last_error(ctx).decode()


def ns_destroy(ctx):
    lib().ns_destroy(ctx)


# ---------------------------------------------------------------------- convenience owner
class Solver:
    """Owns torch device tensors for the fields and the workspace of one context.

    Fields are float64 CUDA tensors with the layouts of include/ns.h.  Every method calls the
    C ABI; nothing is computed in Python or PyTorch.
    """

    def __init__(self, case, u=None, v=None, w=None, p=None, precision=None, device="cuda:0", stream=None,
                 bl=None):
        import torch
        self.torch = torch
        self.case = case
        self.cfg = make_config(case, precision)
        dev = torch.device(device)
        nx, ny, nz = case.nx, case.ny, case.nz

        def put(a, shape):
            if a is None:
                return torch.zeros(shape, dtype=torch.float64, device=dev)
            if isinstance(a, torch.Tensor) and a.device == dev:
                # a device tensor of the right layout is used in place (the context updates it)
                if a.dtype != torch.float64 or tuple(a.shape) != shape or not a.is_contiguous():
                    raise ValueError("device field must be a contiguous float64 tensor of shape %s" % (shape,))
                return a
            t = torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).to(dev)
            assert tuple(t.shape) == shape, (t.shape, shape)
            return t.contiguous()

        self.u = put(u, (nz, ny, nx))
        self.v = put(v, (nz, ny + 1, nx))
        self.w = put(w, (nz, ny, nx))
        self.p = put(p, (nz, ny, nx))
        nbytes = ns_workspace_bytes(self.cfg)
        if nbytes == 0:
            raise NSError(NS_ERR_SIZE, "invalid configuration")
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self.bl = None
        bptr = [None] * 5
        if case.bc_x == 1:
            names = ("u_out", "v_in", "v_out", "w_in", "w_out")
            shapes = {"u_out": (nz, ny), "v_in": (nz, ny + 1), "v_out": (nz, ny + 1), "w_in": (nz, ny),
                      "w_out": (nz, ny)}
            bl = bl or {}
            self.bl = {q: put(bl.get(q), shapes[q]) for q in names}
            bptr = [self.bl[q].data_ptr() for q in names]
        self.fields = ns_fields(self.u.data_ptr(), self.v.data_ptr(), self.w.data_ptr(), self.p.data_ptr(), *bptr)
        self.ctx = ns_init(self.cfg, self.fields, self.ws.data_ptr(), nbytes, self.stream.cuda_stream)
        self.es = 4 if self.cfg.precision == NS_MIXED else 8

    # views of workspace buffers as torch tensors
    def buffer(self, which):
        torch = self.torch
        ptr, n = ns_get_buffer(self.ctx, which)
        off = ptr - self.ws.data_ptr()
        raw = self.ws[off:off + n]
        c = self.case
        if which == NS_BUF_SPEC:
            return raw.view(torch.float64).view(c.nz // 2 + 1, c.ny, c.nx, 2)
        if which == NS_BUF_POIS_MODE:
            return raw.view(c.nz // 2 + 1, c.nx)
        if which == NS_BUF_PHI:
            return raw.view(torch.float64).view(c.nz, c.ny, c.nx)
        dt = torch.float32 if self.es == 4 else torch.float64
        rows = c.ny + 1 if which in (NS_BUF_RV, NS_BUF_NV) else c.ny
        return raw.view(dt).view(c.nz, rows, c.nx)

    def rhs(self, k):
        ns_rhs(self.ctx, k)

    def adi(self, direction, k):
        ns_adi_sweep(self.ctx, direction, k)

    def poisson(self, k):
        ns_poisson_solve(self.ctx, k)

    def project(self, k):
        ns_project(self.ctx, k)

    def substep(self, k):
        ns_substep(self.ctx, k)

    def step(self, n=1):
        ns_step(self.ctx, n)

    def launches_per_step(self):
        n = lib().ns_launches_per_step(self.ctx)
        if n < 0:
            raise NSError(NS_ERR_CUDA, lib().ns_last_error(self.ctx).decode())
        return n

    def step_profiled(self, n=1):
        return ns_step_profiled(self.ctx, n)

    def convective_rate(self):
        return ns_convective_rate(self.ctx)

    def set_dt(self, dt):
        ns_set_dt(self.ctx, dt)

    def step_cfl(self, n, cfl):
        return ns_step_cfl(self.ctx, n, cfl)

    def make_divergence_free(self):
        ns_make_divergence_free(self.ctx)

    def set_partition(self, P, mode=NS_PART_AUTO):
        ns_set_partition(self.ctx, 0, P, mode)

    def partition(self):
        return ns_get_partition(self.ctx, 0)

    def set_line_partition(self, direction, P):
        """y (1) or z (2) lines of the mixed form: P = 0 whole lines, else the built-in shape."""
        ns_set_partition(self.ctx, direction, P, NS_PART_AUTO)

    def line_partition(self, direction):
        return ns_get_partition(self.ctx, direction)

    def autotune(self):
        ns_autotune(self.ctx)

    def sync(self):
        ns_sync(self.ctx)

    def state(self):
        self.sync()
        return tuple(t.cpu().numpy() for t in (self.u, self.v, self.w, self.p))

    def boundary(self):
        self.sync()
        return {q: t.cpu().numpy() for q, t in (self.bl or {}).items()}

    def close(self):
        if getattr(self, "ctx", None) is not None:
            ns_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Owns the device fields of n instances and one batch context (include/ns.h, ns_batch_*)."""

    def __init__(self, cases, fields=None, precision=None, device="cuda:0"):
        import torch
        self.torch = torch
        dev = torch.device(device)
        self.cases = cases
        self.n = len(cases)
        self.cfgs = (ns_config * self.n)()
        self._keep = []
        self.t = []
        flds = (ns_fields * self.n)()
        for q, case in enumerate(cases):
            cfg = make_config(case, precision)
            self._keep.append(cfg)
            self.cfgs[q] = cfg
            nx, ny, nz = case.nx, case.ny, case.nz
            src = fields[q] if fields is not None else (None, None, None, None)
            ts = []
            for a, shape in zip(src, ((nz, ny, nx), (nz, ny + 1, nx), (nz, ny, nx), (nz, ny, nx))):
                if a is None:
                    ts.append(torch.zeros(shape, dtype=torch.float64, device=dev))
                else:
                    ts.append(torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).to(dev).contiguous())
            self.t.append(ts)
            flds[q] = ns_fields(*[x.data_ptr() for x in ts], None, None, None, None, None)
        nbytes = lib().ns_batch_workspace_bytes(self.cfgs, self.n)
        if nbytes == 0:
            raise NSError(NS_ERR_ARG, "invalid batch configuration")
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        self.stream = torch.cuda.current_stream(dev)
        self.b = C.c_void_p()
        s = lib().ns_batch_init(C.byref(self.b), self.cfgs, flds, self.n, self.ws.data_ptr(), nbytes,
                                self.stream.cuda_stream)
        if s != NS_OK:
            raise NSError(s, lib().ns_last_error(None).decode())

    def _chk(self, s):
        if s != NS_OK:
            raise NSError(s, lib().ns_batch_last_error(self.b).decode())

    def step(self, n=1):
        self._chk(lib().ns_batch_step(self.b, n))

    def autotune(self):
        self._chk(lib().ns_batch_autotune(self.b))

    def set_partition(self, i, P, mode=NS_PART_AUTO):
        self._chk(lib().ns_batch_set_partition(self.b, i, P, mode))

    def launches_per_step(self):
        return lib().ns_batch_launches_per_step(self.b)

    def instance(self, i):
        return C.c_void_p(lib().ns_batch_instance(self.b, i))

    def make_divergence_free(self):
        for q in range(self.n):
            ns_make_divergence_free(self.instance(q))

    def sync(self):
        self._chk(lib().ns_batch_sync(self.b))

    def state(self, i):
        self.sync()
        return tuple(x.cpu().numpy() for x in self.t[i])

    def close(self):
        if getattr(self, "b", None) is not None and self.b.value:
            lib().ns_batch_destroy(self.b)
            self.b = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
