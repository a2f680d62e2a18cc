"""y-slab decomposition of the time step (Sec. 3.2 and Algorithm 1) through the C ABI (ns_slab_*).

A slab is one GPU's share of the paper's multi-GPU method: whole x-z planes of the rows [j0, j1)
of y, with one halo row on each side that has a neighbour.  A sub-step is a fixed sequence of
library phases, each followed by one exchange (include/ns.h).  This module holds

* Slab: owns one slab's local device fields, workspace and library handle;
* SUBSTEP / run_steps: the order of phases and exchanges (the same for every driver);
* LocalExchange: the exchanges of p slabs held on one device, as device copies;
* DistExchange: the exchanges of one slab per rank over torch.distributed (NCCL between GPUs,
  gloo on the host): point-to-point between neighbours, all-gather where every slot is read.

Nothing here computes: the phases run the library's kernels, the exchanges only move bytes.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import binding as B

NS_XCH_HALO, NS_XCH_ADIY, NS_XCH_VSTAR, NS_XCH_POIS, NS_XCH_PHI, NS_XCH_FLUX, NS_XCH_RCY, NS_XCH_COUNT = range(8)
NS_SLAB_PACK, NS_SLAB_RHS, NS_SLAB_ADIZ, NS_SLAB_POIS, NS_SLAB_PHI, NS_SLAB_PROJECT = range(6)

# one RK3 sub-step: each phase, then the exchanges that move what it wrote (with the recycling
# inflow, the PACK phase and the PROJECT phase of sub-step 2 are also followed by RCY)
SUBSTEP = ((NS_SLAB_RHS, (NS_XCH_ADIY,)), (NS_SLAB_ADIZ, (NS_XCH_VSTAR, NS_XCH_FLUX)),
           (NS_SLAB_POIS, (NS_XCH_POIS,)), (NS_SLAB_PHI, (NS_XCH_PHI,)), (NS_SLAB_PROJECT, (NS_XCH_HALO,)))


def rows(ny, p, r):
    j0, j1 = C.c_int(), C.c_int()
    if B.lib().ns_slab_rows(ny, p, r, C.byref(j0), C.byref(j1)) != B.NS_OK:
        raise B.NSError(B.NS_ERR_ARG, "invalid slab split")
    return j0.value, j1.value


def slots(p, r, xch, ymode):
    """Slots lo .. hi (inclusive) of its receive buffer that slab r reads in exchange xch."""
    lo, hi = C.c_int(), C.c_int()
    if B.lib().ns_slab_slots(p, r, xch, ymode, C.byref(lo), C.byref(hi)) != B.NS_OK:
        raise B.NSError(B.NS_ERR_ARG, "invalid slot query")
    return lo.value, hi.value


def slot_bytes(cfg, p, xch):
    return B.lib().ns_slab_slot_bytes(C.byref(cfg), p, xch)


def solve_line_host(a, b, c, d, p, mode):
    """ns_slab_solve_line_host: one tridiagonal line solved the slabs' way on the host (no GPU).
    Returns (x, largest coupling PDD drops)."""
    arr = [np.ascontiguousarray(q, dtype=np.float64) for q in (a, b, c, d)]
    n = arr[3].size
    x = np.empty(n)
    drop = C.c_double()
    P = lambda q: q.ctypes.data_as(C.POINTER(C.c_double))
    st = B.lib().ns_slab_solve_line_host(n, *[P(q) for q in arr], p, mode, P(x), C.byref(drop))
    if st != B.NS_OK:
        raise B.NSError(st, "ns_slab_solve_line_host failed")
    return x, drop.value


def run_steps(slabs, exchange, nsteps, first=True):
    """nsteps time steps (three sub-steps each) of the slabs in `slabs` (all p slabs on one device,
    or this rank's one slab), exchanging with exchange(xch) after every phase.  first=True packs and
    exchanges the halo rows (and the recycle plane) before the first sub-step (the fields were just
    filled)."""
    rcy = bool(getattr(getattr(slabs[0], "case", None), "recycle_i", 0))
    if first:
        for s in slabs:
            s.phase(NS_SLAB_PACK, 0)
        exchange(NS_XCH_HALO)
        if rcy:
            exchange(NS_XCH_RCY)
    for _ in range(nsteps):
        for k in range(3):
            for ph, xchs in SUBSTEP:
                for s in slabs:
                    s.phase(ph, k)
                for xch in xchs:
                    exchange(xch)
            if rcy and k == 2:
                exchange(NS_XCH_RCY)


class Slab:
    """Slab r of p of the whole-domain case: its fields (rows j0-hb .. j1+ha-1, v faces
    j0-hb .. j1+ha) are cut from the whole-domain arrays u, v, w, p given (host arrays)."""

    def __init__(self, case, p, r, u, v, w, pr, ymode=B.NS_PART_AUTO, device="cuda:0", stream=None, bl=None):
        import torch
        self.torch = torch
        self.case, self.p, self.r = case, p, r
        self.cfg = B.make_config(case)
        dev = torch.device(device)
        self.j0, self.j1 = rows(case.ny, p, r)
        self.hb, self.ha = int(r > 0), int(r < p - 1)
        lo, hi = self.j0 - self.hb, self.j1 + self.ha
        put = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).to(dev).contiguous()
        self.u = put(u[:, lo:hi])
        self.v = put(v[:, lo:hi + 1])
        self.w = put(w[:, lo:hi])
        self.pr = put(pr[:, lo:hi])
        nbytes = B.lib().ns_slab_workspace_bytes(C.byref(self.cfg), p, r)
        if nbytes == 0:
            raise B.NSError(B.NS_ERR_ARG, "configuration not supported by the slab decomposition")
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        # boundary planes of inflow / outflow x (index k * rows + j), halo rows included
        self.bl = None
        bptr = [None] * 5
        if case.bc_x == 1:
            names = ("u_out", "v_in", "v_out", "w_in", "w_out")
            self.bl = {q: put(bl[q][:, lo:hi + (1 if q[0] == "v" else 0)]) for q in names}
            bptr = [self.bl[q].data_ptr() for q in names]
        self.fields = B.ns_fields(self.u.data_ptr(), self.v.data_ptr(), self.w.data_ptr(), self.pr.data_ptr(), *bptr)
        self.h = C.c_void_p()
        if stream is not None:  # the uploads above ran on the current stream
            torch.cuda.current_stream(dev).synchronize()
        st = B.lib().ns_slab_init(C.byref(self.h), C.byref(self.cfg), p, r, ymode, C.byref(self.fields),
                                  self.ws.data_ptr(), nbytes, self.stream.cuda_stream)
        if st != B.NS_OK:
            raise B.NSError(st, B.lib().ns_last_error(None).decode())
        m, drop = C.c_int(), C.c_double()
        B.lib().ns_slab_mode(self.h, C.byref(m), C.byref(drop))
        self.ymode, self.ydrop = m.value, drop.value
        self.send, self.recv = [], []
        for x in range(NS_XCH_COUNT):
            sp, rp, sb = C.c_void_p(), C.c_void_p(), C.c_size_t()
            B.lib().ns_slab_buffers(self.h, x, C.byref(sp), C.byref(rp), C.byref(sb))
            base = self.ws.data_ptr()
            n = sb.value
            self.send.append(self.ws[sp.value - base:sp.value - base + n])
            self.recv.append(self.ws[rp.value - base:rp.value - base + p * n].view(p, n))

    def slots(self, xch):
        return slots(self.p, self.r, xch, self.ymode)

    def phase(self, ph, k):
        st = B.lib().ns_slab_phase(self.h, ph, k)
        if st != B.NS_OK:
            raise B.NSError(st, B.lib().ns_slab_last_error(self.h).decode())

    def sync(self):
        st = B.lib().ns_slab_sync(self.h)
        if st != B.NS_OK:
            raise B.NSError(st, B.lib().ns_slab_last_error(self.h).decode())

    def owned(self):
        """The owned rows (u, w, p: j0 .. j1-1; v: faces j0 .. j1-1, and the top face for the last
        slab) as host arrays."""
        self.sync()
        a, b = self.hb, self.hb + (self.j1 - self.j0)
        vb = b + (1 if self.r == self.p - 1 else 0)
        return (self.u[:, a:b].cpu().numpy(), self.v[:, a:vb].cpu().numpy(), self.w[:, a:b].cpu().numpy(),
                self.pr[:, a:b].cpu().numpy())

    def owned_planes(self):
        """The owned rows of the boundary planes (inflow / outflow x), as host arrays."""
        self.sync()
        a, b = self.hb, self.hb + (self.j1 - self.j0)
        vb = b + (1 if self.r == self.p - 1 else 0)
        return {q: t[:, a:(vb if q[0] == "v" else b)].cpu().numpy() for q, t in self.bl.items()}

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            B.lib().ns_slab_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class LocalExchange:
    """The exchanges of p slabs held on one device: slot s of every slab that reads it receives
    slab s's send buffer by a device copy on the reading slab's stream.  Slabs may have streams of
    their own (their kernels then overlap, as on separate GPUs): a copy waits for the phase that
    wrote its source, and a slab's next phase waits for every copy of this exchange."""

    def __init__(self, slabs):
        self.slabs = slabs
        self.torch = slabs[0].torch

    def __call__(self, xch):
        torch = self.torch
        written = []
        for s in self.slabs:
            e = torch.cuda.Event()
            e.record(s.stream)
            written.append(e)
        for t in self.slabs:
            lo, hi = t.slots(xch)
            with torch.cuda.stream(t.stream):
                for q in range(lo, hi + 1):
                    if q != t.r:
                        t.stream.wait_event(written[q])
                        t.recv[xch][q].copy_(self.slabs[q].send[xch])
        copied = []
        for t in self.slabs:
            e = torch.cuda.Event()
            e.record(t.stream)
            copied.append(e)
        for s in self.slabs:
            for q, e in enumerate(copied):
                if q != s.r:
                    s.stream.wait_event(e)


class DistExchange:
    """The exchanges of this rank's slab over torch.distributed (one slab per rank, rank = slab
    index, world size = p).  An exchange whose every slot is read by every slab is an all-gather;
    the others are point-to-point sends to the slabs that read this slab's slot and receives from
    the slots this slab reads.  host=True stages device buffers through host memory, for a
    backend that moves host tensors only (gloo)."""

    def __init__(self, dist, p, r, ymode, send, recv, host=False):
        self.dist, self.p, self.r, self.ymode = dist, p, r, ymode
        self.send, self.recv = send, recv   # per exchange: send tensor, (p, slot) receive tensor
        self.host = host
        if host:
            import torch
            self.hsend = [torch.empty(t.shape, dtype=t.dtype) for t in send]
            self.hrecv = [torch.empty(t.shape, dtype=t.dtype) for t in recv]

    def readers(self, xch):
        """Slabs other than this one that read this slab's slot."""
        return [t for t in range(self.p) if t != self.r and slots(self.p, t, xch, self.ymode)[0] <= self.r
                <= slots(self.p, t, xch, self.ymode)[1]]

    def __call__(self, xch):
        if not self.host:
            self._move(xch, self.send[xch], self.recv[xch])
            return
        self.hsend[xch].copy_(self.send[xch])  # waits for the phase that wrote it (same stream)
        self._move(xch, self.hsend[xch], self.hrecv[xch])
        lo, hi = slots(self.p, self.r, xch, self.ymode)
        for s in range(lo, hi + 1):
            if s != self.r:  # this slab's own slot is written by the library
                self.recv[xch][s].copy_(self.hrecv[xch][s])

    def _move(self, xch, send, recv):
        dist, p, r = self.dist, self.p, self.r
        lo, hi = slots(p, r, xch, self.ymode)
        if (lo, hi) == (0, p - 1) and all(slots(p, t, xch, self.ymode) == (0, p - 1) for t in range(p)):
            dist.all_gather(list(recv.unbind(0)), send)
            return
        recvs = [(s, recv[s]) for s in range(lo, hi + 1) if s != r]
        sends = self.readers(xch)
        if dist.get_backend() == "nccl":
            # NCCL point-to-point must be one group: neighbours that each send before they receive
            # would otherwise wait for one another
            ops = [dist.P2POp(dist.irecv, t, s) for s, t in recvs]
            ops += [dist.P2POp(dist.isend, send, t) for t in sends]
            reqs = dist.batch_isend_irecv(ops) if ops else []
        else:
            reqs = [dist.irecv(t, s) for s, t in recvs] + [dist.isend(send, t) for t in sends]
        for q in reqs:
            q.wait()
