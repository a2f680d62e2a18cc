"""Benchmark: grid-point-steps/s of the fractional-step NS step on one GB300 (N replicas, or N y-slabs).

Default workload: the turbulent-channel-sized FP64 step, 256 x 192 x 256 cells, periodic x and z,
tanh-stretched y with no-slip walls, Re_tau = 395 log-law field with 10 % Gaussian fluctuations
(seeded, synthetic), dt fixed from CFL 0.5.  One step = three RK3 sub-steps, each: RHS, ADI x
(PDD/PPT partitioned), ADI y, ADI z (+u*), divergence + z FFT, x FFT, y tridiagonal per (kx, kz),
inverse x FFT, inverse z FFT, projection.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|mixed] [--impl ours|reference]

Prints one JSON line.  N > 1 runs under torch.distributed.run: every rank advances its own
replica (the single-instance path has no data-path exchange), value = cells*steps summed over
ranks / max-over-ranks time.  With --slabs the N ranks instead share the one workload as N
y-slabs (the paper's multi-GPU decomposition, strong scaling; --backend gloo for ranks sharing a
GPU).  --impl reference times the FP64 CPU oracle on the same workload (bounded samples of it) on
the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "grid-point-steps/s at 1 GB300 (FP64 vs mixed) + % HBM roofline per sweep"
UNIT = "grid-point-steps/s"

# Algorithmic work per cell per launch of each kernel (FP64 path):
# bytes = each input read once + each output written once; flops = the per-cell estimates of the
# hot-path scope table (FMA = 2): RHS about 150, ADI about 5 per point per sweep for each of the
# three components (plus the u* = u + delta add of the z sweep), FFTs 5 N log2 N per complex
# transform of length N (2.5 log2 N per real point), the y solve about 10 per complex point, the
# projection about 15.  Complex spectral arrays have (nz/2+1)/nz of a cell each.
def kernel_model(nx, ny, nz, es):
    """(algorithmic bytes, flops) per cell of one launch of each stage.  es = 8: FP64 form, with the
    Poisson spectra in complex128.  es = 4: the mixed form, whose Poisson transforms run in FP32 on
    a complex64 spectrum around an FP64 right-hand side and one FP64 refinement; its Poisson flops
    count the FP64 work only (divergence, residual, y solves), the FP32 transforms being far from
    their pipe's bound."""
    sh = (nz // 2 + 1) / nz
    L = lambda n: math.log2(n)
    m = {
        #                 bytes per cell                       flops per cell
        "rhs":              (4 * 8 + 3 * es + 6 * es,        150.0),
        "adi_x":            (6 * es,                         15.0),
        "adi_y":            (6 * es,                         15.0),
        "adi_z":            (3 * es + 6 * 8,                 18.0),
        "poisson_div_fftz": (3 * 8 + sh * 16,                9.0 + 2.5 * L(nz) + 2.0),
        "poisson_x_fwd":    (2 * sh * 16,                    sh * 5.0 * L(nx)),
        "poisson_tdma_y":   (3 * sh * 16,                    sh * 10.0),
        "poisson_x_inv":    (2 * sh * 16,                    sh * 5.0 * L(nx)),
        # boundary-plane stages (inflow / outflow only): per cell of the volume they are tiny
        "outflow":          (8 * 3.0 * 5 / nx,               8.0 / nx),
        "flux_correct":     (8 * 3.0 / nx,                   3.0 / nx),
        "recycle":          (8 * 3.0 * 4 / nx,               40.0 / nx),
        "poisson_ifftz":    (sh * 16 + 8,                    2.5 * L(nz) + 2.0),
        "poisson_refine":   (0.0,                            0.0),
        "project":          (8 + 8 * 8,                      15.0),
    }
    if es == 4:
        cs = 8  # complex64
        m.update({
            # u, v, w in; bs (FP64) and the spectrum out
            "poisson_div_fftz": (3 * 8 + 8 + sh * cs,        9.0),
            "poisson_x_fwd":    (2 * sh * cs,                0.0),
            # spectrum in and out, the two FP64 factor planes
            "poisson_tdma_y":   (sh * (2 * cs + 16),         sh * 10.0),
            "poisson_x_inv":    (2 * sh * cs,                0.0),
            "poisson_ifftz":    (sh * cs + 4,                0.0),
            # residual (bs, phi1 in, spectrum out), the four stages again, phi = phi1 + phi2
            "poisson_refine":   (24 + 8 * sh * cs + sh * 16, 13.0 + sh * 10.0),
        })
    return m


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured", float(d.get("sm_max_mhz", 2070.0))
    except Exception:
        return 6800.0, "fallback", 2070.0


# FP64 ALU peak from unit counts and clock: 152 SMs x 2 FP64 FMA/clk/SM x 2 flop x f_max (the
# fallback when the live measurement below is not available).
def fp64_peak_tflops(sm_mhz):
    return 152 * 2 * 2 * sm_mhz * 1e6 / 1e12


def measure_fp64_peak(torch, B, dev, reps=5):
    """FP64 FMA throughput (TFLOP/s) of this GPU: the library's probe kernel (8 independent FMA
    chains per thread, 8 blocks of 256 threads per SM), best of `reps` launches, each timed with
    CUDA events on the stream it runs on.  Returns (TFLOP/s, description)."""
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    nb, it = 8 * nsm, 4096
    out = torch.empty(nb * 256, dtype=torch.float64, device=dev)
    st = torch.cuda.Stream(dev)
    flops = 16.0 * it * nb * 256
    best = 0.0
    with torch.cuda.stream(st):
        B.ns_fp64_fma_probe(out.data_ptr(), nb, it, st.cuda_stream)  # warm-up
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            B.ns_fp64_fma_probe(out.data_ptr(), nb, it, st.cuda_stream)
            e1.record(st)
            e1.synchronize()
            best = max(best, flops / (e0.elapsed_time(e1) * 1e-3) / 1e12)
    if not bool(torch.isfinite(out).all()):
        raise RuntimeError("FP64 probe produced non-finite values")
    return best, ("measured live: ns_fp64_fma_probe, %d blocks x 256 threads x 8 chains x %d FMAs, best of %d "
                  "(CUDA events)" % (nb, it, reps))


def fp32_peak_tflops(sm_mhz):
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


def load_traffic(workload, kernel, key="bytes_per_launch"):
    """A counter figure of `kernel` from the committed ncu capture of this workload (DRAM bytes per
    launch by default; "fp64_inst_per_cell": executed FP64 instructions per cell), or None if there
    is none or the kernel's source file changed since the counters were taken."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic_%s.json" % workload)) as fh:
            rec = json.load(fh).get(kernel)
        if rec is None:
            return None
        with open(os.path.join(ROOT, rec["source"]), "rb") as fh:
            if hashlib.sha256(fh.read()).hexdigest()[:16] != rec["source_sha256_16"]:
                return None
        return rec.get(key)
    except Exception:
        return None


def host_cpu():
    """The host CPU's model name from /proc/cpuinfo, else its architecture."""
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                key, _, val = line.partition(":")
                if key.strip().lower() == "model name" and val.strip():
                    return val.strip()
    except OSError:
        pass
    import platform
    return platform.machine() or "unknown"


def max_over_ranks(torch, dist, seconds, device="cpu"):
    """The slowest rank's time: every rank passes its own, every rank gets the maximum.  With
    dist None (one process) it is the time itself."""
    if dist is None:
        return seconds
    t = torch.tensor([seconds], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, cells, steps, seconds):
    """Whole-job grid-point-steps/s: every rank advances its own replica of `cells` cells."""
    return world * cells * steps / seconds


def nvtx_push(torch, name):
    """Marks a timed region, so that an ncu launch list can be restricted to it (--nvtx-include)."""
    try:
        torch.cuda.nvtx.range_push(name)
    except Exception:
        pass


def nvtx_pop(torch):
    try:
        torch.cuda.nvtx.range_pop()
    except Exception:
        pass


# ------------------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = str(gpu_index)
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu, "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                pw.append(float(parts[3]))
            except ValueError:
                continue
            for n, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(pw) if pw else None, "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------------------------ oracle sample
def oracle_sample_substep(O, g, st, k, dt, re, fx, F, part=0):
    """One RK3 sub-step of the FP64 oracle on 1/F of every stage's work, line lengths unchanged:
    RHS, x and y sweeps, x transforms and projection on a z-slab of nz/F planes; z sweeps and z
    transforms on nx/F x-columns (all nz planes); y solves on the slab's nz/F spanwise modes."""
    nz, ny, nx = g.nz, g.ny, g.nx
    nzs = max(1, nz // F)
    k0 = (part * nzs) % nz
    ncol = max(1, nx // F)
    i0 = (part * ncol) % nx
    gs = O.Grid(nx, ny, nzs, g.lx, g.lz * nzs / nz, g.yf, g.ytop)
    sl = slice(k0, k0 + nzs)
    cols = slice(i0, i0 + ncol)
    u, v, w, p = (st[q][sl] for q in ("u", "v", "w", "p"))
    nprev = None if k == 0 else [a[sl] for a in st["nprev"]]
    r, N = O.rhs(gs, u, v, w, p, nprev, k, dt, re, fx)
    beta = O.RK3_ALPHA[k] * dt / (2 * re)
    d = [O.adi_sweep(gs, r[c], 0, c, beta) for c in range(3)]
    d = [O.adi_sweep(gs, d[c], 1, c, beta) for c in range(3)]
    zcols = [st[q][:, :, cols] for q in ("u", "v", "w")]
    [O.adi_sweep(g, zc, 2, c, beta) for c, zc in enumerate(zcols)]
    us, vs, ws = u + d[0], v + d[1], w + d[2]
    b = O.divergence(gs, us, vs, ws) / (O.RK3_ALPHA[k] * dt)
    bh = O.dft(b.astype(np.complex128), 2)
    O.dft(st["p"][:, :, cols].astype(np.complex128), 0)
    a_, c_ = O.poisson_ycoeffs(g)
    lam = O.modified_wavenumbers(nz, g.dz)[sl][:, None] + O.modified_wavenumbers(nx, g.dx)[None, :]
    dd = np.moveaxis(bh, 1, -1)
    B = -(a_ + c_)[None, None, :] - lam[:, :, None]
    ph = np.moveaxis(O.thomas(a_, B, c_, dd), -1, 1)
    O.dft(st["p"][:, :, cols].astype(np.complex128), 0, +1)
    phi = O.dft(ph, 2, +1).real / (nx * nz)
    O.project(gs, us, vs, ws, phi, O.RK3_ALPHA[k] * dt)
    return N


def oracle_baseline(case, u, v, w, p, F, nsub, warm=0):
    """Time nsub sample sub-steps (k = 0, 1, 2, ...) of the oracle; returns (cell-steps/s, seconds)."""
    from oracle import ns_oracle as O
    g = O.Grid.from_case(case)
    st = dict(u=u, v=v, w=w, p=p)
    st["nprev"] = [np.zeros_like(u), np.zeros_like(v), np.zeros_like(w)]
    for q in range(warm):
        oracle_sample_substep(O, g, st, q % 3, case.dt, case.re, case.fx, F, part=q)
    t0 = time.perf_counter()
    for q in range(nsub):
        oracle_sample_substep(O, g, st, q % 3, case.dt, case.re, case.fx, F, part=q)
    t = time.perf_counter() - t0
    # nsub sample sub-steps = nsub / (3 F) full steps of the workload
    return case.cells() * (nsub / (3.0 * F)) / t, t


def bench_cfl(B, dev, case, u0, v0, w0, p0, steps, cells):
    """Steps at a fixed CFL number of 1.0 (the paper's runs): each step's graph reduces the
    convective rate, sets dt and rebuilds every dt table on the device, then steps; the dt log is
    read back once per call.  Host wall clock with a device synchronisation on both sides, beside
    the same number of fixed-dt steps on the same clock."""
    s = B.Solver(case, u0, v0, w0, p0, device=str(dev))
    s.make_divergence_free()
    s.step_cfl(3, 1.0)
    s.sync()
    t0 = time.perf_counter()
    dts = s.step_cfl(steps, 1.0)
    s.sync()
    t = time.perf_counter() - t0
    # the same number of steps at a fixed dt (the last one), same clock
    s.step(1)
    s.sync()
    t1 = time.perf_counter()
    s.step(steps)
    s.sync()
    tf = time.perf_counter() - t1
    s.close()
    return {"cfl": 1.0, "steps": steps, "value": cells * steps / t, "unit": UNIT, "ms_per_step": 1e3 * t / steps,
            "fixed_dt_ms_per_step_same_clock": 1e3 * tf / steps, "dt_min": min(dts), "dt_max": max(dts),
            "timing": "host wall clock around synchronised steps (rate, dt and tables on the device)"}


def bench_ensemble(B, torch, dev, args):
    """64 uneven channel instances: batched (one persistent launch per stage, one graph per step)
    against the same instances stepped one context at a time; FP64 and mixed."""
    from paper_1812_01178_gb300 import inputs as I
    ens = I.ensemble(64)
    cells = sum(e[0].cells() for e in ens)
    out = {"workload": "ensemble_64_channels_32^3_to_128x96x128", "instances": len(ens), "cells": cells}
    steps = max(5, args.steps // 5)
    for prec, tag in ((0, "fp64"), (1, "mixed")):
        for e in ens:
            e[0].precision = prec
        b = B.Batch([e[0] for e in ens], [e[1:] for e in ens], device=str(dev))
        b.autotune()
        b.make_divergence_free()
        b.step(args.warmup)
        b.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(b.stream)
        b.step(steps)
        e1.record(b.stream)
        torch.cuda.synchronize()
        tb = e0.elapsed_time(e1)
        launches = b.launches_per_step()
        parts = [B.ns_get_partition(b.instance(q))[:2] for q in range(len(ens))]
        b.close()
        solvers = [B.Solver(e[0], *e[1:], device=str(dev)) for e in ens]
        seq_launches = sum(s.launches_per_step() for s in solvers)
        for s, pm in zip(solvers, parts):
            s.set_partition(*pm)
            s.make_divergence_free()
            s.step(args.warmup)
        torch.cuda.synchronize()
        e0.record(solvers[0].stream)
        for _ in range(steps):
            for s in solvers:
                s.step(1)
        e1.record(solvers[0].stream)
        torch.cuda.synchronize()
        ts = e0.elapsed_time(e1)
        for s in solvers:
            s.close()
        out[tag] = {"value": cells * steps / (tb * 1e-3), "ms_per_step": tb / steps,
                    "batched_launches_per_step": launches, "sequential_value": cells * steps / (ts * 1e-3),
                    # the kernel nodes of each instance's step graph
                    "sequential_launches_per_step": seq_launches,
                    "speedup_vs_sequential": ts / tb}
    out["mixed_speedup_vs_fp64"] = out["fp64"]["ms_per_step"] / out["mixed"]["ms_per_step"]
    return out


# ------------------------------------------------------------------------------ boundary layers
def device_bl_fields(torch, I, dev, case, slab=8, workers=8):
    """The boundary-layer initial field built a few z planes at a time on the host (threads; each
    slab is bit for bit that plane range of the whole-field generator) and copied into device
    tensors, so host memory holds a few slabs only.  Sets case.dt from CFL 0.5 on that field."""
    from concurrent.futures import ThreadPoolExecutor
    nx, ny, nz = case.nx, case.ny, case.nz
    f64 = dict(dtype=torch.float64, device=dev)
    u = torch.empty((nz, ny, nx), **f64)
    v = torch.empty((nz, ny + 1, nx), **f64)
    w = torch.empty((nz, ny, nx), **f64)
    p = torch.zeros((nz, ny, nx), **f64)
    bl = {q: torch.empty((nz, rows), **f64) for q, rows in
          (("u_out", ny), ("v_in", ny + 1), ("v_out", ny + 1), ("w_in", ny), ("w_out", ny))}

    def gen(k0):
        k1 = min(nz, k0 + slab)
        su, sv, sw, sbl = I.boundary_layer_slab(case, k0, k1)
        return k0, k1, su, sv, sw, sbl, I.boundary_layer_rate(case, su, sv, sw)

    rate = 0.0
    with ThreadPoolExecutor(workers) as ex:
        for k0, k1, su, sv, sw, sbl, r in ex.map(gen, range(0, nz, slab)):
            rate = max(rate, r)
            for t, a in ((u, su), (v, sv), (w, sw)):
                t[k0:k1].copy_(torch.from_numpy(a))
            for q, a in sbl.items():
                bl[q][k0:k1].copy_(torch.from_numpy(a))
    case.dt = 0.5 / rate
    return u, v, w, p, bl


def device_max_divergence(torch, s, case, slab=32):
    """max over cells of |D u| (inflow / outflow x, periodic z), evaluated on the device a few z
    planes at a time (measurement bookkeeping with torch; the solver's work is the library's)."""
    dx, dz = case.lx / case.nx, case.lz / case.nz
    dy = torch.as_tensor(np.diff(case.yf), device=s.u.device)[None, :, None]
    out = 0.0
    nz = case.nz
    for k0 in range(0, nz, slab):
        k1 = min(nz, k0 + slab)
        u, v, w = s.u[k0:k1], s.v[k0:k1], s.w[k0:k1]
        ux = torch.cat([u[:, :, 1:], s.bl["u_out"][k0:k1, :, None]], dim=2)
        wz = s.w[[(k + 1) % nz for k in range(k0, k1)]]
        d = (ux - u) / dx + (v[:, 1:] - v[:, :-1]) / dy + (wz - w) / dz
        out = max(out, float(d.abs().max()))
    return out


def timed_steps(torch, s, start, steps, warmup, gpu_index):
    """warmup steps (graph capture), the projected start restored, then `steps` steps timed with
    CUDA events on the solver's stream and clocks sampled.  Returns (ms, clocks)."""
    s.step(warmup)
    s.sync()
    for t, a in zip(solver_state(s), start):
        t.copy_(a)
    ck = ClockSampler(gpu_index)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ck.start()
    time.sleep(0.3)
    ev0.record(s.stream)
    s.step(steps)
    ev1.record(s.stream)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1), ck.stop()


def solver_state(s):
    """Everything a step reads: u, v, w, p and the boundary planes (N_prev is not read by the
    first sub-step, whose zeta is 0)."""
    return [s.u, s.v, s.w, s.p] + [s.bl[q] for q in sorted(s.bl)]


def kernel_fracs(model, kms, launches, cells, hbm):
    out = {}
    for name, ms in kms.items():
        if ms <= 0.0:
            continue
        per = ms / launches
        gbps = model[name][0] * cells / (per * 1e-3) / 1e9
        out[name] = {"ms_per_launch": round(per, 4), "GBps": round(gbps, 1), "hbm_frac_algorithmic": round(gbps / hbm, 4)}
    return out


def bench_boundary_layer(B, torch, I, dev, gpu_index, nx, ny, nz, steps, fp64_ref, warmup=2):
    """The paper-scale flat-plate workloads (inflow / convective outflow in x, wall and stress-free
    top in y, periodic z), mixed form, `steps` steps timed like the headline.  With fp64_ref, the
    FP64 form also runs the same steps from the same projected start, and the record reports the
    per-field relative L2 difference of the mixed form from it."""
    hbm, _, _ = load_peaks()
    case = I.boundary_layer_case(nx, ny, nz, steps=steps)
    cells = case.cells()
    t0 = time.perf_counter()
    u, v, w, p, bl = device_bl_fields(torch, I, dev, case)
    rec = {"workload": "boundary_layer_%dx%dx%d" % (nx, ny, nz), "cells": cells, "steps": steps, "dt": case.dt,
           "cfl": 0.5, "re": case.re, "bc": "inflow / convective outflow x; wall + stress-free top y; periodic z",
           "inputs_s": round(time.perf_counter() - t0, 1)}
    free0 = torch.cuda.mem_get_info(dev)[0]
    torch.cuda.reset_peak_memory_stats(dev)
    # the start: projected in FP64 (outflow flux corrected first), shared by both forms
    case.precision = 0
    sa = B.Solver(case, u, v, w, p, bl=bl, device=str(dev))
    sa.make_divergence_free()
    sa.sync()
    start = [t.clone() for t in solver_state(sa)]
    ref = None
    if fp64_ref:
        ms, ck = timed_steps(torch, sa, start, steps, warmup, gpu_index)
        ref = [t.clone() for t in (sa.u, sa.v, sa.w, sa.p)]  # after exactly `steps` steps
        rec["fp64"] = {"value": cells * steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps, "clocks": ck,
                       "max_divergence": device_max_divergence(torch, sa, case)}
        rec["fp64"]["kernels"] = kernel_fracs(kernel_model(nx, ny, nz, 8), sa.step_profiled(1), 3, cells, hbm)
    sa.close()
    del sa, u, v, w, p, bl
    # the mixed form from the same start
    case.precision = 1
    sm = B.Solver(case, *[t.clone() for t in start[:4]], bl={q: t.clone() for q, t in zip(sorted(start_bl_names()), start[4:])},
                  device=str(dev))
    sm.autotune()
    for t, a in zip(solver_state(sm), start):
        t.copy_(a)
    P, mode, drop = sm.partition()
    rec["partition_x"] = {"P": P, "rows": nx // P, "mode": "PDD" if mode == B.NS_PART_PDD else "PPT",
                          "pdd_dropped": drop, "chosen_by": "ns_autotune"}
    ms, ck = timed_steps(torch, sm, start, steps, warmup, gpu_index)
    rec["mixed"] = {"value": cells * steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps, "clocks": ck,
                    "max_divergence": device_max_divergence(torch, sm, case)}
    if ref is not None:
        vel = math.sqrt(sum(float(torch.linalg.vector_norm(t)) ** 2 for t in ref[:3]))
        err = {n: float(torch.linalg.vector_norm(getattr(sm, n) - r)) / vel for n, r in zip("uvw", ref[:3])}
        pa = ref[3] - ref[3].mean()
        pb = sm.p - sm.p.mean()
        err["p"] = float(torch.linalg.vector_norm(pb - pa)) / max(float(torch.linalg.vector_norm(pa)),
                                                                  vel * vel / math.sqrt(pa.numel()))
        rec["rel_l2_mixed_vs_fp64_after_%d_steps" % steps] = err
        rec["speedup_mixed_vs_fp64"] = rec["fp64"]["ms_per_step"] / rec["mixed"]["ms_per_step"]
    rec["mixed"]["kernels"] = kernel_fracs(kernel_model(nx, ny, nz, 4), sm.step_profiled(1), 3, cells, hbm)
    state_bytes = sum(t.numel() * 8 for t in solver_state(sm))
    rec["footprint"] = {"state_bytes": state_bytes, "workspace_bytes": sm.ws.numel(),
                        "torch_allocator_peak_bytes": torch.cuda.max_memory_allocated(dev),
                        "device_used_bytes_at_end": free0 - torch.cuda.mem_get_info(dev)[0],
                        "note": "peak includes the saved projected start and, with fp64_ref, the FP64 run"}
    sm.close()
    del sm, start, ref
    torch.cuda.empty_cache()
    return rec


def start_bl_names():
    return ("u_out", "v_in", "v_out", "w_in", "w_out")


# ------------------------------------------------------------------------------ y slabs
def bench_slabs(B, torch, dev, s_single, case, steps=5):
    """The bench workload split into p y-slabs held on this one GPU (the paper's decomposition,
    Sec. 3.2, with the exchanges as device copies): time per step against the single context,
    and the difference of the fields after the timed steps.  This measures what the decomposition
    itself costs (reduced systems, spike corrections, halo rows, exchange copies), not multi-GPU
    scaling."""
    from paper_1812_01178_gb300 import slabs as S
    start = [t.detach().cpu().numpy() for t in (s_single.u, s_single.v, s_single.w, s_single.p)]
    one = B.Solver(case, *start, device=str(dev))
    one.step(1)
    for t, a in zip((one.u, one.v, one.w, one.p), start):
        t.copy_(torch.from_numpy(a))
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(one.stream)
    one.step(steps)
    ev1.record(one.stream)
    torch.cuda.synchronize()
    t_one = ev0.elapsed_time(ev1) / steps
    ref = [t.cpu().numpy() for t in (one.u, one.v, one.w, one.p)]
    one.close()
    out = {"workload": "turbulent_channel_%dx%dx%d_fp64" % (case.nx, case.ny, case.nz), "steps": steps,
           "single_context_ms_per_step": t_one,
           "timing": "CUDA events around steps issued phase by phase from the host, one stream per slab",
           "exchange": "device copies between slabs on one GPU (slabs.LocalExchange), ordered by events"}
    for p in (2, 4):
        # one stream per slab: the slabs' kernels overlap on the GPU as they would on p GPUs
        slabs = [S.Slab(case, p, r, *start, device=str(dev), stream=torch.cuda.Stream(dev)) for r in range(p)]
        ex = S.LocalExchange(slabs)
        S.run_steps(slabs, ex, 1)  # warm-up
        torch.cuda.synchronize()
        for sl in slabs:  # restore the start (halo rows come from the first exchange)
            sl.u.copy_(torch.from_numpy(start[0][:, sl.j0 - sl.hb:sl.j1 + sl.ha].copy()))
            sl.v.copy_(torch.from_numpy(start[1][:, sl.j0 - sl.hb:sl.j1 + sl.ha + 1].copy()))
            sl.w.copy_(torch.from_numpy(start[2][:, sl.j0 - sl.hb:sl.j1 + sl.ha].copy()))
            sl.pr.copy_(torch.from_numpy(start[3][:, sl.j0 - sl.hb:sl.j1 + sl.ha].copy()))
        torch.cuda.synchronize()
        ev0.record(slabs[0].stream)
        for sl in slabs[1:]:
            sl.stream.wait_event(ev0)
        S.run_steps(slabs, ex, steps)
        for sl in slabs[1:]:
            e = torch.cuda.Event()
            e.record(sl.stream)
            slabs[0].stream.wait_event(e)
        ev1.record(slabs[0].stream)
        torch.cuda.synchronize()
        t_p = ev0.elapsed_time(ev1) / steps
        parts = [sl.owned() for sl in slabs]
        got = [np.concatenate([q[f] for q in parts], axis=1) for f in range(4)]
        vel = math.sqrt(sum(float(np.linalg.norm(a)) ** 2 for a in ref[:3]))
        err = {n: float(np.linalg.norm(g - r)) / vel for n, g, r in zip("uvw", got[:3], ref[:3])}
        out["p%d" % p] = {"ms_per_step": t_p, "vs_single_context": t_p / t_one,
                          "y_sweep": "PDD" if slabs[0].ymode == B.NS_PART_PDD else "PPT",
                          "pdd_dropped": slabs[0].ydrop, "rel_l2_vs_single_context": err,
                          "rows_per_slab": [sl.j1 - sl.j0 for sl in slabs]}
        for sl in slabs:
            sl.close()
    return out


def run_slabs_mode(args, torch, B, dev, dist, world, rank, case, u0, v0, w0, p0, config, gpu_index):
    """--slabs: the bench workload cut into `world` y-slabs, one per rank, as the paper's multi-GPU
    method does (Sec. 3.2, Algorithm 1): strong scaling of the one workload.  The exchanges go over
    torch.distributed (NCCL between GPUs; gloo, staged through host memory, for a run whose ranks
    share a GPU).  Every rank projects the same seeded field with one context, keeps its slab, and
    steps; the time is the slowest rank's."""
    from paper_1812_01178_gb300 import slabs as S
    s0 = B.Solver(case, u0, v0, w0, p0, device=str(dev))
    s0.make_divergence_free()
    start = [t.cpu().numpy() for t in (s0.u, s0.v, s0.w, s0.p)]
    s0.close()
    slab = S.Slab(case, world, rank, *start, device=str(dev))
    if dist is None:  # one slab: every slot it reads is its own, which the library writes
        ex = lambda xch: None
    else:
        ex = S.DistExchange(dist, world, rank, slab.ymode, slab.send, slab.recv, host=(args.backend == "gloo"))
    S.run_steps([slab], ex, args.warmup)
    slab.sync()
    if dist:
        dist.barrier()
    clocks = ClockSampler(gpu_index)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    ev0.record(slab.stream)
    S.run_steps([slab], ex, args.steps, first=False)  # the warm-up's last exchange filled the halos
    ev1.record(slab.stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    if dist:
        dist.barrier()
    t_max = max_over_ranks(torch, dist, ev0.elapsed_time(ev1), dev if args.backend == "nccl" else "cpu")
    cells = case.cells()
    rows = [S.rows(case.ny, world, r) for r in range(world)]
    ymode = "PDD" if slab.ymode == B.NS_PART_PDD else "PPT"
    slab.close()
    if rank != 0:
        return
    config = dict(config, parallelism="y-slabs x%d (%s)" % (world, args.backend),
                  slab_rows=[j1 - j0 for j0, j1 in rows], y_sweep=ymode)
    out = {"metric": METRIC, "value": cells * args.steps / (t_max * 1e-3), "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
           "scaling": "strong", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded Re_tau 395 log-law channel field, 10% Gaussian fluctuations, projected)",
           "config": config, "clocks": ck, "e2e": None,
           "note": "one y-slab per rank, exchanges over torch.distributed between phases (host-driven)"}
    print(json.dumps(out))


# ------------------------------------------------------------------------------ main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--no-cfl", action="store_true")
    ap.add_argument("--no-bl", action="store_true", help="skip the 134M- and 604M-cell boundary-layer records")
    ap.add_argument("--no-slabs", action="store_true", help="skip the y-slab record (slabs held on one GPU)")
    ap.add_argument("--slabs", action="store_true",
                    help="N > 1: cut the workload into N y-slabs, one per rank (strong scaling), instead of replicas")
    ap.add_argument("--backend", choices=["nccl", "gloo"], default="nccl",
                    help="process group of --slabs (gloo stages the exchanges through host memory)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference" and rank != 0:
        return  # the reference arm runs on rank 0 alone; the other ranks exit without work

    from paper_1812_01178_gb300 import inputs as I
    case, u0, v0, w0, p0 = I.turbulent_channel()
    case.precision = 1 if args.precision == "mixed" else 0
    cells = case.cells()
    config = {"workload": "turbulent_channel_256x192x256_%s" % args.precision, "nx": case.nx, "ny": case.ny,
              "nz": case.nz, "re_tau": case.re, "dt": case.dt, "cfl": 0.5, "bc": "periodic x,z; no-slip walls y",
              "precision": args.precision, "l2": "inputs larger than L2 (state 0.40 GB + workspace)"}

    if args.impl == "reference":
        import multiprocessing
        F = 1  # every step: one whole RK3 sub-step of the workload (about 3 s on 16 host cores)
        t_all0 = time.perf_counter()
        val, t = oracle_baseline(case, u0, v0, w0, p0, F, args.steps, warm=args.warmup)
        cores = os.cpu_count()
        sample = ("each step: one RK3 sub-step of the FP64 numpy oracle on the whole workload, counted as "
                  "1/3 of a time step")
        out = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
               "data": "synthetic (seeded Re_tau 395 log-law channel field)", "config": config,
               "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "cpu": host_cpu(), "kind": "oracle",
                                "sample": sample},
               "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
               "gpu_launches": 0, "wall_s": time.perf_counter() - t_all0}
        print(json.dumps(out))
        return

    # cpu baseline first, in this process, before any CUDA work
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not args.slabs:
        F = 1  # the whole workload: two RK3 steps, about 18 s on 16 host cores
        val, t = oracle_baseline(case, u0, v0, w0, p0, F, 6)
        cpu = {"value": val, "unit": UNIT, "cores": os.cpu_count(), "cpu": host_cpu(), "kind": "oracle",
               "sample": "two RK3 steps (6 sub-steps) of the FP64 numpy oracle on the whole workload; %.1f s" % t}

    import torch
    from paper_1812_01178_gb300 import binding as B
    import __graft_entry__
    __graft_entry__.build()

    # ranks sharing a GPU (only with --slabs --backend gloo) take it modulo the visible devices
    local = local % max(1, torch.cuda.device_count()) if args.backend == "gloo" else local
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        if args.backend == "gloo":
            dist.init_process_group("gloo")
        else:
            dist.init_process_group("nccl", device_id=dev)
    if args.slabs:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        run_slabs_mode(args, torch, B, dev, dist, world, rank, case, u0, v0, w0, p0, config,
                       vis.split(",")[local] if vis else str(local))
        if dist:
            dist.destroy_process_group()
        return

    fp64_live = None
    try:
        fp64_live = measure_fp64_peak(torch, B, dev)
    except Exception as exc:  # the derived figure stands in, and the line says so
        sys.stderr.write("FP64 probe failed: %s\n" % exc)

    s = B.Solver(case, u0, v0, w0, p0, device=str(dev))
    s.make_divergence_free()
    s.step(args.warmup)
    s.step_profiled(1)
    s.sync()
    launches_step = s.launches_per_step()
    P, mode, drop = s.partition()
    config["partition_x"] = {"P": P, "mode": "PDD" if mode == B.NS_PART_PDD else "PPT", "pdd_dropped": drop}

    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    gpu_index = vis.split(",")[local] if vis else str(local)
    clocks = ClockSampler(gpu_index)
    stream = s.stream
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    nvtx_push(torch, "bench_timed")
    ev0.record(stream)
    kms = s.step_profiled(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    nvtx_pop(torch)
    ck = clocks.stop()
    if dist:
        dist.barrier()
    t_ms = ev0.elapsed_time(ev1)
    t_max = max_over_ranks(torch, dist, t_ms, dev)
    value = job_throughput(world, cells, args.steps, t_max * 1e-3)

    # per-kernel roofline of the dominant kernel
    hbm, hbm_kind, smax = load_peaks()
    es = 4 if args.precision == "mixed" else 8
    model = kernel_model(case.nx, case.ny, case.nz, es)
    launches = 3 * args.steps
    kern = {}
    for name, ms in kms.items():
        if ms <= 0.0:
            continue  # stage not launched in this configuration
        per = ms / launches
        b, f = model[name]
        gbps = b * cells / (per * 1e-3) / 1e9
        kern[name] = {"ms_per_launch": per, "share": ms / max(sum(kms.values()), 1e-9),
                      "GBps": gbps, "GFLOPps": f * cells / (per * 1e-3) / 1e9,
                      # % of the HBM roofline: algorithmic bytes, and the ncu DRAM bytes of the
                      # committed capture (null once the kernel's source has changed)
                      "hbm_frac_algorithmic": gbps / hbm}
        tr = load_traffic(config["workload"], name)
        kern[name]["hbm_frac_measured"] = (tr / (per * 1e-3) / 1e9 / hbm) if tr else None
    top = max(kms, key=kms.get)
    b, f = model[top]
    per = kms[top] / launches
    fp64 = not (args.precision == "mixed" and top in ("rhs", "adi_x", "adi_y"))
    if fp64 and fp64_live:
        alu_peak, alu_src = fp64_live[0] * 1e12, fp64_live[1]
    else:
        alu_peak = (fp64_peak_tflops(smax) if fp64 else fp32_peak_tflops(smax)) * 1e12
        alu_src = "derived: 152 SMs x %s FMA/clk/SM x 2 x %.0f MHz" % ("2 FP64" if fp64 else "128 FP32", smax)
    t_alu = f * cells / alu_peak
    t_mem = b * cells / (hbm * 1e9)
    traffic = load_traffic(config["workload"], top)
    if t_alu >= t_mem:
        ach = f * cells / (per * 1e-3) / 1e12
        roof = {"kernel": top, "bound": "alu", "achieved": ach, "peak": alu_peak / 1e12, "unit": "TFLOP/s",
                "frac": ach / (alu_peak / 1e12), "traffic": traffic, "peak_source": alu_src,
                "algorithmic_flops_per_cell": f, "cells_per_launch": cells,
                "algorithmic_flops_per_launch": f * cells, "ms_per_launch": per}
        # executed FP64 instructions per cell (ncu opcode counters of the committed capture) against
        # the pipe's instruction rate, which is half the FMA flop rate
        ipc = load_traffic(config["workload"], top, "fp64_inst_per_cell") if fp64 else None
        roof["fp64_inst_per_cell"] = ipc
        roof["fp64_issue_frac"] = (ipc * cells / (per * 1e-3) / (alu_peak / 2.0)) if ipc else None
    else:
        ach = b * cells / (per * 1e-3) / 1e9
        roof = {"kernel": top, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                "frac": ach / hbm, "traffic": traffic, "peak_source": "%s hbm_gbs" % hbm_kind,
                "algorithmic_bytes_per_launch": b * cells}

    # end to end through the host-buffer entry point (pinned host memory)
    hu = torch.from_numpy(np.ascontiguousarray(u0)).pin_memory().numpy()
    hv = torch.from_numpy(np.ascontiguousarray(v0)).pin_memory().numpy()
    hw = torch.from_numpy(np.ascontiguousarray(w0)).pin_memory().numpy()
    hp = torch.from_numpy(np.ascontiguousarray(p0)).pin_memory().numpy()
    e2e = None
    if args.e2e_steps > 0:
        B.ns_step_host(s.ctx, hu, hv, hw, hp, 1)
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            B.ns_step_host(s.ctx, hu, hv, hw, hp, 1)
        te = max_over_ranks(torch, dist, time.perf_counter() - t0, dev)
        nbytes = (hu.nbytes + hv.nbytes + hw.nbytes + hp.nbytes)
        e2e = {"value": job_throughput(world, cells, args.e2e_steps, te), "unit": UNIT, "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes, "steps": args.e2e_steps,
               "path": "ns_step_host: pinned host state -> device, one step, device -> host, sync"}
    # mixed precision on the same workload: throughput, speedup, and difference from FP64
    mixed = None
    if args.precision == "fp64" and not args.no_mixed:
        sm = B.Solver(case, u0, v0, w0, p0, precision=B.NS_MIXED, device=str(dev))
        sm.make_divergence_free()
        sm.step(args.warmup)
        sm.sync()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        nvtx_push(torch, "bench_timed_mixed")
        ev0.record(sm.stream)
        sm.step(args.steps)
        ev1.record(sm.stream)
        torch.cuda.synchronize()
        nvtx_pop(torch)
        tm = max_over_ranks(torch, dist, ev0.elapsed_time(ev1), dev)
        kmix = sm.step_profiled(max(3, args.steps // 5))
        sm.close()
        # accuracy: both forms from the same projected state, 10 steps
        sa = B.Solver(case, u0, v0, w0, p0, device=str(dev))
        sb = B.Solver(case, u0, v0, w0, p0, precision=B.NS_MIXED, device=str(dev))
        sa.make_divergence_free()
        sb.make_divergence_free()
        sa.step(10)
        sb.step(10)
        sa.sync()
        sb.sync()
        vel = math.sqrt(sum(float(torch.linalg.vector_norm(t)) ** 2 for t in (sa.u, sa.v, sa.w)))
        err = {n: float(torch.linalg.vector_norm(getattr(sb, n) - getattr(sa, n))) / vel for n in ("u", "v", "w")}
        pa = sa.p - sa.p.mean()
        pb = sb.p - sb.p.mean()
        err["p"] = float(torch.linalg.vector_norm(pb - pa)) / max(float(torch.linalg.vector_norm(pa)),
                                                                  vel * vel / math.sqrt(pa.numel()))
        sa.close()
        sb.close()
        mixed = {"value": job_throughput(world, cells, args.steps, tm * 1e-3), "ms_per_step": tm / args.steps,
                 "speedup_vs_fp64": t_max / tm, "rel_l2_vs_fp64_after_10_steps": err,
                 "dtype": "f32 increments (rhs, adi) on f64 state; f64 divergence, y solves and projection; f32 poisson transforms with one f64 refinement",
                 "kernel_ms_per_step": {k: v / max(3, args.steps // 5) for k, v in kmix.items() if v > 0}}

    # fixed-CFL stepping (dt from a device max-reduction before every step)
    cflsec = None
    if args.precision == "fp64" and not args.no_cfl:
        cflsec = bench_cfl(B, dev, case, u0, v0, w0, p0, min(args.steps, 20), cells)

    # batched ensemble of uneven instances (64 laminar channels, 32^3 .. 128x96x128)
    ensemble = None
    if not args.no_ensemble:
        ensemble = bench_ensemble(B, torch, dev, args)

    # the paper-scale boundary layers (one GPU only: the records are single-GPU figures)
    bls = None
    if args.precision == "fp64" and not args.no_bl and world == 1:
        from paper_1812_01178_gb300 import inputs as I
        bls = {"1024x256x512": bench_boundary_layer(B, torch, I, dev, gpu_index, 1024, 256, 512, 50, True),
               "2048x288x1024": bench_boundary_layer(B, torch, I, dev, gpu_index, 2048, 288, 1024, 20, False)}

    # the y-slab decomposition with its slabs on this GPU (one GPU only)
    slabrec = None
    if args.precision == "fp64" and not args.no_slabs and world == 1:
        slabrec = bench_slabs(B, torch, dev, s, case)

    s.close()
    if dist:
        dist.destroy_process_group()
    if rank != 0:
        return
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f64+f32",
           "data": "synthetic (seeded Re_tau 395 log-law channel field, 10% Gaussian fluctuations, projected)",
           "config": config, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
           "fp64_peak": ({"tflops": fp64_live[0], "source": fp64_live[1]} if fp64_live else None),
           "gpu_launches": launches_step * args.steps, "clocks": ck, "mixed": mixed, "fixed_cfl": cflsec, "ensemble": ensemble, "boundary_layer": bls, "slabs_one_gpu": slabrec,
           "kernels": {k: {kk: (round(vv, 4) if vv is not None else None) for kk, vv in d.items()}
                       for k, d in kern.items()}}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
