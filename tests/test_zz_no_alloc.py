"""The allocation-free Poisson entry point (ns_poisson_solve_static) against ns_poisson_solve.

Some callers cannot call cudaMalloc: a plugin whose host framework owns all device memory through
its own pool, or a fixed-latency loop that must not allocate after start-up.
ns_poisson_solve_static keeps its scratch in a static device array and takes only the caller's
inputs and output.  This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

from tests.gpu_common import B, need_gpu, to_np, torch
from paper_1812_01178_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _reference_phi(case, u, v, w, p, k):
    s = B.Solver(case, u, v, w, p)
    s.poisson(k)
    phi = to_np(s.buffer(B.NS_BUF_PHI))
    dev = (s.u, s.v, s.w)
    return s, phi, dev


def _static(cfg, du, dv, dw, out, k):
    B.ns_poisson_solve_static(cfg, du.data_ptr(), dv.data_ptr(), dw.data_ptr(), out.data_ptr(), k,
                              torch.cuda.current_stream().cuda_stream)


# two calls in a row on different grids and sub-steps (the second reuses the array the first left)
@pytest.mark.parametrize("calls", [(((64, 37, 32), 1), ((32, 20, 16), -1)),
                                   (((32, 20, 16), 0), ((64, 37, 32), 2))])
def test_static_poisson_matches_context_path_twice(calls):
    need_gpu()
    for n, (shape, k) in enumerate(calls):
        case, u, v, w, p = I.small_channel(*shape, seed=20 + n)
        s, phi_ref, (du, dv, dw) = _reference_phi(case, u, v, w, p, k)
        out = torch.full((case.nz, case.ny, case.nx), float("nan"), dtype=torch.float64, device=du.device)
        _static(B.make_config(case), du, dv, dw, out, k)
        got = to_np(out)
        assert np.isfinite(got).all()
        np.testing.assert_allclose(got, phi_ref, rtol=0, atol=1e-12 * np.abs(phi_ref).max())
        s.close()


def test_static_poisson_allocates_no_device_memory():
    """After a first call (which looks up the array's address and loads the kernels), a call on the
    same grid leaves the driver's free device memory unchanged."""
    need_gpu()
    case, u, v, w, p = I.small_channel(64, 37, 32, seed=31)
    du, dv, dw = (torch.from_numpy(a.copy()).cuda() for a in (u, v, w))
    out = torch.empty((case.nz, case.ny, case.nx), dtype=torch.float64, device="cuda")
    cfg = B.make_config(case)
    _static(cfg, du, dv, dw, out, 0)
    first = out.clone()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    _static(cfg, du, dv, dw, out, 0)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.equal(out, first)


def test_static_poisson_rejects_grids_beyond_the_scratch():
    need_gpu()
    case, u, v, w, p = I.small_channel(512, 64, 512)
    cfg = B.make_config(case)
    t = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(B.NSError) as ei:
        _static(cfg, t, t, t, t, 0)
    assert ei.value.status == B.NS_ERR_SIZE
    assert "scratch" in str(ei.value)


def test_static_poisson_rejects_mixed_precision_and_misaligned_pointers():
    need_gpu()
    case, u, v, w, p = I.small_channel(32, 20, 16, seed=5)
    n = case.nz * (case.ny + 1) * case.nx
    t = torch.zeros(n + 64, dtype=torch.float64, device="cuda")
    with pytest.raises(B.NSError) as ei:
        _static(B.make_config(case, precision=B.NS_MIXED), t, t, t, t, 0)
    assert ei.value.status == B.NS_ERR_UNSUPPORTED
    assert "FP64" in str(ei.value)
    cfg = B.make_config(case)
    for q in range(4):
        args = [t, t, t, t]
        args[q] = t[1:]  # 8 bytes past a 256-byte boundary
        with pytest.raises(B.NSError) as ei:
            _static(cfg, *args, 0)
        assert ei.value.status == B.NS_ERR_ARG
        assert "aligned" in str(ei.value)
