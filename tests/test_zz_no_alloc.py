"""The allocation-free Poisson entry point (ns_poisson_solve_static) against ns_poisson_solve.

Some callers cannot call cudaMalloc (an application with a stream capture open, a plugin whose
host framework owns all device memory, a fixed-latency loop).  ns_poisson_solve_static keeps its
scratch in a static device array and takes only the caller's inputs and output.  This file is
collected last so that a run stopping at the first failure has already run every other test; it
also passes alone in a fresh process.
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


@pytest.mark.parametrize("shapes", [((64, 37, 32), (32, 20, 16))])
def test_static_poisson_matches_context_path_twice(shapes):
    need_gpu()
    stream = torch.cuda.current_stream().cuda_stream
    for call, (shape, k) in enumerate(zip(shapes, (1, -1))):
        case, u, v, w, p = I.small_channel(*shape, seed=20 + call)
        s, phi_ref, (du, dv, dw) = _reference_phi(case, u, v, w, p, k)
        out = torch.full((case.nz, case.ny, case.nx), float("nan"), dtype=torch.float64, device=du.device)
        cfg = B.make_config(case)
        B.ns_poisson_solve_static(cfg, du.data_ptr(), dv.data_ptr(), dw.data_ptr(), out.data_ptr(), k, stream)
        got = to_np(out)
        assert np.isfinite(got).all()
        np.testing.assert_allclose(got, phi_ref, rtol=0, atol=1e-12 * np.abs(phi_ref).max())
        s.close()


def test_static_poisson_rejects_grids_beyond_the_scratch():
    need_gpu()
    case, u, v, w, p = I.small_channel(512, 64, 512)
    cfg = B.make_config(case)
    t = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(B.NSError) as ei:
        B.ns_poisson_solve_static(cfg, t.data_ptr(), t.data_ptr(), t.data_ptr(), t.data_ptr(), 0,
                                  torch.cuda.current_stream().cuda_stream)
    assert ei.value.status == B.NS_ERR_SIZE
    assert "scratch" in str(ei.value)
