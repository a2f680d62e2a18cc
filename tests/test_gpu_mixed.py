"""Mixed precision (FP32 RHS and ADI increments on an FP64 state; FP64 divergence, Poisson,
projection and accumulation) against the FP64 oracle: per-field bounds and divergence."""
import numpy as np
import pytest

from tests.gpu_common import B, O, field_rel_errors, need_gpu
from paper_1812_01178_gb300 import inputs as I

pytestmark = pytest.mark.gpu

# Stated bounds of the mixed form after the given number of steps (relative L2 as in
# field_rel_errors); divergence stays at FP64 round-off because the projection is FP64.
BOUNDS = {"u": 1e-7, "v": 1e-7, "w": 1e-7, "p": 1e-6}


@pytest.mark.parametrize("which", ["laminar", "random"])
def test_mixed_vs_oracle(which):
    need_gpu()
    if which == "laminar":
        case, u, v, w, p = I.laminar_channel()
        nsteps = case.steps
    else:
        case, u, v, w, p = I.small_channel(64, 37, 32, amp=0.3)
        case.dt = 1e-3
        nsteps = 5
    g = O.Grid.from_case(case)
    u, v, w = O.make_divergence_free(g, u, v, w)
    ref = O.step(g, dict(u=u, v=v, w=w, p=p), case.dt, case.re, case.fx, nsteps=nsteps)
    s = B.Solver(case, u, v, w, p, precision=B.NS_MIXED)
    s.step(nsteps)
    gu, gv, gw, gp = s.state()
    errs = field_rel_errors((gu, gv, gw, gp), (ref["u"], ref["v"], ref["w"], ref["p"]))
    print("mixed vs FP64 oracle (%s, %d steps): %s" % (which, nsteps, errs))
    for k, bnd in BOUNDS.items():
        assert errs[k] < bnd, (k, errs)
    div = np.abs(O.divergence(g, gu, gv, gw)).max()
    assert div <= 1e-10, div
    s.close()


def test_mixed_rhs_and_adi_are_fp32_close():
    """Stage level: mixed RHS / ADI x on the same input agree with the oracle to FP32 accuracy."""
    need_gpu()
    case, u, v, w, p = I.small_channel(64, 37, 32)
    g = O.Grid.from_case(case)
    s = B.Solver(case, u, v, w, p, precision=B.NS_MIXED)
    r0, N0 = O.rhs(g, u, v, w, p, None, 0, case.dt, case.re, case.fx)
    s.rhs(0)
    for q, bi in enumerate([B.NS_BUF_RU, B.NS_BUF_RV, B.NS_BUF_RW]):
        got = s.buffer(bi).double().cpu().numpy()
        assert s.buffer(bi).dtype.itemsize == 4
        err = np.abs(got - r0[q]).max() / np.abs(r0[q]).max()
        assert err < 2e-5, (q, err)
    s.close()
