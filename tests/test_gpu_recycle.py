"""Recycling inflow: the CUDA path through the C ABI against the FP64 oracle."""
import numpy as np
import pytest

from tests.gpu_common import B, O, field_rel_errors, need_gpu
from paper_1812_01178_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def _case(nx=64, ny=24, nz=16, ir=40, delta_in=1.1, seed=5, precision=0):
    case, u, v, w, p, bl = I.boundary_layer(nx, ny, nz, amp=0.05, seed=seed, re=300.0, precision=precision)
    case.recycle_i = ir
    case.delta_in = delta_in
    g = O.Grid.from_case(case)
    u, v, w, bl = O.make_divergence_free_bl(g, u, v, w, bl)
    return case, g, u, v, w, p, bl


@pytest.mark.parametrize("shape,ir,delta_in", [((64, 24, 16), 40, 1.1), ((32, 13, 8), 5, 0.6), ((96, 20, 24), 95, 2.0)])
def test_recycled_inflow_planes_match_the_oracle(shape, ir, delta_in):
    """After sub-step 0 the inflow planes are the recycled ones of the initial fields (the inflow
    face and v_in, w_in are not changed by the rest of the sub-step)."""
    case, g, u, v, w, p, bl = _case(*shape, ir=ir, delta_in=delta_in)
    s = B.Solver(case, u, v, w, p, bl=bl)
    s.substep(0)
    ui, vi, wi = O.recycle_inflow(g, u, v, w, ir, delta_in, case.re, case.u_conv)
    gu = s.state()[0]
    gb = s.boundary()
    np.testing.assert_allclose(gu[:, :, 0], ui, rtol=0, atol=1e-13 * np.abs(ui).max())
    np.testing.assert_allclose(gb["v_in"], vi, rtol=0, atol=1e-13 * (np.abs(vi).max() + 1e-300))
    np.testing.assert_allclose(gb["w_in"], wi, rtol=0, atol=1e-13 * (np.abs(wi).max() + 1e-300))
    assert not np.allclose(ui, u[:, :, 0])
    s.close()


@pytest.mark.parametrize("prec,bound", [(B.NS_FP64, 1e-11), (B.NS_MIXED, 1e-6)])
def test_recycled_steps_match_the_oracle(prec, bound):
    case, g, u, v, w, p, bl = _case(precision=prec)
    s = B.Solver(case, u, v, w, p, bl=bl)
    s.step(3)
    ref = O.step_bl_recycled(g, dict(u=u, v=v, w=w, p=p, bl=bl), case.dt, case.re, case.fx, case.recycle_i,
                             case.delta_in, nsteps=3, u_conv=case.u_conv)
    errs = field_rel_errors(s.state(), (ref["u"], ref["v"], ref["w"], ref["p"]))
    for name in ("u", "v", "w", "p"):
        assert errs[name] < bound, (name, errs)
    gb = s.boundary()
    for q in ("v_in", "w_in", "u_out"):
        np.testing.assert_allclose(gb[q], ref["bl"][q], rtol=0, atol=10 * bound * (np.abs(ref["bl"][q]).max() + 1e-300))
    wgt = g.dy[None, :] * g.dz
    gu = s.state()[0]
    assert abs((gu[:, :, 0] * wgt).sum() - (gb["u_out"] * wgt).sum()) < 1e-10
    s.close()
