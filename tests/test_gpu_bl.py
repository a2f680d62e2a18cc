"""Inflow / convective-outflow (flat-plate) configuration: CUDA path vs the FP64 oracle."""
import numpy as np
import pytest

from tests.gpu_common import B, O, field_rel_errors, need_gpu, to_np, torch
from paper_1812_01178_gb300 import inputs as I

pytestmark = pytest.mark.gpu

SHAPES = [(64, 20, 16), (32, 13, 8), (128, 9, 32)]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def _case(nx, ny, nz, seed=3, amp=0.05):
    case, u, v, w, p, bl = I.boundary_layer(nx, ny, nz, amp=amp, seed=seed, re=200.0)
    return case, u, v, w, p, bl


@pytest.mark.parametrize("shape", SHAPES)
def test_bl_rhs_parity(shape):
    case, u, v, w, p, bl = _case(*shape)
    g = O.Grid.from_case(case)
    s = B.Solver(case, u, v, w, p, bl=bl)
    r0, N0 = O.rhs_bl(g, u, v, w, p, None, bl, 0, case.dt, case.re, case.fx)
    s.rhs(0)
    for q, (bi, bn) in enumerate([(B.NS_BUF_RU, B.NS_BUF_NU), (B.NS_BUF_RV, B.NS_BUF_NV),
                                  (B.NS_BUF_RW, B.NS_BUF_NW)]):
        np.testing.assert_allclose(to_np(s.buffer(bi)), r0[q], rtol=0, atol=1e-12 * np.abs(r0[q]).max())
        # the library stores N pre-multiplied by the sub-step's convection weight -dt gamma_k
        cn = -case.dt * O.RK3_GAMMA[0]
        np.testing.assert_allclose(to_np(s.buffer(bn)), cn * N0[q], rtol=0, atol=1e-12 * np.abs(cn * N0[q]).max())
    s.close()


@pytest.mark.parametrize("shape", SHAPES)
def test_bl_poisson_projection_parity(shape):
    case, u, v, w, p, bl = _case(*shape)
    g = O.Grid.from_case(case)
    s = B.Solver(case, u, v, w, p, bl=bl)
    s.make_divergence_free()
    gu, gv, gw, gp = s.state()
    gbl = s.boundary()
    ru, rv, rw, rbl = O.make_divergence_free_bl(g, u, v, w, bl)
    np.testing.assert_allclose(gbl["u_out"], rbl["u_out"], rtol=0, atol=1e-13)
    for a_, b_ in ((gu, ru), (gv, rv), (gw, rw)):
        np.testing.assert_allclose(a_, b_, rtol=0, atol=1e-11 * np.abs(b_).max())
    assert np.abs(O.divergence_bl(g, gu, gv, gw, gbl)).max() < 1e-11
    s.close()


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("mode", [B.NS_PART_PPT, B.NS_PART_PDD])
def test_bl_steps_parity(shape, mode):
    case, u, v, w, p, bl = _case(*shape)
    g = O.Grid.from_case(case)
    u, v, w, bl = O.make_divergence_free_bl(g, u, v, w, bl)
    ref = O.step_bl(g, dict(u=u, v=v, w=w, p=p, bl=bl), case.dt, case.re, case.fx, nsteps=3, u_conv=case.u_conv)
    s = B.Solver(case, u, v, w, p, bl=bl)
    s.set_partition(s.partition()[0], mode)
    s.step(3)
    errs = field_rel_errors(s.state(), (ref["u"], ref["v"], ref["w"], ref["p"]))
    for name in ("u", "v", "w", "p"):
        assert errs[name] < 1e-11, (name, errs)
    gbl = s.boundary()
    for q in ("u_out", "v_out", "w_out"):
        np.testing.assert_allclose(gbl[q], ref["bl"][q], rtol=0, atol=1e-12 * (np.abs(ref["bl"][q]).max() + 1e-300))
    s.close()


def test_bl_long_lines_and_mixed():
    """1024-long x-lines (long-line solver with inflow / outflow rows), FP64 and mixed."""
    case, u, v, w, p, bl = _case(1024, 8, 8)
    g = O.Grid.from_case(case)
    u, v, w, bl = O.make_divergence_free_bl(g, u, v, w, bl)
    ref = O.step_bl(g, dict(u=u, v=v, w=w, p=p, bl=bl), case.dt, case.re, case.fx, nsteps=1, u_conv=case.u_conv)
    for prec, bound in ((B.NS_FP64, 1e-11), (B.NS_MIXED, 1e-6)):
        s = B.Solver(case, u, v, w, p, bl=bl, precision=prec)
        s.step(1)
        errs = field_rel_errors(s.state(), (ref["u"], ref["v"], ref["w"], ref["p"]))
        for name in ("u", "v", "w", "p"):
            assert errs[name] < bound, (prec, name, errs)
        s.close()
