"""The Poisson solve of the mixed form (FP32 transforms, FP64 right-hand side, y solves in FP64
arithmetic, one refinement on the FP64 residual) against the FP64 oracle: phi, the projected
fields and the divergence, for periodic and inflow / outflow x, power-of-two and radix-3 sizes,
and a right-hand side dominated by the lowest wavenumbers."""
import math

import numpy as np
import pytest

from tests.gpu_common import B, O, need_gpu, to_np
from paper_1812_01178_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def _smooth_push(case, g, u, amp):
    """u += amp * (1 - y^2) cos(2 pi x / Lx) cos(2 pi z / Lz): a divergence in the lowest
    (kx, kz) = (1, 1) modes, amp times the scale of the random field."""
    x = np.arange(case.nx) * g.dx
    z = (np.arange(case.nz) + 0.5) * g.dz
    yc = 0.5 * (g.yf[1:] + g.yf[:-1])
    yy = (yc - yc.min()) / (yc.max() - yc.min()) * 2.0 - 1.0
    return u + amp * np.cos(2 * math.pi * z / case.lz)[:, None, None] * (1 - yy ** 2)[None, :, None] * \
        np.cos(2 * math.pi * x / case.lx)[None, None, :]


@pytest.mark.parametrize("shape,low", [((64, 37, 32), 0.0), ((48, 20, 24), 0.0), ((64, 37, 32), 30.0),
                                       ((32, 16, 96), 30.0)])
@pytest.mark.parametrize("k", [-1, 1])
def test_mixed_poisson_and_projection(shape, low, k):
    case, u, v, w, p = I.small_channel(*shape, seed=4, amp=0.2)
    g = O.Grid.from_case(case)
    if low:
        u = _smooth_push(case, g, u, low)
    s = B.Solver(case, u, v, w, p, precision=B.NS_MIXED)
    scale = 1.0 if k < 0 else O.RK3_ALPHA[k] * case.dt
    b = O.divergence(g, u, v, w)
    phi_ref = O.poisson_solve(g, b / scale)
    s.poisson(k)
    phi = to_np(s.buffer(B.NS_BUF_PHI))
    err = np.abs((phi - phi.mean()) - (phi_ref - phi_ref.mean())).max() / np.abs(phi_ref).max()
    assert err < 1e-10, err
    s.project(k)
    gu, gv, gw, gp = s.state()
    ru, rv, rw = O.project(g, u, v, w, phi_ref, scale)
    for a_, b_ in ((gu, ru), (gv, rv), (gw, rw)):
        np.testing.assert_allclose(a_, b_, rtol=0, atol=1e-10 * np.abs(b_).max())
    div = np.abs(O.divergence(g, gu, gv, gw)).max()
    assert div < 1e-10 * np.abs(b).max() + 1e-13, (div, np.abs(b).max())
    s.close()


@pytest.mark.parametrize("shape", [(64, 20, 16), (96, 13, 24)])
def test_mixed_poisson_boundary_layer(shape):
    """Inflow / outflow x: the FP32 cosine transforms and the Neumann-x residual."""
    case, u, v, w, p, bl = I.boundary_layer(*shape, amp=0.05, seed=3, re=200.0, precision=1)
    g = O.Grid.from_case(case)
    s = B.Solver(case, u, v, w, p, bl=bl)
    assert s.es == 4
    s.make_divergence_free()
    gu, gv, gw, gp = s.state()
    gbl = s.boundary()
    ru, rv, rw, rbl = O.make_divergence_free_bl(g, u, v, w, bl)
    for a_, b_ in ((gu, ru), (gv, rv), (gw, rw)):
        np.testing.assert_allclose(a_, b_, rtol=0, atol=1e-10 * np.abs(b_).max())
    assert np.abs(O.divergence_bl(g, gu, gv, gw, gbl)).max() < 1e-11
    s.close()


def test_mixed_step_profile_has_the_refinement():
    """The mixed form launches the refinement slot; the FP64 form leaves it idle."""
    case, u, v, w, p = I.small_channel(32, 16, 32, seed=2)
    for prec, active in ((B.NS_FP64, False), (B.NS_MIXED, True)):
        s = B.Solver(case, u, v, w, p, precision=prec)
        ms = s.step_profiled(2)
        assert (ms["poisson_refine"] > 0) == active, ms
        s.close()
