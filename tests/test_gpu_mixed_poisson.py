"""The Poisson solve of the mixed form (FP32 transforms, FP64 right-hand side, y solves in FP32
arithmetic on the well-conditioned modes and in FP64 on the rest (float-float in the staged
tiles), one refinement on the FP64 residual) against the FP64 oracle: phi, the projected fields
and the divergence, for periodic and inflow / outflow x, power-of-two and radix-3 sizes, and a
right-hand side dominated by the lowest wavenumbers; and the per-mode choice of arithmetic."""
import math

import numpy as np
import pytest

from tests.gpu_common import B, O, need_gpu, to_np
from tests import poisson_modes as PM
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


# nx = 24: not a multiple of 16, the y solves take the register form (the others are staged)
@pytest.mark.parametrize("shape,low", [((64, 37, 32), 0.0), ((48, 20, 24), 0.0), ((64, 37, 32), 30.0),
                                       ((32, 16, 96), 30.0), ((24, 20, 24), 30.0)])
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


@pytest.mark.parametrize("kind", ["channel_256x192x256", "bl_256x64x128", "channel_64x37x32"])
def test_mixed_poisson_mode_flags(kind):
    """The mixed form's y-solve arithmetic per (kx, kz) mode, as the library reports it
    (NS_BUF_POIS_MODE): FP64 for kz = 0 and wherever the Skeel condition number the host finds
    from the oracle's operator exceeds 4096, FP32 elsewhere (a flip is allowed only within 1e-9
    of the threshold).  Most modes take FP32; on the bench grid the lowest take FP64."""
    if kind.startswith("bl"):
        case, u, v, w, p, bl = I.boundary_layer(256, 64, 128, amp=0.0, seed=3, re=200.0, precision=1)
        s = B.Solver(case, u, v, w, p, bl=bl)
    else:
        nx, ny, nz = (int(q) for q in kind.split("_")[1].split("x"))
        if nx == 256:  # the bench grid; the field values do not enter the flags
            case = I.Case("channel", nx, ny, nz, 2 * math.pi, math.pi, I.channel_faces(ny, 2.0), re=395.0,
                          fx=1.0, dt=1e-3, precision=1)
            u, v, w, p = (np.zeros(sh) for sh in I.field_shapes(case))
        else:
            case, u, v, w, p = I.small_channel(nx, ny, nz, seed=4)
        s = B.Solver(case, u, v, w, p, precision=B.NS_MIXED)
    g = O.Grid.from_case(case)
    flags = to_np(s.buffer(B.NS_BUF_POIS_MODE)).astype(bool)
    want, kap = PM.fp32_modes(g, kind.startswith("bl"))
    assert flags.shape == want.shape
    assert not flags[0].any()
    diff = flags != want
    assert np.all(np.abs(kap[diff] / PM.KAPPA_MAX - 1.0) < 1e-9), np.argwhere(diff)[:8]
    assert flags.mean() > 0.75, flags.mean()
    if kind.startswith("channel_256"):
        assert not flags[1, 0] and not flags[1, 1]
    s.close()


def test_fp64_context_has_no_mode_flags():
    case, u, v, w, p = I.small_channel(32, 16, 32, seed=2)
    s = B.Solver(case, u, v, w, p, precision=B.NS_FP64)
    with pytest.raises(B.NSError):
        s.buffer(B.NS_BUF_POIS_MODE)
    s.close()


def test_launches_per_step():
    """ns_launches_per_step counts the step graph's kernels: 10 per sub-step in FP64, 15 in the
    mixed form (the refinement's five), with the y solve staged (nx a multiple of 16) or not."""
    case, u, v, w, p = I.small_channel(32, 16, 32, seed=2)
    s = B.Solver(case, u, v, w, p, precision=B.NS_FP64)
    assert s.launches_per_step() == 30
    s.close()
    for nx in (64, 24):
        case, u, v, w, p = I.small_channel(nx, 37, 32, seed=2)
        s = B.Solver(case, u, v, w, p, precision=B.NS_MIXED)
        assert s.launches_per_step() == 45
        s.step(1)
        s.sync()
        s.close()
