"""Pins of the oracle's RK3 / ADI / projection time step (Sec. 2.2)."""
import math

import numpy as np
import pytest

from oracle import ns_oracle as O
from paper_1812_01178_gb300 import inputs as I


def test_rk3_constants():
    """Low-storage RK3: alpha = gamma + zeta, sum alpha = 1, and the explicit part
    reproduces exp(z) to third order on y' = lambda y."""
    for k in range(3):
        assert abs(O.RK3_ALPHA[k] - O.RK3_GAMMA[k] - O.RK3_ZETA[k]) < 1e-15
    assert abs(sum(O.RK3_ALPHA) - 1.0) < 1e-15
    for z in (1e-2, 2e-2):
        y, yprev = 1.0, 0.0
        for k in range(3):
            ynew = y + z * (O.RK3_GAMMA[k] * y + O.RK3_ZETA[k] * yprev)
            yprev, y = y, ynew
        assert abs(y - (1 + z + z * z / 2 + z ** 3 / 6)) < 2 * z ** 4


def test_poiseuille_steady():
    """Laminar Poiseuille flow with f = 3/Re stays steady to round-off (10 steps)."""
    case, u, v, w, p = I.laminar_channel(16, 16, 8, amp=0.0)
    g = O.Grid.from_case(case)
    s = O.step(g, dict(u=u, v=v, w=w, p=p), case.dt, case.re, case.fx, nsteps=10)
    assert np.abs(s["u"] - u).max() < 1e-13
    assert np.abs(s["v"]).max() < 1e-13 and np.abs(s["w"]).max() < 1e-13
    assert np.abs(s["p"] - s["p"].mean()).max() < 1e-12


def test_stokes_mode_closed_form_decay():
    """u = U(y) sin(2 pi z/Lz), v = w = 0 with U an eigenvector of the discrete
    y operator: convection and pressure vanish, and each sub-step multiplies u by
    1 - 2 b (my + mz) / ((1 + b my)(1 + b mz)), b = alpha_k dt/(2 Re)."""
    nx, ny, nz = 4, 12, 8
    yf = I.channel_faces(ny, 1.7)
    g = O.Grid(nx, ny, nz, 2 * math.pi, math.pi, yf)
    A, C = O.yrows_centre(g)
    M = np.diag(-(A + C)) + np.diag(A[1:], -1) + np.diag(C[:-1], 1)
    ev, vecs = np.linalg.eig(M)
    q = np.argmax(ev.real)                              # slowest-decaying mode
    my = -ev[q].real
    U = vecs[:, q].real
    zc = (np.arange(nz) + 0.5) * g.dz
    mz = O.modified_wavenumbers(nz, g.dz)[1]
    u = U[None, :, None] * np.sin(2 * math.pi * zc / g.lz)[:, None, None] * np.ones((nz, ny, nx))
    v = np.zeros((nz, ny + 1, nx))
    w = np.zeros((nz, ny, nx))
    p = np.zeros((nz, ny, nx))
    re, dt = 50.0, 0.01
    s = O.step(g, dict(u=u, v=v, w=w, p=p), dt, re, 0.0, nsteps=3)
    amp = 1.0
    for _ in range(3):
        for k in range(3):
            b = O.RK3_ALPHA[k] * dt / (2 * re)
            amp *= 1 - 2 * b * (my + mz) / ((1 + b * my) * (1 + b * mz))
    np.testing.assert_allclose(s["u"], amp * u, atol=1e-13)
    assert np.abs(s["v"]).max() < 1e-13 and np.abs(s["w"]).max() < 1e-13


def _smooth_divfree(g):
    xf = np.arange(g.nx) * g.dx
    xc = xf + 0.5 * g.dx
    zc = (np.arange(g.nz) + 0.5) * g.dz
    kx = 2 * math.pi / g.lx
    Z, Y, X = np.meshgrid(zc, g.yc, xf, indexing="ij")
    u = np.sin(kx * X) * (-4 * Y * (1 - Y ** 2)) + 0.3 * np.cos(2 * math.pi * Z / g.lz)
    Z, Y, X = np.meshgrid(zc, g.yf, xc, indexing="ij")
    v = -kx * np.cos(kx * X) * (1 - Y ** 2) ** 2
    v[:, 0] = 0
    v[:, -1] = 0
    Z, Y, X = np.meshgrid(np.arange(g.nz) * g.dz, g.yc, xc, indexing="ij")
    w = 0.5 * np.sin(2 * math.pi * Z / g.lz) * np.cos(kx * X) * (1 - Y ** 2)
    return O.make_divergence_free(g, u, v, w)


@pytest.mark.slow
def test_rk3_third_order_in_time_inviscid():
    """With Re = inf the velocity follows low-storage RK3 on du/dt = -P N(u), so
    errors shrink 8x per halving of dt."""
    yf = I.channel_faces(8, 1.0)
    g = O.Grid(8, 8, 4, 2 * math.pi, math.pi, yf)
    u, v, w = _smooth_divfree(g)
    T = 0.24
    sols = []
    for dt in (0.04, 0.02, 0.01, 0.0025):
        s = dict(u=u, v=v, w=w, p=np.zeros((g.nz, g.ny, g.nx)))
        s = O.step(g, s, dt, float("inf"), 0.0, nsteps=int(round(T / dt)))
        sols.append(s["u"])
    e = [np.abs(sols[i] - sols[-1]).max() for i in range(3)]
    assert e[0] / e[1] > 6.5 and e[1] / e[2] > 7.0, e


def test_divergence_after_each_substep():
    case, u, v, w, p = I.small_channel(16, 12, 8, amp=0.3)
    g = O.Grid.from_case(case)
    u, v, w = O.make_divergence_free(g, u, v, w)
    s = dict(u=u, v=v, w=w, p=p)
    for k in range(3):
        s = O.substep(g, s, k, case.dt, case.re, case.fx)
        d = O.divergence(g, s["u"], s["v"], s["w"])
        assert np.abs(d).max() < 1e-12


@pytest.mark.parametrize("k", [1, 2])
def test_an_irrotational_field_is_removed_and_becomes_pressure(k):
    """Projection (Sec. 2.2): an intermediate field that is a discrete gradient, u* = G psi, is
    removed completely by the projection u = u* - alpha_k dt G phi, and the pressure increment
    is phi = psi / (alpha_k dt) up to a constant.  Driven through a whole inviscid sub-step from
    u = eps G psi at rest otherwise (no force, no N_prev): the convection term is O(eps^2), so
    the velocity left is O(eps^2) and p - mean(p) = eps (psi - mean(psi)) / (alpha_k dt) to
    relative O(eps).  Sub-steps 1 and 2, where alpha_k differs from gamma_k."""
    case, *_ = I.small_channel(16, 12, 8, seed=3)
    g = O.Grid.from_case(case)
    rng = np.random.default_rng(8)
    psi = rng.standard_normal((g.nz, g.ny, g.nx))
    eps, dt = 1e-6, 1e-2
    gx, gy, gz = O.gradient(g, psi)
    state = dict(u=eps * gx, v=eps * gy, w=eps * gz, p=np.zeros_like(psi),
                 nprev=[np.zeros_like(gx), np.zeros_like(gy), np.zeros_like(gz)])
    s = O.substep(g, state, k, dt, float("inf"), 0.0)
    want = eps * (psi - psi.mean()) / (O.RK3_ALPHA[k] * dt)
    got = s["p"] - s["p"].mean()
    assert np.abs(got - want).max() < 1e-5 * np.abs(want).max()
    for f in ("u", "v", "w"):
        assert np.abs(s[f]).max() < 1e-4 * eps * np.abs(gx).max()
