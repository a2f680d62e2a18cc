"""Pins of the oracle's inflow / convective-outflow (flat-plate) configuration."""
import math

import numpy as np
import pytest

from oracle import ns_oracle as O
from paper_1812_01178_gb300 import inputs as I


def _grid(nx=8, ny=6, nz=4, ly=3.0):
    yf = I.boundary_layer_faces(ny, 1.5, ly)
    return O.Grid(nx, ny, nz, 6.0, 2.0, yf, ytop=1)


def _fields(g, seed=0, amp=1.0):
    rng = np.random.default_rng(seed)
    u = 1.0 + amp * rng.standard_normal((g.nz, g.ny, g.nx))
    v = amp * rng.standard_normal((g.nz, g.ny + 1, g.nx))
    v[:, 0] = 0
    v[:, -1] = 0
    w = amp * rng.standard_normal((g.nz, g.ny, g.nx))
    bl = dict(u_out=1.0 + amp * rng.standard_normal((g.nz, g.ny)),
              v_in=amp * rng.standard_normal((g.nz, g.ny + 1)),
              v_out=amp * rng.standard_normal((g.nz, g.ny + 1)),
              w_in=amp * rng.standard_normal((g.nz, g.ny)),
              w_out=amp * rng.standard_normal((g.nz, g.ny)))
    for q in ("v_in", "v_out"):
        bl[q][:, 0] = 0
        bl[q][:, -1] = 0
    return u, v, w, bl


@pytest.mark.parametrize("n", [1, 2, 5, 8, 16])
def test_dct_matrices_match_library(n):
    sp = pytest.importorskip("scipy.fft")
    x = np.random.default_rng(n).standard_normal((3, n))
    X = x @ O.dct2_matrix(n).T
    np.testing.assert_allclose(X, 0.5 * sp.dct(x, type=2, axis=1), atol=1e-13 * n)
    np.testing.assert_allclose(X @ O.dct3_inverse_matrix(n).T, x, atol=1e-13 * n)


@pytest.mark.parametrize("n", [3, 6, 11])
def test_neumann_modified_wavenumbers(n):
    h = 0.7
    M = np.zeros((n, n))
    for i in range(n):
        if i > 0:
            M[i, i] += 1 / h ** 2
            M[i, i - 1] -= 1 / h ** 2
        if i < n - 1:
            M[i, i] += 1 / h ** 2
            M[i, i + 1] -= 1 / h ** 2
    lam = (2 / h ** 2) * (1 - np.cos(math.pi * np.arange(n) / n))
    np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(M)), np.sort(lam), atol=1e-10 / h ** 2)
    # the DCT-II basis vectors are its eigenvectors
    C = O.dct2_matrix(n)
    np.testing.assert_allclose(M @ C.T, C.T * lam[None, :], atol=1e-10 / h ** 2)


def test_poisson_bl_matches_dense_solve():
    g = _grid(5, 4, 4)
    n = g.nx * g.ny * g.nz
    zero_bl = dict(u_out=np.zeros((g.nz, g.ny)))
    M = np.zeros((n, n))
    for q in range(n):
        e = np.zeros(n)
        e[q] = 1.0
        gx, gy, gz = O.gradient_bl(g, e.reshape(g.nz, g.ny, g.nx))
        M[:, q] = O.divergence_bl(g, gx, gy, gz, zero_bl).ravel()
    u, v, w, bl = _fields(g, 1)
    bl["u_out"] = O.flux_correct_outflow(g, u[:, :, 0], bl["u_out"])
    b = O.divergence_bl(g, u, v, w, bl)
    ref = np.linalg.lstsq(M, b.ravel(), rcond=None)[0].reshape(b.shape)
    phi = O.poisson_solve_bl(g, b)
    np.testing.assert_allclose(phi - phi.mean(), ref - ref.mean(), atol=1e-11)


def test_projection_and_flux_correction():
    g = _grid(16, 10, 8)
    u, v, w, bl = _fields(g, 2)
    u2, v2, w2, bl2 = O.make_divergence_free_bl(g, u, v, w, bl)
    d = O.divergence_bl(g, u2, v2, w2, bl2)
    assert np.abs(d).max() < 1e-12 * np.abs(O.divergence_bl(g, u, v, w, bl)).max()
    # net flux through the outflow equals the inflow flux; inflow face untouched by the projection
    wgt = g.dy[None, :] * g.dz
    assert abs((u2[:, :, 0] * wgt).sum() - (bl2["u_out"] * wgt).sum()) < 1e-12 * np.abs(u).sum()
    assert np.array_equal(u2[:, :, 0], u[:, :, 0])


@pytest.mark.parametrize("comp", [0, 1, 2])
def test_adi_x_bl_rows_invert_the_ghost_operator(comp):
    """The x sweep with inflow/outflow solves (I - beta delta_xx) delta = r where delta_xx is the
    explicit operator with the boundary increments (inflow 0, outflow inc) in the ghosts."""
    g = _grid(12, 6, 4)
    rng = np.random.default_rng(3 + comp)
    shape = (g.nz, g.ny + 1, g.nx) if comp == 1 else (g.nz, g.ny, g.nx)
    r = rng.standard_normal(shape)
    if comp == 0:
        r[:, :, 0] = 0.0
    inc = rng.standard_normal(shape[:2])
    beta = 0.3
    x = O.adi_sweep_x_bl(g, r, comp, beta, inc)
    h2 = g.dx ** 2
    if comp == 0:
        xn = O._xnext_u(x, dict(u_out=inc))
        lap = (xn - 2 * x + O._xprev_u(x)) / h2
        lap[:, :, 0] = 0.0
    else:
        lap = (O._xnext_c(x, inc) - 2 * x + O._xprev_c(x, np.zeros_like(inc))) / h2
    np.testing.assert_allclose(x - beta * lap, r, atol=1e-12)


def test_uniform_inviscid_stream_is_steady():
    g = _grid(16, 8, 8)
    u = np.ones((g.nz, g.ny, g.nx))
    v = np.zeros((g.nz, g.ny + 1, g.nx))
    w = np.zeros((g.nz, g.ny, g.nx))
    bl = dict(u_out=np.ones((g.nz, g.ny)), v_in=np.zeros((g.nz, g.ny + 1)), v_out=np.zeros((g.nz, g.ny + 1)),
              w_in=np.zeros((g.nz, g.ny)), w_out=np.zeros((g.nz, g.ny)))
    s = O.step_bl(g, dict(u=u, v=v, w=w, p=np.zeros_like(u), bl=bl), 0.05, float("inf"), 0.0, nsteps=3)
    assert np.abs(s["u"] - 1).max() < 1e-14 and np.abs(s["v"]).max() < 1e-14
    assert np.abs(s["bl"]["u_out"] - 1).max() < 1e-14


def test_bl_step_keeps_divergence_and_mass_balance():
    case, u, v, w, p, bl = I.boundary_layer(16, 12, 8, seed=4)
    g = O.Grid.from_case(case)
    u, v, w, bl = O.make_divergence_free_bl(g, u, v, w, bl)
    s = dict(u=u, v=v, w=w, p=p, bl=bl)
    wgt = g.dy[None, :] * g.dz
    for k in range(3):
        s = O.substep_bl(g, s, k, case.dt, case.re, case.fx, case.u_conv)
        assert np.abs(O.divergence_bl(g, s["u"], s["v"], s["w"], s["bl"])).max() < 1e-11
        assert abs((s["u"][:, :, 0] * wgt).sum() - (s["bl"]["u_out"] * wgt).sum()) < 1e-11
        assert np.array_equal(s["u"][:, :, 0], u[:, :, 0])


def test_bl_convection_telescopes_to_boundary_fluxes():
    """Divergence form with inflow/outflow: volume sums of N_v and N_w reduce exactly to the
    momentum fluxes through the inflow and outflow faces (plus, for v, the wall-adjacent
    centre terms), with face values u v and u w built here independently of the oracle."""
    g = _grid(10, 7, 6)
    u, v, w, bl = _fields(g, 5)
    Nu, Nv, Nw = O.convection_bl(g, u, v, w, bl)
    u_in = u[:, :, 0]

    def u_at_yfaces(col):   # linear interpolation in y, zero at the walls (v = 0 there)
        out = np.zeros((g.nz, g.ny + 1))
        for k in range(g.nz):
            out[k, 1:-1] = np.interp(g.yf[1:-1], g.yc, col[k])
        return out

    flux_v = u_at_yfaces(bl["u_out"]) * bl["v_out"] - u_at_yfaces(u_in) * bl["v_in"]
    hv = np.zeros(g.ny + 1)
    hv[1:-1] = g.hc
    vc = 0.5 * (v[:, :-1] + v[:, 1:])
    expect_v = g.dz * (hv[None, :] * flux_v).sum() + g.dx * g.dz * (vc[:, -1] ** 2 - vc[:, 0] ** 2).sum()
    got_v = (Nv * hv[None, :, None]).sum() * g.dx * g.dz
    assert abs(got_v - expect_v) < 1e-12 * np.abs(Nv).sum() * g.dx * g.dz * 10

    def zface(a):   # average of planes k-1 and k (periodic z)
        return 0.5 * (np.roll(a, 1, axis=0) + a)

    flux_w = zface(bl["u_out"]) * bl["w_out"] - zface(u_in) * bl["w_in"]
    expect_w = g.dz * (g.dy[None, :] * flux_w).sum()
    got_w = (Nw * g.dy[None, :, None]).sum() * g.dx * g.dz
    assert abs(got_w - expect_w) < 1e-12 * np.abs(Nw).sum() * g.dx * g.dz * 10


def test_outflow_update_advects_a_linear_profile_exactly():
    """The convective outflow condition df/dt + U_c df/dx = 0 (Sec. 2.1), one upwind step of
    alpha_k dt: for a field linear in x the one-sided difference between the outflow plane
    (x = Lx) and the last interior point is the exact slope, whatever their distance (dx from the
    last u face, dx/2 from the last v, w centre), so each plane moves by exactly -U_c (alpha dt)
    slope.  The wall rows of v stay zero."""
    g = _grid()
    a, b = 0.3, -0.7
    xf = np.arange(g.nx) * g.dx             # u faces 0..nx-1 (face 0 the inflow)
    xc = (np.arange(g.nx) + 0.5) * g.dx     # centres
    lx = g.nx * g.dx
    u = np.broadcast_to(a + b * xf, (g.nz, g.ny, g.nx)).copy()
    v = np.broadcast_to(a + b * xc, (g.nz, g.ny + 1, g.nx)).copy()
    w = np.broadcast_to(a + b * xc, (g.nz, g.ny, g.nx)).copy()
    bl = dict(u_out=np.full((g.nz, g.ny), a + b * lx), v_out=np.full((g.nz, g.ny + 1), a + b * lx),
              w_out=np.full((g.nz, g.ny), a + b * lx), v_in=np.zeros((g.nz, g.ny + 1)),
              w_in=np.zeros((g.nz, g.ny)))
    scale, uc = 0.013, 1.3
    new, inc = O.outflow_update(g, u, v, w, bl, scale, uc)
    want = a + b * lx - uc * scale * b
    np.testing.assert_allclose(new["u_out"], want, rtol=0, atol=1e-14)
    np.testing.assert_allclose(new["w_out"], want, rtol=0, atol=1e-14)
    np.testing.assert_allclose(new["v_out"][:, 1:-1], want, rtol=0, atol=1e-14)
    assert np.all(new["v_out"][:, 0] == 0) and np.all(new["v_out"][:, -1] == 0)
    for q in ("u_out", "v_out", "w_out"):
        np.testing.assert_array_equal(inc[q], new[q] - bl[q])


def test_divergence_telescopes_to_the_boundary_fluxes():
    """Discrete Gauss theorem: the volume sum of D u equals the net flux through the boundary,
    the outflow plane u_out at x = Lx minus the inflow face u_0 at x = 0 (periodic z, v = 0 on
    the walls of a channel-like box here, so only x contributes besides the y faces given)."""
    g = _grid(12, 7, 6)
    u, v, w, bl = _fields(g, 5)
    d = O.divergence_bl(g, u, v, w, bl)
    vol = g.dx * g.dy[None, :, None] * g.dz
    wy = g.dy[None, :] * g.dz
    net = ((bl["u_out"] - u[:, :, 0]) * wy).sum() + ((v[:, -1, :] - v[:, 0, :]) * g.dx * g.dz).sum()
    assert abs((d * vol).sum() - net) < 1e-12 * np.abs(u).sum()


def test_step_from_unbalanced_outflow_keeps_divergence_and_inflow():
    """Sub-steps from a random field that is neither solenoidal nor mass-balanced: the outflow flux
    correction makes the Poisson problem compatible, so every sub-step ends divergence-free to
    round-off with the outflow flux equal to the inflow flux.  The inflow face of u stays fixed
    (a Dirichlet condition) even under a body force."""
    g = _grid(16, 10, 8)
    u, v, w, bl = _fields(g, 9, amp=0.5)  # not projected: the first sub-step must balance it
    p = np.zeros_like(u)
    s = dict(u=u, v=v, w=w, p=p, bl=bl)
    wgt = g.dy[None, :] * g.dz
    for k in range(3):
        s = O.substep_bl(g, s, k, 2e-3, 50.0, 0.7, 1.0)
        assert np.abs(O.divergence_bl(g, s["u"], s["v"], s["w"], s["bl"])).max() < 1e-10
        assert abs((s["u"][:, :, 0] * wgt).sum() - (s["bl"]["u_out"] * wgt).sum()) < 1e-11
        assert np.array_equal(s["u"][:, :, 0], u[:, :, 0])


def test_viscous_operator_with_ghosts_is_exact_for_linear_x_profiles():
    """The inflow / outflow ghosts (2 f_in - f_0, 2 f_out - f_{nx-1}) extrapolate linearly, so the
    x second difference vanishes on fields linear in x: for f = (a + b x) phi(y), the viscous
    operator equals (a + b x) / a times its value on a phi(y), cell by cell, for u, v and w."""
    g = _grid(12, 7, 4)
    rng = np.random.default_rng(3)
    pc = rng.standard_normal(g.ny)
    pf = rng.standard_normal(g.ny + 1)
    pf[0] = pf[-1] = 0.0
    xf = np.arange(g.nx) * g.dx
    xc = (np.arange(g.nx) + 0.5) * g.dx
    lx = g.nx * g.dx

    def fields(a, b):
        u = np.broadcast_to((a + b * xf)[None, None, :] * pc[None, :, None], (g.nz, g.ny, g.nx)).copy()
        v = np.broadcast_to((a + b * xc)[None, None, :] * pf[None, :, None], (g.nz, g.ny + 1, g.nx)).copy()
        w = np.broadcast_to((a + b * xc)[None, None, :] * pc[None, :, None], (g.nz, g.ny, g.nx)).copy()
        bl = dict(u_out=np.broadcast_to((a + b * lx) * pc, (g.nz, g.ny)).copy(),
                  v_in=np.broadcast_to(a * pf, (g.nz, g.ny + 1)).copy(),
                  v_out=np.broadcast_to((a + b * lx) * pf, (g.nz, g.ny + 1)).copy(),
                  w_in=np.broadcast_to(a * pc, (g.nz, g.ny)).copy(),
                  w_out=np.broadcast_to((a + b * lx) * pc, (g.nz, g.ny)).copy())
        return u, v, w, bl

    a, b = 1.5, -0.4
    L1 = O.laplacian_bl(g, *fields(a, b))
    L0 = O.laplacian_bl(g, *fields(a, 0.0))
    for comp, x in ((0, xf), (1, xc), (2, xc)):
        want = ((a + b * x) / a)[None, None, :] * L0[comp]
        if comp == 0:
            want[:, :, 0] = 0.0  # the inflow face of u takes no viscous term
        np.testing.assert_allclose(L1[comp], want, rtol=0, atol=1e-10 * np.abs(L0[comp]).max())


@pytest.mark.parametrize("bl", [False, True])
def test_poisson_gauge_zero_mean_on_the_first_row(bl):
    """The singular (kx, kz) = (0, 0) mode is gauged by phi_hat(j = 0) = 0: the solution's mean
    over the first y row of cells is zero."""
    g = _grid(8, 6, 4)
    rng = np.random.default_rng(4)
    rhs = rng.standard_normal((g.nz, g.ny, g.nx))
    rhs -= (rhs * g.dy[None, :, None]).sum() / (g.dy.sum() * g.nx * g.nz)  # compatible
    phi = O.poisson_solve_bl(g, rhs) if bl else O.poisson_solve(g, rhs)
    assert abs(phi[:, 0, :].mean()) < 1e-12 * np.abs(phi).max()
