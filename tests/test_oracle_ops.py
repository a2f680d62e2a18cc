"""Pins of the oracle's spatial operators, transforms and Poisson solver (Sec. 2.1-2.2)."""
import math

import numpy as np
import pytest

from oracle import ns_oracle as O
from paper_1812_01178_gb300 import inputs as I


def _grid(nx=8, ny=6, nz=4, beta=1.5, ytop=0, uniform=False):
    yf = np.linspace(-1, 1, ny + 1) if uniform else I.channel_faces(ny, beta)
    return O.Grid(nx, ny, nz, 2 * math.pi, math.pi, yf, ytop)


def _rand_fields(g, seed=0):
    rng = np.random.default_rng(seed)
    u = rng.standard_normal((g.nz, g.ny, g.nx))
    v = rng.standard_normal((g.nz, g.ny + 1, g.nx))
    v[:, 0] = 0
    v[:, -1] = 0
    w = rng.standard_normal((g.nz, g.ny, g.nx))
    p = rng.standard_normal((g.nz, g.ny, g.nx))
    return u, v, w, p


# ---------------------------------------------------------------- transforms
@pytest.mark.parametrize("n", [1, 2, 8, 12, 17])
def test_dft_matches_library_fft(n):
    rng = np.random.default_rng(n)
    f = rng.standard_normal((3, n)) + 1j * rng.standard_normal((3, n))
    np.testing.assert_allclose(O.dft(f, 1), np.fft.fft(f, axis=1), atol=1e-12 * n)
    np.testing.assert_allclose(O.dft(f, 1, +1), np.fft.ifft(f, axis=1) * n, atol=1e-12 * n)
    # Parseval
    F = O.dft(f, 1)
    np.testing.assert_allclose((np.abs(F) ** 2).sum(1), n * (np.abs(f) ** 2).sum(1), rtol=1e-12)


@pytest.mark.parametrize("n", [72, 96, 128, 256])
def test_dft_above_the_naive_limit_equals_the_definition(n):
    """Lines longer than NAIVE_DFT_MAX go through numpy's FFT: the same sums as the definition
    F_k = sum_m f_m exp(sign 2 pi i k m / N), written out here as a matrix product, along both
    axes used by the solver (0 and 2), forward and unnormalised inverse."""
    assert n > O.NAIVE_DFT_MAX
    rng = np.random.default_rng(n)
    f = rng.standard_normal((n, 3, n)) + 1j * rng.standard_normal((n, 3, n))
    k = np.arange(n)
    for sign in (-1, +1):
        M = np.exp(sign * 2j * np.pi * np.outer(k, k) / n)
        by_def2 = np.einsum("km,zym->zyk", M, f)
        by_def0 = np.einsum("km,myx->kyx", M, f)
        scale = np.abs(by_def2).max()
        np.testing.assert_allclose(O.dft(f, 2, sign), by_def2, rtol=0, atol=1e-12 * scale)
        np.testing.assert_allclose(O.dft(f, 0, sign), by_def0, rtol=0, atol=1e-12 * scale)
    # round trip: the inverse is unnormalised, so it returns n f
    np.testing.assert_allclose(O.dft(O.dft(f, 2), 2, +1), n * f, rtol=0, atol=1e-12 * n * np.abs(f).max())


@pytest.mark.parametrize("n", [4, 7, 16])
def test_modified_wavenumbers_are_eigenvalues(n):
    h = 0.3
    M = np.zeros((n, n))
    for i in range(n):
        M[i, i] = 2 / h ** 2
        M[i, (i + 1) % n] -= 1 / h ** 2
        M[i, (i - 1) % n] -= 1 / h ** 2
    ev = np.sort(np.linalg.eigvalsh(M))
    np.testing.assert_allclose(np.sort(O.modified_wavenumbers(n, h)), ev, atol=1e-10 / h ** 2)


# ---------------------------------------------------------------- gradient / divergence
def test_gradient_is_minus_adjoint_of_divergence():
    """sum_c p (D u) dV_c = - sum_f u . (G p) dV_f (summation by parts, walls v = 0)."""
    g = _grid(7, 5, 6)
    u, v, w, p = _rand_fields(g, 1)
    cu, cv, cw, cp = g.volumes()
    lhs = (p * O.divergence(g, u, v, w) * cp).sum()
    gx, gy, gz = O.gradient(g, p)
    rhs = -((u * gx * cu).sum() + (v * gy * cv).sum() + (w * gz * cw).sum())
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1)


def test_divergence_of_uniform_translation_is_zero():
    g = _grid()
    u = np.full((g.nz, g.ny, g.nx), 1.3)
    v = np.zeros((g.nz, g.ny + 1, g.nx))
    w = np.full((g.nz, g.ny, g.nx), -0.4)
    assert np.abs(O.divergence(g, u, v, w)).max() == 0.0


# ---------------------------------------------------------------- convection
def test_convection_conserves_momentum():
    """Divergence form: fluxes telescope, so volume sums of N vanish (any field)."""
    g = _grid(6, 7, 5)
    u, v, w, _ = _rand_fields(g, 2)
    Nu, Nv, Nw = O.convection(g, u, v, w)
    cu, cv, cw, _ = g.volumes()
    scale = np.abs(Nu * cu).sum()
    assert abs((Nu * cu).sum()) < 1e-13 * scale
    assert abs((Nw * cw).sum()) < 1e-13 * scale
    # v control volumes end at the first / last cell centres, where the flux v^2
    # is not zero: the sum telescopes to exactly that boundary term.
    vc = 0.5 * (v[:, :-1] + v[:, 1:])
    boundary = g.dx * g.dz * (vc[:, -1] ** 2 - vc[:, 0] ** 2).sum()
    assert abs((Nv * cv).sum() - boundary) < 1e-13 * scale


def test_convection_conserves_energy_on_uniform_grid():
    """On a uniform staggered grid the divergence form conserves kinetic energy
    when D u = 0 (Morinishi et al. 1998): sum u.N(u) dV = 0."""
    g = _grid(8, 6, 6, uniform=True)
    u, v, w, _ = _rand_fields(g, 3)
    u, v, w = O.make_divergence_free(g, u, v, w)
    assert np.abs(O.divergence(g, u, v, w)).max() < 1e-11
    Nu, Nv, Nw = O.convection(g, u, v, w)
    cu, cv, cw, _ = g.volumes()
    e = (u * Nu * cu).sum() + (v * Nv * cv).sum() + (w * Nw * cw).sum()
    scale = np.abs(u * Nu * cu).sum()
    assert abs(e) < 1e-12 * scale


def test_convection_y_interpolation_exact_for_linear_profiles():
    """Linear interpolation to y-faces is exact for fields linear in y, on any grid:
    with u = a + b y and v = V on the interior faces, d(uv)/dy = V b in every cell
    away from the walls (rough random spacing, so weights must be the distances)."""
    rng = np.random.default_rng(11)
    ny = 9
    yf = np.concatenate([[-1.0], np.sort(rng.uniform(-1, 1, ny - 1)), [1.0]])
    g = O.Grid(4, ny, 4, 2 * math.pi, math.pi, yf)
    a, b, V = 0.3, 1.7, -0.6
    u = (a + b * g.yc)[None, :, None] * np.ones((g.nz, g.ny, g.nx))
    v = np.full((g.nz, g.ny + 1, g.nx), V)
    v[:, 0] = 0
    v[:, -1] = 0
    w = np.zeros((g.nz, g.ny, g.nx))
    Nu, Nv, Nw = O.convection(g, u, v, w)
    np.testing.assert_allclose(Nu[:, 1:-1], V * b, rtol=1e-12)
    # the same for w, and for the x-flux of v-momentum (u interpolated to y-faces)
    Nu, Nv, Nw = O.convection(g, np.zeros_like(u), v, u)
    np.testing.assert_allclose(Nw[:, 1:-1], V * b, rtol=1e-12)
    xf = np.arange(g.nx) * g.dx
    uu = (a + b * g.yc)[None, :, None] * np.cos(xf)[None, None, :] * np.ones((g.nz, 1, 1))
    Nu, Nv, Nw = O.convection(g, uu, v, w)
    lin_f = (a + b * g.yf[1:-1])[None, :, None]
    cosr = np.cos(np.roll(xf, -1))[None, None, :]
    expect = V * lin_f * (cosr - np.cos(xf)[None, None, :]) / g.dx
    vc = 0.5 * (v[:, :-1] + v[:, 1:])
    expect = expect + (vc[:, 1:] ** 2 - vc[:, :-1] ** 2) / g.hc[None, :, None]
    np.testing.assert_allclose(Nv[:, 1:-1], expect, rtol=1e-11, atol=1e-12)


def test_convection_is_quadratic():
    g = _grid()
    u, v, w, _ = _rand_fields(g, 4)
    N1 = O.convection(g, u, v, w)
    N2 = O.convection(g, 3 * u, 3 * v, 3 * w)
    for a, b in zip(N1, N2):
        np.testing.assert_allclose(b, 9 * a, rtol=1e-13, atol=1e-12)


def _analytic_fields(g):
    """Smooth fields vanishing at y = +-1 and their analytic d(u_i u_j)/dx_j."""
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z")
    U = sp.sin(x) * sp.cos(2 * z) * (1 - y ** 2) + 0.5 * (1 - y ** 2)
    V = sp.cos(x) * sp.sin(2 * z) * (1 - y ** 2) ** 2
    W = sp.sin(x + 2 * z) * (1 - y ** 2)
    Nu = sp.diff(U * U, x) + sp.diff(U * V, y) + sp.diff(U * W, z)
    Nv = sp.diff(U * V, x) + sp.diff(V * V, y) + sp.diff(V * W, z)
    Nw = sp.diff(U * W, x) + sp.diff(V * W, y) + sp.diff(W * W, z)
    LU = sp.diff(U, x, 2) + sp.diff(U, y, 2) + sp.diff(U, z, 2)
    f = [sp.lambdify((x, y, z), e, "numpy") for e in (U, V, W, Nu, Nv, Nw, LU)]
    xf = np.arange(g.nx) * g.dx
    xc = xf + 0.5 * g.dx
    zf = np.arange(g.nz) * g.dz
    zc = zf + 0.5 * g.dz

    def ev(fun, X, Y, Z):
        Zg, Yg, Xg = np.meshgrid(Z, Y, X, indexing="ij")
        return np.broadcast_to(fun(Xg, Yg, Zg), Xg.shape).astype(float)

    u = ev(f[0], xf, g.yc, zc)
    v = ev(f[1], xc, g.yf, zc)
    w = ev(f[2], xc, g.yc, zf)
    return (u, v, w), (ev(f[3], xf, g.yc, zc), ev(f[4], xc, g.yf, zc), ev(f[5], xc, g.yc, zf)), \
        ev(f[6], xf, g.yc, zc)


def test_convection_and_viscous_second_order():
    """N(u) and L(u) converge at 2nd order to the analytic operators on stretched grids."""
    errs, lerrs = [], []
    for n in (16, 32, 64):
        yf = I.channel_faces(n, 1.2)
        g = O.Grid(n, n, n // 2, 2 * math.pi, math.pi, yf)
        (u, v, w), (Nu, Nv, Nw), LU = _analytic_fields(g)
        N = O.convection(g, u, v, w)
        e = max(np.abs(N[0] - Nu).max(), np.abs(N[1][:, 1:-1] - Nv[:, 1:-1]).max(),
                np.abs(N[2] - Nw).max())
        errs.append(e)
        L = O.laplacian(g, u, v, w)
        lerrs.append(np.abs(L[0] - LU).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert r1 > 3.3 and r2 > 3.5, errs
    l1, l2 = lerrs[0] / lerrs[1], lerrs[1] / lerrs[2]
    assert l1 > 3.0 and l2 > 3.3, lerrs


# ---------------------------------------------------------------- viscous / ADI rows
@pytest.mark.parametrize("ytop", [0, 1])
def test_dyy_exact_for_quadratics(ytop):
    g = _grid(4, 9, 4, beta=2.0, ytop=ytop)
    if ytop == 0:
        f = (1 - g.yc ** 2)[None, :, None] * np.ones((g.nz, g.ny, g.nx))
        L = O.laplacian(g, f, np.zeros((g.nz, g.ny + 1, g.nx)), f)
        np.testing.assert_allclose(L[0], -2.0, rtol=1e-12)
    # faces: v = 1 - y^2 vanishes at both walls
    v = (1 - g.yf ** 2)[None, :, None] * np.ones((g.nz, g.ny + 1, g.nx))
    z = np.zeros((g.nz, g.ny, g.nx))
    L = O.laplacian(g, z, v, z)
    np.testing.assert_allclose(L[1][:, 1:-1], -2.0, rtol=1e-11)


def test_stress_free_top_has_zero_flux():
    """A field constant in y has zero y-curvature everywhere under a stress-free
    top except next to the no-slip bottom wall."""
    g = _grid(4, 8, 4, ytop=1)
    f = np.ones((g.nz, g.ny, g.nx))
    L = O.laplacian(g, f, np.zeros((g.nz, g.ny + 1, g.nx)), f)
    assert np.abs(L[0][:, 1:]).max() < 1e-10
    assert np.all(L[0][:, 0] < 0)


@pytest.mark.parametrize("direction,comp", [(0, 0), (1, 0), (1, 1), (2, 2)])
def test_adi_rows_identity(direction, comp):
    """Interior ADI rows satisfy |b| = |a| + |c| + 1 (Sec. 3.2)."""
    g = _grid(8, 10, 6)
    a, b, c = O.adi_rows(g, direction, comp, 0.37)
    s = slice(1, -1)
    np.testing.assert_allclose(np.abs(b[s]), np.abs(a[s]) + np.abs(c[s]) + 1.0, rtol=1e-14)


def test_adi_sweep_inverts_factor():
    """Each sweep solves its factor: (I - beta delta_dd) applied to the result gives r."""
    g = _grid(8, 7, 6)
    rng = np.random.default_rng(9)
    beta = 0.05
    r = rng.standard_normal((g.nz, g.ny, g.nx))
    zeros_v = np.zeros((g.nz, g.ny + 1, g.nx))
    zeros_c = np.zeros((g.nz, g.ny, g.nx))
    # x
    x = O.adi_sweep(g, r, 0, 0, beta)
    back = x - beta * (np.roll(x, -1, 2) - 2 * x + np.roll(x, 1, 2)) / g.dx ** 2
    np.testing.assert_allclose(back, r, atol=1e-12)
    # z
    x = O.adi_sweep(g, r, 2, 2, beta)
    back = x - beta * (np.roll(x, -1, 0) - 2 * x + np.roll(x, 1, 0)) / g.dz ** 2
    np.testing.assert_allclose(back, r, atol=1e-12)
    # y (u): the laplacian restricted to y-curvature, from a field constant in x, z
    rc = np.broadcast_to(r[:1, :, :1], r.shape).copy()
    x = O.adi_sweep(g, rc, 1, 0, beta)
    Lx = O.laplacian(g, x, zeros_v, zeros_c)[0]
    np.testing.assert_allclose(x - beta * Lx, rc, atol=1e-11)
    # y (v)
    rv = rng.standard_normal((1, g.ny + 1, 1)) * np.ones((g.nz, g.ny + 1, g.nx))
    rv[:, 0] = 0
    rv[:, -1] = 0
    x = O.adi_sweep(g, rv, 1, 1, beta)
    Lv = O.laplacian(g, zeros_c, x, zeros_c)[1]
    np.testing.assert_allclose(x - beta * Lv, rv, atol=1e-11)


# ---------------------------------------------------------------- Poisson
def test_poisson_matches_dense_solve():
    """Brute force: assemble D G as a dense matrix on a tiny grid and solve it."""
    g = _grid(4, 5, 4)
    n = g.nx * g.ny * g.nz
    M = np.zeros((n, n))
    for q in range(n):
        e = np.zeros(n)
        e[q] = 1.0
        gx, gy, gz = O.gradient(g, e.reshape(g.nz, g.ny, g.nx))
        M[:, q] = O.divergence(g, gx, gy, gz).ravel()
    u, v, w, _ = _rand_fields(g, 5)
    b = O.divergence(g, u, v, w)
    ref = np.linalg.lstsq(M, b.ravel(), rcond=None)[0].reshape(b.shape)
    phi = O.poisson_solve(g, b)
    np.testing.assert_allclose(phi - phi.mean(), ref - ref.mean(), atol=1e-11)


def test_poisson_discrete_residual():
    g = _grid(16, 12, 8, beta=2.0)
    u, v, w, _ = _rand_fields(g, 6)
    b = O.divergence(g, u, v, w)
    phi = O.poisson_solve(g, b)
    gx, gy, gz = O.gradient(g, phi)
    res = O.divergence(g, gx, gy, gz) - b
    assert np.abs(res).max() < 1e-11 * np.abs(b).max()


def test_poisson_manufactured_second_order():
    """phi = cos(2 pi x/Lx) cos(2 pi z/Lz) cos(pi (y+1)/2), Neumann at y = +-1."""
    errs = []
    for n in (8, 16, 32):
        yf = I.channel_faces(n, 1.2)
        g = O.Grid(n, n, n, 2 * math.pi, math.pi, yf)
        xc = (np.arange(g.nx) + 0.5) * g.dx
        zc = (np.arange(g.nz) + 0.5) * g.dz
        Z, Y, X = np.meshgrid(zc, g.yc, xc, indexing="ij")
        kx, kz, ky = 2 * math.pi / g.lx, 2 * math.pi / g.lz, math.pi / 2
        ex = np.cos(kx * X) * np.cos(kz * Z) * np.cos(ky * (Y + 1))
        b = -(kx ** 2 + ky ** 2 + kz ** 2) * ex
        phi = O.poisson_solve(g, b)
        errs.append(np.abs((phi - phi.mean()) - (ex - ex.mean())).max())
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.7, errs


def test_projection_divergence_roundoff():
    g = _grid(16, 12, 8, beta=2.0)
    u, v, w, _ = _rand_fields(g, 7)
    u2, v2, w2 = O.make_divergence_free(g, u, v, w)
    assert np.abs(O.divergence(g, u2, v2, w2)).max() < 1e-12 * np.abs(O.divergence(g, u, v, w)).max()
    # idempotent
    u3, v3, w3 = O.make_divergence_free(g, u2, v2, w2)
    assert np.abs(u3 - u2).max() < 1e-12 and np.abs(v3 - v2).max() < 1e-12
