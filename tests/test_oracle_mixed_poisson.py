"""The reading behind the mixed form's Poisson solve, checked on the CPU with the oracle's
operators: transforms carried in FP32 leave a residual of the discrete Poisson equation near the
FP32 rounding level (too large for a divergence of 1e-10 after projection), and one refinement
on the residual formed in FP64 brings it back to the FP64 level.  The FP32 transforms here are
scipy's single-precision FFTs; the y solves are the oracle's Thomas in FP64, as on the GPU."""
import math

import numpy as np
import pytest

from oracle import ns_oracle as O
from paper_1812_01178_gb300 import inputs as I
from tests import poisson_modes as PM

sf = pytest.importorskip("scipy.fft")


def _poisson(g, rhs, fp32, y32=None):
    """D G phi = rhs: z real transform, x transform, y Thomas per (kx, kz) in FP64, inverses;
    with fp32 the transforms and the spectrum are single precision (phi returned in FP32); y32, a
    [kz, kx] mask, runs those modes' y solves in FP32 arithmetic (the mixed form's split)."""
    a, c = O.poisson_ycoeffs(g)
    lx = O.modified_wavenumbers(g.nx, g.dx)
    lz = O.modified_wavenumbers(g.nz, g.dz)[: g.nz // 2 + 1]
    x = rhs.astype(np.float32) if fp32 else rhs
    bh = sf.fft(sf.rfft(x, axis=0), axis=2).astype(np.complex128)
    d = np.moveaxis(bh, 1, -1)
    A = np.broadcast_to(a, d.shape).copy()
    C = np.broadcast_to(c, d.shape).copy()
    B = np.array(np.broadcast_to(-(a + c)[None, None, :] - (lz[:, None] + lx[None, :])[:, :, None], d.shape))
    B[0, 0, 0], C[0, 0, 0] = 1.0, 0.0
    d = d.copy()
    d[0, 0, 0] = 0.0
    ph = O.thomas(A, B, C, d)
    if y32 is not None:
        ph[y32] = PM.thomas32(A[y32], B[y32], C[y32], d[y32], cp_from_ip=True)  # as the staged form
    ph = np.moveaxis(ph, -1, 1)
    if fp32:
        ph = ph.astype(np.complex64)
    phi = sf.irfft(sf.ifft(ph, axis=2), n=g.nz, axis=0)
    return phi.astype(np.float32) if fp32 else phi


def _lap(g, phi):
    return O.divergence(g, *O.gradient(g, phi))


@pytest.mark.parametrize("y32", [False, True])
@pytest.mark.parametrize("low", [0.0, 20.0])
def test_fp32_transforms_need_one_fp64_refinement(low, y32):
    """Also with the y solves of the well-conditioned modes (kz > 0, Skeel condition <= 4096) in
    FP32 arithmetic, as the mixed form runs them: one refinement still reaches the FP64 level."""
    case, u, v, w, p = I.small_channel(32, 24, 32, seed=12, amp=0.3)
    g = O.Grid.from_case(case)
    if low:  # add a divergence in the lowest (kx, kz) modes
        x = np.arange(case.nx) * g.dx
        z = (np.arange(case.nz) + 0.5) * g.dz
        yc = 0.5 * (g.yf[1:] + g.yf[:-1])
        u = u + low * np.cos(2 * math.pi * z / case.lz)[:, None, None] * (1 - yc ** 2)[None, :, None] * \
            np.cos(2 * math.pi * x / case.lx)[None, None, :]
    b = O.divergence(g, u, v, w)
    b = b - (b * g.dy[None, :, None]).sum() / (g.dy.sum() * case.nx * case.nz)  # compatible
    nb = np.abs(b).max()
    phi64 = _poisson(g, b, False)
    assert np.abs(b - _lap(g, phi64)).max() < 1e-12 * nb
    sel = None
    if y32:
        sel, _ = PM.fp32_modes(g, False)
        assert 0.5 < sel.mean() < 1.0 and not sel[0].any()
    phi1 = _poisson(g, b, True, sel).astype(np.float64)
    r1 = b - _lap(g, phi1)
    assert 1e-9 * nb < np.abs(r1).max() < 1e-4 * nb  # the FP32 level: not good enough alone
    phi = phi1 + _poisson(g, r1, True, sel).astype(np.float64)
    r2 = b - _lap(g, phi)
    assert np.abs(r2).max() < 1e-10 * nb
    assert np.abs(r2).max() < 1e-3 * np.abs(r1).max()
    # the refined phi equals the FP64 solve up to the gauge constant
    e = (phi - phi.mean()) - (phi64 - phi64.mean())
    assert np.abs(e).max() < 1e-9 * np.abs(phi64).max()


@pytest.mark.parametrize("bl", [False, True])
def test_skeel_condition_by_one_solve_and_fp32_line_solves(bl):
    """The mode selection's two parts on the stretched y grids of the 256x192x256 channel and of
    the 1024x256x512 boundary layer: (1) kappa by one Thomas solve equals the definition
    || |A^-1| |A| 1 ||_inf by a dense inverse; (2) the FP32 sweep with rounded FP64 factors (c/pivot
    stored, or formed from the float 1/pivot as the staged form does) solves a mode's system to the
    FP32 level, and one refinement on the FP64 residual to the FP64 level (1e-12 where kappa <=
    4096);
    (3) kappa falls with the wavenumber, so the FP64 modes are the lowest ones."""
    if bl:
        g = O.Grid.from_case(I.boundary_layer_case(1024, 256, 512))
    else:
        g = O.Grid(256, 192, 256, 2 * math.pi, math.pi, I.channel_faces(192, 2.0))
    a, c = O.poisson_ycoeffs(g)
    lam = PM.mode_lambdas(g, bl)
    rng = np.random.default_rng(7)
    kz_kx = [(1, 0), (1, 1), (5, 3), (10, 10), (40, 40), (60, 100)]
    kaps = []
    for kz, kx in kz_kx:
        L = lam[kz, kx]
        k1 = PM.skeel(a, c, np.array([L]))[0]
        assert abs(k1 - PM.skeel_dense(a, c, L)) < 1e-9 * k1
        kaps.append(k1)
        A = np.diag(-(a + c) - L) + np.diag(a[1:], -1) + np.diag(c[:-1], 1)
        d = rng.standard_normal(g.ny) + 1j * rng.standard_normal(g.ny)
        x = np.linalg.solve(A, d)
        Bd = (-(a + c) - L)[None, :]
        for from_ip in (False, True):  # the register form's stored c/pivot, the staged form's c * (1/pivot)
            x1 = PM.thomas32(a[None, :], Bd, c[None, :], d[None, :], from_ip)[0].astype(np.complex128)
            x2 = x1 + PM.thomas32(a[None, :], Bd, c[None, :], (d - A @ x1)[None, :], from_ip)[0].astype(np.complex128)
            e1 = np.abs(x1 - x).max() / np.abs(x).max()
            e2 = np.abs(x2 - x).max() / np.abs(x).max()
            assert 1e-9 < e1 < 2e-6, (kz, kx, from_ip, e1)
            assert e2 < (1e-11 if k1 > PM.KAPPA_MAX else 1e-12), (kz, kx, from_ip, e2)
    assert all(k0 > k1 for k0, k1 in zip(kaps, kaps[1:]))
    assert kaps[0] > 1e4 and kaps[-1] < PM.KAPPA_MAX


@pytest.mark.parametrize("bl", [False, True])
def test_float_float_sweep_of_the_fp64_modes(bl):
    """The staged form sweeps its FP64 modes (kz = 0 and Skeel condition > 4096) in float-float
    arithmetic: on those modes of the stretched channel and boundary-layer grids its error on a
    random right-hand side stays within 1.5 times that of the FP64-arithmetic sweep (both store
    the rows in float), before and after one refinement on the FP64 residual (the refined error
    of a mode is set by its conditioning and the float rows, the same for both)."""
    if bl:
        g = O.Grid.from_case(I.boundary_layer_case(1024, 256, 512))
    else:
        g = O.Grid(256, 192, 256, 2 * math.pi, math.pi, I.channel_faces(192, 2.0))
    a, c = O.poisson_ycoeffs(g)
    lam = PM.mode_lambdas(g, bl)
    rng = np.random.default_rng(11)
    for kz, kx in [(0, 1), (0, 7), (1, 0), (1, 1), (2, 2)]:
        L = lam[kz, kx]
        if kz > 0:
            assert PM.skeel(a, c, np.array([L]))[0] > PM.KAPPA_MAX  # an FP64 mode
        B = -(a + c) - L
        A = np.diag(B) + np.diag(a[1:], -1) + np.diag(c[:-1], 1)
        d = rng.standard_normal(g.ny).astype(np.float32).astype(np.float64)
        x = np.linalg.solve(A, d)
        err = lambda y: np.abs(y - x).max() / np.abs(x).max()
        xf = PM.thomas_ff(a, B, c, d).astype(np.float64)
        x6 = PM.thomas64_stored32(a, B, c, d).astype(np.float64)
        assert err(xf) <= 1.5 * err(x6) + 1e-12, (kz, kx, err(xf), err(x6))
        x2 = xf + PM.thomas_ff(a, B, c, d - A @ xf).astype(np.float64)
        y2 = x6 + PM.thomas64_stored32(a, B, c, d - A @ x6).astype(np.float64)
        assert err(x2) <= 1.5 * err(y2) + 1e-14, (kz, kx, err(x2), err(y2))
        assert err(x2) < 1e-2 * err(xf), (kz, kx, err(x2), err(xf))

