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

sf = pytest.importorskip("scipy.fft")


def _poisson(g, rhs, fp32):
    """D G phi = rhs: z real transform, x transform, y Thomas per (kx, kz) in FP64, inverses;
    with fp32 the transforms and the spectrum are single precision (phi returned in FP32)."""
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
    ph = np.moveaxis(O.thomas(A, B, C, d), -1, 1)
    if fp32:
        ph = ph.astype(np.complex64)
    phi = sf.irfft(sf.ifft(ph, axis=2), n=g.nz, axis=0)
    return phi.astype(np.float32) if fp32 else phi


def _lap(g, phi):
    return O.divergence(g, *O.gradient(g, phi))


@pytest.mark.parametrize("low", [0.0, 20.0])
def test_fp32_transforms_need_one_fp64_refinement(low):
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
    phi1 = _poisson(g, b, True).astype(np.float64)
    r1 = b - _lap(g, phi1)
    assert 1e-9 * nb < np.abs(r1).max() < 1e-4 * nb  # the FP32 level: not good enough alone
    phi = phi1 + _poisson(g, r1, True).astype(np.float64)
    r2 = b - _lap(g, phi)
    assert np.abs(r2).max() < 1e-10 * nb
    assert np.abs(r2).max() < 1e-3 * np.abs(r1).max()
    # the refined phi equals the FP64 solve up to the gauge constant
    e = (phi - phi.mean()) - (phi64 - phi64.mean())
    assert np.abs(e).max() < 1e-9 * np.abs(phi64).max()
