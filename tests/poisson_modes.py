"""Which Poisson modes the mixed form may solve in FP32 arithmetic, restated for the tests: the
Skeel condition number kappa = || |A^-1| |A| 1 ||_inf of each (kx, kz) mode's y matrix A (rows
a_j, -(a_j + c_j) - lam, c_j of the oracle's operator), and the FP32 Thomas sweep the mixed form
runs on the modes with kz > 0 and kappa <= 4096 (factors formed in FP64 and rounded to float)."""
import math

import numpy as np

from oracle import ns_oracle as O

KAPPA_MAX = 4096.0


def mode_lambdas(g, bl):
    """lam[kz, kx] = lam_x + lam_z: periodic x (DFT) or the cosine transform of inflow / outflow x."""
    if bl:
        lx = (2.0 / (g.dx * g.dx)) * (1.0 - np.cos(math.pi * np.arange(g.nx) / g.nx))
    else:
        lx = O.modified_wavenumbers(g.nx, g.dx)
    lz = O.modified_wavenumbers(g.nz, g.dz)[: g.nz // 2 + 1]
    return lz[:, None] + lx[None, :]


def skeel_dense(a, c, lam):
    """kappa of one mode from the definition: dense inverse, absolute values, row sums."""
    A = np.diag(-(a + c) - lam) + np.diag(a[1:], -1) + np.diag(c[:-1], 1)
    return (np.abs(np.linalg.inv(A)) @ np.abs(A) @ np.ones(len(a))).max()


def skeel(a, c, lam):
    """kappa of every mode by one Thomas solve each: -A is an M-matrix (a_j, c_j >= 0), so A^-1
    has one sign and |A^-1| |A| 1 = y with -A y = |A| 1 = 2 (a_j + c_j) + lam."""
    L = np.asarray(lam, dtype=float).reshape(-1)
    Bm = (a + c)[None, :] + L[:, None]
    rhs = 2.0 * (a + c)[None, :] + L[:, None]
    y = O.thomas(np.broadcast_to(-a, Bm.shape).copy(), Bm, np.broadcast_to(-c, Bm.shape).copy(), rhs)
    return np.abs(y).max(axis=1).reshape(np.shape(lam))


def fp32_modes(g, bl):
    """The modes the mixed form solves in FP32: kz > 0 and kappa <= KAPPA_MAX (and the kappa)."""
    a, c = O.poisson_ycoeffs(g)
    lam = mode_lambdas(g, bl)
    kap = np.full(lam.shape, np.inf)
    kap[1:] = skeel(a, c, lam[1:])
    return kap <= KAPPA_MAX, kap


def thomas32(a, b, c, d, cp_from_ip=False):
    """Thomas sweeps in FP32 on complex64 data, with the factors 1/pivot and c/pivot formed in
    FP64 and rounded to float.  a, b, c: (..., ny) real; d: (..., ny) complex.  cp_from_ip: the
    staged form's backward factor, c_j rounded to float times the float 1/pivot (rounded again),
    instead of the rounded FP64 c/pivot."""
    ny = d.shape[-1]
    ip = np.empty(b.shape)
    cp = np.empty(b.shape)
    prev = np.zeros(b.shape[:-1])
    for j in range(ny):
        ip[..., j] = 1.0 / (b[..., j] - a[..., j] * prev)
        prev = c[..., j] * ip[..., j]
        cp[..., j] = prev
    ip, cp, a32 = ip.astype(np.float32), cp.astype(np.float32), a.astype(np.float32)
    if cp_from_ip:
        cp = (np.asarray(c, dtype=np.float32) * ip).astype(np.float32)
    x = d.astype(np.complex64)
    p = np.zeros(d.shape[:-1], np.complex64)
    for j in range(ny):
        p = ((x[..., j] - a32[..., j] * p) * ip[..., j]).astype(np.complex64)
        x[..., j] = p
    for j in range(ny - 2, -1, -1):
        x[..., j] = x[..., j] - cp[..., j] * x[..., j + 1]
    return x
