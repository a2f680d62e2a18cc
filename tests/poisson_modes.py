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


def _fma32(a, b, c):
    """a b + c rounded once to float (float inputs: the product is exact in float64)."""
    return np.float32(np.float64(a) * np.float64(b) + np.float64(c))


def _ff_norm(s, e):
    h = np.float32(s + e)
    return h, np.float32(e - np.float32(h - s))


def _ff_mul(a, b):
    p = np.float32(a[0] * b[0])
    e = _fma32(a[0], b[0], -p)
    e = _fma32(a[0], b[1], _fma32(a[1], b[0], e))
    return _ff_norm(p, e)


def _ff_sub(x, b):
    s = np.float32(x - b[0])
    bb = np.float32(s - x)
    e = np.float32(np.float32(x - np.float32(s - bb)) + np.float32(-b[0] - bb))
    return _ff_norm(s, np.float32(e - b[1]))


def _ff_split(x):
    h = np.float32(x)
    return h, np.float32(x - np.float64(h))


def thomas_ff(a, b, c, d):
    """The staged form's sweep of an FP64 mode in float-float arithmetic, one real line: factors
    1/pivot and c/pivot formed in FP64 and split into two floats, a_j split likewise, the
    recurrences carried as float pairs, every row stored rounded to float (the spectrum is
    float).  a, b, c, d: (ny,) real; returns float32 (ny,)."""
    ny = len(d)
    ip, cp = np.empty(ny), np.empty(ny)
    prev = 0.0
    for j in range(ny):
        ip[j] = 1.0 / (b[j] - a[j] * prev)
        prev = c[j] * ip[j]
        cp[j] = prev
    out = np.empty(ny, np.float32)
    p = (np.float32(0), np.float32(0))
    for j in range(ny):
        p = _ff_mul(_ff_sub(np.float32(d[j]), _ff_mul(_ff_split(a[j]), p)), _ff_split(ip[j]))
        out[j] = p[0]
    n = p
    for j in range(ny - 2, -1, -1):
        n = _ff_sub(out[j], _ff_mul(_ff_split(cp[j]), n))
        out[j] = n[0]
    return out


def thomas64_stored32(a, b, c, d):
    """The same sweep in FP64 arithmetic with every row stored rounded to float (the FP64-mode
    sweep of the register form)."""
    ny = len(d)
    ip, cp = np.empty(ny), np.empty(ny)
    prev = 0.0
    for j in range(ny):
        ip[j] = 1.0 / (b[j] - a[j] * prev)
        prev = c[j] * ip[j]
        cp[j] = prev
    out = np.empty(ny, np.float32)
    p = 0.0
    for j in range(ny):
        p = (np.float64(np.float32(d[j])) - a[j] * p) * ip[j]
        out[j] = np.float32(p)
    n = p
    for j in range(ny - 2, -1, -1):
        n = np.float64(out[j]) - cp[j] * n
        out[j] = np.float32(n)
    return out

