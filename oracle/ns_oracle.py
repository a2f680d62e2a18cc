"""FP64 CPU oracle of the fractional-step Navier-Stokes step (test infrastructure).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
bench's cpu_baseline / reference legs may import this module.  It shares no
code with the CUDA path; both sides take their inputs from
paper_1812_01178_gb300.inputs, which holds none of the method's arithmetic.

What it computes, with the paper's sections/equations (Ha, Park & You,
"A scalable multi-GPU method for semi-implicit fractional-step integration
of incompressible Navier-Stokes equations"):

* Sec. 2.1, Eq. (NScontinuity), Eq. (NSmomentum): incompressible NS on a
  staggered grid (velocities on faces, pressure at centres), uniform x and
  z, stretched y, no-slip wall(s), periodic z (and x for the channel).
* Sec. 2.2: low-storage RK3 for convection + Crank-Nicolson for viscous
  terms, 2nd-order central differences, ADI factorisation into three
  tridiagonal solves per velocity component, Poisson equation by Fourier
  transforms in x and z and (complex) tridiagonal solves in y, then the
  pseudo-pressure phi projects the velocity.
* Sec. 3.2, Eqs. (smidentity)-(xppt): the partitioned (PDD / PPT) solve of a
  tridiagonal system, written with the dense matrices A~, V, E, Y, Z, P, Z-bar
  exactly as the section defines them (used to pin the GPU's partitioned
  solver; the time step itself uses whole-line Thomas).

The paper leaves the discretisation details to an earlier work that is not
available; the readings used here (stencils, BC rows, RK3 constants,
interpolation weights, gauge) are stated in each function.  Every tridiagonal
system is solved by whole-line Thomas (cyclic lines by Sherman-Morrison),
every transform by a naive O(N^2) DFT from its definition.

Parity unpinned: the complete multi-step time integration is pinned only by
invariants (steady Poiseuille flow, closed-form decay of a Stokes mode,
third-order temporal convergence, divergence at round-off), not by a printed
result, because the paper prints none.

Array layout: numpy shape (nz, ny, nx) with x fastest; v has ny+1 rows
(rows 0 and ny are the walls, v = 0 there).
"""
from __future__ import annotations

import math

import numpy as np

# Low-storage RK3 (Sec. 2.2 names the scheme; constants are the standard set
# of Spalart, Moser & Rogers 1991 / Le & Moin 1991).  alpha_k = gamma_k + zeta_k.
RK3_GAMMA = (8.0 / 15.0, 5.0 / 12.0, 3.0 / 4.0)
RK3_ZETA = (0.0, -17.0 / 60.0, -5.0 / 12.0)
RK3_ALPHA = (8.0 / 15.0, 2.0 / 15.0, 1.0 / 3.0)


class Grid:
    """Staggered grid of Sec. 2.1: uniform x, z; face coordinates yf in y.

    ytop: 0 = no-slip wall at the top, 1 = stress-free top (v = 0,
    du/dy = dw/dy = 0).  The bottom is always a no-slip wall.  x and z are
    periodic.
    """

    def __init__(self, nx, ny, nz, lx, lz, yf, ytop=0):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.lx, self.lz = float(lx), float(lz)
        self.yf = np.asarray(yf, dtype=np.float64).copy()
        assert self.yf.shape == (self.ny + 1,)
        self.ytop = int(ytop)
        self.dx = self.lx / self.nx
        self.dz = self.lz / self.nz
        self.yc = 0.5 * (self.yf[:-1] + self.yf[1:])      # ny centres
        self.dy = self.yf[1:] - self.yf[:-1]              # ny cell heights
        self.hc = self.yc[1:] - self.yc[:-1]              # centre spacing across faces 1..ny-1

    @staticmethod
    def from_case(case):
        return Grid(case.nx, case.ny, case.nz, case.lx, case.lz, case.yf, case.bc_ytop)

    def volumes(self):
        """Control-volume sizes of u, v, w, p points (for weighted sums)."""
        cu = (self.dx * self.dz) * self.dy[None, :, None] * np.ones((self.nz, self.ny, self.nx))
        hv = np.zeros(self.ny + 1)
        hv[1:-1] = self.hc
        cv = (self.dx * self.dz) * hv[None, :, None] * np.ones((self.nz, self.ny + 1, self.nx))
        return cu, cv, cu.copy(), cu.copy()


# ----------------------------------------------------------------------------
# neighbour access (periodic x: axis 2, periodic z: axis 0)
# ----------------------------------------------------------------------------

def _xp(f):
    return np.roll(f, -1, axis=2)


def _xm(f):
    return np.roll(f, 1, axis=2)


def _zp(f):
    return np.roll(f, -1, axis=0)


def _zm(f):
    return np.roll(f, 1, axis=0)


def _centre_to_yface(g, f):
    """Linear interpolation of a centre quantity to y-faces 0..ny.

    Face j lies between centres j-1 and j; the weights are the distances
    (Sec. 2.2: 2nd-order central differences on the stretched grid).  The wall
    faces (0 and ny) get 0: every flux through them is multiplied by v = 0.
    """
    nz, ny, nx = f.shape
    out = np.zeros((nz, ny + 1, nx))
    whi = (g.yf[1:-1] - g.yc[:-1]) / g.hc          # weight of centre j at face j
    wlo = 1.0 - whi                                 # weight of centre j-1
    out[:, 1:-1, :] = wlo[None, :, None] * f[:, :-1, :] + whi[None, :, None] * f[:, 1:, :]
    return out


# ----------------------------------------------------------------------------
# spatial operators (Sec. 2.1 / 2.2)
# ----------------------------------------------------------------------------

def convection(g, u, v, w):
    """Divergence-form convection d(u_i u_j)/dx_j of Eq. (NSmomentum).

    Central differences of face/edge fluxes; velocities are averaged
    arithmetically in x and z and interpolated linearly in y.  Returns
    (Nu, Nv, Nw) at the u, v, w points; Nv rows 0 and ny are 0.
    """
    dx, dz = g.dx, g.dz
    dy = g.dy[None, :, None]
    hc = g.hc[None, :, None]
    # ---- Nu at (xf_i, yc_j, zc_k)
    uc = 0.5 * (u + _xp(u))                                   # u at centre i
    nux = (uc * uc - _xm(uc) * _xm(uc)) / dx
    u_yf = _centre_to_yface(g, u)                             # u at (xf_i, yf_j)
    v_xf = 0.5 * (_xm(v) + v)                                 # v at (xf_i, yf_j)
    fuv = u_yf * v_xf
    nuy = (fuv[:, 1:, :] - fuv[:, :-1, :]) / dy
    u_zf = 0.5 * (_zm(u) + u)                                 # u at (xf_i, zf_k)
    w_xf = 0.5 * (_xm(w) + w)                                 # w at (xf_i, zf_k)
    fuw = u_zf * w_xf                                         # edge (xf_i, yc_j, zf_k)
    nuz = (_zp(fuw) - fuw) / dz
    Nu = nux + nuy + nuz
    # ---- Nv at (xc_i, yf_j, zc_k), j = 1..ny-1
    nvx = (_xp(fuv) - fuv) / dx
    vc = 0.5 * (v[:, :-1, :] + v[:, 1:, :])                   # v at centres
    nvy = np.zeros_like(v)
    nvy[:, 1:-1, :] = (vc[:, 1:, :] ** 2 - vc[:, :-1, :] ** 2) / hc
    v_zf = 0.5 * (_zm(v) + v)                                 # v at (yf_j, zf_k)
    w_yf = _centre_to_yface(g, w)                             # w at (yf_j, zf_k)
    fvw = v_zf * w_yf
    nvz = (_zp(fvw) - fvw) / dz
    Nv = nvx + nvy + nvz
    Nv[:, 0, :] = 0.0
    Nv[:, -1, :] = 0.0
    # ---- Nw at (xc_i, yc_j, zf_k)
    nwx = (_xp(fuw) - fuw) / dx
    nwy = (fvw[:, 1:, :] - fvw[:, :-1, :]) / dy
    wc = 0.5 * (w + _zp(w))
    nwz = (wc * wc - _zm(wc) * _zm(wc)) / dz
    Nw = nwx + nwy + nwz
    return Nu, Nv, Nw


def gradient(g, p):
    """Pressure gradient G p at the u, v, w points (v rows 0, ny are 0)."""
    gx = (p - _xm(p)) / g.dx
    gy = np.zeros((g.nz, g.ny + 1, g.nx))
    gy[:, 1:-1, :] = (p[:, 1:, :] - p[:, :-1, :]) / g.hc[None, :, None]
    gz = (p - _zm(p)) / g.dz
    return gx, gy, gz


def divergence(g, u, v, w):
    """Discrete divergence D u at cell centres (continuity, Eq. NScontinuity)."""
    return ((_xp(u) - u) / g.dx
            + (v[:, 1:, :] - v[:, :-1, :]) / g.dy[None, :, None]
            + (_zp(w) - w) / g.dz)


def yrows_centre(g):
    """Coefficients (A, C) of the y second derivative at centres.

    d2f/dy2 at centre j ~ A_j f_{j-1} - (A_j + C_j) f_j + C_j f_{j+1}, the
    three-point formula on non-uniform spacing (exact for quadratics).  Below
    centre 0 the neighbour is the wall at yf_0 (value 0, no slip).  At the
    top: a no-slip wall at yf_ny, or, for a stress-free top, zero flux
    (C_{ny-1} = 0).  The wall neighbour's coefficient is kept in the diagonal.
    """
    ny = g.ny
    hm = np.empty(ny)
    hp = np.empty(ny)
    hm[0] = g.yc[0] - g.yf[0]
    hm[1:] = g.hc
    hp[:-1] = g.hc
    hp[-1] = g.yf[-1] - g.yc[-1]
    A = 2.0 / (hm * (hm + hp))
    C = 2.0 / (hp * (hm + hp))
    if g.ytop == 1:
        C[-1] = 0.0
    return A, C


def yrows_face(g):
    """Coefficients (A, C) of the y second derivative at interior faces 1..ny-1.

    Same three-point formula with spacings dy_{j-1}, dy_j; v = 0 at both
    boundary faces.
    """
    hm = g.dy[:-1]
    hp = g.dy[1:]
    A = 2.0 / (hm * (hm + hp))
    C = 2.0 / (hp * (hm + hp))
    return A, C


def _dyy_centre(g, f):
    A, C = yrows_centre(g)
    fm = np.zeros_like(f)
    fp = np.zeros_like(f)
    fm[:, 1:, :] = f[:, :-1, :]
    fp[:, :-1, :] = f[:, 1:, :]
    return A[None, :, None] * fm - (A + C)[None, :, None] * f + C[None, :, None] * fp


def _dyy_face(g, f):
    A, C = yrows_face(g)
    out = np.zeros_like(f)
    out[:, 1:-1, :] = (A[None, :, None] * f[:, :-2, :] - (A + C)[None, :, None] * f[:, 1:-1, :]
                       + C[None, :, None] * f[:, 2:, :])
    return out


def laplacian(g, u, v, w):
    """Viscous operator (delta_xx + delta_yy + delta_zz) of each component."""
    def dxx(f):
        return (_xp(f) - 2.0 * f + _xm(f)) / (g.dx * g.dx)

    def dzz(f):
        return (_zp(f) - 2.0 * f + _zm(f)) / (g.dz * g.dz)

    Lu = dxx(u) + _dyy_centre(g, u) + dzz(u)
    Lv = dxx(v) + _dyy_face(g, v) + dzz(v)
    Lv[:, 0, :] = 0.0
    Lv[:, -1, :] = 0.0
    Lw = dxx(w) + _dyy_centre(g, w) + dzz(w)
    return Lu, Lv, Lw


# ----------------------------------------------------------------------------
# tridiagonal solvers
# ----------------------------------------------------------------------------

def thomas(a, b, c, d):
    """Thomas algorithm for a_j x_{j-1} + b_j x_j + c_j x_{j+1} = d_j.

    The line runs along the last axis of d; a, b, c broadcast against d
    (a_0 and c_{n-1} are ignored).  Forward elimination then back
    substitution, no pivoting.  A 1-D a, b or c holds the same rows for every
    line; when all three are 1-D the pivots and c'_j are computed once for all
    lines.  The operations on each element are the same either way.  The
    recurrences run over the rows of an array with the row index first, so that
    each step works on one slice of all lines.
    """
    d = np.asarray(d)
    n = d.shape[-1]
    D = np.moveaxis(d, -1, 0)
    A, Bm, Cm = (np.asarray(q) if np.ndim(q) == 1 else np.moveaxis(np.broadcast_to(q, d.shape), -1, 0)
                 for q in (a, b, c))
    shared = A.ndim == Bm.ndim == Cm.ndim == 1
    cp = np.empty(Bm.shape if shared else D.shape, dtype=np.result_type(Bm, Cm, np.float64))
    dp = np.empty(D.shape, dtype=np.result_type(D, Bm, Cm, np.float64))
    den = Bm[0]
    cp[0] = Cm[0] / den
    dp[0] = D[0] / den
    for j in range(1, n):
        den = Bm[j] - A[j] * cp[j - 1]
        cp[j] = Cm[j] / den
        dp[j] = (D[j] - A[j] * dp[j - 1]) / den
    x = np.empty_like(dp)
    x[n - 1] = dp[n - 1]
    for j in range(n - 2, -1, -1):
        x[j] = dp[j] - cp[j] * x[j + 1]
    return np.moveaxis(x, 0, -1)


def thomas_cyclic(a, b, c, d):
    """Periodic tridiagonal solve (a_0 couples x_{n-1}, c_{n-1} couples x_0).

    Sherman-Morrison on top of Thomas: A = B + s t^T with s = (g,0..0,c_{n-1}),
    t = (1,0..0,a_0/g), g = -b_0; x = y - (t.y)/(1 + t.q) q with B y = d, B q = s.
    With 1-D a, b, c (the same rows for every line) q is one vector shared by all lines.
    """
    d = np.asarray(d)
    n = d.shape[-1]
    shp = (n,) if all(np.ndim(q) == 1 for q in (a, b, c)) else d.shape
    a = np.array(np.broadcast_to(a, shp), dtype=np.float64)
    b = np.array(np.broadcast_to(b, shp), dtype=np.float64)
    c = np.array(np.broadcast_to(c, shp), dtype=np.float64)
    gam = -b[..., 0]
    alpha = c[..., n - 1]       # A[n-1, 0]
    beta = a[..., 0]            # A[0, n-1]
    bb = b.copy()
    bb[..., 0] = b[..., 0] - gam
    bb[..., n - 1] = b[..., n - 1] - alpha * beta / gam
    y = thomas(a, bb, c, d)
    s = np.zeros(shp)
    s[..., 0] = gam
    s[..., n - 1] = alpha
    q = thomas(a, bb, c, s)
    fac = (y[..., 0] + beta / gam * y[..., n - 1]) / (1.0 + q[..., 0] + beta / gam * q[..., n - 1])
    return y - fac[..., None] * q


# ----------------------------------------------------------------------------
# Sec. 3.2: partitioned solve (PDD / PPT) with the paper's dense matrices
# ----------------------------------------------------------------------------

def tridiag_dense(a, b, c, cyclic=False):
    n = len(b)
    A = np.diag(np.asarray(b, dtype=np.float64))
    for j in range(1, n):
        A[j, j - 1] = a[j]
        A[j - 1, j] = c[j - 1]
    if cyclic and n > 2:
        A[0, n - 1] = a[0]
        A[n - 1, 0] = c[n - 1]
    return A


def partition_matrices(a, b, c, p, cyclic=False):
    """A = A~ + V E^T of Sec. 3.2 for p partitions of m = n/p rows.

    A~ is A with the couplings between partitions removed (block-tridiagonal);
    for interface r (between partition r and r+1, and p-1 -> 0 if cyclic)
    the two cut couplings are c at the last row of r and a at the first row
    of r+1.  Columns of V / rows of E^T come in pairs per interface, in the
    order of y = E^T x = (x^{(r)}_m, x^{(r+1)}_1): V's first column of the pair
    is a_{first(r+1)} e_{first(r+1)} (it pairs with x^{(r)}_m), the second is
    c_{last(r)} e_{last(r)} (it pairs with x^{(r+1)}_1).
    """
    n = len(b)
    assert n % p == 0
    m = n // p
    A = tridiag_dense(a, b, c, cyclic)
    nif = p if cyclic else p - 1
    V = np.zeros((n, 2 * nif))
    E = np.zeros((n, 2 * nif))
    for r in range(nif):
        last = r * m + m - 1
        first = ((r + 1) % p) * m
        V[first, 2 * r] = A[first, last]
        E[last, 2 * r] = 1.0
        V[last, 2 * r + 1] = A[last, first]
        E[first, 2 * r + 1] = 1.0
    At = A - V @ E.T
    return A, At, V, E


def swap_permutation(k):
    """The permutation P = P^{-1} of Sec. 3.2 that swaps entries 2r and 2r+1."""
    P = np.zeros((k, k))
    for r in range(0, k, 2):
        P[r, r + 1] = 1.0
        P[r + 1, r] = 1.0
    return P


def ppt_solve(a, b, c, d, p, cyclic=False):
    """PPT of Sec. 3.2: A~ x~ = d (Eq. blockAx), A~ Ybar = V P (Eq. blockAYbar),
    Zbar y = E^T x~ (Eq. Zppt) with Zbar = P + E^T A~^{-1} V P, x = x~ - Ybar y
    (Eq. xppt).  Exact.  Dense solves stand in for the per-block solves."""
    A, At, V, E = partition_matrices(a, b, c, p, cyclic)
    xt = np.linalg.solve(At, d)
    P = swap_permutation(V.shape[1])
    Ybar = np.linalg.solve(At, V @ P)
    Zbar = P + E.T @ Ybar
    y = np.linalg.solve(Zbar, E.T @ xt)
    return xt - Ybar @ y


def pdd_solve(a, b, c, d, p, cyclic=False):
    """PDD of Sec. 3.2: A~ x~ = d, A~ Y = V (Eq. blockAY), then Z y = E^T x~
    (Eq. Zpdd) with Z = I + E^T Y reduced to its 2x2 diagonal blocks (the
    couplings v_m, w_1 between interfaces dropped), x = x~ - Y y (Eq. xpdd)."""
    A, At, V, E = partition_matrices(a, b, c, p, cyclic)
    xt = np.linalg.solve(At, d)
    Y = np.linalg.solve(At, V)
    Z = np.eye(V.shape[1]) + E.T @ Y
    Zb = np.zeros_like(Z)
    for r in range(0, Z.shape[0], 2):
        Zb[r:r + 2, r:r + 2] = Z[r:r + 2, r:r + 2]
    y = np.linalg.solve(Zb, E.T @ xt)
    return xt - Y @ y


def pdd_dropped_coupling(a, b, c, p, cyclic=False):
    """Largest entry of Z outside its 2x2 diagonal blocks (what PDD drops)."""
    A, At, V, E = partition_matrices(a, b, c, p, cyclic)
    Z = np.eye(V.shape[1]) + E.T @ np.linalg.solve(At, V)
    Zo = Z.copy()
    for r in range(0, Z.shape[0], 2):
        Zo[r:r + 2, r:r + 2] = 0.0
    return float(np.abs(Zo).max()) if Zo.size else 0.0


# ----------------------------------------------------------------------------
# ADI (Sec. 2.2): (I - b d_xx)(I - b d_yy)(I - b d_zz) delta = r
# ----------------------------------------------------------------------------

def adi_rows(g, direction, comp, beta):
    """(a, b, c) of one line of (I - beta*delta_dd), as 1-D arrays.

    x, z: a = c = -beta/h^2, b = 1 + 2 beta/h^2 (periodic, cyclic).
    y: a = -beta A_j, c = -beta C_j, b = 1 + beta (A_j + C_j) from
    yrows_centre (u, w) or yrows_face (v: the ny-1 interior faces).
    """
    if direction in (0, 2):
        h = g.dx if direction == 0 else g.dz
        n = g.nx if direction == 0 else g.nz
        r = beta / (h * h)
        return (np.full(n, -r), np.full(n, 1.0 + 2.0 * r), np.full(n, -r))
    A, C = yrows_face(g) if comp == 1 else yrows_centre(g)
    return (-beta * A, 1.0 + beta * (A + C), -beta * C)


def adi_sweep(g, r, direction, comp, beta):
    """Solve (I - beta delta_dd) x = r along one direction for one component."""
    a, b, c = adi_rows(g, direction, comp, beta)
    if direction == 0:
        return thomas_cyclic(a, b, c, r)
    if direction == 2:
        return np.moveaxis(thomas_cyclic(a, b, c, np.moveaxis(r, 0, -1)), -1, 0)
    if comp == 1:
        out = np.zeros_like(r)
        out[:, 1:-1, :] = np.moveaxis(thomas(a, b, c, np.moveaxis(r[:, 1:-1, :], 1, -1)), -1, 1)
        return out
    return np.moveaxis(thomas(a, b, c, np.moveaxis(r, 1, -1)), -1, 1)


def adi_solve(g, r3, beta):
    """x, then y, then z sweep on each component (delta form)."""
    out = []
    for comp, r in enumerate(r3):
        x = adi_sweep(g, r, 0, comp, beta)
        x = adi_sweep(g, x, 1, comp, beta)
        x = adi_sweep(g, x, 2, comp, beta)
        out.append(x)
    return out


# ----------------------------------------------------------------------------
# Poisson (Sec. 2.2): transforms in x and z, tridiagonal in y
# ----------------------------------------------------------------------------

def dft_matrix(n, sign=-1):
    k = np.arange(n)
    return np.exp(sign * 2j * math.pi * np.outer(k, k) / n)


# Lines longer than this are transformed by numpy's FFT (the same sums, O(N log N)); shorter
# ones by the definition.  The FFT is pinned against the definition at lengths above the limit.
NAIVE_DFT_MAX = 64


def dft(f, axis, sign=-1):
    """DFT along an axis: F_k = sum_n f_n exp(sign 2 pi i k n / N), unnormalised in both
    directions.  Naive O(N^2) matrix product for N <= NAIVE_DFT_MAX, numpy's FFT above."""
    n = f.shape[axis]
    if n > NAIVE_DFT_MAX:
        if sign < 0:
            return np.fft.fft(f, axis=axis)
        return np.fft.ifft(f, axis=axis, norm="forward")
    M = dft_matrix(n, sign)
    return np.moveaxis(np.moveaxis(f, axis, -1) @ M.T, -1, axis)


def poisson_ycoeffs(g):
    """y rows of the Poisson operator D G: a_j phi_{j-1} + diag phi_j + c_j phi_{j+1}.

    a_j = 1/(dy_j hc_j), c_j = 1/(dy_j hc_{j+1}); zero normal gradient at both
    y boundaries (a_0 = c_{ny-1} = 0).  Returns (a, c).
    """
    ny = g.ny
    a = np.zeros(ny)
    c = np.zeros(ny)
    a[1:] = 1.0 / (g.dy[1:] * g.hc)
    c[:-1] = 1.0 / (g.dy[:-1] * g.hc)
    return a, c


def modified_wavenumbers(n, h):
    """Eigenvalues of -(f_{i+1} - 2 f_i + f_{i-1})/h^2 on a periodic line."""
    l = np.arange(n)
    return (2.0 / (h * h)) * (1.0 - np.cos(2.0 * math.pi * l / n))


def poisson_solve(g, rhs):
    """Solve D G phi = rhs (pure Neumann in y, periodic x, z).

    Forward DFT in x and z, one complex tridiagonal solve per (l, m) in y,
    inverse DFT.  Gauge for the singular (0, 0) mode: its row j = 0 is
    replaced by phi_0 = 0.
    """
    bh = dft(dft(rhs.astype(np.complex128), 2), 0)              # (nz, ny, nx)
    a, c = poisson_ycoeffs(g)
    lx = modified_wavenumbers(g.nx, g.dx)
    lz = modified_wavenumbers(g.nz, g.dz)
    lam = lz[:, None] + lx[None, :]                              # (nz, nx)
    d = np.moveaxis(bh, 1, -1)                                   # (nz, nx, ny)
    A = np.broadcast_to(a, d.shape).copy()
    C = np.broadcast_to(c, d.shape).copy()
    B = -(a + c)[None, None, :] - lam[:, :, None]
    B = np.array(np.broadcast_to(B, d.shape))
    B[0, 0, 0] = 1.0
    C[0, 0, 0] = 0.0
    d = d.copy()
    d[0, 0, 0] = 0.0
    ph = thomas(A, B, C, d)
    ph = np.moveaxis(ph, -1, 1)
    phi = dft(dft(ph, 0, +1), 2, +1) / (g.nx * g.nz)
    return phi.real.copy()


def project(g, u, v, w, phi, scale):
    """u <- u - scale * G phi (Sec. 2.2, the projection with the pseudo-pressure)."""
    gx, gy, gz = gradient(g, phi)
    return u - scale * gx, v - scale * gy, w - scale * gz


def make_divergence_free(g, u, v, w):
    """Project an initial field: solve D G phi = D u and subtract G phi."""
    phi = poisson_solve(g, divergence(g, u, v, w))
    return project(g, u, v, w, phi, 1.0)


# ----------------------------------------------------------------------------
# RK3 sub-step and full step (Sec. 2.2)
# ----------------------------------------------------------------------------

def rhs(g, u, v, w, p, nprev, k, dt, re, fx):
    """Explicit right-hand side of sub-step k in delta form.

    r = dt [ -gamma_k N(u) - zeta_k N_prev - alpha_k G p
             + (alpha_k/Re) L(u) + alpha_k f ]
    with f = (fx, 0, 0).  Returns (r, N(u)); N(u) becomes N_prev of the next
    sub-step.  inv_re = 0 is allowed (re = inf).
    """
    gam, zet, alp = RK3_GAMMA[k], RK3_ZETA[k], RK3_ALPHA[k]
    N = convection(g, u, v, w)
    G = gradient(g, p)
    L = laplacian(g, u, v, w)
    inv_re = 0.0 if not np.isfinite(re) else 1.0 / re
    r = []
    for comp in range(3):
        t = -gam * N[comp] - alp * G[comp] + (alp * inv_re) * L[comp]
        if zet != 0.0:
            t = t - zet * nprev[comp]
        if comp == 0:
            t = t + alp * fx
        t = dt * t
        if comp == 1:
            t[:, 0, :] = 0.0
            t[:, -1, :] = 0.0
        r.append(t)
    return r, N


def pressure_update(p, phi, lap_phi, beta, pressure):
    """p = p + phi (pressure="delta"), or the Kim & Moin (J. Comput. Phys. 59, 1985) form
    p = p + phi - beta_k L phi with L = D G, the operator of the Poisson solve
    (pressure="kim_moin")."""
    if pressure == "delta":
        return p + phi
    if pressure == "kim_moin":
        return p + phi - beta * lap_phi
    raise ValueError(pressure)


def substep(g, state, k, dt, re, fx, pressure="delta"):
    """One RK3 sub-step: RHS, ADI (x, y, z), u* = u + delta, Poisson, projection.

    state = dict(u, v, w, p, nprev); returns a new dict.  beta_k = alpha_k dt/(2 Re);
    the Poisson right-hand side is D u* / (alpha_k dt); u = u* - alpha_k dt G phi;
    p = p + phi (or the Kim-Moin form, pressure_update).
    """
    u, v, w, p = state["u"], state["v"], state["w"], state["p"]
    r, N = rhs(g, u, v, w, p, state.get("nprev"), k, dt, re, fx)
    inv_re = 0.0 if not np.isfinite(re) else 1.0 / re
    beta = RK3_ALPHA[k] * dt * inv_re / 2.0
    du, dv, dw = adi_solve(g, r, beta)
    us, vs, ws = u + du, v + dv, w + dw
    scale = RK3_ALPHA[k] * dt
    phi = poisson_solve(g, divergence(g, us, vs, ws) / scale)
    un, vn, wn = project(g, us, vs, ws, phi, scale)
    lap = divergence(g, *gradient(g, phi)) if pressure != "delta" else None
    return dict(u=un, v=vn, w=wn, p=pressure_update(p, phi, lap, beta, pressure), nprev=N, phi=phi)


def step(g, state, dt, re, fx, nsteps=1, pressure="delta"):
    """nsteps full time steps of three RK3 sub-steps each."""
    s = dict(state)
    for _ in range(nsteps):
        for k in range(3):
            s = substep(g, s, k, dt, re, fx, pressure)
    return s


# ----------------------------------------------------------------------------
# Time step at a fixed CFL number (the paper's runs hold CFL = 1.0, Sec. 4)
# ----------------------------------------------------------------------------
# Reading: the paper gives no formula for its CFL number.  Here it is the convective one,
# dt max over cells of |u|/dx + |v_c|/dy_j + |w|/dz, with u and w the values on the cell's lower
# x and z faces and v_c the average of its two y faces; dt is set before every step from the
# velocity at the start of the step and held for the three sub-steps.

def convective_rate(g, u, v, w):
    """max over cells of |u|/dx + |v_c|/dy_j + |w|/dz (so that CFL = dt * rate)."""
    vc = 0.5 * (v[:, :-1, :] + v[:, 1:, :])
    c = np.abs(u) / g.dx + np.abs(vc) / g.dy[None, :, None] + np.abs(w) / g.dz
    return float(c.max())


def step_cfl(g, state, cfl, re, fx, nsteps=1, pressure="delta", bl=False, u_conv=1.0):
    """nsteps steps, each with dt = cfl / convective_rate(velocity at the start of the step).
    Returns (state, list of the dt of each step)."""
    s = dict(state)
    dts = []
    for _ in range(nsteps):
        dt = cfl / convective_rate(g, s["u"], s["v"], s["w"])
        dts.append(dt)
        if bl:
            s = step_bl(g, s, dt, re, fx, 1, u_conv, pressure)
        else:
            s = step(g, s, dt, re, fx, 1, pressure)
    return s, dts


# ----------------------------------------------------------------------------
# Inflow / convective outflow in x (the flat-plate configuration of Sec. 2.1)
# ----------------------------------------------------------------------------
# Readings (the paper gives the boundary conditions in words only, Sec. 2.1):
# * u is stored on faces 0..nx-1 (face 0 = inflow, fixed); the outflow face nx lives in the
#   plane bl["u_out"] (nz, ny).  v and w keep their values on the inflow / outflow faces in
#   bl["v_in"], bl["v_out"] (nz, ny+1) and bl["w_in"], bl["w_out"] (nz, ny).
# * v and w see the boundary faces through linear ghost cells, f_ghost = 2 f_b - f_adjacent,
#   so every interior stencil keeps its form (the face average of ghost and neighbour is f_b).
# * Convective outflow df/dt + U_c df/dx = 0: one first-order upwind step of alpha_k dt per
#   sub-step, with the interior neighbour at distance dx (u) or dx/2 (v, w).
# * Before the Poisson solve the outflow u is shifted uniformly so that the outflow volume flux
#   equals the inflow flux (no flux through the walls / stress-free top), which makes the pure
#   Neumann problem compatible.
# * The Poisson operator has zero normal gradient at x = 0 and x = Lx as well: it is
#   diagonalised by the DCT-II in x (the half-range cosine transform of Sec. 2.2).

def _xnext_u(u, bl):
    """u at face i+1 (face nx from the outflow plane)."""
    return np.concatenate([u[:, :, 1:], bl["u_out"][:, :, None]], axis=2)


def _xprev_u(u):
    """u at face i-1 (face -1 does not exist: 0, never used for an unknown)."""
    return np.concatenate([np.zeros_like(u[:, :, :1]), u[:, :, :-1]], axis=2)


def _xnext_c(f, f_out):
    """Centre value at i+1 with the outflow ghost 2 f_out - f_{nx-1}."""
    return np.concatenate([f[:, :, 1:], (2.0 * f_out - f[:, :, -1])[:, :, None]], axis=2)


def _xprev_c(f, f_in):
    """Centre value at i-1 with the inflow ghost 2 f_in - f_0."""
    return np.concatenate([(2.0 * f_in - f[:, :, 0])[:, :, None], f[:, :, :-1]], axis=2)


def convection_bl(g, u, v, w, bl):
    """Divergence-form convection with inflow / outflow in x (same stencils as convection())."""
    dx, dz = g.dx, g.dz
    dy = g.dy[None, :, None]
    hc = g.hc[None, :, None]
    ux = _xnext_u(u, bl)
    uc = 0.5 * (u + ux)                                        # u at centres 0..nx-1
    nux = (uc * uc - _xprev_c(uc, np.zeros_like(uc[:, :, 0])) ** 2) / dx
    u_yf = _centre_to_yface(g, u)
    v_xf = 0.5 * (_xprev_c(v, bl["v_in"]) + v)                  # v at x-faces 0..nx-1
    fuv = u_yf * v_xf
    nuy = (fuv[:, 1:, :] - fuv[:, :-1, :]) / dy
    u_zf = 0.5 * (_zm(u) + u)
    w_xf = 0.5 * (_xprev_c(w, bl["w_in"]) + w)
    fuw = u_zf * w_xf
    nuz = (_zp(fuw) - fuw) / dz
    Nu = nux + nuy + nuz
    Nu[:, :, 0] = 0.0                                           # inflow face: fixed
    # edge fluxes on the outflow face nx
    uo_yf = _centre_to_yface(g, bl["u_out"][:, :, None])[:, :, 0]
    fuv_out = uo_yf * bl["v_out"]
    uo_zf = 0.5 * (_zm(bl["u_out"]) + bl["u_out"])
    fuw_out = uo_zf * bl["w_out"]
    fuv_n = np.concatenate([fuv[:, :, 1:], fuv_out[:, :, None]], axis=2)
    fuw_n = np.concatenate([fuw[:, :, 1:], fuw_out[:, :, None]], axis=2)
    nvx = (fuv_n - fuv) / dx
    vc = 0.5 * (v[:, :-1, :] + v[:, 1:, :])
    nvy = np.zeros_like(v)
    nvy[:, 1:-1, :] = (vc[:, 1:, :] ** 2 - vc[:, :-1, :] ** 2) / hc
    v_zf = 0.5 * (_zm(v) + v)
    w_yf = _centre_to_yface(g, w)
    fvw = v_zf * w_yf
    nvz = (_zp(fvw) - fvw) / dz
    Nv = nvx + nvy + nvz
    Nv[:, 0, :] = 0.0
    Nv[:, -1, :] = 0.0
    nwx = (fuw_n - fuw) / dx
    nwy = (fvw[:, 1:, :] - fvw[:, :-1, :]) / dy
    wc = 0.5 * (w + _zp(w))
    nwz = (wc * wc - _zm(wc) * _zm(wc)) / dz
    Nw = nwx + nwy + nwz
    return Nu, Nv, Nw


def gradient_bl(g, p):
    """G p with no correction on the inflow face (u fixed there)."""
    gx = (p - _xm(p)) / g.dx
    gx[:, :, 0] = 0.0
    gy = np.zeros((g.nz, g.ny + 1, g.nx))
    gy[:, 1:-1, :] = (p[:, 1:, :] - p[:, :-1, :]) / g.hc[None, :, None]
    gz = (p - _zm(p)) / g.dz
    return gx, gy, gz


def divergence_bl(g, u, v, w, bl):
    return ((_xnext_u(u, bl) - u) / g.dx
            + (v[:, 1:, :] - v[:, :-1, :]) / g.dy[None, :, None]
            + (_zp(w) - w) / g.dz)


def laplacian_bl(g, u, v, w, bl):
    def dzz(f):
        return (_zp(f) - 2.0 * f + _zm(f)) / (g.dz * g.dz)
    h2 = g.dx * g.dx
    Lu = (_xnext_u(u, bl) - 2.0 * u + _xprev_u(u)) / h2 + _dyy_centre(g, u) + dzz(u)
    Lu[:, :, 0] = 0.0
    Lv = (_xnext_c(v, bl["v_out"]) - 2.0 * v + _xprev_c(v, bl["v_in"])) / h2 + _dyy_face(g, v) + dzz(v)
    Lv[:, 0, :] = 0.0
    Lv[:, -1, :] = 0.0
    Lw = (_xnext_c(w, bl["w_out"]) - 2.0 * w + _xprev_c(w, bl["w_in"])) / h2 + _dyy_centre(g, w) + dzz(w)
    return Lu, Lv, Lw


def rhs_bl(g, u, v, w, p, nprev, bl, k, dt, re, fx):
    """rhs() with inflow / outflow in x: the inflow face of u gets r = 0."""
    gam, zet, alp = RK3_GAMMA[k], RK3_ZETA[k], RK3_ALPHA[k]
    N = convection_bl(g, u, v, w, bl)
    G = gradient_bl(g, p)
    L = laplacian_bl(g, u, v, w, bl)
    inv_re = 0.0 if not np.isfinite(re) else 1.0 / re
    r = []
    for comp in range(3):
        t = -gam * N[comp] - alp * G[comp] + (alp * inv_re) * L[comp]
        if zet != 0.0:
            t = t - zet * nprev[comp]
        if comp == 0:
            t = t + alp * fx
        t = dt * t
        if comp == 0:
            t[:, :, 0] = 0.0
        if comp == 1:
            t[:, 0, :] = 0.0
            t[:, -1, :] = 0.0
        r.append(t)
    return r, N


def outflow_update(g, u, v, w, bl, scale, u_conv):
    """One upwind step (scale = alpha_k dt) of df/dt + U_c df/dx = 0 on the outflow planes.
    Returns the new planes and their increments."""
    new = dict(bl)
    c = scale * u_conv
    new["u_out"] = bl["u_out"] - c * (bl["u_out"] - u[:, :, -1]) / g.dx
    new["v_out"] = bl["v_out"] - c * (bl["v_out"] - v[:, :, -1]) / (0.5 * g.dx)
    new["w_out"] = bl["w_out"] - c * (bl["w_out"] - w[:, :, -1]) / (0.5 * g.dx)
    new["v_out"][:, 0] = 0.0
    new["v_out"][:, -1] = 0.0
    inc = {q: new[q] - bl[q] for q in ("u_out", "v_out", "w_out")}
    return new, inc


def adi_rows_x_bl(g, comp, beta):
    """Rows of (I - beta delta_xx) with inflow / outflow.  u: faces 0..nx-1, row 0 is the fixed
    inflow face (identity).  v, w: centres with ghost rows at both ends (b = 1 + 3r)."""
    n = g.nx
    r = beta / (g.dx * g.dx)
    a = np.full(n, -r)
    b = np.full(n, 1.0 + 2.0 * r)
    c = np.full(n, -r)
    if comp == 0:
        a[0], b[0], c[0] = 0.0, 1.0, 0.0
    else:
        b[0] = 1.0 + 3.0 * r
        b[-1] = 1.0 + 3.0 * r
    a[0] = 0.0
    c[-1] = 0.0
    return a, b, c


def adi_sweep_x_bl(g, rr, comp, beta, inc_out):
    """x sweep with inflow / outflow: the outflow increment enters the last row's right-hand side
    (coefficient r for u, 2r for the ghost of v, w; the inflow increment is zero)."""
    a, b, c = adi_rows_x_bl(g, comp, beta)
    r = beta / (g.dx * g.dx)
    d = rr.copy()
    d[:, :, -1] += (r if comp == 0 else 2.0 * r) * inc_out
    return thomas(a, b, c, d)


def flux_correct_outflow(g, u_in, u_out):
    """Shift u_out uniformly so that its volume flux equals the inflow flux."""
    area = (g.yf[-1] - g.yf[0]) * g.lz
    w = g.dy[None, :] * g.dz
    q_in = float((u_in * w).sum())
    q_out = float((u_out * w).sum())
    return u_out + (q_in - q_out) / area


def dct2_matrix(n):
    """DCT-II: X_l = sum_i x_i cos(pi l (2 i + 1) / (2 n))."""
    l = np.arange(n)[:, None]
    i = np.arange(n)[None, :]
    return np.cos(math.pi * l * (2 * i + 1) / (2 * n))


def dct3_inverse_matrix(n):
    """Inverse of dct2_matrix: x_i = (X_0 + 2 sum_{l>0} X_l cos(pi l (2 i + 1)/(2 n))) / n."""
    C = dct2_matrix(n).T.copy()
    C[:, 1:] *= 2.0
    return C / n


def poisson_solve_bl(g, rhs):
    """D G phi = rhs with zero normal gradient on all non-periodic boundaries: DCT-II in x,
    DFT in z, tridiagonal in y, inverses; (0, 0) mode gauged by phi_0 = 0."""
    Cx = dct2_matrix(g.nx)
    bh = dft(np.moveaxis(np.moveaxis(rhs, 2, -1) @ Cx.T, -1, 2).astype(np.complex128), 0)
    a, c = poisson_ycoeffs(g)
    lx = (2.0 / (g.dx * g.dx)) * (1.0 - np.cos(math.pi * np.arange(g.nx) / g.nx))
    lz = modified_wavenumbers(g.nz, g.dz)
    lam = lz[:, None] + lx[None, :]
    d = np.moveaxis(bh, 1, -1)
    A = np.broadcast_to(a, d.shape).copy()
    C = np.broadcast_to(c, d.shape).copy()
    B = np.array(np.broadcast_to(-(a + c)[None, None, :] - lam[:, :, None], d.shape))
    B[0, 0, 0] = 1.0
    C[0, 0, 0] = 0.0
    d = d.copy()
    d[0, 0, 0] = 0.0
    ph = np.moveaxis(thomas(A, B, C, d), -1, 1)
    ph = dft(ph, 0, +1) / g.nz
    Ci = dct3_inverse_matrix(g.nx)
    phi = np.moveaxis(np.moveaxis(ph, 2, -1) @ Ci.T, -1, 2)
    return phi.real.copy()


def project_bl(g, u, v, w, phi, scale):
    gx, gy, gz = gradient_bl(g, phi)
    return u - scale * gx, v - scale * gy, w - scale * gz


def make_divergence_free_bl(g, u, v, w, bl):
    """Flux-correct the outflow plane, then project (scale 1)."""
    bl = dict(bl)
    bl["u_out"] = flux_correct_outflow(g, u[:, :, 0], bl["u_out"])
    phi = poisson_solve_bl(g, divergence_bl(g, u, v, w, bl))
    u2, v2, w2 = project_bl(g, u, v, w, phi, 1.0)
    return u2, v2, w2, bl


def substep_bl(g, state, k, dt, re, fx, u_conv=1.0, pressure="delta"):
    """One RK3 sub-step with inflow / convective outflow in x.  Order: RHS (boundary planes of the
    previous level), outflow update, ADI x (outflow increment on the last row) / y / z,
    u* = u + delta, outflow flux correction, Poisson, projection of interior faces, p += phi."""
    u, v, w, p, bl = state["u"], state["v"], state["w"], state["p"], state["bl"]
    r, N = rhs_bl(g, u, v, w, p, state.get("nprev"), bl, k, dt, re, fx)
    scale = RK3_ALPHA[k] * dt
    bl_new, inc = outflow_update(g, u, v, w, bl, scale, u_conv)
    inv_re = 0.0 if not np.isfinite(re) else 1.0 / re
    beta = scale * inv_re / 2.0
    out = []
    for comp, (rc, ic) in enumerate(zip(r, (inc["u_out"], inc["v_out"], inc["w_out"]))):
        x = adi_sweep_x_bl(g, rc, comp, beta, ic)
        x = adi_sweep(g, x, 1, comp, beta)
        x = adi_sweep(g, x, 2, comp, beta)
        out.append(x)
    us, vs, ws = u + out[0], v + out[1], w + out[2]
    bl_new["u_out"] = flux_correct_outflow(g, u[:, :, 0], bl_new["u_out"])
    phi = poisson_solve_bl(g, divergence_bl(g, us, vs, ws, bl_new) / scale)
    un, vn, wn = project_bl(g, us, vs, ws, phi, scale)
    lap = None
    if pressure != "delta":  # D G phi with zero normal gradient at the inflow and outflow faces
        lap = divergence_bl(g, *gradient_bl(g, phi), dict(u_out=np.zeros((g.nz, g.ny))))
    return dict(u=un, v=vn, w=wn, p=pressure_update(p, phi, lap, beta, pressure), nprev=N, phi=phi, bl=bl_new)


def step_bl(g, state, dt, re, fx, nsteps=1, u_conv=1.0, pressure="delta"):
    s = dict(state)
    for _ in range(nsteps):
        for k in range(3):
            s = substep_bl(g, s, k, dt, re, fx, u_conv, pressure)
    return s


# ----------------------------------------------------------------------------
# Recycling inflow (Sec. 2.1: turbulent inflow by the recycling method of Lund, Wu & Squires,
# J. Comput. Phys. 140, 1998), restated from that method's description.
# ----------------------------------------------------------------------------
# Readings (the paper cites the method only):
# * The recycle plane is the u face i_r (1 <= i_r < nx); v and w there are the averages of the
#   centres i_r - 1 and i_r.  Means are spanwise averages of that plane at the current step (no
#   running time average); fluctuations are the plane minus its means.
# * delta_rec: the first y where the recycled mean U reaches 0.99 U_inf (linear between centres;
#   the top centre if never reached).  The friction velocities enter only through their ratio,
#   gamma = u_tau,inl / u_tau,rec = (delta_rec / delta_inl)^(1/8) (the 1/5 power law:
#   delta ~ x^(4/5), u_tau ~ x^(-1/10)).
# * Inlet row at height y takes the recycled profiles at y gamma (inner: same y+) and at
#   y delta_rec / delta_inl (outer: same eta = y / delta), by linear interpolation in y over the
#   plane's points with the wall value (u, w: 0 at y = 0; v: its face values) and the top value
#   held above.  Inner mean U: gamma U_rec; outer: gamma U_rec + (1 - gamma) U_inf; mean V
#   unscaled; mean W = 0; fluctuations times gamma.  Blend (1 - W) inner + W outer with
#   W(eta) = (1 + tanh(a (eta - b) / ((1 - 2b) eta + b)) / tanh a) / 2, a = 4, b = 0.2, W = 1 for
#   eta > 1.
# * The inflow planes (u on face 0, v_in, w_in) are set this way once at the start of every step.
# * Parity unpinned: the blending constant a = 4 (b = 0.2 is pinned through the weight's
#   inflection point); no independent value of a is available.

def lund_weight(eta, a=4.0, b=0.2):
    """Weight W(eta) of the outer profile in the composite inflow of Lund, Wu & Squires
    (J. Comput. Phys. 140, 1998): the tanh weighting function with which their rescaling blends
    the inner and outer profiles, W(b) = 1/2 at eta = b, W = 1 above eta = 1.  a = 4 and b = 0.2
    are the constants given with that function.  Parity unpinned for a (see the section header)."""
    eta = np.asarray(eta, dtype=np.float64)
    wgt = 0.5 * (1.0 + np.tanh(a * (eta - b) / ((1.0 - 2.0 * b) * eta + b)) / math.tanh(a))
    return np.where(eta > 1.0, 1.0, wgt)


def _interp_rows(yq, ys, f):
    """Linear interpolation along axis 1 of f (nz, n) given at ys (increasing), at heights yq;
    values beyond the ends are the end values."""
    out = np.empty((f.shape[0], yq.size))
    for k in range(f.shape[0]):
        out[k] = np.interp(yq, ys, f[k])
    return out


def delta99(yc, U, u_inf=1.0):
    """First height where U reaches 0.99 u_inf (linear between centres); yc[-1] if never."""
    target = 0.99 * u_inf
    for j in range(len(U)):
        if U[j] >= target:
            if j == 0:
                return yc[0] * target / U[0]
            return yc[j - 1] + (target - U[j - 1]) * (yc[j] - yc[j - 1]) / (U[j] - U[j - 1])
    return yc[-1]


def rescale_inflow(g, u_r, v_r, w_r, gamma, delta_rec, delta_inl, u_inf=1.0):
    """Inlet planes from recycle-plane values u_r (nz, ny) at centres, v_r (nz, ny+1) at faces,
    w_r (nz, ny) at centres, given gamma and the two thicknesses."""
    yc, yf = g.yc, g.yf
    # sample points with the wall value: centres plus y = 0 for u, w; faces for v
    ys_c = np.concatenate([[yf[0]], yc])
    U = u_r.mean(axis=0)
    V = v_r.mean(axis=0)
    Wm = w_r.mean(axis=0)
    up = u_r - U[None, :]
    vp = v_r - V[None, :]
    wp = w_r - Wm[None, :]
    def sample_c(f2d, yq):
        z1 = np.zeros((f2d.shape[0], 1))
        return _interp_rows(yq, ys_c, np.concatenate([z1, f2d], axis=1))

    def blend(inner, outer, y):
        wgt = lund_weight(y / delta_inl)[None, :]
        return (1.0 - wgt) * inner + wgt * outer

    r = delta_rec / delta_inl
    # u (centres)
    Ui = gamma * sample_c(U[None, :], gamma * yc)
    Uo = gamma * sample_c(U[None, :], r * yc) + (1.0 - gamma) * u_inf
    ui = gamma * sample_c(up, gamma * yc)
    uo = gamma * sample_c(up, r * yc)
    u_in = blend(Ui + ui, Uo + uo, yc)
    # w (centres; mean W = 0 at the inlet)
    w_in = blend(gamma * sample_c(wp, gamma * yc), gamma * sample_c(wp, r * yc), yc)
    # v (faces, wall and top rows kept at 0)
    Vi = _interp_rows(gamma * yf, yf, V[None, :])
    Vo = _interp_rows(r * yf, yf, V[None, :])
    vi = gamma * _interp_rows(gamma * yf, yf, vp)
    vo = gamma * _interp_rows(r * yf, yf, vp)
    v_in = blend(Vi + vi, Vo + vo, yf)
    v_in[:, 0] = 0.0
    v_in[:, -1] = 0.0
    return u_in, v_in, w_in


def recycle_inflow(g, u, v, w, i_r, delta_inl, re, u_inf=1.0):
    """The inflow planes (u face 0, v_in, w_in) recycled from the u face i_r."""
    u_r = u[:, :, i_r]
    v_r = 0.5 * (v[:, :, i_r - 1] + v[:, :, i_r])
    w_r = 0.5 * (w[:, :, i_r - 1] + w[:, :, i_r])
    U = u_r.mean(axis=0)
    delta_rec = delta99(g.yc, U, u_inf)
    gamma = (delta_rec / delta_inl) ** 0.125
    return rescale_inflow(g, u_r, v_r, w_r, gamma, delta_rec, delta_inl, u_inf)


def step_bl_recycled(g, state, dt, re, fx, i_r, delta_inl, nsteps=1, u_conv=1.0, pressure="delta"):
    """step_bl with the inflow planes recycled from face i_r at the start of every step."""
    s = dict(state)
    for _ in range(nsteps):
        u_in, v_in, w_in = recycle_inflow(g, s["u"], s["v"], s["w"], i_r, delta_inl, re, u_conv)
        u = s["u"].copy()
        u[:, :, 0] = u_in
        bl = dict(s["bl"])
        bl["v_in"] = v_in
        bl["w_in"] = w_in
        s = dict(s, u=u, bl=bl)
        s = step_bl(g, s, dt, re, fx, 1, u_conv, pressure)
    return s
