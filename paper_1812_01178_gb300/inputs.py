"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module holds no arithmetic of the numerical method.  It makes the
inputs the method is run on:

* a counter-based random generator (splitmix64, Steele, Lea & Flood 2014;
  normals by the Box-Muller transform), so any element can be regenerated
  from (seed, index) alone;
* wall-normal grid face coordinates with tanh clustering near the wall(s)
  (the paper's Sec. 2.1 says only that the y grid is clustered near the
  wall, so the stretching function is a chosen input recipe, not a step of
  the method);
* the initial velocity fields of the workloads (laminar channel, turbulent-
  channel-shaped field, boundary-layer-shaped field) and their sizes.

Arrays use the device layout: x fastest, then y, then z, i.e. numpy shape
(nz, ny or ny+1, nx).  u lives on x-faces, v on y-faces (ny+1 rows, rows 0 and
ny are walls), w on z-faces, p at cell centres (Sec. 2.1).  With inflow /
outflow in x, u holds faces 0..nx-1 (face 0 is the inflow) and the outflow face
and the inflow / outflow values of v, w are separate planes.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Return n outputs of splitmix64 for counters offset..offset+n-1."""
    with np.errstate(over="ignore"):
        idx = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of splitmix64."""
    return (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Standard normals by Box-Muller on pairs of uniforms."""
    m = (n + 1) // 2
    u = uniform01(seed, 2 * m, 2 * offset)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    out = np.empty(2 * m)
    out[0::2] = r * np.cos(2.0 * math.pi * u2)
    out[1::2] = r * np.sin(2.0 * math.pi * u2)
    return out[:n]


def normal_range(seed: int, e0: int, n: int) -> np.ndarray:
    """Elements e0 .. e0+n-1 of the sequence normal(seed, N, 0) (any N >= e0 + n), without
    generating the elements before e0: element e uses the uniforms of counters 2(e // 2) and
    2(e // 2) + 1, so a range that starts on an even element is normal(seed, n, e0 / 2)."""
    s = e0 - (e0 % 2)
    return normal(seed, n + (e0 - s), s // 2)[e0 - s:]


# ----------------------------------------------------------------------------
# grids
# ----------------------------------------------------------------------------

def channel_faces(ny: int, beta: float) -> np.ndarray:
    """Face coordinates y_0..y_ny on [-1, 1], clustered at both walls."""
    j = np.arange(ny + 1, dtype=np.float64)
    y = np.tanh(beta * (2.0 * j / ny - 1.0)) / math.tanh(beta)
    y[0], y[-1] = -1.0, 1.0
    return y


def boundary_layer_faces(ny: int, beta: float, ly: float) -> np.ndarray:
    """Face coordinates on [0, ly], clustered at the wall y=0."""
    j = np.arange(ny + 1, dtype=np.float64)
    y = ly * (1.0 + np.tanh(beta * (j / ny - 1.0)) / math.tanh(beta))
    y[0], y[-1] = 0.0, ly
    return y


@dataclass
class Case:
    """One workload: sizes, domain, physics constants and step count."""
    name: str
    nx: int
    ny: int
    nz: int
    lx: float
    lz: float
    yf: np.ndarray = field(repr=False)
    re: float = 1.0
    fx: float = 0.0
    dt: float = 1e-3
    steps: int = 10
    bc_x: int = 0          # 0 periodic, 1 inflow / convective outflow
    bc_ytop: int = 0       # 0 no-slip wall, 1 stress-free
    precision: int = 0     # 0 FP64, 1 mixed
    u_conv: float = 1.0
    pressure_update: int = 0  # 0: p += phi; 1: Kim-Moin form
    recycle_i: int = 0        # u face recycled to the inflow (0: fixed inflow planes)
    delta_in: float = 0.0     # inlet boundary-layer thickness of the recycling

    def cells(self) -> int:
        return self.nx * self.ny * self.nz

    def describe(self) -> dict:
        d = {k: v for k, v in asdict(self).items() if k != "yf"}
        return d


def _centres(yf: np.ndarray) -> np.ndarray:
    return 0.5 * (yf[:-1] + yf[1:])


def laminar_channel(nx=64, ny=64, nz=32, beta=2.0, re_b=2000.0, amp=1e-3,
                    dt=1e-3, steps=10, seed=1812, lx=2 * math.pi, lz=math.pi):
    """Poiseuille profile 1.5(1-y^2) plus uniform noise U(-amp, amp) on u, v, w.

    The body force 3/Re_b holds the laminar profile steady.  Returns
    (case, u, v, w, p); the fields are not yet divergence-free.
    """
    yf = channel_faces(ny, beta)
    case = Case("laminar_channel_%dx%dx%d" % (nx, ny, nz), nx, ny, nz, lx, lz, yf,
                re=re_b, fx=3.0 / re_b, dt=dt, steps=steps)
    yc = _centres(yf)
    n = nx * ny * nz
    u = 1.5 * (1.0 - yc ** 2)[None, :, None] * np.ones((nz, ny, nx))
    u = u + amp * (2.0 * uniform01(seed, n, 0).reshape(nz, ny, nx) - 1.0)
    v = amp * (2.0 * uniform01(seed, nz * (ny + 1) * nx, n).reshape(nz, ny + 1, nx) - 1.0)
    v[:, 0, :] = 0.0
    v[:, ny, :] = 0.0
    w = amp * (2.0 * uniform01(seed, n, n + nz * (ny + 1) * nx).reshape(nz, ny, nx) - 1.0)
    p = np.zeros((nz, ny, nx))
    return case, u, v, w, p


def loglaw_mean(yplus: np.ndarray) -> np.ndarray:
    """Mean velocity U+ = y+ below y+ = 11, else (1/0.41) ln y+ + 5.2."""
    yp = np.maximum(yplus, 1e-300)
    return np.where(yp < 11.0, yp, np.log(yp) / 0.41 + 5.2)


def turbulent_channel(nx=256, ny=192, nz=256, beta=2.0, re_tau=395.0, rms=0.1,
                      cfl=0.5, steps=100, seed=1812, lx=2 * math.pi, lz=math.pi):
    """Log-law mean in wall units plus Gaussian fluctuations (10 % of the local mean).

    Units: u_tau = 1, half-height 1, so Re = re_tau and the driving body
    force is 1.  dt is fixed from the CFL number on the initial field.
    Returns (case, u, v, w, p); the fields are not yet divergence-free.
    """
    yf = channel_faces(ny, beta)
    yc = _centres(yf)
    yplus_c = (1.0 - np.abs(yc)) * re_tau
    umean = loglaw_mean(yplus_c)
    n = nx * ny * nz
    sig = rms * umean
    u = umean[None, :, None] + sig[None, :, None] * normal(seed, n, 0).reshape(nz, ny, nx)
    yplus_f = (1.0 - np.abs(yf)) * re_tau
    sig_f = rms * loglaw_mean(yplus_f)
    v = sig_f[None, :, None] * normal(seed + 1, nz * (ny + 1) * nx, 0).reshape(nz, ny + 1, nx)
    v[:, 0, :] = 0.0
    v[:, ny, :] = 0.0
    w = sig[None, :, None] * normal(seed + 2, n, 0).reshape(nz, ny, nx)
    p = np.zeros((nz, ny, nx))
    dx, dz = lx / nx, lz / nz
    dy = np.diff(yf)
    c = (np.abs(u) / dx + np.abs(0.5 * (v[:, :-1] + v[:, 1:])) / dy[None, :, None]
         + np.abs(w) / dz)
    dt = cfl / float(c.max())
    case = Case("turbulent_channel_%dx%dx%d" % (nx, ny, nz), nx, ny, nz, lx, lz, yf,
                re=re_tau, fx=1.0, dt=dt, steps=steps)
    return case, u, v, w, p


def field_shapes(case: Case):
    """numpy shapes of u, v, w, p for a case (x fastest, then y, then z)."""
    return ((case.nz, case.ny, case.nx), (case.nz, case.ny + 1, case.nx),
            (case.nz, case.ny, case.nx), (case.nz, case.ny, case.nx))


def small_channel(nx, ny, nz, seed=7, amp=0.1, re=100.0, dt=2e-3, beta=1.5,
                  lx=2 * math.pi, lz=math.pi):
    """Small channel with O(amp) random fields, for parity cases of any size."""
    yf = channel_faces(ny, beta)
    case = Case("channel_%dx%dx%d" % (nx, ny, nz), nx, ny, nz, lx, lz, yf,
                re=re, fx=3.0 / re, dt=dt, steps=2)
    yc = _centres(yf)
    n = nx * ny * nz
    u = 1.5 * (1.0 - yc ** 2)[None, :, None] + amp * normal(seed, n, 0).reshape(nz, ny, nx)
    v = amp * normal(seed + 1, nz * (ny + 1) * nx, 0).reshape(nz, ny + 1, nx)
    v[:, 0, :] = 0.0
    v[:, ny, :] = 0.0
    w = amp * normal(seed + 2, n, 0).reshape(nz, ny, nx)
    p = amp * normal(seed + 3, n, 0).reshape(nz, ny, nx)
    return case, u, v, w, p


def boundary_layer_case(nx=1024, ny=256, nz=512, beta=2.0, re=1000.0, steps=50, lx=None, ly=None, lz=None,
                        precision=0):
    """The boundary-layer workload's sizes and constants (dt is set from the initial field by
    boundary_layer / boundary_layer_dt).  Units: inlet thickness and free-stream speed; domain
    Lx = 200, Ly = 20, Lz = 30 by default (scaled down for small grids)."""
    lx = lx if lx is not None else (200.0 if nx >= 256 else 0.2 * nx)
    ly = ly if ly is not None else (20.0 if ny >= 64 else 0.3 * ny)
    lz = lz if lz is not None else (30.0 if nz >= 128 else 0.25 * nz)
    yf = boundary_layer_faces(ny, beta, ly)
    return Case("boundary_layer_%dx%dx%d" % (nx, ny, nz), nx, ny, nz, lx, lz, yf, re=re, fx=0.0,
                steps=steps, bc_x=1, bc_ytop=1, precision=precision, u_conv=1.0)


def boundary_layer_slab(case: Case, k0: int, k1: int, amp=1e-2, seed=1812):
    """Planes k0 <= k < k1 of the boundary-layer initial field: (u, v, w, bl) with u, v, w of shape
    (k1-k0, ny or ny+1, nx) and the boundary planes of those rows.  The planes are exactly those
    of the whole field (every value comes from its own counter), so a field can be built slab by
    slab with little host memory."""
    nx, ny = case.nx, case.ny
    nk = k1 - k0
    prof = np.tanh(2.0 * _centres(case.yf))
    u = prof[None, :, None] + amp * normal_range(seed, k0 * ny * nx, nk * ny * nx).reshape(nk, ny, nx)
    v = amp * normal_range(seed + 1, k0 * (ny + 1) * nx, nk * (ny + 1) * nx).reshape(nk, ny + 1, nx)
    v[:, 0, :] = 0.0
    v[:, ny, :] = 0.0
    w = amp * normal_range(seed + 2, k0 * ny * nx, nk * ny * nx).reshape(nk, ny, nx)
    # inflow planes (face 0 of u; v, w on the inflow face), fixed in time
    u[:, :, 0] = prof[None, :] + amp * normal_range(seed + 3, k0 * ny, nk * ny).reshape(nk, ny)
    v_in = amp * normal_range(seed + 4, k0 * (ny + 1), nk * (ny + 1)).reshape(nk, ny + 1)
    v_in[:, 0] = 0.0
    v_in[:, ny] = 0.0
    w_in = amp * normal_range(seed + 5, k0 * ny, nk * ny).reshape(nk, ny)
    bl = dict(u_out=u[:, :, -1].copy(), v_in=v_in, v_out=v[:, :, -1].copy(), w_in=w_in, w_out=w[:, :, -1].copy())
    return u, v, w, bl


def boundary_layer_rate(case: Case, u, v, w) -> float:
    """max |u|/dx + |v_c|/dy + |w|/dz of (a slab of) the initial field: the CFL recipe of dt."""
    dx, dz = case.lx / case.nx, case.lz / case.nz
    dy = np.diff(case.yf)
    c = np.abs(u) / dx + np.abs(0.5 * (v[:, :-1] + v[:, 1:])) / dy[None, :, None] + np.abs(w) / dz
    return float(c.max())


def boundary_layer(nx=1024, ny=256, nz=512, beta=2.0, re=1000.0, amp=1e-2, cfl=0.5, steps=50, seed=1812,
                   lx=None, ly=None, lz=None, precision=0):
    """Boundary-layer-shaped field with inflow / convective outflow in x.

    Units: inlet thickness and free-stream speed.  Domain Lx = 200, Ly = 20, Lz = 30 by default
    (scaled down for small grids).  Inflow u = tanh(2 y) plus seeded perturbations of amplitude
    amp on u, v, w (time-invariant); the interior starts from the same profile plus its own
    perturbations; the outflow planes start as the last interior column.  No-slip wall at y = 0,
    stress-free top, periodic z, U_c = 1.  dt from the CFL number on the initial field.  Returns
    (case, u, v, w, p, bl) with u holding faces 0..nx-1 (face 0 = inflow) and bl the boundary
    planes u_out, v_in, v_out, w_in, w_out.
    """
    case = boundary_layer_case(nx, ny, nz, beta, re, steps, lx, ly, lz, precision)
    u, v, w, bl = boundary_layer_slab(case, 0, nz, amp, seed)
    p = np.zeros((nz, ny, nx))
    case.dt = cfl / boundary_layer_rate(case, u, v, w)
    return case, u, v, w, p, bl


def ensemble(n=64, seed=1812, amp=1e-3, steps=10, sizes_x=(32, 64, 128), sizes_y=(32, 48, 64, 96),
             re_range=(1000.0, 5000.0), beta=2.0, dt=2e-3):
    """Uneven laminar-channel instances (32x32x32 up to 128x96x128): instance i draws nx, nz from
    sizes_x, ny from sizes_y and Re_b uniformly from re_range with seed + i.  Returns a list of
    (case, u, v, w, p)."""
    out = []
    for i in range(n):
        r = uniform01(seed + i, 4)
        nx = sizes_x[int(r[0] * len(sizes_x))]
        nz = sizes_x[int(r[1] * len(sizes_x))]
        ny = sizes_y[int(r[2] * len(sizes_y))]
        re_b = re_range[0] + (re_range[1] - re_range[0]) * float(r[3])
        case, u, v, w, p = laminar_channel(nx, ny, nz, beta=beta, re_b=re_b, amp=amp, dt=dt, steps=steps,
                                           seed=seed + 1000 + i)
        case.name = "ensemble_%d_%dx%dx%d" % (i, nx, ny, nz)
        out.append((case, u, v, w, p))
    return out
