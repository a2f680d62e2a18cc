// Explicit right-hand side of one RK3 sub-step (Sec. 2.2, delta form):
//   r_i = dt [ -gamma_k N_i(u) - zeta_k N_prev_i - alpha_k G_i p + (alpha_k / Re) L u_i + alpha_k f_i ]
// N is the divergence-form convection of Eq. (NSmomentum) with 2nd-order central differences on
// the staggered grid: fluxes at faces / edges from arithmetic averages in x and z and
// distance-weighted linear interpolation in y.  L is the viscous operator (uniform second
// differences in x and z, the three-point non-uniform formula in y).  G is the pressure gradient.
//
// One thread per (i, j) of one z-plane, j = 0..ny (row ny only writes the v wall row).  T is the
// arithmetic type (double, or float for the mixed form), TR the storage type of r and N.
#include "ns_internal.cuh"

namespace {

struct RhsArgs {
  const double* __restrict__ u;
  const double* __restrict__ v;
  const double* __restrict__ w;
  const double* __restrict__ p;
  void* ru;
  void* rv;
  void* rw;
  void* nu;
  void* nv;
  void* nw;
  const double* __restrict__ gc;
  int nx, ny, nz;
  double idx, idz, idx2, idz2;
  double dt, gam, zet, alp, inv_re, fx;
};

template <typename T, typename TR>
__global__ void __launch_bounds__(128) rhs_kernel(RhsArgs a) {
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const long plane = (long)nx * (ny + 1);
  const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= plane) return;
  const int j = (int)(q / nx);
  const int i = (int)(q - (long)j * nx);
  const int k = blockIdx.y;
  const int ip = (i + 1 == nx) ? 0 : i + 1;
  const int im = (i == 0) ? nx - 1 : i - 1;
  const int kp = (k + 1 == nz) ? 0 : k + 1;
  const int km = (k == 0) ? nz - 1 : k - 1;
  const int ny1 = ny + 1;
  const int G = ny + 1;  // stride of the coefficient arrays

  auto U = [&](int ii, int jj, int kk) -> T { return (T)__ldg(a.u + ((long)kk * ny + jj) * nx + ii); };
  auto V = [&](int ii, int jj, int kk) -> T { return (T)__ldg(a.v + ((long)kk * ny1 + jj) * nx + ii); };
  auto W = [&](int ii, int jj, int kk) -> T { return (T)__ldg(a.w + ((long)kk * ny + jj) * nx + ii); };
  auto Pp = [&](int ii, int jj, int kk) -> T { return (T)__ldg(a.p + ((long)kk * ny + jj) * nx + ii); };
  auto C = [&](int f, int jj) -> T { return (T)__ldg(a.gc + f * G + jj); };

  const T idx = (T)a.idx, idz = (T)a.idz, idx2 = (T)a.idx2, idz2 = (T)a.idz2;
  const T dt = (T)a.dt, gam = (T)a.gam, zet = (T)a.zet, alp = (T)a.alp;
  const T avis = (T)(a.alp * a.inv_re);
  const T half = (T)0.5, quarter = (T)0.25, two = (T)2;

  TR* ru = (TR*)a.ru;
  TR* rv = (TR*)a.rv;
  TR* rw = (TR*)a.rw;
  TR* nu = (TR*)a.nu;
  TR* nv = (TR*)a.nv;
  TR* nw = (TR*)a.nw;

  if (j < ny) {
    const long cc = ((long)k * ny + j) * nx + i;
    const T idy = C(GC_IDY, j);
    // ---------------- u at (xf_i, yc_j, zc_k)
    {
      const T u0 = U(i, j, k), uxp = U(ip, j, k), uxm = U(im, j, k);
      const T uzp = U(i, j, kp), uzm = U(i, j, km);
      const T uyp = (j + 1 < ny) ? U(i, j + 1, k) : (T)0;
      const T uym = (j > 0) ? U(i, j - 1, k) : (T)0;
      const T sr = u0 + uxp, sl = uxm + u0;
      const T nux = (sr * sr - sl * sl) * (quarter * idx);
      T ft = 0, fb = 0;
      if (j + 1 < ny) {
        const T ut = C(GC_WLO, j + 1) * u0 + C(GC_WHI, j + 1) * uyp;
        ft = ut * (V(im, j + 1, k) + V(i, j + 1, k));
      }
      if (j > 0) {
        const T ub = C(GC_WLO, j) * uym + C(GC_WHI, j) * u0;
        fb = ub * (V(im, j, k) + V(i, j, k));
      }
      const T nuy = (ft - fb) * (half * idy);
      const T nuz = ((u0 + uzp) * (W(im, j, kp) + W(i, j, kp)) - (uzm + u0) * (W(im, j, k) + W(i, j, k))) *
                    (quarter * idz);
      const T n = nux + nuy + nuz;
      const T ac = C(GC_AC, j), cy = C(GC_CC, j);
      const T lap = (uxp - two * u0 + uxm) * idx2 + (uzp - two * u0 + uzm) * idz2 + ac * uym -
                    (ac + cy) * u0 + cy * uyp;
      const T gp = (Pp(i, j, k) - Pp(im, j, k)) * idx;
      T r = -gam * n - alp * gp + avis * lap + (T)(a.alp * a.fx);
      if (a.zet != 0.0) r -= zet * (T)nu[cc];
      ru[cc] = (TR)(dt * r);
      nu[cc] = (TR)n;
    }
    // ---------------- w at (xc_i, yc_j, zf_k)
    {
      const T w0 = W(i, j, k), wxp = W(ip, j, k), wxm = W(im, j, k);
      const T wzp = W(i, j, kp), wzm = W(i, j, km);
      const T wyp = (j + 1 < ny) ? W(i, j + 1, k) : (T)0;
      const T wym = (j > 0) ? W(i, j - 1, k) : (T)0;
      const T fr = (U(ip, j, km) + U(ip, j, k)) * (w0 + wxp);
      const T fl = (U(i, j, km) + U(i, j, k)) * (wxm + w0);
      const T nwx = (fr - fl) * (quarter * idx);
      T gt = 0, gb = 0;
      if (j + 1 < ny) gt = (V(i, j + 1, km) + V(i, j + 1, k)) * (C(GC_WLO, j + 1) * w0 + C(GC_WHI, j + 1) * wyp);
      if (j > 0) gb = (V(i, j, km) + V(i, j, k)) * (C(GC_WLO, j) * wym + C(GC_WHI, j) * w0);
      const T nwy = (gt - gb) * (half * idy);
      const T cf = w0 + wzp, cb = wzm + w0;
      const T nwz = (cf * cf - cb * cb) * (quarter * idz);
      const T n = nwx + nwy + nwz;
      const T ac = C(GC_AC, j), cy = C(GC_CC, j);
      const T lap = (wxp - two * w0 + wxm) * idx2 + (wzp - two * w0 + wzm) * idz2 + ac * wym -
                    (ac + cy) * w0 + cy * wyp;
      const T gp = (Pp(i, j, k) - Pp(i, j, km)) * idz;
      T r = -gam * n - alp * gp + avis * lap;
      if (a.zet != 0.0) r -= zet * (T)nw[cc];
      rw[cc] = (TR)(dt * r);
      nw[cc] = (TR)n;
    }
  }
  // ---------------- v at (xc_i, yf_j, zc_k)
  {
    const long cf = ((long)k * ny1 + j) * nx + i;
    if (j == 0 || j == ny) {
      rv[cf] = (TR)0;
      nv[cf] = (TR)0;
      return;
    }
    const T v0 = V(i, j, k), vxp = V(ip, j, k), vxm = V(im, j, k);
    const T vzp = V(i, j, kp), vzm = V(i, j, km);
    const T vyp = V(i, j + 1, k), vym = V(i, j - 1, k);
    const T wl = C(GC_WLO, j), wh = C(GC_WHI, j);
    const T fr = (wl * U(ip, j - 1, k) + wh * U(ip, j, k)) * (v0 + vxp);
    const T fl = (wl * U(i, j - 1, k) + wh * U(i, j, k)) * (vxm + v0);
    const T nvx = (fr - fl) * (half * idx);
    const T ct = v0 + vyp, cb = vym + v0;
    const T ihc = C(GC_IHC, j);
    const T nvy = (ct * ct - cb * cb) * (quarter * ihc);
    const T gf = (v0 + vzp) * (wl * W(i, j - 1, kp) + wh * W(i, j, kp));
    const T gb = (vzm + v0) * (wl * W(i, j - 1, k) + wh * W(i, j, k));
    const T nvz = (gf - gb) * (half * idz);
    const T n = nvx + nvy + nvz;
    const T af = C(GC_AF, j), cyf = C(GC_CF, j);
    const T lap = (vxp - two * v0 + vxm) * idx2 + (vzp - two * v0 + vzm) * idz2 + af * vym -
                  (af + cyf) * v0 + cyf * vyp;
    const T gp = (Pp(i, j, k) - Pp(i, j - 1, k)) * ihc;
    T r = -gam * n - alp * gp + avis * lap;
    if (a.zet != 0.0) r -= zet * (T)nv[cf];
    rv[cf] = (TR)(dt * r);
    nv[cf] = (TR)n;
  }
}

}  // namespace

cudaError_t launch_rhs(ns_ctx* c, int k) {
  RhsArgs a;
  a.u = c->f.u;
  a.v = c->f.v;
  a.w = c->f.w;
  a.p = c->f.p;
  a.ru = c->ru;
  a.rv = c->rv;
  a.rw = c->rw;
  a.nu = c->nu;
  a.nv = c->nv;
  a.nw = c->nw;
  a.gc = c->gc;
  a.nx = c->cfg.nx;
  a.ny = c->cfg.ny;
  a.nz = c->cfg.nz;
  a.idx = 1.0 / c->dx;
  a.idz = 1.0 / c->dz;
  a.idx2 = a.idx * a.idx;
  a.idz2 = a.idz * a.idz;
  a.dt = c->cfg.dt;
  a.gam = NS_GAMMA[k];
  a.zet = NS_ZETA[k];
  a.alp = NS_ALPHA[k];
  a.inv_re = c->cfg.re > 0 ? 1.0 / c->cfg.re : 0.0;
  a.fx = c->cfg.fx;
  const long plane = (long)a.nx * (a.ny + 1);
  dim3 grid((unsigned)((plane + 127) / 128), (unsigned)a.nz);
  if (c->cfg.precision == NS_MIXED)
    rhs_kernel<float, float><<<grid, 128, 0, c->launch>>>(a);
  else
    rhs_kernel<double, double><<<grid, 128, 0, c->launch>>>(a);
  return cudaGetLastError();
}
