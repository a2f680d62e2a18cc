// Explicit right-hand side of one RK3 sub-step (Sec. 2.2, delta form):
//   r_i = dt [ -gamma_k N_i(u) - zeta_k N_prev_i - alpha_k G_i p + (alpha_k / Re) L u_i + alpha_k f_i ]
// N is the divergence-form convection of Eq. (NSmomentum) with 2nd-order central differences on
// the staggered grid: fluxes at faces / edges from arithmetic averages in x and z and
// distance-weighted linear interpolation in y.  L is the viscous operator (uniform second
// differences in x and z, the three-point non-uniform formula in y).  G is the pressure gradient.
//
// rhs_kernel: one thread per (i, j) of one z-plane, j = 0..ny (row ny only writes the v wall row),
// used when nx is not a multiple of 32 or nz not a multiple of 8; rhs_tiled_kernel otherwise.
// T is the arithmetic type (double, or float for the mixed form), TR the storage type of r and N.
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
  const double* __restrict__ rt;  // per-j assembly coefficients of this sub-step (RT_* rows)
  const float* __restrict__ rtf;  // the same rows in float (read by the FP32 form)
  // inflow / outflow in x (bl = 1): boundary planes, index k * rows + j
  int bl;
  const double* __restrict__ u_out;
  const double* __restrict__ v_in;
  const double* __restrict__ v_out;
  const double* __restrict__ w_in;
  const double* __restrict__ w_out;
  int nx, ny, nz;
  double idx, idz, idx2, idz2;
  double dt, gam, zet, alp, inv_re, fx;
  double cprev;     // zeta_k / gamma_(k-1): weight of the stored (pre-multiplied) N of sub-step k-1
  const StepK* sk;  // dt-dependent constants of this sub-step (device; read by the Dyn variants)
  StepK kc;         // the same values as kernel arguments (read by the fixed-dt variants)
};

}  // namespace

namespace {

// Dyn: the sub-step constants are read from device memory (a step graph that outlives changes of
// dt); otherwise from the kernel arguments, where they cost no registers.
template <typename T, typename TR, bool Dyn>
struct RhsK {
  struct Args {
    RhsArgs a;
  };
  static constexpr int kThreads = 128;
  static constexpr int kMinBlocks = 7;
  static Args make(RhsArgs a) { return Args{a}; }
  static __device__ __forceinline__ void run(const Args& a_, const dim3 bid_, const dim3 gdim_) {
    const RhsArgs& a = a_.a;

  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const long plane = (long)nx * (ny + 1);
  const long q = (long)bid_.x * blockDim.x + threadIdx.x;
  if (q >= plane) return;
  const int j = (int)(q / nx);
  const int i = (int)(q - (long)j * nx);
  const int k = bid_.y;
  const int ip = (i + 1 == nx) ? 0 : i + 1;
  const int im = (i == 0) ? nx - 1 : i - 1;
  const int kp = (k + 1 == nz) ? 0 : k + 1;
  const int km = (k == 0) ? nz - 1 : k - 1;
  const int ny1 = ny + 1;
  const int G = ny + 1;  // stride of the coefficient arrays

  // x-neighbours: periodic wrap, or (bl) the outflow plane / linear ghosts of the boundary faces
  const bool bl = a.bl != 0;
  const int ipx = bl ? i + 1 : ip, imx = bl ? i - 1 : im;
  auto U = [&](int ii, int jj, int kk) -> T {
    if (ii == nx) return from_double<T>(__ldg(a.u_out + (long)kk * ny + jj));
    if (ii < 0) return (T)0;
    return from_double<T>(__ldg(a.u + ((long)kk * ny + jj) * nx + ii));
  };
  auto V = [&](int ii, int jj, int kk) -> T {
    if (ii == nx) return from_double<T>(2.0 * __ldg(a.v_out + (long)kk * ny1 + jj) - __ldg(a.v + ((long)kk * ny1 + jj) * nx + nx - 1));
    if (ii < 0) return from_double<T>(2.0 * __ldg(a.v_in + (long)kk * ny1 + jj) - __ldg(a.v + ((long)kk * ny1 + jj) * nx));
    return from_double<T>(__ldg(a.v + ((long)kk * ny1 + jj) * nx + ii));
  };
  auto W = [&](int ii, int jj, int kk) -> T {
    if (ii == nx) return from_double<T>(2.0 * __ldg(a.w_out + (long)kk * ny + jj) - __ldg(a.w + ((long)kk * ny + jj) * nx + nx - 1));
    if (ii < 0) return from_double<T>(2.0 * __ldg(a.w_in + (long)kk * ny + jj) - __ldg(a.w + ((long)kk * ny + jj) * nx));
    return from_double<T>(__ldg(a.w + ((long)kk * ny + jj) * nx + ii));
  };
  auto Pp = [&](int ii, int jj, int kk) -> T {
    if (ii < 0 || ii == nx) return (T)0;
    return from_double<T>(__ldg(a.p + ((long)kk * ny + jj) * nx + ii));
  };
  auto C = [&](int f, int jj) -> T { return from_double<T>(__ldg(a.gc + f * G + jj)); };

  const T idx = (T)a.idx, idz = (T)a.idz, idx2 = (T)a.idx2, idz2 = (T)a.idz2;
  const T dt = (T)(Dyn ? a.sk->dt : a.kc.dt), alp = (T)a.alp;
  const T avis = (T)(a.alp * a.inv_re);
  // N is stored pre-multiplied by cn = -dt gamma_k, as in the tiled form; the stored N of the
  // previous sub-step enters with zeta_k / gamma_(k-1)
  const T cn = -dt * (T)a.gam, cpn = (T)a.cprev;
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
      const T u0 = U(i, j, k), uxp = U(ipx, j, k), uxm = U(imx, j, k);
      const T uzp = U(i, j, kp), uzm = U(i, j, km);
      const T uyp = (j + 1 < ny) ? U(i, j + 1, k) : (T)0;
      const T uym = (j > 0) ? U(i, j - 1, k) : (T)0;
      const T sr = u0 + uxp, sl = uxm + u0;
      const T nux = (sr * sr - sl * sl) * (quarter * idx);
      T ft = 0, fb = 0;
      if (j + 1 < ny) {
        const T ut = C(GC_WLO, j + 1) * u0 + C(GC_WHI, j + 1) * uyp;
        ft = ut * (V(imx, j + 1, k) + V(i, j + 1, k));
      }
      if (j > 0) {
        const T ub = C(GC_WLO, j) * uym + C(GC_WHI, j) * u0;
        fb = ub * (V(imx, j, k) + V(i, j, k));
      }
      const T nuy = (ft - fb) * (half * idy);
      const T nuz = ((u0 + uzp) * (W(imx, j, kp) + W(i, j, kp)) - (uzm + u0) * (W(imx, j, k) + W(i, j, k))) *
                    (quarter * idz);
      const T n = nux + nuy + nuz;
      const T ac = C(GC_AC, j), cy = C(GC_CC, j);
      const T lap = (uxp - two * u0 + uxm) * idx2 + (uzp - two * u0 + uzm) * idz2 + ac * uym -
                    (ac + cy) * u0 + cy * uyp;
      const T gp = (Pp(i, j, k) - Pp(imx, j, k)) * idx;
      const T nt = cn * n;
      T r = dt * (-alp * gp + avis * lap + (T)(a.alp * a.fx)) + nt;
      if (a.zet != 0.0) r += cpn * (T)nu[cc];
      const bool fixed = bl && i == 0;  // inflow face
      ru[cc] = fixed ? (TR)0 : (TR)r;
      nu[cc] = fixed ? (TR)0 : (TR)nt;
    }
    // ---------------- w at (xc_i, yc_j, zf_k)
    {
      const T w0 = W(i, j, k), wxp = W(ipx, j, k), wxm = W(imx, j, k);
      const T wzp = W(i, j, kp), wzm = W(i, j, km);
      const T wyp = (j + 1 < ny) ? W(i, j + 1, k) : (T)0;
      const T wym = (j > 0) ? W(i, j - 1, k) : (T)0;
      const T fr = (U(ipx, j, km) + U(ipx, j, k)) * (w0 + wxp);
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
      const T nt = cn * n;
      T r = dt * (-alp * gp + avis * lap) + nt;
      if (a.zet != 0.0) r += cpn * (T)nw[cc];
      rw[cc] = (TR)r;
      nw[cc] = (TR)nt;
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
    const T v0 = V(i, j, k), vxp = V(ipx, j, k), vxm = V(imx, j, k);
    const T vzp = V(i, j, kp), vzm = V(i, j, km);
    const T vyp = V(i, j + 1, k), vym = V(i, j - 1, k);
    const T wl = C(GC_WLO, j), wh = C(GC_WHI, j);
    const T fr = (wl * U(ipx, j - 1, k) + wh * U(ipx, j, k)) * (v0 + vxp);
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
    const T nt = cn * n;
    T r = dt * (-alp * gp + avis * lap) + nt;
    if (a.zet != 0.0) r += cpn * (T)nv[cf];
    rv[cf] = (TR)r;
    nv[cf] = (TR)nt;
  }

  }
};

// ---------------------------------------------------------------------------------------------
// Tiled form of the same right-hand side.  A block of TX x TZ threads owns a TX (x) by TZ (z)
// column of cells and marches along y over [jb, je).  Four rolling planes of u, v, w, p (with a
// one-cell halo in x and z, periodic wrap) sit in shared memory.  Every product the
// divergence-form convection needs is computed once per tile and then differenced:
//   centre squares  Q1 = (u_i + u_{i+1})^2, Q2 = (v_j + v_{j+1})^2, Q3 = (w_k + w_{k+1})^2
//   edge fluxes     Fuv = u(yf_j) (v_{i-1} + v_i)       at (xf_i, yf_j)
//                   Fuw = (u_{k-1} + u_k)(w_{i-1} + w_i) at (xf_i, zf_k)
//                   Fvw = (v_{k-1} + v_k) w(yf_j)       at (yf_j, zf_k)
// (factors 1/2, 1/4 of the averages are folded into the difference weights).  y-face fluxes of
// face j+1 become those of face j in the next step; Q2 of centre j is kept in a register.
// ---------------------------------------------------------------------------------------------
constexpr int RT_X = 32;
constexpr int RT_Z = 8;
constexpr int RT_PX = RT_X + 2;   // plane pitch (x halo on both sides)
constexpr int RT_PZ = RT_Z + 2;
constexpr int RT_PLANE = RT_PX * RT_PZ;
constexpr int RT_NPL = 4;         // rolling planes per field

template <typename T>
struct RhsTile {
  T pl[4][RT_NPL][RT_PLANE];                 // u, v, w, p planes (j mod 4), index (kk+1)*RT_PX + (ii+1)
  T fuv[2][RT_Z][RT_X + 1];                  // Fuv on y-face (parity), x = i0 .. i0+TX
  T fvw[2][RT_Z + 1][RT_X];                  // Fvw on y-face (parity), z = k0 .. k0+TZ
  T q1[RT_Z][RT_X + 1];                      // x = i0-1 .. i0+TX-1
  T q3[RT_Z + 1][RT_X];                      // z = k0-1 .. k0+TZ-1
  T fuw[RT_Z + 1][RT_X + 1];                 // x = i0 .. i0+TX, z = k0 .. k0+TZ
  T rt[RT_NPL][RT_COUNT];                    // per-row assembly coefficients of row j (j mod 4)
  T wf[RT_NPL];                              // RHO = WHI / WLO of face j (j mod 4), zero at the walls
};

// State values entering the FP32 tile: the hardware conversion (one instruction on the FP64
// pipe, which the FP32 RHS leaves idle) instead of the integer-pipe d2f_rn (about a dozen
// instructions on the issue-bound FP32 RHS).
template <typename T>
__device__ __forceinline__ T plane_cvt(double x) {
  if constexpr (sizeof(T) == 4) return __double2float_rn(x);
  else return x;
}

// 8-byte global -> shared copy that completes asynchronously (cp.async, waited for by
// cp.async.wait_all); with valid false nothing is read and the 8 bytes are zero-filled
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem, bool valid) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(gmem), "r"(valid ? 8 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit8() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all8() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <typename T, typename TR, bool Dyn>
struct RhsTiledK {
  struct Args {
    RhsArgs a;
    int jchunk;
  };
  static constexpr int kThreads = RT_X * RT_Z;
  // FP64: shared memory allows 3 resident blocks, so up to 85 registers cost nothing.  FP32: 6
  // blocks of up to 40 registers (the kernel waits on memory and shared memory, so occupancy pays
  // more than registers: 0.314 ms at 6 blocks against 0.338 at 5, 0.352 at 4 and 0.434 at 3), or 4
  // of up to 64 when the sub-step constants come from device memory (fewer spill)
  static constexpr int kMinBlocks = sizeof(T) == 8 ? 3 : (Dyn ? 4 : 6);
  static Args make(RhsArgs a, int jchunk) { return Args{a, jchunk}; }
  static __device__ __forceinline__ void run(const Args& a_, const dim3 bid_, const dim3 gdim_) {
    const RhsArgs& a = a_.a;
    const int i0 = bid_.x * RT_X, k0 = bid_.y * RT_Z;
    const int jb = bid_.z * a_.jchunk;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  RhsTile<T>& S = *reinterpret_cast<RhsTile<T>*>(smem_raw);
  const int nx = a.nx, ny = a.ny, nz = a.nz, ny1 = ny + 1, G = ny + 1;
  const int tx = threadIdx.x, tz = threadIdx.y, tid = tz * RT_X + tx;
  const int je = min(jb + a_.jchunk, ny);
  const int jlast = (je == ny) ? ny : je - 1;  // v rows: the last chunk also writes face ny

  auto P = [&](int f, int j, int kk, int ii) -> T& { return S.pl[f][j & 3][(kk + 1) * RT_PX + ii + 1]; };

  // Plane loads.  Each thread owns up to two positions of the (RT_PZ x RT_PX) halo plane and
  // loads all four fields there, so the index arithmetic (wrap, offsets) is done once per thread
  // and only j changes between planes.  u, w, p share the offset of a centre; v has its own.
  // Positions on the x boundary of an inflow / outflow domain take the boundary planes instead.
  constexpr int kPos = (RT_PLANE + RT_X * RT_Z - 1) / (RT_X * RT_Z);
  long oc[kPos], ov[kPos];
  int pos[kPos];  // plane index e, -1 if unused, or -(e + 2) for an x-boundary halo position
#pragma unroll
  for (int r = 0; r < kPos; ++r) {
    const int e = tid + r * RT_X * RT_Z;
    pos[r] = -1;
    oc[r] = 0;
    ov[r] = 0;
    if (e < RT_PLANE) {
      const int kk = e / RT_PX - 1, ii = e % RT_PX - 1;
      int gi = i0 + ii, gk = k0 + kk;
      gk = gk < 0 ? gk + nz : (gk >= nz ? gk - nz : gk);
      if (a.bl && (gi < 0 || gi >= nx)) {
        pos[r] = -(e + 2);
        oc[r] = gk;
      } else {
        gi = gi < 0 ? gi + nx : (gi >= nx ? gi - nx : gi);
        pos[r] = e;
        oc[r] = (long)gk * ny * nx + gi;
        ov[r] = (long)gk * ny1 * nx + gi;
      }
    }
  }
  // FP64: planes are copied global -> shared by cp.async one step ahead (plane j + 2 is issued in
  // step j, after the barrier that ends every read of plane j - 2 in its buffer, and waited for in
  // step j + 1), so that no block stalls on its own plane loads; x-boundary halo positions are
  // formed by plain loads.  FP32 converts on the way and loads through registers.
  constexpr bool kAsync = sizeof(T) == 8;
  auto load_plane = [&](int j) {
    const bool jc = j >= 0 && j < ny, jv = j >= 0 && j <= ny;
    const long jo = (long)j * nx;
#pragma unroll
    for (int r = 0; r < kPos; ++r) {
      if (kAsync && pos[r] >= 0) {
        const int e = pos[r];
        const long o = oc[r] + jo, q = ov[r] + jo;
        cp_async8(&S.pl[0][j & 3][e], a.u + (jc ? o : 0), jc);
        cp_async8(&S.pl[1][j & 3][e], a.v + (jv ? q : 0), jv);
        cp_async8(&S.pl[2][j & 3][e], a.w + (jc ? o : 0), jc);
        cp_async8(&S.pl[3][j & 3][e], a.p + (jc ? o : 0), jc);
      } else if (pos[r] >= 0) {
        const int e = pos[r];
        const long o = oc[r] + jo, q = ov[r] + jo;
        T vu = (T)0, vv = (T)0, vw = (T)0, vp = (T)0;
        if (jc) {
          vu = plane_cvt<T>(__ldg(a.u + o));
          vw = plane_cvt<T>(__ldg(a.w + o));
          vp = plane_cvt<T>(__ldg(a.p + o));
        }
        if (jv) vv = plane_cvt<T>(__ldg(a.v + q));
        S.pl[0][j & 3][e] = vu;
        S.pl[1][j & 3][e] = vv;
        S.pl[2][j & 3][e] = vw;
        S.pl[3][j & 3][e] = vp;
      } else if (pos[r] < -1) {
        // x-boundary halo: outflow plane of u, linear ghosts of v and w, nothing for p
        const int e = -pos[r] - 2;
        const int gk = (int)oc[r];
        const bool out = i0 + e % RT_PX - 1 >= nx;
        T vu = (T)0, vv = (T)0, vw = (T)0;
        if (out && jc) vu = from_double<T>(__ldg(a.u_out + (long)gk * ny + j));
        if (jv) {
          const double b = __ldg((out ? a.v_out : a.v_in) + (long)gk * ny1 + j);
          vv = from_double<T>(2.0 * b - __ldg(a.v + ((long)gk * ny1 + j) * nx + (out ? nx - 1 : 0)));
        }
        if (jc) {
          const double b = __ldg((out ? a.w_out : a.w_in) + (long)gk * ny + j);
          vw = from_double<T>(2.0 * b - __ldg(a.w + ((long)gk * ny + j) * nx + (out ? nx - 1 : 0)));
        }
        S.pl[0][j & 3][e] = vu;
        S.pl[1][j & 3][e] = vv;
        S.pl[2][j & 3][e] = vw;
        S.pl[3][j & 3][e] = (T)0;
      }
    }
    if (kAsync) cp_async_commit8();
  };
  // Each product loop gives every thread the item q = tid first (every loop has at least 256
  // items).  In the FP32 form that item's tile offsets are worked out once, before the march in y,
  // and only the few items q >= 256 take the general index arithmetic: the FP32 RHS is
  // issue-bound.  (The FP64 form takes the general index arithmetic for both: the offsets cost it
  // registers.)
  constexpr bool kHoist = sizeof(T) == 4;
  const int hk = tid / (RT_X + 1), hi = tid % (RT_X + 1);   // items of the (RT_X + 1)-wide loops
  const int gk = tid / RT_X, gi = tid % RT_X;               // items of the RT_X-wide loops
  const int eA = (hk + 1) * RT_PX + hi + 1, fA = hk * (RT_X + 1) + hi;
  const int eB = (gk + 1) * RT_PX + gi + 1, fB = gk * RT_X + gi;
  auto PL = [&](int f, int j) -> T* { return S.pl[f][j & 3]; };
  // y-face fluxes on face jf, zero on the walls, each divided by the interpolation weight WLO_jf
  // (which the difference weights carry): Fuv = (u_{j-1} + RHO u_j)(v_{i-1} + v_i) and
  // Fvw = (v_{k-1} + v_k)(w_{j-1} + RHO w_j), one FMA, one add and one product each
  // Every product loop has NT <= n < 2 NT items: thread tid takes item tid.  In the FP32 form the
  // n - NT items past NT go to the threads from `off` on: Fuv and Q1's extra items to warp 0,
  // Fvw and Q3's to warp 1 and Fuw's to warps 2 and 3, so that the four SM sub-partitions (warp w
  // issues on sub-partition w mod 4) share them (FP32 RHS 0.242 -> 0.237 ms).  The FP64 form keeps
  // them on the first threads (spread, it took 74 registers instead of 67 and 1.58 ms instead of
  // 1.55).
  constexpr int NT = RT_X * RT_Z;
  auto second = [&](int n, int off) {
    const int x = tid - off;
    return (x >= 0 && x < n - NT) ? NT + x : -1;
  };
  auto face_fluxes = [&](int jf) {
    const bool inner = jf >= 1 && jf <= ny - 1;
    const T rho = S.wf[jf & 3];
    auto fuv_at = [&](int q) {
      const int kk = q / (RT_X + 1), ii = q % (RT_X + 1);
      T f = 0;
      if (inner)
        f = (P(0, jf - 1, kk, ii) + rho * P(0, jf, kk, ii)) * (P(1, jf, kk, ii - 1) + P(1, jf, kk, ii));
      S.fuv[jf & 1][kk][ii] = f;
    };
    auto fvw_at = [&](int q) {
      const int kk = q / RT_X, ii = q % RT_X;
      T f = 0;
      if (inner)
        f = (P(1, jf, kk - 1, ii) + P(1, jf, kk, ii)) * (P(2, jf - 1, kk, ii) + rho * P(2, jf, kk, ii));
      S.fvw[jf & 1][kk][ii] = f;
    };
    if constexpr (kHoist) {
      const T* u0 = PL(0, jf - 1);
      const T* u1 = PL(0, jf);
      const T* v1 = PL(1, jf);
      const T* w0 = PL(2, jf - 1);
      const T* w1 = PL(2, jf);
      (&S.fuv[jf & 1][0][0])[fA] = inner ? (u0[eA] + rho * u1[eA]) * (v1[eA - 1] + v1[eA]) : (T)0;
      (&S.fvw[jf & 1][0][0])[fB] = inner ? (v1[eB - RT_PX] + v1[eB]) * (w0[eB] + rho * w1[eB]) : (T)0;
      if (const int q = second(RT_Z * (RT_X + 1), 0); q >= 0) fuv_at(q);
      if (const int q = second((RT_Z + 1) * RT_X, 32); q >= 0) fvw_at(q);
    } else {
      for (int q = tid; q < RT_Z * (RT_X + 1); q += NT) fuv_at(q);
      for (int q = tid; q < (RT_Z + 1) * RT_X; q += NT) fvw_at(q);
    }
  };
  // centre-plane products of plane j (Q1, Q3, Fuw)
  auto centre_products = [&](int j) {
    auto q1_at = [&](int q) {
      const int kk = q / (RT_X + 1), ii = q % (RT_X + 1) - 1;
      const T s = P(0, j, kk, ii) + P(0, j, kk, ii + 1);
      S.q1[kk][ii + 1] = s * s;
    };
    auto q3_at = [&](int q) {
      const int kk = q / RT_X - 1, ii = q % RT_X;
      const T s = P(2, j, kk, ii) + P(2, j, kk + 1, ii);
      S.q3[kk + 1][ii] = s * s;
    };
    auto fuw_at = [&](int q) {
      const int kk = q / (RT_X + 1), ii = q % (RT_X + 1);
      S.fuw[kk][ii] = (P(0, j, kk - 1, ii) + P(0, j, kk, ii)) * (P(2, j, kk, ii - 1) + P(2, j, kk, ii));
    };
    if constexpr (kHoist) {
      const T* u = PL(0, j);
      const T* w = PL(2, j);
      const T s1 = u[eA - 1] + u[eA];  // Q1 item: x = i0 - 1 + hi, z row hk
      (&S.q1[0][0])[fA] = s1 * s1;
      const T s3 = w[eB - RT_PX] + w[eB];  // Q3 item: z = k0 - 1 + gk
      (&S.q3[0][0])[fB] = s3 * s3;
      (&S.fuw[0][0])[fA] = (u[eA - RT_PX] + u[eA]) * (w[eA - 1] + w[eA]);
      if (const int q = second(RT_Z * (RT_X + 1), 0); q >= 0) q1_at(q);
      if (const int q = second((RT_Z + 1) * RT_X, 32); q >= 0) q3_at(q);
      if (const int q = second((RT_Z + 1) * (RT_X + 1), 64); q >= 0) fuw_at(q);
    } else {
      for (int q = tid; q < RT_Z * (RT_X + 1); q += NT) q1_at(q);
      for (int q = tid; q < (RT_Z + 1) * RT_X; q += NT) q3_at(q);
      for (int q = tid; q < (RT_Z + 1) * (RT_X + 1); q += NT) fuw_at(q);
    }
  };

  // r = cn N + cp N_prev + cgx (p_i - p_{i-1}) + cx (f_{i+1} + f_{i-1}) + cz (f_{k+1} + f_{k-1})
  //     + cA f_{j-1} + cC f_{j+1} + cD f (+ cb for u), with every constant pre-multiplied by dt;
  // cn N is formed directly (the difference weights carry cn) and stored as the next N_prev
  auto K = [&](int q) -> T {
    const StepK& sk = Dyn ? *a.sk : a.kc;
    if constexpr (sizeof(T) == 4) return sk.kf[q];
    else return sk.kd[q];
  };
  const T qidx = K(RK_QIDX), qidz = K(RK_QIDZ);
  const T cp = K(RK_CP), cgx = K(RK_CGX), cgz = K(RK_CGZ), cx = K(RK_CX), cz = K(RK_CZ);
  const T cb = K(RK_CB);
  const bool use_prev = a.zet != 0.0;
  auto R = [&](int f, int jj) -> T {
    if constexpr (sizeof(T) == 4) return __ldg(a.rtf + f * G + jj);
    else return (T)__ldg(a.rt + f * G + jj);
  };
  TR* ru = (TR*)a.ru;
  TR* rv = (TR*)a.rv;
  TR* rw = (TR*)a.rw;
  TR* nu = (TR*)a.nu;
  TR* nv = (TR*)a.nv;
  TR* nw = (TR*)a.nw;
  const int i = i0 + tx, k = k0 + tz;

  // The per-row coefficients every thread of the block reads (R, and the face weights of the
  // y fluxes) are fetched by a few threads into a small ring in shared memory, one step ahead of
  // their use, instead of by every thread through the read-only path.
  auto fetch_face = [&](int jf) { S.wf[jf & 3] = (jf >= 1 && jf <= ny - 1) ? R(RT_RHO, jf) : (T)0; };
  // prologue: planes jb-1, jb (jb+1 in flight); fluxes of face jb; Q2 of centre jb-1
  load_plane(jb - 1);
  load_plane(jb);
  if (kAsync) cp_async_wait_all8();
  if (tid == 0) fetch_face(jb);
  __syncthreads();
  if (kAsync) load_plane(jb + 1);
  face_fluxes(jb);
  T q2prev = 0;
  {
    const T s = P(1, jb - 1, tz, tx) + P(1, jb, tz, tx);
    q2prev = (jb >= 1) ? s * s : (T)0;
  }
  for (int j = jb; j <= jlast; ++j) {
    if (tid < RT_COUNT) S.rt[j & 3][tid] = R(tid, j);
    else if (tid == RT_COUNT) fetch_face(j + 1);
    if (kAsync) cp_async_wait_all8();  // this thread's copies of plane j + 1
    else load_plane(j + 1);
    __syncthreads();
    if (kAsync && j + 1 <= jlast) load_plane(j + 2);
    face_fluxes(j + 1);
    centre_products(j);
    __syncthreads();
    // The three components are assembled in one straight-line block (v also on the wall faces
    // and u, w also on the face row j = ny, where the planes read are zero and the results are
    // not stored), so that the compiler can interleave their three FP64 chains.
    const bool vrow = j > 0 && j < ny;  // interior v face
    const bool crow = j < ny;           // a row of cells
    const long cf = ((long)k * ny1 + j) * nx + i;
    const long cc = ((long)k * ny + (crow ? j : 0)) * nx + i;
    const T* rt = S.rt[j & 3];
    // ---------------- v at face j
    const T sv = P(1, j, tz, tx) + P(1, j + 1, tz, tx);
    const T q2 = sv * sv;  // Q2 of centre j (zero planes beyond the top)
    const T nvv = (S.fuv[j & 1][tz][tx + 1] - S.fuv[j & 1][tz][tx]) * rt[RT_HXW] + (q2 - q2prev) * rt[RT_QIHC] +
                  (S.fvw[j & 1][tz + 1][tx] - S.fvw[j & 1][tz][tx]) * rt[RT_HZW];
    q2prev = q2;
    const T v0 = P(1, j, tz, tx);
    T rv_ = nvv + rt[RT_CGY] * (P(3, j, tz, tx) - P(3, j - 1, tz, tx));
    rv_ += cx * (P(1, j, tz, tx + 1) + P(1, j, tz, tx - 1));
    rv_ += cz * (P(1, j, tz + 1, tx) + P(1, j, tz - 1, tx));
    // one FMA per term on r (a sum of the three products first would add an instruction)
    rv_ += rt[RT_AF] * P(1, j - 1, tz, tx);
    rv_ += rt[RT_CF] * P(1, j + 1, tz, tx);
    rv_ += rt[RT_DF] * v0;
    // ---------------- u at (xf_i, yc_j, zc_k)
    const T hym = rt[RT_HYM], hyp = rt[RT_HYP];
    const T cA = rt[RT_AC], cC = rt[RT_CC], cD = rt[RT_DC];
    const T u0 = P(0, j, tz, tx);
    const T nuu = (S.q1[tz][tx + 1] - S.q1[tz][tx]) * qidx +
                  S.fuv[(j + 1) & 1][tz][tx] * hyp + S.fuv[j & 1][tz][tx] * hym +
                  (S.fuw[tz + 1][tx] - S.fuw[tz][tx]) * qidz;
    T ru_ = nuu + cb + cgx * (P(3, j, tz, tx) - P(3, j, tz, tx - 1));
    ru_ += cx * (P(0, j, tz, tx + 1) + P(0, j, tz, tx - 1));
    ru_ += cz * (P(0, j, tz + 1, tx) + P(0, j, tz - 1, tx));
    ru_ += cA * P(0, j - 1, tz, tx);
    ru_ += cC * P(0, j + 1, tz, tx);
    ru_ += cD * u0;
    // ---------------- w at (xc_i, yc_j, zf_k)
    const T w0 = P(2, j, tz, tx);
    const T nww = (S.fuw[tz][tx + 1] - S.fuw[tz][tx]) * qidx +
                  S.fvw[(j + 1) & 1][tz][tx] * hyp + S.fvw[j & 1][tz][tx] * hym +
                  (S.q3[tz + 1][tx] - S.q3[tz][tx]) * qidz;
    T rw_ = nww + cgz * (P(3, j, tz, tx) - P(3, j, tz - 1, tx));
    rw_ += cx * (P(2, j, tz, tx + 1) + P(2, j, tz, tx - 1));
    rw_ += cz * (P(2, j, tz + 1, tx) + P(2, j, tz - 1, tx));
    rw_ += cA * P(2, j - 1, tz, tx);
    rw_ += cC * P(2, j + 1, tz, tx);
    rw_ += cD * w0;
    if (use_prev) {
      if (vrow) rv_ += cp * (T)nv[cf];
      if (crow) {
        ru_ += cp * (T)nu[cc];
        rw_ += cp * (T)nw[cc];
      }
    }
    rv[cf] = vrow ? (TR)rv_ : (TR)0;
    nv[cf] = vrow ? (TR)nvv : (TR)0;
    if (crow) {
      const bool fixed = a.bl && i == 0;  // inflow face of u
      ru[cc] = fixed ? (TR)0 : (TR)ru_;
      nu[cc] = fixed ? (TR)0 : (TR)nuu;
      rw[cc] = (TR)rw_;
      nw[cc] = (TR)nww;
    }
  }

  }
};

}  // namespace

template <typename T, bool Dyn>
cudaError_t rhs_attributes(int* bps) {
  using K = RhsTiledK<T, T, Dyn>;
  const cudaError_t e = set_smem_limit<K>((int)sizeof(RhsTile<T>));
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, single_kernel<K>, RT_X * RT_Z, sizeof(RhsTile<T>));
}

cudaError_t rhs_set_attributes(int* bps) {
  cudaError_t e;
  if ((e = rhs_attributes<double, false>(bps + 0)) != cudaSuccess ||
      (e = rhs_attributes<double, true>(bps + 1)) != cudaSuccess ||
      (e = rhs_attributes<float, false>(bps + 2)) != cudaSuccess)
    return e;
  return rhs_attributes<float, true>(bps + 3);
}

cudaError_t launch_rhs(ns_ctx* c, int k) {
  LaunchSink s{c, nullptr};
  return stage_rhs(s, k);
}

template <typename T, bool Dyn>
cudaError_t emit_tiled(LaunchSink& s, const RhsArgs& a) {
  // split y into chunks (each re-derives one face and two planes) so that the blocks fill whole
  // waves of the resident capacity: minimise waves * (planes per chunk + prologue).  (Chunks of
  // equal rows in one single wave, some spanning two tiles, were slower on both forms: neighbouring
  // tiles then march at different y.)
  ns_ctx* c = s.c;
  const int tiles = (a.nx / RT_X) * (a.nz / RT_Z);
  const int resident = c->num_sms * std::max(c->rhs_bps[(sizeof(T) == 4 ? 2 : 0) + (Dyn ? 1 : 0)], 1);
  int best_nch = 1;
  double best = 1e300;
  for (int nch = 1; nch <= (a.ny + 5) / 6 && nch <= 64; ++nch) {
    const int jc = (a.ny + nch - 1) / nch;
    const long nb = (long)tiles * ((a.ny + jc - 1) / jc);
    const long waves = (nb + resident - 1) / resident;
    const double cost = (double)waves * (jc + 2.0);
    if (cost < best - 1e-9) {
      best = cost;
      best_nch = nch;
    }
  }
  const int jchunk = (a.ny + best_nch - 1) / best_nch;
  const int nch = (a.ny + jchunk - 1) / jchunk;
  return emit<RhsTiledK<T, T, Dyn>>(s, RhsTiledK<T, T, Dyn>::make(a, jchunk), dim3(a.nx / RT_X, a.nz / RT_Z, nch),
                                    dim3(RT_X, RT_Z), sizeof(RhsTile<T>));
}

cudaError_t stage_rhs(LaunchSink& s, int k) {
  ns_ctx* c = s.c;
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
  a.cprev = k > 0 ? NS_ZETA[k] / NS_GAMMA[k - 1] : 0.0;
  a.alp = NS_ALPHA[k];
  a.inv_re = c->cfg.re > 0 ? 1.0 / c->cfg.re : 0.0;
  a.fx = c->cfg.fx;
  a.rt = c->rtab[k];
  a.rtf = c->rtabf[k];
  a.bl = c->bl;
  a.u_out = c->f.u_out;
  a.v_in = c->f.v_in;
  a.v_out = c->f.v_out;
  a.w_in = c->f.w_in;
  a.w_out = c->f.w_out;
  a.sk = c->stepk + k;
  a.kc = c->stepk_h[k];
  if (a.nx % RT_X == 0 && a.nz % RT_Z == 0) {
    if (c->cfg.precision == NS_MIXED)
      return c->dyn_consts ? emit_tiled<float, true>(s, a) : emit_tiled<float, false>(s, a);
    // FP64 always reads them from device memory: the register allocation of that variant is
    // faster than the one with constant-bank operands on this kernel
    return emit_tiled<double, true>(s, a);
  }
  const long plane = (long)a.nx * (a.ny + 1);
  dim3 grid((unsigned)((plane + 127) / 128), (unsigned)a.nz);
  if (c->cfg.precision == NS_MIXED)
    return c->dyn_consts ? emit<RhsK<float, float, true>>(s, RhsK<float, float, true>::make(a), grid, 128, 0)
                         : emit<RhsK<float, float, false>>(s, RhsK<float, float, false>::make(a), grid, 128, 0);
  return c->dyn_consts ? emit<RhsK<double, double, true>>(s, RhsK<double, double, true>::make(a), grid, 128, 0)
                       : emit<RhsK<double, double, false>>(s, RhsK<double, double, false>::make(a), grid, 128, 0);
}
