// ADI factors of the momentum increment (Sec. 2.2):  (I - b d_xx)(I - b d_yy)(I - b d_zz) delta = r.
//
// x: lines are contiguous and periodic.  Each line is split into P partitions of M rows, one
//    partition per lane of a team of P lanes (Sec. 3.2, the PDD / PPT divide-and-conquer scheme
//    moved from MPI ranks to warp lanes):
//      A~ x~ = d                 (Eq. blockAx)  block Thomas with precomputed factors
//      A~ Y  = V                 (Eq. blockAY)  spikes v, w: line-independent, precomputed
//      Z y   = E^T x~            (Eq. Zpdd)     interface unknowns y = (x^{(r)}_m, x^{(r+1)}_1)
//      x     = x~ - Y y          (Eq. xpdd)
//    PDD keeps only the 2x2 diagonal blocks of Z; PPT solves all of Z exactly by block parallel
//    cyclic reduction over the team with warp shuffles (line-independent eliminators).
// y: lines have stride nx; one thread per line, Thomas with precomputed factors.
// z: lines have stride nx*ny and are periodic; one thread per line, Thomas on the Sherman-
//    Morrison-modified matrix plus the rank-one correction; then u* = u + delta (FP64).
#include "ns_internal.cuh"

namespace {

// ----------------------------------------------------------------------------------------------
// x: partitioned solve
// ----------------------------------------------------------------------------------------------
template <typename T>
struct AdiXArgs {
  const T* __restrict__ tab[2];  // table of the u lines [0] and of the v, w lines [1]
  T* r[3];
  int nx, ny, nz, P;
  long nlines;  // nz*ny (u) + nz*(ny-1) (v) + nz*ny (w)
  // inflow / outflow in x: the outflow-plane increment of component c enters the last row as
  // + sk->xcf[c] * dout[c][k * rows + j]
  int bl;
  const double* __restrict__ dout[3];
  const StepK* sk;  // reduction levels L (0: PDD) and the outflow weights of this sub-step
};

// xcf[comp] * dout[comp][plane] in the arithmetic type
template <typename T>
__device__ __forceinline__ T outflow_term(const AdiXArgs<T>& a, int comp, long plane) {
  const double* d = comp == 0 ? a.dout[0] : (comp == 1 ? a.dout[1] : a.dout[2]);
  T cf;
  if constexpr (sizeof(T) == 4) cf = a.sk->xcff[comp];
  else cf = a.sk->xcf[comp];
  return cf * (T)__ldg(d + plane);
}

// component, boundary-plane index and row pointer of x-line number `line`
template <typename T>
__device__ __forceinline__ T* x_line(const AdiXArgs<T>& a, long line, int* comp, long* plane) {
  const int nx = a.nx, ny = a.ny;
  const long Lu = (long)a.nz * ny;
  const long Lv = (long)a.nz * (ny - 1);
  if (line < Lu) {
    *comp = 0;
    *plane = line;
    return a.r[0] + line * nx;
  }
  if (line < Lu + Lv) {
    const long q = line - Lu;
    const long kk = q / (ny - 1);
    const long jj = 1 + (q - kk * (ny - 1));
    *comp = 1;
    *plane = kk * (ny + 1) + jj;
    return a.r[1] + *plane * nx;
  }
  *comp = 2;
  *plane = line - Lu - Lv;
  return a.r[2] + *plane * nx;
}

template <typename T, int M>
__device__ __forceinline__ void load_part(const T* __restrict__ src, T (&d)[M]) {
  if constexpr (sizeof(T) * M % 16 == 0) {
    constexpr int V = 16 / sizeof(T);
#pragma unroll
    for (int e = 0; e < M; e += V) {
      if constexpr (sizeof(T) == 8) {
        const double2 t = *reinterpret_cast<const double2*>(src + e);
        d[e] = t.x;
        d[e + 1] = t.y;
      } else {
        const float4 t = *reinterpret_cast<const float4*>(src + e);
        d[e] = t.x;
        d[e + 1] = t.y;
        d[e + 2] = t.z;
        d[e + 3] = t.w;
      }
    }
  } else {
#pragma unroll
    for (int e = 0; e < M; ++e) d[e] = src[e];
  }
}

template <typename T, int M>
__device__ __forceinline__ void store_part(T* __restrict__ dst, const T (&d)[M]) {
  if constexpr (sizeof(T) * M % 16 == 0) {
    constexpr int V = 16 / sizeof(T);
#pragma unroll
    for (int e = 0; e < M; e += V) {
      if constexpr (sizeof(T) == 8) {
        *reinterpret_cast<double2*>(dst + e) = make_double2(d[e], d[e + 1]);
      } else {
        *reinterpret_cast<float4*>(dst + e) = make_float4(d[e], d[e + 1], d[e + 2], d[e + 3]);
      }
    }
  } else {
#pragma unroll
    for (int e = 0; e < M; ++e) dst[e] = d[e];
  }
}

template <typename T, int M>
struct AdiXK {
  struct Args {
    AdiXArgs<T> a;
  };
  static constexpr int kThreads = 256;
  // FP32 is bandwidth-bound: occupancy.  At 8 rows, 4 blocks of 64 registers (a 24-byte spill)
  // beat 3 of 80 (0.071 -> 0.066 ms on 256-row lines)
  static constexpr int kMinBlocks = sizeof(T) == 4 ? (M == 8 ? 4 : 3) : 2;
  static Args make(AdiXArgs<T> a) { return Args{a}; }
  static __device__ __forceinline__ void run(const Args& a_, const dim3 bid_, const dim3 gdim_) {
    const AdiXArgs<T>& a = a_.a;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* st = reinterpret_cast<T*>(smem_raw);
  const int P = a.P, L = a.sk->L;
  const int ntab = (int)xtab_count(M, P, L);
  const int ncls = a.bl ? 2 : 1;
  for (int q = threadIdx.x; q < ntab * ncls; q += blockDim.x) st[q] = q < ntab ? a.tab[0][q] : a.tab[1][q - ntab];
  __syncthreads();

  const int lane = threadIdx.x & 31;
  const int r = lane & (P - 1);
  const int team = lane / P;
  const int teams = 32 / P;
  const long warp = ((long)bid_.x * blockDim.x + threadIdx.x) >> 5;
  const long nwarps = ((long)gdim_.x * blockDim.x) >> 5;

  for (long l0 = warp * teams; l0 < a.nlines; l0 += nwarps * teams) {
    const long line = l0 + team;
    const bool valid = line < a.nlines;
    T* row = nullptr;
    int comp = 0;
    long plane = 0;
    if (valid) row = x_line(a, line, &comp, &plane);
    const T* tb = st + (a.bl && comp != 0 ? ntab : 0);
    const T* INV = tb + XT_INV * M * P;
    const T* AINV = tb + XT_AINV * M * P;
    const T* CP = tb + XT_CP * M * P;
    const T* SV = tb + XT_V * M * P;
    const T* SW = tb + XT_W * M * P;
    const T* DINV = tb + XT_NF * M * P;
    const T* ML = DINV + 4 * P;
    const T* MU = ML + 4 * L * P;
    T d[M];
    if (valid) {
      load_part<T, M>(row + r * M, d);
      if (a.bl && r == P - 1) d[M - 1] += outflow_term(a, comp, plane);
    } else {
#pragma unroll
      for (int e = 0; e < M; ++e) d[e] = (T)0;
    }
    // A~ x~ = d on this partition (forward elimination, back substitution)
    d[0] = d[0] * INV[r];
#pragma unroll
    for (int e = 1; e < M; ++e) d[e] = d[e] * INV[e * P + r] - AINV[e * P + r] * d[e - 1];
#pragma unroll
    for (int e = M - 2; e >= 0; --e) d[e] = d[e] - CP[e * P + r] * d[e + 1];
    // interface r: g = (x~^{(r)}_m, x~^{(r+1)}_1)
    T g0 = d[M - 1];
    T g1 = __shfl_sync(NS_FULL_MASK, d[0], r + 1, P);
    // reduced system: block PCR (PPT) over the team; L = 0 gives PDD
    for (int lv = 0, s = 1; lv < L; ++lv, s <<= 1) {
      const T h0 = __shfl_sync(NS_FULL_MASK, g0, r - s + P, P);
      const T h1 = __shfl_sync(NS_FULL_MASK, g1, r - s + P, P);
      const T k0 = __shfl_sync(NS_FULL_MASK, g0, r + s, P);
      const T k1 = __shfl_sync(NS_FULL_MASK, g1, r + s, P);
      const T* ml = ML + 4 * lv * P;
      const T* mu = MU + 4 * lv * P;
      const T n0 = g0 - ml[r] * h0 - ml[P + r] * h1 - mu[r] * k0 - mu[P + r] * k1;
      const T n1 = g1 - ml[2 * P + r] * h0 - ml[3 * P + r] * h1 - mu[2 * P + r] * k0 - mu[3 * P + r] * k1;
      g0 = n0;
      g1 = n1;
    }
    const T y0 = DINV[r] * g0 + DINV[P + r] * g1;      // x^{(r)}_m
    const T y1 = DINV[2 * P + r] * g0 + DINV[3 * P + r] * g1;  // x^{(r+1)}_1
    const T left = __shfl_sync(NS_FULL_MASK, y0, r - 1 + P, P);  // x^{(r-1)}_m
    // x = x~ - v x^{(r-1)}_m - w x^{(r+1)}_1; when the tables say the back half of v and the front
    // half of w are below the truncation tolerance (StepK::xhalf), each row keeps one term
    if (a.sk->xhalf[a.bl && comp != 0 ? 1 : 0]) {
#pragma unroll
      for (int e = 0; e < M / 2; ++e) d[e] = d[e] - SV[e * P + r] * left;
#pragma unroll
      for (int e = M / 2; e < M; ++e) d[e] = d[e] - SW[e * P + r] * y1;
    } else {
#pragma unroll
      for (int e = 0; e < M; ++e) d[e] = d[e] - SV[e * P + r] * left - SW[e * P + r] * y1;
    }
    if (valid) store_part<T, M>(row + r * M, d);
  }

  }
};

// ----------------------------------------------------------------------------------------------
// x, long lines (M = 24 ... 128 rows per partition, P = 32): the same algebra with each warp's line
// staged in shared memory at stride M+1 per partition (conflict-free for 8-byte elements), the
// per-partition tables read through L1.  One warp per line, four warps per block.
// ----------------------------------------------------------------------------------------------
template <typename T, int M>
struct AdiXLongK {
  struct Args {
    AdiXArgs<T> a;
  };
  static constexpr int kThreads = 128;
  static constexpr int kMinBlocks = 8;
  static Args make(AdiXArgs<T> a) { return Args{a}; }
  static __device__ __forceinline__ void run(const Args& a_, const dim3 bid_, const dim3 gdim_) {
    const AdiXArgs<T>& a = a_.a;

  constexpr int P = 32;
  constexpr int LS = P * (M + 1);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* line_buf = reinterpret_cast<T*>(smem_raw) + (threadIdx.x >> 5) * LS;
  const int r = threadIdx.x & 31;
  const int L = a.sk->L;
  const long warp = ((long)bid_.x * blockDim.x + threadIdx.x) >> 5;
  const long nwarps = ((long)gdim_.x * blockDim.x) >> 5;
  T* my = line_buf + r * (M + 1);
  for (long line = warp; line < a.nlines; line += nwarps) {
    int comp;
    long plane;
    T* row = x_line(a, line, &comp, &plane);
    const T* tb = (a.bl && comp != 0) ? a.tab[1] : a.tab[0];
    const T* INV = tb + XT_INV * M * P;
    const T* AINV = tb + XT_AINV * M * P;
    const T* CP = tb + XT_CP * M * P;
    const T* SV = tb + XT_V * M * P;
    const T* SW = tb + XT_W * M * P;
    const T* DINV = tb + XT_NF * M * P;
    const T* ML = DINV + 4 * P;
    const T* MU = ML + 4 * L * P;
    // coalesced load: element g = q*32 + lane goes to partition g / M, row g % M
#pragma unroll 4
    for (int q = 0; q < M; ++q) {
      const int g = q * 32 + r;
      line_buf[(g / M) * (M + 1) + (g % M)] = row[g];
    }
    __syncwarp();
    if (a.bl && r == P - 1) my[M - 1] += outflow_term(a, comp, plane);
    // A~ x~ = d on partition r
    T prev = my[0] * __ldg(INV + r);
    my[0] = prev;
    for (int e = 1; e < M; ++e) {
      prev = my[e] * __ldg(INV + e * P + r) - __ldg(AINV + e * P + r) * prev;
      my[e] = prev;
    }
    T next = prev;
    for (int e = M - 2; e >= 0; --e) {
      next = my[e] - __ldg(CP + e * P + r) * next;
      my[e] = next;
    }
    T g0 = prev;
    T g1 = __shfl_sync(NS_FULL_MASK, next, r + 1, P);
    for (int lv = 0, s = 1; lv < L; ++lv, s <<= 1) {
      const T h0 = __shfl_sync(NS_FULL_MASK, g0, r - s + P, P);
      const T h1 = __shfl_sync(NS_FULL_MASK, g1, r - s + P, P);
      const T k0 = __shfl_sync(NS_FULL_MASK, g0, r + s, P);
      const T k1 = __shfl_sync(NS_FULL_MASK, g1, r + s, P);
      const T* ml = ML + 4 * lv * P;
      const T* mu = MU + 4 * lv * P;
      const T n0 = g0 - __ldg(ml + r) * h0 - __ldg(ml + P + r) * h1 - __ldg(mu + r) * k0 - __ldg(mu + P + r) * k1;
      const T n1 = g1 - __ldg(ml + 2 * P + r) * h0 - __ldg(ml + 3 * P + r) * h1 - __ldg(mu + 2 * P + r) * k0 -
                   __ldg(mu + 3 * P + r) * k1;
      g0 = n0;
      g1 = n1;
    }
    const T y0 = __ldg(DINV + r) * g0 + __ldg(DINV + P + r) * g1;
    const T y1 = __ldg(DINV + 2 * P + r) * g0 + __ldg(DINV + 3 * P + r) * g1;
    const T left = __shfl_sync(NS_FULL_MASK, y0, r - 1 + P, P);
    for (int e = 0; e < M; ++e) my[e] = my[e] - __ldg(SV + e * P + r) * left - __ldg(SW + e * P + r) * y1;
    __syncwarp();
#pragma unroll 4
    for (int q = 0; q < M; ++q) {
      const int g = q * 32 + r;
      row[g] = line_buf[(g / M) * (M + 1) + (g % M)];
    }
    __syncwarp();
  }

  }
};

// ----------------------------------------------------------------------------------------------
// y and z lines of the mixed form, partitioned (Sec. 3.2, the paper's own use of PDD/PPT on the
// wall-normal lines): a block holds 32 consecutive lines (x) by P partitions of M rows, and
// thread (tx, r) keeps rows rM .. rM+M-1 of line tx in registers.  Each element is loaded and
// stored once, coalesced across tx, instead of the forward sweep's write and the back sweep's
// re-read of the thread-per-line solver.  The P interfaces of a line form the same 2x2-block
// reduced system as on x-lines (Eq. Zpdd); it is solved through shared memory, by block PCR
// (L levels) or, when its dropped coupling is negligible, by its diagonal blocks (PDD, L = 0).
// Tables: the x-solver layout (xtab_count) built by the host for the rows of each direction:
// y centres (u, w), y faces (v; the wall row 0 enters as an identity row), z (cyclic).  The z
// lines end with u* = u + delta in FP64.
// ----------------------------------------------------------------------------------------------
template <int P, int M, bool ZDIR>
struct AdiLinePK {
  struct Args {
    float* r[3];
    double* f[3];
    const float* tab[2];  // y: [0] centres, [1] faces; z: [0]
    const StepK* sk;      // levels Ly / Lz of this sub-step
    int nx, ny, nz;
  };
  static constexpr int kThreads = 32 * P;
  // P = 8 (256 threads): 4 blocks per SM where 64 registers hold the rows without spilling (z,
  // and y up to 16 rows), else 3; the latency of the strided rows is hidden by occupancy
  // (z 8 x 32: 0.156 ms at 2 blocks, 0.137 at 3, 0.130 at 4)
  static constexpr int kMinBlocks = P == 8 ? ((ZDIR || M <= 16) ? 4 : 3) : 1;
  static Args make(float* ru, float* rv, float* rw, double* u, double* v, double* w, const float* t0, const float* t1,
                   const StepK* sk, int nx, int ny, int nz) {
    return Args{{ru, rv, rw}, {u, v, w}, {t0, t1}, sk, nx, ny, nz};
  }
  static __device__ __forceinline__ void run(const Args& a, const dim3 bid_, const dim3 gdim_) {
    constexpr int LMAX = P == 8 ? 3 : (P == 16 ? 4 : 5);
    const int nx = a.nx, ny = a.ny;
    const int comp = bid_.z;
    const int tx = threadIdx.x & 31, r = threadIdx.x >> 5;
    const int i = bid_.x * 32 + tx;
    int L;
    long base, stride;
    const float* gtab;
    if constexpr (ZDIR) {
      const int j = bid_.y + (comp == 1 ? 1 : 0);
      if (comp == 1 && j > ny - 1) return;  // uniform over the block
      base = (long)j * nx + i;
      stride = (long)(comp == 1 ? ny + 1 : ny) * nx;
      gtab = a.tab[0];
      L = a.sk->Lz;
    } else {
      const int k = bid_.y;
      base = (long)k * (comp == 1 ? ny + 1 : ny) * nx + i;
      stride = nx;
      gtab = a.tab[comp == 1 ? 1 : 0];
      L = a.sk->Ly;
    }
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* st = reinterpret_cast<float*>(smem_raw);
    float* ex0 = st + xtab_count(M, P, LMAX);  // [P][32]
    float* ex1 = ex0 + P * 32;
    const int ntab = (int)xtab_count(M, P, L);
    for (int q = threadIdx.x; q < ntab; q += blockDim.x) st[q] = __ldg(gtab + q);
    float* line = (comp == 0 ? a.r[0] : comp == 1 ? a.r[1] : a.r[2]) + base;
    float d[M];
#pragma unroll
    for (int e = 0; e < M; ++e) d[e] = line[(long)(r * M + e) * stride];
    __syncthreads();
    const float* INV = st + XT_INV * M * P;
    const float* AINV = st + XT_AINV * M * P;
    const float* CP = st + XT_CP * M * P;
    const float* SV = st + XT_V * M * P;
    const float* SW = st + XT_W * M * P;
    const float* DINV = st + XT_NF * M * P;
    const float* ML = DINV + 4 * P;
    const float* MU = ML + 4 * L * P;
    // A~ x~ = d on this partition
    d[0] = d[0] * INV[r];
#pragma unroll
    for (int e = 1; e < M; ++e) d[e] = d[e] * INV[e * P + r] - AINV[e * P + r] * d[e - 1];
#pragma unroll
    for (int e = M - 2; e >= 0; --e) d[e] = d[e] - CP[e * P + r] * d[e + 1];
    // interface r: g = (x~^{(r)}_m, x~^{(r+1)}_1)
    ex0[r * 32 + tx] = d[0];
    __syncthreads();
    float g0 = d[M - 1];
    float g1 = ex0[((r + 1) % P) * 32 + tx];
    for (int lv = 0, sd = 1; lv < L; ++lv, sd <<= 1) {
      __syncthreads();
      ex0[r * 32 + tx] = g0;
      ex1[r * 32 + tx] = g1;
      __syncthreads();
      const int rm = (r - sd + P) % P, rp = (r + sd) % P;
      const float h0 = ex0[rm * 32 + tx], h1 = ex1[rm * 32 + tx];
      const float k0 = ex0[rp * 32 + tx], k1 = ex1[rp * 32 + tx];
      const float* ml = ML + 4 * lv * P;
      const float* mu = MU + 4 * lv * P;
      const float n0 = g0 - ml[r] * h0 - ml[P + r] * h1 - mu[r] * k0 - mu[P + r] * k1;
      const float n1 = g1 - ml[2 * P + r] * h0 - ml[3 * P + r] * h1 - mu[2 * P + r] * k0 - mu[3 * P + r] * k1;
      g0 = n0;
      g1 = n1;
    }
    const float y0 = DINV[r] * g0 + DINV[P + r] * g1;          // x^{(r)}_m
    const float y1 = DINV[2 * P + r] * g0 + DINV[3 * P + r] * g1;  // x^{(r+1)}_1
    __syncthreads();
    ex0[r * 32 + tx] = y0;
    __syncthreads();
    const float left = ex0[((r + P - 1) % P) * 32 + tx];  // x^{(r-1)}_m
#pragma unroll
    for (int e = 0; e < M; ++e) d[e] = d[e] - SV[e * P + r] * left - SW[e * P + r] * y1;
    if constexpr (ZDIR) {
      double* f = (comp == 0 ? a.f[0] : comp == 1 ? a.f[1] : a.f[2]) + base;
      constexpr int U = 8;  // u rows in flight at a time (bounds the registers of the FP64 values)
#pragma unroll
      for (int e0 = 0; e0 < M; e0 += U) {
        double fv[U];
#pragma unroll
        for (int q = 0; q < U; ++q)
          if (e0 + q < M) fv[q] = f[(long)(r * M + e0 + q) * stride];
#pragma unroll
        for (int q = 0; q < U; ++q)
          if (e0 + q < M) f[(long)(r * M + e0 + q) * stride] = fv[q] + f2d(d[e0 + q]);
      }
    } else {
#pragma unroll
      for (int e = 0; e < M; ++e) line[(long)(r * M + e) * stride] = d[e];
    }
  }
};

// ----------------------------------------------------------------------------------------------
// y: one thread per line, Thomas with precomputed factors [INV, AINV, CP][n]
// ----------------------------------------------------------------------------------------------
template <typename T>
struct AdiYK {
  struct Args {
    T* ru;
    T* rv;
    T* rw;
    const T* tc;
    const T* tf;
    int nx;
    int ny;
    int nz;
  };
  static constexpr int kThreads = 128;
  static constexpr int kMinBlocks = 12;  // room for the rows fetched ahead
  static Args make(T* ru, T* rv, T* rw, const T* tc, const T* tf, int nx, int ny, int nz) { return Args{ru, rv, rw, tc, tf, nx, ny, nz}; }
  static __device__ __forceinline__ void run(const Args& a_, const dim3 bid_, const dim3 gdim_) {
    T* __restrict__ ru = a_.ru;
    T* __restrict__ rv = a_.rv;
    T* __restrict__ rw = a_.rw;
    const T* __restrict__ tc = a_.tc;
    const T* __restrict__ tf = a_.tf;
    int nx = a_.nx;
    int ny = a_.ny;
    int nz = a_.nz;

  const int comp = bid_.z;
  const int i = bid_.x * blockDim.x + threadIdx.x;
  const int k = bid_.y;
  if (i >= nx) return;
  T* line;
  const T* tab;
  int n;
  if (comp == 1) {
    line = rv + ((long)k * (ny + 1) + 1) * nx + i;
    tab = tf;
    n = ny - 1;
  } else {
    line = (comp == 0 ? ru : rw) + (long)k * ny * nx + i;
    tab = tc;
    n = ny;
  }
  const T* INV = tab;
  const T* AINV = tab + n;
  const T* CP = tab + 2 * n;
  // rows are fetched U at a time ahead of the dependent recurrence (memory-level parallelism)
  constexpr int U = 4;
  T prev = (T)0;
  for (int j0 = 0; j0 < n; j0 += U) {
    T dv[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (j0 + u < n) dv[u] = line[(long)(j0 + u) * nx];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (j0 + u < n) {
        prev = dv[u] * __ldg(INV + j0 + u) - __ldg(AINV + j0 + u) * prev;  // AINV[0] = 0
        line[(long)(j0 + u) * nx] = prev;
      }
  }
  T next = prev;
  for (int j1 = n - 2; j1 >= 0; j1 -= U) {
    T dv[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (j1 - u >= 0) dv[u] = line[(long)(j1 - u) * nx];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (j1 - u >= 0) {
        next = dv[u] - __ldg(CP + j1 - u) * next;
        line[(long)(j1 - u) * nx] = next;
      }
  }
  }
};

// ----------------------------------------------------------------------------------------------
// z: one thread per line, cyclic (Sherman-Morrison), then u* = u + delta.
// table: [INV, AINV, CP, Q][nz] then (FAC, BG)
// ----------------------------------------------------------------------------------------------
template <typename T>
struct AdiZK {
  struct Args {
    T* ru;
    T* rv;
    T* rw;
    double* u;
    double* v;
    double* w;
    const T* tab;
    int nx;
    int ny;
    int nz;
  };
  static constexpr int kThreads = 128;
  static constexpr int kMinBlocks = 10;  // room for the rows fetched ahead
  static Args make(T* ru, T* rv, T* rw, double* u, double* v, double* w, const T* tab, int nx, int ny, int nz) { return Args{ru, rv, rw, u, v, w, tab, nx, ny, nz}; }
  static __device__ __forceinline__ void run(const Args& a_, const dim3 bid_, const dim3 gdim_) {
    T* __restrict__ ru = a_.ru;
    T* __restrict__ rv = a_.rv;
    T* __restrict__ rw = a_.rw;
    double* __restrict__ u = a_.u;
    double* __restrict__ v = a_.v;
    double* __restrict__ w = a_.w;
    const T* __restrict__ tab = a_.tab;
    int nx = a_.nx;
    int ny = a_.ny;
    int nz = a_.nz;

  const int comp = bid_.z;
  const int i = bid_.x * blockDim.x + threadIdx.x;
  const int j = bid_.y + (comp == 1 ? 1 : 0);
  if (i >= nx) return;
  if (comp == 1 && j > ny - 1) return;
  const int rows = comp == 1 ? ny + 1 : ny;
  const long stride = (long)rows * nx;
  const long base = (long)j * nx + i;
  T* line = (comp == 0 ? ru : comp == 1 ? rv : rw) + base;
  double* f = (comp == 0 ? u : comp == 1 ? v : w) + base;
  constexpr int U = 4;
  if constexpr (sizeof(T) == 8) {
    const T* Z = tab + 4 * nz + 2;
    if (__ldg(Z + 2) != 0.0) {  // uniform over the grid: the factorised circulant form (dt_ztab)
      const double lam = __ldg(Z), ia = __ldg(Z + 1);
      const int K = (int)__ldg(Z + 3);
      const T* LP = Z + 4;  // lam^1 .. lam^KMAX
      // forward recurrence t_j = d_j + lam t_{j-1} from t_0 = d_0 + sum_k lam^k d_{nz-k}
      double t = line[0];
#pragma unroll
      for (int q = 1; q <= NS_ZF_KMAX; ++q)
        if (q <= K) t = fma(__ldg(LP + q - 1), line[(long)(nz - q) * stride], t);
      line[0] = t;
      for (int k0 = 1; k0 < nz; k0 += U) {
        double dv[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (k0 + u < nz) dv[u] = line[(long)(k0 + u) * stride];
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (k0 + u < nz) {
            t = fma(lam, t, dv[u]);
            line[(long)(k0 + u) * stride] = t;
          }
      }
      // backward recurrence x_j = t_j + lam x_{j+1} from x_{nz-1} = t_{nz-1} + sum_k lam^k t_{k-1};
      // u* = u + x / alpha
      // (t_0 .. t_{K-1} are read back from the line: this thread wrote them)
      double x = t;
#pragma unroll
      for (int q = 1; q <= NS_ZF_KMAX; ++q)
        if (q <= K) x = fma(__ldg(LP + q - 1), line[(long)(q - 1) * stride], x);
      f[(long)(nz - 1) * stride] = fma(x, ia, f[(long)(nz - 1) * stride]);
      for (int k1 = nz - 2; k1 >= 0; k1 -= U) {
        double dv[U], fv[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (k1 - u >= 0) {
            dv[u] = line[(long)(k1 - u) * stride];
            fv[u] = f[(long)(k1 - u) * stride];
          }
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (k1 - u >= 0) {
            x = fma(lam, x, dv[u]);
            f[(long)(k1 - u) * stride] = fma(x, ia, fv[u]);
          }
      }
      return;
    }
  }
  const T* INV = tab;
  const T* AINV = tab + nz;
  const T* CP = tab + 2 * nz;
  const T* Q = tab + 3 * nz;
  const T fac = __ldg(tab + 4 * nz);
  const T bg = __ldg(tab + 4 * nz + 1);
  // Thomas on the Sherman-Morrison-modified matrix, rows fetched U at a time ahead
  T prev = (T)0;
  for (int k0 = 0; k0 < nz; k0 += U) {
    T dv[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (k0 + u < nz) dv[u] = line[(long)(k0 + u) * stride];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (k0 + u < nz) {
        prev = dv[u] * __ldg(INV + k0 + u) - __ldg(AINV + k0 + u) * prev;
        line[(long)(k0 + u) * stride] = prev;
      }
  }
  const T ylast = prev;
  T next = prev;
  for (int k1 = nz - 2; k1 >= 0; k1 -= U) {
    T dv[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (k1 - u >= 0) dv[u] = line[(long)(k1 - u) * stride];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (k1 - u >= 0) {
        next = dv[u] - __ldg(CP + k1 - u) * next;
        line[(long)(k1 - u) * stride] = next;
      }
  }
  // rank-one correction, then u* = u + delta in FP64
  const T corr = (next + bg * ylast) * fac;
  for (int k0 = 0; k0 < nz; k0 += U) {
    T yv[U];
    double fv[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (k0 + u < nz) {
        yv[u] = line[(long)(k0 + u) * stride];
        fv[u] = f[(long)(k0 + u) * stride];
      }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (k0 + u < nz) {
        const T x = yv[u] - corr * __ldg(Q + k0 + u);
        double xd;
        if constexpr (sizeof(T) == 4) xd = f2d(x);
        else xd = x;
        f[(long)(k0 + u) * stride] = fv[u] + xd;
      }
  }
  }
};

template <typename T>
void fill_x_args(ns_ctx* c, int k, AdiXArgs<T>& a) {
  a.tab[0] = (const T*)c->xtab[k][0];
  a.tab[1] = (const T*)c->xtab[k][1];
  a.bl = c->bl;
  a.sk = c->stepk + k;
  for (int q = 0; q < 3; ++q) a.dout[q] = c->dout[q];
}

template <typename T, int M>
cudaError_t launch_x_t(LaunchSink& s, int k) {
  ns_ctx* c = s.c;
  AdiXArgs<T> a;
  fill_x_args(c, k, a);
  a.r[0] = (T*)c->ru;
  a.r[1] = (T*)c->rv;
  a.r[2] = (T*)c->rw;
  a.nx = c->cfg.nx;
  a.ny = c->cfg.ny;
  a.nz = c->cfg.nz;
  a.P = c->P;
  a.nlines = (long)a.nz * a.ny * 2 + (long)a.nz * (a.ny - 1);
  // room for the PPT tables: the levels are read from device memory and follow the mode in use
  int lmax = 0;
  while ((1 << lmax) < a.P) ++lmax;
  const size_t smem = xtab_count(M, a.P, lmax) * sizeof(T) * (a.bl ? 2 : 1);
  const long teams_per_block = 8L * (32 / a.P);
  long blocks = (a.nlines + teams_per_block - 1) / teams_per_block;
  if (blocks > 152L * 16) blocks = 152L * 16;
  return emit<AdiXK<T, M>>(s, AdiXK<T, M>::make(a), dim3((unsigned)blocks), dim3(256), smem);
}

template <typename T, int M>
cudaError_t launch_x_long_t(LaunchSink& s, int k) {
  ns_ctx* c = s.c;
  AdiXArgs<T> a;
  fill_x_args(c, k, a);
  a.r[0] = (T*)c->ru;
  a.r[1] = (T*)c->rv;
  a.r[2] = (T*)c->rw;
  a.nx = c->cfg.nx;
  a.ny = c->cfg.ny;
  a.nz = c->cfg.nz;
  a.P = c->P;
  a.nlines = (long)a.nz * a.ny * 2 + (long)a.nz * (a.ny - 1);
  const size_t smem = (size_t)4 * 32 * (M + 1) * sizeof(T);
  long blocks = (a.nlines + 3) / 4;
  if (blocks > 152L * 16) blocks = 152L * 16;
  return emit<AdiXLongK<T, M>>(s, AdiXLongK<T, M>::make(a), dim3((unsigned)blocks), dim3(128), smem);
}

template <typename T>
cudaError_t launch_x_m(LaunchSink& s, int k) {
  ns_ctx* c = s.c;
  if (!x_partition_ok(c->P, c->M)) return cudaErrorInvalidValue;
  switch (c->M) {
    case 1: return launch_x_t<T, 1>(s, k);
    case 2: return launch_x_t<T, 2>(s, k);
    case 3: return launch_x_t<T, 3>(s, k);
    case 4: return launch_x_t<T, 4>(s, k);
    case 6: return launch_x_t<T, 6>(s, k);
    case 8: return launch_x_t<T, 8>(s, k);
    case 9: return launch_x_t<T, 9>(s, k);
    case 12: return launch_x_t<T, 12>(s, k);
    case 16: return launch_x_t<T, 16>(s, k);
    case 24: return launch_x_long_t<T, 24>(s, k);
    case 32: return launch_x_long_t<T, 32>(s, k);
    case 48: return launch_x_long_t<T, 48>(s, k);
    case 64: return launch_x_long_t<T, 64>(s, k);
    case 96: return launch_x_long_t<T, 96>(s, k);
    case 128: return launch_x_long_t<T, 128>(s, k);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t stage_adi_x(LaunchSink& s, int k) {
  if (s.c->cfg.precision == NS_MIXED) return launch_x_m<float>(s, k);
  return launch_x_m<double>(s, k);
}

template <int P, int M, bool ZDIR>
cudaError_t emit_line_part(LaunchSink& s, int k) {
  ns_ctx* c = s.c;
  const int nx = c->cfg.nx, ny = c->cfg.ny, nz = c->cfg.nz;
  constexpr int LMAX = P == 8 ? 3 : (P == 16 ? 4 : 5);
  const size_t smem = (xtab_count(M, P, LMAX) + 2 * P * 32) * sizeof(float);
  const dim3 grid(nx / 32, ZDIR ? ny : nz, 3);
  const float* t0 = (const float*)c->ptab[k][ZDIR ? 2 : 0];
  const float* t1 = (const float*)c->ptab[k][ZDIR ? 2 : 1];
  return emit<AdiLinePK<P, M, ZDIR>>(s, AdiLinePK<P, M, ZDIR>::make((float*)c->ru, (float*)c->rv, (float*)c->rw,
                                                                    c->f.u, c->f.v, c->f.w, t0, t1, c->stepk + k, nx,
                                                                    ny, nz),
                                     grid, dim3(32 * P), smem);
}

// the partitioned y / z line solver of shape (P, n / P), if one is built
template <bool ZDIR>
cudaError_t launch_line_part(LaunchSink& s, int k, int P, int n) {
  const int M = n / P;
  switch (P * 1000 + M) {
    case 8004: return emit_line_part<8, 4, ZDIR>(s, k);
    case 8006: return emit_line_part<8, 6, ZDIR>(s, k);
    case 8008: return emit_line_part<8, 8, ZDIR>(s, k);
    case 8012: return emit_line_part<8, 12, ZDIR>(s, k);
    case 8016: return emit_line_part<8, 16, ZDIR>(s, k);
    case 8024: return emit_line_part<8, 24, ZDIR>(s, k);
    case 8032: return emit_line_part<8, 32, ZDIR>(s, k);
    case 16018: return emit_line_part<16, 18, ZDIR>(s, k);
    case 16032: return emit_line_part<16, 32, ZDIR>(s, k);
    case 32032: return emit_line_part<32, 32, ZDIR>(s, k);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t stage_adi_y(LaunchSink& s, int k) {
  ns_ctx* c = s.c;
  const int nx = c->cfg.nx, ny = c->cfg.ny, nz = c->cfg.nz;
  if (c->yP) return launch_line_part<false>(s, k, c->yP, ny);
  dim3 grid((nx + 127) / 128, nz, 3);
  if (c->cfg.precision == NS_MIXED)
    return emit<AdiYK<float>>(s, AdiYK<float>::make((float*)c->ru, (float*)c->rv, (float*)c->rw,
                                                    (const float*)c->ytab[k][0], (const float*)c->ytab[k][1], nx,
                                                    ny, nz), grid, 128, 0);
  return emit<AdiYK<double>>(s, AdiYK<double>::make((double*)c->ru, (double*)c->rv, (double*)c->rw,
                                                    (const double*)c->ytab[k][0], (const double*)c->ytab[k][1],
                                                    nx, ny, nz), grid, 128, 0);
}

cudaError_t stage_adi_z(LaunchSink& s, int k) {
  ns_ctx* c = s.c;
  const int nx = c->cfg.nx, ny = c->cfg.ny, nz = c->cfg.nz;
  if (c->zP) return launch_line_part<true>(s, k, c->zP, nz);
  dim3 grid((nx + 127) / 128, ny, 3);
  if (c->cfg.precision == NS_MIXED)
    return emit<AdiZK<float>>(s, AdiZK<float>::make((float*)c->ru, (float*)c->rv, (float*)c->rw, c->f.u, c->f.v,
                                                    c->f.w, (const float*)c->ztab[k], nx, ny, nz), grid, 128, 0);
  return emit<AdiZK<double>>(s, AdiZK<double>::make((double*)c->ru, (double*)c->rv, (double*)c->rw, c->f.u,
                                                    c->f.v, c->f.w, (const double*)c->ztab[k], nx, ny, nz),
                             grid, 128, 0);
}

cudaError_t launch_adi_x(ns_ctx* c, int k) {
  LaunchSink s{c, nullptr};
  return stage_adi_x(s, k);
}

cudaError_t launch_adi_y(ns_ctx* c, int k) {
  LaunchSink s{c, nullptr};
  return stage_adi_y(s, k);
}

cudaError_t launch_adi_z(ns_ctx* c, int k) {
  LaunchSink s{c, nullptr};
  return stage_adi_z(s, k);
}

template <typename T, int M>
cudaError_t short_attr() {
  return set_smem_limit<AdiXK<T, M>>(2 * 48 * 1024);
}

template <typename T>
cudaError_t x_attributes() {
  cudaError_t e;
  if ((e = short_attr<T, 1>()) != cudaSuccess || (e = short_attr<T, 2>()) != cudaSuccess ||
      (e = short_attr<T, 3>()) != cudaSuccess || (e = short_attr<T, 4>()) != cudaSuccess ||
      (e = short_attr<T, 6>()) != cudaSuccess || (e = short_attr<T, 8>()) != cudaSuccess ||
      (e = short_attr<T, 9>()) != cudaSuccess || (e = short_attr<T, 12>()) != cudaSuccess ||
      (e = short_attr<T, 16>()) != cudaSuccess)
    return e;
  if ((e = set_smem_limit<AdiXLongK<T, 24>>(4 * 32 * 25 * (int)sizeof(T))) != cudaSuccess ||
      (e = set_smem_limit<AdiXLongK<T, 32>>(4 * 32 * 33 * (int)sizeof(T))) != cudaSuccess ||
      (e = set_smem_limit<AdiXLongK<T, 48>>(4 * 32 * 49 * (int)sizeof(T))) != cudaSuccess ||
      (e = set_smem_limit<AdiXLongK<T, 64>>(4 * 32 * 65 * (int)sizeof(T))) != cudaSuccess ||
      (e = set_smem_limit<AdiXLongK<T, 96>>(4 * 32 * 97 * (int)sizeof(T))) != cudaSuccess)
    return e;
  return set_smem_limit<AdiXLongK<T, 128>>(4 * 32 * 129 * (int)sizeof(T));
}

template <int P, int M>
cudaError_t line_attr() {
  constexpr int LMAX = P == 8 ? 3 : (P == 16 ? 4 : 5);
  const int bytes = (int)((xtab_count(M, P, LMAX) + 2 * P * 32) * sizeof(float));
  cudaError_t e = set_smem_limit<AdiLinePK<P, M, false>>(bytes);
  if (e != cudaSuccess) return e;
  return set_smem_limit<AdiLinePK<P, M, true>>(bytes);
}

cudaError_t adi_set_attributes() {
  cudaError_t e = x_attributes<double>();
  if (e != cudaSuccess) return e;
  if ((e = line_attr<8, 4>()) != cudaSuccess || (e = line_attr<8, 6>()) != cudaSuccess ||
      (e = line_attr<8, 8>()) != cudaSuccess || (e = line_attr<8, 12>()) != cudaSuccess ||
      (e = line_attr<8, 16>()) != cudaSuccess || (e = line_attr<8, 24>()) != cudaSuccess ||
      (e = line_attr<8, 32>()) != cudaSuccess || (e = line_attr<16, 18>()) != cudaSuccess ||
      (e = line_attr<16, 32>()) != cudaSuccess || (e = line_attr<32, 32>()) != cudaSuccess)
    return e;
  return x_attributes<float>();
}

size_t adi_y_tab_count(int ny) { return 3 * (size_t)ny; }
size_t adi_z_tab_count(int nz) { return ztab_entries(nz); }
