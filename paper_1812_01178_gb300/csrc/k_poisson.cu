// Pressure Poisson solve and projection (Sec. 2.2), FP64 throughout.
//
//   b = D u* / (alpha_k dt)                      divergence at cell centres
//   b^(kx, j, kz) = FFT_x FFT_z b                 real FFT along z (two real columns packed into
//                                                 one complex sequence), complex FFT along x
//   for every (kx, kz): complex tridiagonal solve in y with rows
//     a_j phi_{j-1} - (a_j + c_j + lam_x + lam_z) phi_j + c_j phi_{j+1} = b_j
//   (zero normal gradient at both y boundaries; for (0,0) row 0 is replaced by phi_0 = 0)
//   phi = IFFT_z IFFT_x phi^ / (nx nz)   (the 1/(nx nz) is applied to b before the transforms)
//   u = u* - alpha_k dt G phi,  p = p + phi
//
// FFTs are mixed radix-2/4/3 Stockham autosort transforms (decimation in time) in shared memory
// with a precomputed table of FMA-form twiddles (fft_twiddles); nx and nz are 2^a 3^b.  The y factors (1/pivot, c/pivot) of every (kx, kz)
// system are precomputed once by pois_factor_kernel (the operator does not change).
#include <algorithm>

#include "ns_internal.cuh"

namespace {

// complex arithmetic on double2 (FP64 path) and float2 (the transforms of the mixed form)
template <typename C> struct Cplx;
template <> struct Cplx<double2> {
  using R = double;
  static __device__ __forceinline__ double2 mk(double x, double y) { return make_double2(x, y); }
};
template <> struct Cplx<float2> {
  using R = float;
  static __device__ __forceinline__ float2 mk(float x, float y) { return make_float2(x, y); }
};
__device__ __forceinline__ double fmaT(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmaT(float a, float b, float c) { return fmaf(a, b, c); }
// error-free transformations (Knuth's TwoSum; TwoProd by one FMA): s + e = a + b, p + e = a b
__device__ __forceinline__ void ff_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void ff_two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}
template <typename C>
__device__ __forceinline__ C cadd(C a, C b) { return Cplx<C>::mk(a.x + b.x, a.y + b.y); }
template <typename C>
__device__ __forceinline__ C csub(C a, C b) { return Cplx<C>::mk(a.x - b.x, a.y - b.y); }

// Stockham autosort FFT on nseq sequences of length N = 2^a 3^b stored contiguously in A
// ([seq][N]); plan = a | (b << 8) (fft_plan).  B is scratch of the same size.  SIGN = -1 forward,
// +1 inverse (unscaled).  Decimation in time: one twiddle-free radix-2 stage first when a is odd,
// then a/2 radix-4 stages, then b radix-3 stages.  A radix-R stage that follows stages combining
// sub-transforms of length Ns reads, for j < N/R and k = j mod Ns, the R inputs at j + r N/R,
// multiplies input r by w^(r k) (w = exp(-2 pi i / (R Ns)), conjugated for the inverse), takes the
// R-point DFT and writes output r to (j / Ns) R Ns + k + r Ns.
//
// The FP64 pipe is the bound here, so the twiddled butterflies use the tangent factorisation of
// Goedecker (SIAM J. Sci. Comput. 18, 1997): b w = cos(th) (b.x + tan(th) b.y, b.y - tan(th) b.x)
// costs two FMAs, and the cosine is folded into the following additions; inputs 1 and 3 (radix
// 4) or 1 and 2 (radix 3) share one scale through the ratio of their cosines.  A twiddled radix-4
// butterfly is 22 FMAs (instead of 28 instructions), a radix-3 one 16.  tw holds six doubles per
// entry Ns + k (fft_twiddles): radix 4, th = 2 pi k / (4 Ns): {tan th, cos th}, {tan 2th, cos 2th},
// {tan 3th, cos 3th / cos th}; radix 3, th = 2 pi k / (3 Ns): {tan th, cos th},
// {tan 2th, cos 2th / cos th}, {cos th / 2, (sqrt 3 / 2) cos th}.  cos th is never exactly zero in
// floating point, so every factor is finite.  Returns the buffer that holds the result.  All
// threads of the block take part.
template <int SIGN, typename C = double2>
__device__ C* stockham(C* A, C* B, int N, int plan, int nseq, const C* __restrict__ tw) {
  using R = typename Cplx<C>::R;
  auto mk = [](R x, R y) { return Cplx<C>::mk(x, y); };
  const int a2 = plan & 0xff, b3 = plan >> 8;
  const bool p2 = b3 == 0;  // N a power of two: index arithmetic by shifts
  int Ns = 1;
  if (a2 & 1) {  // radix-2, Ns = 1: no twiddles
    const int half = N >> 1;
    const int total = nseq * half;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
      const int sq = p2 ? idx >> (a2 - 1) : idx / half;
      const int j = idx - sq * half;
      const C* X = A + sq * N;
      C* Y = B + sq * N;
      const C a = X[j], b = X[j + half];
      Y[2 * j] = cadd(a, b);
      Y[2 * j + 1] = csub(a, b);
    }
    __syncthreads();
    C* t = A;
    A = B;
    B = t;
    Ns = 2;
  }
  const int quarter = N >> 2;
  for (int st = 0; st < (a2 >> 1); ++st, Ns <<= 2) {
    const int ls = __ffs(Ns) - 1;  // Ns is a power of two in the radix-4 stages
    const int total = nseq * quarter;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
      const int sq = p2 ? idx >> (a2 - 2) : idx / quarter;
      const int j = idx - sq * quarter;
      const int k = j & (Ns - 1);
      const C* X = A + sq * N + j;
      C* Y = B + sq * N + ((j >> ls) << (ls + 2)) + k;
      const C a = X[0], b = X[quarter], c = X[2 * quarter], d = X[3 * quarter];
      C y0, y1, y2, y3;
      if (Ns == 1) {
        const C t0 = cadd(a, c), t1 = csub(a, c), t2 = cadd(b, d), t3 = csub(b, d);
        // -i t3 (forward) or +i t3 (inverse)
        const C r3 = SIGN < 0 ? mk(t3.y, -t3.x) : mk(-t3.y, t3.x);
        y0 = cadd(t0, t2);
        y2 = csub(t0, t2);
        y1 = cadd(t1, r3);
        y3 = csub(t1, r3);
      } else {
        const C e1 = __ldg(tw + 3 * (Ns + k)), e2 = __ldg(tw + 3 * (Ns + k) + 1), e3 = __ldg(tw + 3 * (Ns + k) + 2);
        const R t1 = SIGN < 0 ? e1.x : -e1.x, t2 = SIGN < 0 ? e2.x : -e2.x, t3 = SIGN < 0 ? e3.x : -e3.x;
        const R c1 = e1.y, c2 = e2.y, r = e3.y;
        // b, c, d times their twiddles, each up to its cosine
        const C bb = mk(fmaT(t1, b.y, b.x), fmaT(-t1, b.x, b.y));
        const C cc = mk(fmaT(t2, c.y, c.x), fmaT(-t2, c.x, c.y));
        const C dd = mk(fmaT(t3, d.y, d.x), fmaT(-t3, d.x, d.y));
        const C T0 = mk(fmaT(c2, cc.x, a.x), fmaT(c2, cc.y, a.y));    // a + c w^2k
        const C T1 = mk(fmaT(-c2, cc.x, a.x), fmaT(-c2, cc.y, a.y));  // a - c w^2k
        const C S = mk(fmaT(r, dd.x, bb.x), fmaT(r, dd.y, bb.y));    // (b w^k + d w^3k) / cos th
        const C D = mk(fmaT(-r, dd.x, bb.x), fmaT(-r, dd.y, bb.y));  // (b w^k - d w^3k) / cos th
        y0 = mk(fmaT(c1, S.x, T0.x), fmaT(c1, S.y, T0.y));
        y2 = mk(fmaT(-c1, S.x, T0.x), fmaT(-c1, S.y, T0.y));
        // y1 = T1 - i (v1 - v3), y3 = T1 + i (v1 - v3) forward; signs of i swap for the inverse
        const R s1 = SIGN < 0 ? c1 : -c1;
        y1 = mk(fmaT(s1, D.y, T1.x), fmaT(-s1, D.x, T1.y));
        y3 = mk(fmaT(-s1, D.y, T1.x), fmaT(s1, D.x, T1.y));
      }
      Y[0] = y0;
      Y[Ns] = y1;
      Y[2 * Ns] = y2;
      Y[3 * Ns] = y3;
    }
    __syncthreads();
    C* t = A;
    A = B;
    B = t;
  }
  const int third = N / 3;
  const R kS3 = (R)0.86602540378443864676;  // sqrt(3) / 2
  for (int st = 0; st < b3; ++st, Ns *= 3) {
    const int total = nseq * third;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
      const int sq = idx / third;
      const int j = idx - sq * third;
      const int g = j / Ns;
      const int k = j - g * Ns;
      const C* X = A + sq * N + j;
      C* Y = B + sq * N + g * 3 * Ns + k;
      const C a = X[0], b = X[third], c = X[2 * third];
      C S, D, y0, T;
      R gs;
      if (Ns == 1) {
        S = cadd(b, c);
        D = csub(b, c);
        y0 = cadd(a, S);
        T = mk(fmaT((R)-0.5, S.x, a.x), fmaT((R)-0.5, S.y, a.y));
        gs = SIGN < 0 ? kS3 : -kS3;
      } else {
        const C e1 = __ldg(tw + 3 * (Ns + k)), e2 = __ldg(tw + 3 * (Ns + k) + 1), e3 = __ldg(tw + 3 * (Ns + k) + 2);
        const R t1 = SIGN < 0 ? e1.x : -e1.x, t2 = SIGN < 0 ? e2.x : -e2.x;
        const R c1 = e1.y, r = e2.y, h = e3.x;
        const C bb = mk(fmaT(t1, b.y, b.x), fmaT(-t1, b.x, b.y));
        const C cc = mk(fmaT(t2, c.y, c.x), fmaT(-t2, c.x, c.y));
        S = mk(fmaT(r, cc.x, bb.x), fmaT(r, cc.y, bb.y));    // (b w^k + c w^2k) / cos th
        D = mk(fmaT(-r, cc.x, bb.x), fmaT(-r, cc.y, bb.y));  // (b w^k - c w^2k) / cos th
        y0 = mk(fmaT(c1, S.x, a.x), fmaT(c1, S.y, a.y));
        T = mk(fmaT(-h, S.x, a.x), fmaT(-h, S.y, a.y));      // a - (v1 + v2) / 2
        gs = SIGN < 0 ? e3.y : -e3.y;                                // (sqrt 3 / 2) cos th
      }
      // y1 = T - i (sqrt 3 / 2)(v1 - v2), y2 = T + i (sqrt 3 / 2)(v1 - v2) forward
      Y[0] = y0;
      Y[Ns] = mk(fmaT(gs, D.y, T.x), fmaT(-gs, D.x, T.y));
      Y[2 * Ns] = mk(fmaT(-gs, D.y, T.x), fmaT(gs, D.x, T.y));
    }
    __syncthreads();
    C* t = A;
    A = B;
    B = t;
  }
  return A;
}

// ------------------------------------------------------------------------------------------
// divergence + forward z FFT.  Block = (x-tile of TX columns, row j).  Output spec[kz][j][i].
// ------------------------------------------------------------------------------------------
struct DivzK {
  struct Args {
    const double* u;
    const double* v;
    const double* w;
    const double* gc;
    const double2* twz;
    double2* spec;
    int nx;
    int ny;
    int nz;
    int pz;  // fft_plan(nz)
    int TX;
    double idx;
    double idz;
    const StepK* sk;  // pscale = 1 / (alpha_k dt nx nz)
    const double* u_out;
  };
  static constexpr int kThreads = 256;
  static constexpr int kMinBlocks = 4;  // shared memory limits residency to ~3 blocks anyway
  static Args make(const double* u, const double* v, const double* w, const double* gc, const double2* twz, double2* spec, int nx, int ny, int nz, int pz, int TX, double idx, double idz, const StepK* sk, const double* u_out) { return Args{u, v, w, gc, twz, spec, nx, ny, nz, pz, TX, idx, idz, sk, u_out}; }
  static __device__ __forceinline__ void run(const Args& a_, const dim3 bid_, const dim3 gdim_) {
    const double* __restrict__ u = a_.u;
    const double* __restrict__ v = a_.v;
    const double* __restrict__ w = a_.w;
    const double* __restrict__ gc = a_.gc;
    const double2* __restrict__ twz = a_.twz;
    double2* __restrict__ spec = a_.spec;
    int nx = a_.nx;
    int ny = a_.ny;
    int nz = a_.nz;
    int pz = a_.pz;
    int TX = a_.TX;
    double idx = a_.idx;
    double idz = a_.idz;
    const double scale = a_.sk->pscale;
    const double* __restrict__ u_out = a_.u_out;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nseq = TX >> 1;
  double2* A = reinterpret_cast<double2*>(smem_raw);
  double2* B = A + nseq * nz;
  const int i0 = bid_.x * TX;
  const int j = bid_.y;
  // the 1/2 of the two-real-sequence unpack below is folded into the scale here
  const double hs = 0.5 * scale;
  const double idy = __ldg(gc + GC_IDY * (ny + 1) + j) * hs;
  idx *= hs;
  idz *= hs;
  const long pl = (long)ny * nx, plv = (long)(ny + 1) * nx;
  for (int q = threadIdx.x; q < TX * nz; q += blockDim.x) {
    const int il = q % TX;
    const int k = q / TX;
    const int i = i0 + il;
    const int ip = (i + 1 == nx) ? 0 : i + 1;
    const int kp = (k + 1 == nz) ? 0 : k + 1;
    const long c = k * pl + (long)j * nx;
    // u on face i+1: periodic wrap, or the outflow plane (u_out != NULL) for the last cell
    const double uip = (u_out && i + 1 == nx) ? __ldg(u_out + (long)k * ny + j) : __ldg(u + c + ip);
    const double du = uip - __ldg(u + c + i);
    const double dv = __ldg(v + k * plv + (long)(j + 1) * nx + i) - __ldg(v + k * plv + (long)j * nx + i);
    const double dw = __ldg(w + kp * pl + (long)j * nx + i) - __ldg(w + c + i);
    const double b = fma(du, idx, fma(dv, idy, dw * idz));  // scale folded into idx, idy, idz
    double* slot = reinterpret_cast<double*>(A + (il >> 1) * nz + k);
    slot[il & 1] = b;
  }
  __syncthreads();
  double2* R = stockham<-1>(A, B, nz, pz, nseq, twz);
  // unpack the two real transforms of each packed pair; write kz = 0..nz/2
  const int nh = (nz >> 1) + 1;
  for (int q = threadIdx.x; q < nh * TX; q += blockDim.x) {
    const int il = q % TX;
    const int m = q / TX;
    const int c = il >> 1;
    const double2 zm = R[c * nz + m];
    const double2 zn = R[c * nz + (m == 0 ? 0 : nz - m)];
    double2 X;
    if ((il & 1) == 0)
      X = make_double2(zm.x + zn.x, zm.y - zn.y);
    else
      X = make_double2(zm.y + zn.y, zn.x - zm.x);
    spec[((long)m * ny + j) * nx + i0 + il] = X;
  }

  }
};

// ------------------------------------------------------------------------------------------
// complex FFT along x of R rows per block (rows are contiguous, length nx), in place.
// ------------------------------------------------------------------------------------------
template <int SIGN, typename C = double2>
struct FftxK {
  using R_ = typename Cplx<C>::R;
  struct Args {
    C* spec;
    const C* twx;
    long nrows;
    int nx;
    int px;  // fft_plan(nx)
    int R;
    R_ scale;
  };
  static constexpr int kThreads = 256;
  static constexpr int kMinBlocks = 4;  // shared memory limits residency to ~3 blocks anyway
  static Args make(C* spec, const C* twx, long nrows, int nx, int px, int R, R_ scale) { return Args{spec, twx, nrows, nx, px, R, scale}; }
  static __device__ __forceinline__ void run(const Args& a_, const dim3 bid_, const dim3 gdim_) {
    C* __restrict__ spec = a_.spec;
    const C* __restrict__ twx = a_.twx;
    long nrows = a_.nrows;
    int nx = a_.nx;
    int px = a_.px;
    int R = a_.R;
    R_ scale = a_.scale;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* A = reinterpret_cast<C*>(smem_raw);
  C* B = A + R * nx;
  const long row0 = (long)bid_.x * R;
  const int nr = (int)min((long)R, nrows - row0);
  C* g = spec + row0 * nx;
  for (int q = threadIdx.x; q < nr * nx; q += blockDim.x) A[q] = g[q];
  for (int q = nr * nx + threadIdx.x; q < R * nx; q += blockDim.x) A[q] = Cplx<C>::mk(0, 0);
  __syncthreads();
  C* Rb = stockham<SIGN, C>(A, B, nx, px, R, twx);
  if (scale == (R_)1) {
    for (int q = threadIdx.x; q < nr * nx; q += blockDim.x) g[q] = Rb[q];
  } else {
    for (int q = threadIdx.x; q < nr * nx; q += blockDim.x) {
      const C t = Rb[q];
      g[q] = Cplx<C>::mk(t.x * scale, t.y * scale);
    }
  }

  }
};

// The forward and backward sweeps of the y system of one (kx, kz) line (one of its real and
// imaginary parts), rows d[j * sd], with the factor planes finv (1/pivot) and fcp (c/pivot) and the
// sub-diagonal pa; T is the storage type of the spectrum (double, or float in the mixed form; the
// arithmetic is FP64).  The loads of the next U rows are issued before the current U rows are
// computed and stored (other rows, so no hazard), and their latency overlaps the recurrence.
__device__ __forceinline__ double tdma_cv(double x) { return x; }
__device__ __forceinline__ double tdma_cv(float x) { return f2d(x); }
__device__ __forceinline__ void tdma_st(double* p, double x) { *p = x; }
__device__ __forceinline__ void tdma_st(float* p, double x) { *p = d2f_rn(x); }

template <typename T, int U = 4>
__device__ __forceinline__ void tdma_line(T* d, long sd, const double* __restrict__ finv,
                                          const double* __restrict__ fcp, const double* __restrict__ pa, int nx,
                                          int ny, bool gauge) {
  // two register sets, A and B, take turns: no copies between them (a copy of a register whose
  // load is in flight would wait for it)
  // (the spectrum values stay in their storage type until used: a conversion right after the load
  // would wait for it)
  T Ad[U] = {}, Bd[U] = {};
  double Af[U] = {}, Aa[U] = {}, Bf[U] = {}, Ba[U] = {};
  auto load_f = [&](int j0, T* D, double* F, double* A) {
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (j0 + u < ny) {
        D[u] = d[(long)(j0 + u) * sd];
        F[u] = __ldg(finv + (long)(j0 + u) * nx);
        A[u] = __ldg(pa + j0 + u);  // a_0 = 0
      }
  };
  double prev = 0.0;
  auto sweep_f = [&](int j0, const T* D, const double* F, const double* A) {
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (j0 + u < ny) {
        const double dj = (gauge && j0 + u == 0) ? 0.0 : tdma_cv(D[u]);  // the gauge row phi_0 = 0
        prev = fma(-A[u], prev, dj) * F[u];
        tdma_st(d + (long)(j0 + u) * sd, prev);
      }
  };
  load_f(0, Ad, Af, Aa);
  for (int j0 = 0; j0 < ny; j0 += 2 * U) {
    load_f(j0 + U, Bd, Bf, Ba);
    sweep_f(j0, Ad, Af, Aa);
    load_f(j0 + 2 * U, Ad, Af, Aa);
    sweep_f(j0 + U, Bd, Bf, Ba);
  }
  double next = prev;
  auto load_b = [&](int j1, T* D, double* C) {
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (j1 - u >= 0) {
        D[u] = d[(long)(j1 - u) * sd];
        C[u] = __ldg(fcp + (long)(j1 - u) * nx);
      }
  };
  auto sweep_b = [&](int j1, const T* D, const double* C) {
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (j1 - u >= 0) {
        next = fma(-C[u], next, tdma_cv(D[u]));
        tdma_st(d + (long)(j1 - u) * sd, next);
      }
  };
  load_b(ny - 2, Ad, Af);
  for (int j1 = ny - 2; j1 >= 0; j1 -= 2 * U) {
    load_b(j1 - U, Bd, Bf);
    sweep_b(j1, Ad, Af);
    load_b(j1 - 2 * U, Ad, Af);
    sweep_b(j1 - U, Bd, Bf);
  }
}

// ------------------------------------------------------------------------------------------
// The FP32 x transform of the mixed form, persistent and double-buffered: each block walks
// batches of R contiguous rows; the next batch is copied into shared memory by asynchronous
// 16-byte copies (cp.async, waited for by cp.async.wait_group: no spin on a flag) while the
// current batch is transformed and stored.  Rows of a batch are consecutive in the spectrum,
// so a batch is one contiguous range (nx a multiple of 8: every row starts on 64 bytes).
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <int SIGN>
struct FftxPK {
  struct Args {
    float2* spec;
    const float2* twx;
    long nrows;
    int nx, px, R;
    long nbatch;
  };
  static constexpr int kThreads = 256;
  static constexpr int kMinBlocks = 2;
  static __device__ __forceinline__ void run(const Args& a, const dim3 bid_, const dim3 gdim_) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nx = a.nx, R = a.R;
    const int rn = R * nx;  // float2 per buffer
    float2* buf = reinterpret_cast<float2*>(smem_raw);  // [stage 0: data, scratch][stage 1: data, scratch]
    auto issue = [&](long b, int st) {
      if (b < a.nbatch) {
        const long row0 = b * R;
        const int nr = (int)min((long)R, a.nrows - row0);
        const float4* src = reinterpret_cast<const float4*>(a.spec + row0 * nx);
        float4* dst = reinterpret_cast<float4*>(buf + (2 * st) * rn);
        for (int q = threadIdx.x; q < (nr * nx) / 2; q += blockDim.x) cp_async16(dst + q, src + q);
      }
      cp_async_commit();  // a group per call, empty or not, so that the waits count alike
    };
    long b = bid_.x;
    issue(b, 0);
    for (int it = 0; b < a.nbatch; ++it, b += gdim_.x) {
      const int st = it & 1;
      issue(b + gdim_.x, st ^ 1);
      cp_async_wait<1>();  // every group but the newest: batch b has landed
      __syncthreads();
      const float2* X = stockham<SIGN, float2>(buf + (2 * st) * rn, buf + (2 * st + 1) * rn, nx, a.px, R, a.twx);
      const long row0 = b * R;
      const int nr = (int)min((long)R, a.nrows - row0);
      float2* g = a.spec + row0 * nx;
      for (int q = threadIdx.x; q < nr * nx; q += blockDim.x) g[q] = X[q];
      __syncthreads();  // stage st is read out before the next iteration refills it
    }
    cp_async_wait<0>();
  }
};

// The same line solve in FP32 arithmetic (mixed form, on the (kx, kz) modes pois_factor_kernel
// marks): factors 1/pivot and c/pivot are the FP64 ones rounded to float, a_j in float.  No gauge
// row: the (0, 0) mode always takes the FP64 solve.  Global: the factors and a_j are read through
// the read-only path (else they sit in shared memory); nx is the factors' row stride.
template <bool Global, int U>
__device__ __forceinline__ void tdma_line32(float* d, long sd, const float* __restrict__ finv,
                                            const float* __restrict__ fcp, const float* __restrict__ pa, int nx,
                                            int ny) {
  auto ld = [](const float* p) { return Global ? __ldg(p) : *p; };
  float Ad[U] = {}, Bd[U] = {}, Af[U] = {}, Aa[U] = {}, Bf[U] = {}, Ba[U] = {};
  auto load_f = [&](int j0, float* D, float* F, float* A) {
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (j0 + u < ny) {
        D[u] = d[(long)(j0 + u) * sd];
        F[u] = ld(finv + (long)(j0 + u) * nx);
        A[u] = ld(pa + j0 + u);  // a_0 = 0
      }
  };
  float prev = 0.0f;
  auto sweep_f = [&](int j0, const float* D, const float* F, const float* A) {
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (j0 + u < ny) {
        prev = __fmul_rn(__fmaf_rn(-A[u], prev, D[u]), F[u]);
        d[(long)(j0 + u) * sd] = prev;
      }
  };
  load_f(0, Ad, Af, Aa);
  for (int j0 = 0; j0 < ny; j0 += 2 * U) {
    load_f(j0 + U, Bd, Bf, Ba);
    sweep_f(j0, Ad, Af, Aa);
    load_f(j0 + 2 * U, Ad, Af, Aa);
    sweep_f(j0 + U, Bd, Bf, Ba);
  }
  float next = prev;
  auto load_b = [&](int j1, float* D, float* C) {
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (j1 - u >= 0) {
        D[u] = d[(long)(j1 - u) * sd];
        C[u] = ld(fcp + (long)(j1 - u) * nx);
      }
  };
  auto sweep_b = [&](int j1, const float* D, const float* C) {
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (j1 - u >= 0) {
        next = __fmaf_rn(-C[u], next, D[u]);
        d[(long)(j1 - u) * sd] = next;
      }
  };
  load_b(ny - 2, Ad, Af);
  for (int j1 = ny - 2; j1 >= 0; j1 -= 2 * U) {
    load_b(j1 - U, Bd, Bf);
    sweep_b(j1, Ad, Af);
    load_b(j1 - 2 * U, Ad, Af);
    sweep_b(j1 - U, Bd, Bf);
  }
}

// ------------------------------------------------------------------------------------------
// y tridiagonal per (kx, kz), two threads per line (real, imaginary part), factors 1/pivot and
// c/pivot precomputed in two planes (each sweep reads only the one it uses).
// ------------------------------------------------------------------------------------------
struct TdmaK {
  struct Args {
    double2* spec;
    const double2* fac;
    const double* gc;
    int nx;
    int ny;
    int nzh;
  };
  static constexpr int kThreads = 128;
  static constexpr int kMinBlocks = 4;  // nx*(nz/2+1) lines: occupancy is set by the line count, not registers
  static Args make(double2* spec, const double2* fac, const double* gc, int nx, int ny, int nzh) { return Args{spec, fac, gc, nx, ny, nzh}; }
  static __device__ __forceinline__ void run(const Args& a_, const dim3 bid_, const dim3 gdim_) {
    double2* __restrict__ spec = a_.spec;
    const double2* __restrict__ fac = a_.fac;
    const double* __restrict__ gc = a_.gc;
    int nx = a_.nx;
    int ny = a_.ny;

  // two threads per (kx, kz) line: the real and the imaginary part are independent systems
  // with the same real matrix (twice the parallelism of a thread per line, same traffic)
  const int t = bid_.x * blockDim.x + threadIdx.x;
  const int i = t >> 1, part = t & 1;
  const int kz = bid_.y;
  if (i >= nx) return;
  const long base = (long)kz * ny * nx + i;
  double* d = reinterpret_cast<double*>(spec + base) + part;
  const long sd = 2L * nx;  // row stride in doubles
  // factor planes: 1/pivot, then c/pivot (pois_factor_kernel), nzh * ny * nx doubles each
  const double* finv = reinterpret_cast<const double*>(fac) + base;
  const double* fcp = finv + (long)a_.nzh * ny * nx;
  const double* pa = gc + GC_PA * (ny + 1);
  // the (0,0) mode's row 0 is the gauge phi_0 = 0 (its factor row is 1, 0)
  tdma_line(d, sd, finv, fcp, pa, nx, ny, i == 0 && kz == 0);
  }
};

// ------------------------------------------------------------------------------------------
// inverse z FFT (complex-to-real on the half spectrum) -> phi.  Block = (x-tile, row j).
// ------------------------------------------------------------------------------------------
struct IfftzK {
  struct Args {
    const double2* spec;
    const double2* twz;
    double* phi;
    int nx;
    int ny;
    int nz;
    int pz;  // fft_plan(nz)
    int TX;
    double scale;
  };
  static constexpr int kThreads = 256;
  static constexpr int kMinBlocks = 4;  // shared memory limits residency to ~3 blocks anyway
  static Args make(const double2* spec, const double2* twz, double* phi, int nx, int ny, int nz, int pz, int TX, double scale) { return Args{spec, twz, phi, nx, ny, nz, pz, TX, scale}; }
  static __device__ __forceinline__ void run(const Args& a_, const dim3 bid_, const dim3 gdim_) {
    const double2* __restrict__ spec = a_.spec;
    const double2* __restrict__ twz = a_.twz;
    double* __restrict__ phi = a_.phi;
    int nx = a_.nx;
    int ny = a_.ny;
    int nz = a_.nz;
    int pz = a_.pz;
    int TX = a_.TX;
    double scale = a_.scale;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nseq = TX >> 1;
  double2* A = reinterpret_cast<double2*>(smem_raw);
  double2* B = A + nseq * nz;
  const int i0 = bid_.x * TX;
  const int j = bid_.y;
  const int nh = nz >> 1;
  // Z[m] = Xa[m] + i Xb[m] (m <= nz/2), Z[nz-m] = conj(Xa[m]) + i conj(Xb[m]); the m = 0 and
  // m = nz/2 coefficients of a real sequence are real, so only their real parts are used.
  for (int q = threadIdx.x; q < nseq * (nh + 1); q += blockDim.x) {
    const int c = q % nseq;
    const int m = q / nseq;
    const long o = ((long)m * ny + j) * nx + i0 + 2 * c;
    double2 xa = spec[o];
    double2 xb = spec[o + 1];
    if (m == 0 || m == nh) {
      xa.y = 0.0;
      xb.y = 0.0;
    }
    A[c * nz + m] = make_double2(xa.x - xb.y, xa.y + xb.x);
    if (m > 0 && m < nh) A[c * nz + nz - m] = make_double2(xa.x + xb.y, xb.x - xa.y);
  }
  __syncthreads();
  const double2* R = stockham<1>(A, B, nz, pz, nseq, twz);
  const long pl = (long)ny * nx;
  for (int q = threadIdx.x; q < TX * nz; q += blockDim.x) {
    const int il = q % TX;
    const int k = q / TX;
    const double2 t = R[(il >> 1) * nz + k];
    const double val = (il & 1) ? t.y : t.x;
    phi[k * pl + (long)j * nx + i0 + il] = (scale == 1.0) ? val : val * scale;
  }

  }
};

// ------------------------------------------------------------------------------------------
// The Poisson solve of the mixed form: FP32 transforms, one FP64 refinement.
//   pass 1: bs = D u* / (alpha_k dt nx nz) in FP64 (stored), its transforms in FP32 (complex64
//           spectrum), the y solves in FP64 arithmetic on that spectrum, phi1 = inverse (FP32)
//   pass 2: rs = bs - (D G phi1) / (nx nz) in FP64, with D G the operator the solve inverts
//           (periodic or Neumann x, the PA / PC rows in y, periodic z), the same FP32 pipeline on
//           rs, and phi = phi1 + phi2 in FP64
// The FP32 transforms leave relative errors near 1e-6 in phi1; the residual, formed in FP64 from
// the stored phi1, carries them into phi2, whose own FP32 error is then near 1e-12 of phi: the
// projected divergence stays at the level of the FP64 solve.  Conversions between FP64 and FP32
// go through the integer pipe (d2f_rn, f2d).
// ------------------------------------------------------------------------------------------
template <bool RES>
struct DivzMK {
  struct Args {
    const double* u;
    const double* v;
    const double* w;
    const double* gc;
    const float2* twz;
    float2* spec;
    double* bs;         // pass 1 writes it, pass 2 reads it
    const float* phi1;  // pass 2
    int nx, ny, nz, pz, TX, bl;
    double idx, idz, idx2, idz2, inv_nxnz;
    const StepK* sk;  // pscale = 1 / (alpha_k dt nx nz)
    const double* u_out;
  };
  static constexpr int kThreads = 256;
  static constexpr int kMinBlocks = 5;  // 48 registers: 5 blocks of 32 KB (0.173 -> 0.166 ms at 4 -> 5)
  static __device__ __forceinline__ void run(const Args& a, const dim3 bid_, const dim3) {
    const int nx = a.nx, ny = a.ny, nz = a.nz, TX = a.TX;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nseq = TX >> 1;
    float2* A = reinterpret_cast<float2*>(smem_raw);
    float2* B = A + nseq * nz;
    const int i0 = bid_.x * TX;
    const int j = bid_.y;
    const long pl = (long)ny * nx, plv = (long)(ny + 1) * nx;
    if (!RES) {
      const double scale = a.sk->pscale;
      const double idy = __ldg(a.gc + GC_IDY * (ny + 1) + j) * scale, idx = a.idx * scale, idz = a.idz * scale;
      for (int q = threadIdx.x; q < TX * nz; q += blockDim.x) {
        const int il = q % TX, k = q / TX, i = i0 + il;
        const int ip = (i + 1 == nx) ? 0 : i + 1;
        const int kp = (k + 1 == nz) ? 0 : k + 1;
        const long c = k * pl + (long)j * nx;
        const double uip = (a.u_out && i + 1 == nx) ? __ldg(a.u_out + (long)k * ny + j) : __ldg(a.u + c + ip);
        const double du = uip - __ldg(a.u + c + i);
        const double dv = __ldg(a.v + k * plv + (long)(j + 1) * nx + i) - __ldg(a.v + k * plv + (long)j * nx + i);
        const double dw = __ldg(a.w + kp * pl + (long)j * nx + i) - __ldg(a.w + c + i);
        const double b = fma(du, idx, fma(dv, idy, dw * idz));
        a.bs[c + i] = b;
        reinterpret_cast<float*>(A + (il >> 1) * nz + k)[il & 1] = 0.5f * d2f_rn(b);  // 1/2 of the unpack
      }
    } else {
      // rs = bs - (D G phi1) / (nx nz) with D G phi = idx2 (phi_E + phi_W) + idz2 (phi_U + phi_D)
      //   + PA_j phi_S + PC_j phi_N - (2 idx2 + 2 idz2 + PA_j + PC_j) phi; a missing neighbour (the
      //   Neumann x faces, the walls, where PA_0 = PC_{ny-1} = 0) takes the value phi itself, and
      //   the 1/(nx nz) is folded into the weights.  phi1 is FP32, so the stencil is summed in
      //   float-float arithmetic on the FP32 pipe (pair sums exact by TwoSum, products exact by
      //   TwoProd, weights split into two floats, error terms gathered in one float); only the
      //   final bs + S + C is FP64.  Its error is about 2^-46 of the largest stencil term.
      const double inv = a.inv_nxnz;
      const double paj = __ldg(a.gc + GC_PA * (ny + 1) + j), pcj = __ldg(a.gc + GC_PC * (ny + 1) + j);
      float wh[5], wl[5];
      {
        const double w[5] = {(2.0 * a.idx2 + 2.0 * a.idz2 + paj + pcj) * inv, a.idx2 * inv, a.idz2 * inv,
                             paj * inv, pcj * inv};
#pragma unroll
        for (int q = 0; q < 5; ++q) {
          wh[q] = d2f_rn(w[q]);
          wl[q] = d2f_rn(w[q] - f2d(wh[q]));
        }
      }
      const float* __restrict__ f = a.phi1;
      // two elements per thread and pass, their loads all issued before either is used
      constexpr int G = 2;
      const int nq = TX * nz;
      for (int q0 = threadIdx.x; q0 < nq; q0 += G * blockDim.x) {
      float F0[G], FE[G], FW[G], FS[G], FN[G], FU[G], FD[G];
      double BS[G];
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const int q = min(q0 + g * (int)blockDim.x, nq - 1);
        const int il = q % TX, k = q / TX, i = i0 + il;
        const long row = k * pl + (long)j * nx, cc = row + i;
        F0[g] = __ldg(f + cc);
        if (a.bl) {
          FE[g] = __ldg(f + cc + ((i + 1 < nx) ? 1 : 0));
          FW[g] = __ldg(f + cc - ((i > 0) ? 1 : 0));
        } else {
          FE[g] = __ldg(f + row + ((i + 1 == nx) ? 0 : i + 1));
          FW[g] = __ldg(f + row + ((i == 0) ? nx - 1 : i - 1));
        }
        FS[g] = __ldg(f + cc - (j > 0 ? nx : 0));
        FN[g] = __ldg(f + cc + (j + 1 < ny ? nx : 0));
        const int kp = (k + 1 == nz) ? 0 : k + 1, km = (k == 0) ? nz - 1 : k - 1;
        FU[g] = __ldg(f + kp * pl + (long)j * nx + i);
        FD[g] = __ldg(f + km * pl + (long)j * nx + i);
        BS[g] = __ldg(a.bs + cc);
      }
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const int q = q0 + g * blockDim.x;
        if (q >= nq) break;
        const int il = q % TX, k = q / TX;
        const float f0 = F0[g], fe = FE[g], fw = FW[g], fs = FS[g], fn = FN[g], fu = FU[g], fd = FD[g];
        float sxh, sxl, szh, szl;
        ff_two_sum(fe, fw, sxh, sxl);
        ff_two_sum(fu, fd, szh, szl);
        // S + C = w0 phi - wx sx - wz sz - wa phi_S - wc phi_N
        float S, C, p, e, t;
        ff_two_prod(wh[0], f0, S, C);
        C = __fmaf_rn(wl[0], f0, C);
        ff_two_prod(wh[1], sxh, p, e);
        e = __fmaf_rn(wh[1], sxl, __fmaf_rn(wl[1], sxh, e));
        ff_two_sum(S, -p, S, t);
        C = __fsub_rn(__fadd_rn(C, t), e);
        ff_two_prod(wh[2], szh, p, e);
        e = __fmaf_rn(wh[2], szl, __fmaf_rn(wl[2], szh, e));
        ff_two_sum(S, -p, S, t);
        C = __fsub_rn(__fadd_rn(C, t), e);
        ff_two_prod(wh[3], fs, p, e);
        e = __fmaf_rn(wl[3], fs, e);
        ff_two_sum(S, -p, S, t);
        C = __fsub_rn(__fadd_rn(C, t), e);
        ff_two_prod(wh[4], fn, p, e);
        e = __fmaf_rn(wl[4], fn, e);
        ff_two_sum(S, -p, S, t);
        C = __fsub_rn(__fadd_rn(C, t), e);
        const double r = (BS[g] + f2d(S)) + f2d(C);
        reinterpret_cast<float*>(A + (il >> 1) * nz + k)[il & 1] = 0.5f * d2f_rn(r);
      }
      }
    }
    __syncthreads();
    const float2* R = stockham<-1, float2>(A, B, nz, a.pz, nseq, a.twz);
    const int nh = (nz >> 1) + 1;
    for (int q = threadIdx.x; q < nh * TX; q += blockDim.x) {
      const int il = q % TX, m = q / TX, c = il >> 1;
      const float2 zm = R[c * nz + m];
      const float2 zn = R[c * nz + (m == 0 ? 0 : nz - m)];
      const float2 X = (il & 1) == 0 ? make_float2(zm.x + zn.x, zm.y - zn.y) : make_float2(zm.y + zn.y, zn.x - zm.x);
      a.spec[((long)m * ny + j) * nx + i0 + il] = X;
    }
  }
};

// y tridiagonal per (kx, kz) of the mixed form on the complex64 spectrum: FP64 arithmetic and
// factors (the same recurrences as TdmaK) on the kz = 0 modes and the ill-conditioned low modes,
// FP32 on the rest (mode[kz][kx] = 1, set by pois_factor_kernel)
struct TdmaMK {
  struct Args {
    float2* spec;
    const double2* fac;
    const double* gc;
    int nx, ny, nzh;
    const float* fac32;         // 1/pivot and c/pivot planes in float, nzh * ny * nx each
    const float* pa32;          // a_j in float
    const unsigned char* mode;  // nzh * nx: 1 = FP32 solve
  };
  static constexpr int kThreads = 128;
  static constexpr int kMinBlocks = 6;
  static __device__ __forceinline__ void run(const Args& a, const dim3 bid_, const dim3) {
    const int nx = a.nx, ny = a.ny;
    const int t = bid_.x * blockDim.x + threadIdx.x;
    const int i = t >> 1, part = t & 1;
    const int kz = bid_.y;
    if (i >= nx) return;
    const long base = (long)kz * ny * nx + i;
    float* d = reinterpret_cast<float*>(a.spec + base) + part;
    const long sd = 2L * nx;
    if (a.mode[(long)kz * nx + i]) {
      const float* f32 = a.fac32 + base;
      tdma_line32<true, 4>(d, sd, f32, f32 + (long)a.nzh * ny * nx, a.pa32, nx, ny);
      return;
    }
    const double* finv = reinterpret_cast<const double*>(a.fac) + base;
    const double* fcp = finv + (long)a.nzh * ny * nx;
    const double* pa = a.gc + GC_PA * (ny + 1);
    tdma_line(d, sd, finv, fcp, pa, nx, ny, i == 0 && kz == 0);
  }
};

// Float-float values h + l (|l| <= ulp(h) / 2 once renormalised), for the staged y solve's FP64
// tiles: the recurrences of those ill-conditioned modes carried in about 48 bits on the FP32 pipe
// (a warp's FP64 instruction streams through a unit of two lanes per clock, and a sweep's
// dependent FP64 operations set the launch's length).
struct FF {
  float h, l;
};
// Fast2Sum (|s| >= |e|, or s = 0)
__device__ __forceinline__ FF ff_norm(float s, float e) {
  const float h = __fadd_rn(s, e);
  return FF{h, __fsub_rn(e, __fsub_rn(h, s))};
}
// a b: the exact product of the high parts (TwoProd) plus the cross terms
__device__ __forceinline__ FF ff_mul(FF a, FF b) {
  float p, e;
  ff_two_prod(a.h, b.h, p, e);
  e = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, e));
  return ff_norm(p, e);
}
// x - b for a float x
__device__ __forceinline__ FF ff_sub(float x, FF b) {
  float s, e;
  ff_two_sum(x, -b.h, s, e);
  return ff_norm(s, __fsub_rn(e, b.l));
}

// Sweeps of the staged y solve's FP64 tiles over a range of rows, with the factor plane they
// read staged in shared memory as float-float pairs (f[(j - fo) * sf]: 1/pivot for the forward
// sweep, c/pivot for the backward one), a_j as rows[j].x + rows[j].w, and the spectrum column d
// (float, row stride sd).  Forward prev = (d_j - a_j prev) / pivot_j (the gauge row d_0 = 0),
// backward next = d_j - (c_j / pivot_j) next from the forward sweep's last value; each row is
// stored rounded to float (the high part).  prev / next carry from one range to the next.  Rows
// are loaded U ahead into two register sets taking turns.
template <int U>
__device__ __forceinline__ void tdma_fwd_ff(float* d, int sd, const float2* f, int fo, int sf, const float4* rows,
                                            int jb, int je, bool gauge, FF& prev) {
  float Ad[U] = {}, Bd[U] = {};
  float2 Af[U] = {}, Bf[U] = {}, Aa[U] = {}, Ba[U] = {};
  auto load = [&](int j0, float* D, float2* F, float2* A) {
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (j0 + u < je) {
        D[u] = d[(j0 + u) * sd];
        F[u] = f[(j0 + u - fo) * sf];
        const float4 r = rows[j0 + u];  // a_0 = 0
        A[u] = make_float2(r.x, r.w);
      }
  };
  auto sweep = [&](int j0, const float* D, const float2* F, const float2* A) {
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (j0 + u < je) {
        const float dj = (gauge && j0 + u == 0) ? 0.0f : D[u];  // the gauge row phi_0 = 0
        const FF t = ff_sub(dj, ff_mul(FF{A[u].x, A[u].y}, prev));
        prev = ff_mul(t, FF{F[u].x, F[u].y});
        d[(j0 + u) * sd] = prev.h;
      }
  };
  load(jb, Ad, Af, Aa);
  for (int j0 = jb; j0 < je; j0 += 2 * U) {
    load(j0 + U, Bd, Bf, Ba);
    sweep(j0, Ad, Af, Aa);
    load(j0 + 2 * U, Ad, Af, Aa);
    sweep(j0 + U, Bd, Bf, Ba);
  }
}

// rows jhi down to jlo
template <int U>
__device__ __forceinline__ void tdma_bwd_ff(float* d, int sd, const float2* f, int fo, int sf, int jlo, int jhi,
                                            FF& next) {
  float Ad[U] = {}, Bd[U] = {};
  float2 Ac[U] = {}, Bc[U] = {};
  auto load = [&](int j1, float* D, float2* C) {
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (j1 - u >= jlo) {
        D[u] = d[(j1 - u) * sd];
        C[u] = f[(j1 - u - fo) * sf];
      }
  };
  auto sweep = [&](int j1, const float* D, const float2* C) {
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (j1 - u >= jlo) {
        next = ff_sub(D[u], ff_mul(FF{C[u].x, C[u].y}, next));
        d[(j1 - u) * sd] = next.h;
      }
  };
  load(jhi, Ad, Ac);
  for (int j1 = jhi; j1 >= jlo; j1 -= 2 * U) {
    load(j1 - U, Bd, Bc);
    sweep(j1, Ad, Ac);
    load(j1 - 2 * U, Ad, Ac);
    sweep(j1 - U, Bd, Bc);
  }
}

// The FP32 sweep of one mode from its staged 1/pivot column (ip, stride sip: the FP64 factor
// rounded to float) and rows[j] = (a_j, c_j, ., .) in float (a_0 = 0, c_{ny-1} = 0): the forward
// sweep as tdma_line32, the backward one with c_j / pivot_j formed as c_j * ip_j in FP32 (one
// rounding more than the stored factor, which saves staging a second factor plane).
template <int U>
__device__ __forceinline__ void tdma_line32_ip(float* d, int sd, const float* ip, int sip, const float4* rows,
                                               int ny) {
  float Ad[U] = {}, Bd[U] = {}, Af[U] = {}, Bf[U] = {};
  float4 Ar[U] = {}, Br[U] = {};
  auto load_f = [&](int j0, float* D, float* F, float4* R) {
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (j0 + u < ny) {
        D[u] = d[(j0 + u) * sd];
        F[u] = ip[(j0 + u) * sip];
        R[u] = rows[j0 + u];
      }
  };
  float prev = 0.0f;
  auto sweep_f = [&](int j0, const float* D, const float* F, const float4* R) {
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (j0 + u < ny) {
        prev = __fmul_rn(__fmaf_rn(-R[u].x, prev, D[u]), F[u]);
        d[(j0 + u) * sd] = prev;
      }
  };
  load_f(0, Ad, Af, Ar);
  for (int j0 = 0; j0 < ny; j0 += 2 * U) {
    load_f(j0 + U, Bd, Bf, Br);
    sweep_f(j0, Ad, Af, Ar);
    load_f(j0 + 2 * U, Ad, Af, Ar);
    sweep_f(j0 + U, Bd, Bf, Br);
  }
  float next = prev;
  auto load_b = [&](int j1, float* D, float* F, float4* R) {
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (j1 - u >= 0) {
        D[u] = d[(j1 - u) * sd];
        F[u] = ip[(j1 - u) * sip];
        R[u] = rows[j1 - u];
      }
  };
  auto sweep_b = [&](int j1, const float* D, const float* F, const float4* R) {
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (j1 - u >= 0) {
        next = __fmaf_rn(-__fmul_rn(R[u].y, F[u]), next, D[u]);
        d[(j1 - u) * sd] = next;
      }
  };
  load_b(ny - 2, Ad, Af, Ar);
  for (int j1 = ny - 2; j1 >= 0; j1 -= 2 * U) {
    load_b(j1 - U, Bd, Bf, Br);
    sweep_b(j1, Ad, Af, Ar);
    load_b(j1 - 2 * U, Ad, Af, Ar);
    sweep_b(j1 - U, Bd, Bf, Br);
  }
}

// ------------------------------------------------------------------------------------------
// Staged y solve of the mixed form: a block of two warps takes a tile of TL consecutive kx of one
// kz.  The tile's spectrum columns, [ny][TL] complex64, are copied into shared memory (cp.async),
// one warp sweeps the TL lines (a lane per real / imaginary part) and the tile is written back.
// FP32 tiles (every mode kz > 0 with Skeel condition <= NS_POIS_FP32_KAPPA) also stage the float
// 1/pivot plane and form c/pivot from it (tdma_line32_ip).  (Factors formed in FP32 on the way,
// with no plane staged, lose accuracy in proportion to the Skeel condition: about 5e-6 instead of
// 2e-7 at 3600 on the stretched channel grid.)  FP64 tiles (kz = 0 and the ill-conditioned
// lowest modes; the n64 tiles first in the launch) read the FP64 factor planes, staged in shared
// memory half a plane at a time (1/pivot rows [0, hy), [hy, ny), then c/pivot rows [hy, ny),
// [0, hy)) and split there into float-float pairs, and sweep in float-float arithmetic
// (tdma_fwd_ff / tdma_bwd_ff).
// ------------------------------------------------------------------------------------------
struct TdmaSK {
  struct Args {
    float2* spec;
    const double* fac64;   // 1/pivot and c/pivot planes in FP64, nzh * ny * nx each
    const float* fac32;    // 1/pivot in float, nzh * ny * nx
    const float4* rows32;  // (a_j, c_j, -(a_j + c_j), a_j - (float)a_j) in float
    const int* tiles;      // tile q: kz * (nx / TL) + x tile; the n64 FP64 tiles first
    int n64;
    int nx, ny, nzh;
  };
  static constexpr int TL = 16;
  static constexpr int kThreads = 64;
  static constexpr int kMinBlocks = 5;
  // D [ny][TL] float2, then one region of ny * 80 + 64 bytes: FP32 tiles' 1/pivot [ny][TL] float
  // and rows [ny] float4; FP64 tiles' half factor plane [(ny + 1) / 2][TL] double (then float2
  // pairs in place) and rows [ny] float4
  static size_t smem_bytes(int ny) { return (size_t)ny * TL * 8 + (size_t)ny * 80 + 64; }
  static __device__ __forceinline__ void run(const Args& a, const dim3 bid_, const dim3) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nx = a.nx, ny = a.ny;
    const int ntx = nx / TL;
    const int tile = __ldg(a.tiles + bid_.x);
    const bool f64 = (int)bid_.x < a.n64;
    const int kz = tile / ntx, i0 = (tile - kz * ntx) * TL;
    float2* D = reinterpret_cast<float2*>(smem_raw);                     // [ny][TL]
    unsigned char* X = smem_raw + (size_t)ny * TL * 8;                   // the region
    float* IP = reinterpret_cast<float*>(X);                             // [ny][TL]
    float4* ROWS = reinterpret_cast<float4*>(X + (size_t)ny * TL * 4);   // [ny]
    double* F64 = reinterpret_cast<double*>(X);                          // [(ny + 1) / 2][TL]
    float2* F2 = reinterpret_cast<float2*>(X);                           // the same, split
    float4* ROWS64 = reinterpret_cast<float4*>(X + (size_t)((ny + 1) >> 1) * TL * 8);  // [ny]
    const long plane = (long)a.nzh * ny * nx;
    const long row0 = (long)kz * ny * nx + i0;
    constexpr int dq = TL * 8 / 16, gq = TL * 8 / 16, fq = TL * 4 / 16;  // 16-byte pieces per row of D, F64, IP
    for (int q = threadIdx.x; q < ny * dq; q += blockDim.x) {
      const int j = q / dq, r = q - j * dq;
      cp_async16(reinterpret_cast<float4*>(D + (size_t)j * TL) + r,
                 reinterpret_cast<const float4*>(a.spec + row0 + (long)j * nx) + r);
    }
    // rows [j0, j1) of an FP64 factor plane into F64
    auto stage64 = [&](const double* src, int j0, int j1) {
      for (int q = threadIdx.x; q < (j1 - j0) * gq; q += blockDim.x) {
        const int j = q / gq, r = q - j * gq;
        cp_async16(reinterpret_cast<float4*>(F64 + (size_t)j * TL) + r,
                   reinterpret_cast<const float4*>(src + row0 + (long)(j0 + j) * nx) + r);
      }
    };
    auto landed = [&]() {
      cp_async_commit();
      cp_async_wait<0>();
      __syncthreads();
    };
    // the staged rows [0, n) of F64 split in place into float-float pairs (x = h + l to about
    // 2^-48 of x)
    auto split = [&](int n) {
      for (int q = threadIdx.x; q < n * TL; q += blockDim.x) {
        const double x = F64[q];
        const float h = __double2float_rn(x);
        F2[q] = make_float2(h, __double2float_rn(x - (double)h));
      }
      __syncthreads();
    };
    const int hy = (ny + 1) >> 1;
    if (f64) {
      stage64(a.fac64, 0, hy);
      for (int j = threadIdx.x; j < ny; j += blockDim.x) cp_async16(ROWS64 + j, a.rows32 + j);
    } else {
      for (int q = threadIdx.x; q < ny * fq; q += blockDim.x) {
        const int j = q / fq, r = q - j * fq;
        cp_async16(reinterpret_cast<float4*>(IP + (size_t)j * TL) + r,
                   reinterpret_cast<const float4*>(a.fac32 + row0 + (long)j * nx) + r);
      }
      for (int j = threadIdx.x; j < ny; j += blockDim.x) cp_async16(ROWS + j, a.rows32 + j);
    }
    landed();
    const int l = threadIdx.x >> 1, part = threadIdx.x & 1;
    float* d = reinterpret_cast<float*>(D) + 2 * l + part;  // row stride 2 TL floats
    const bool sweeper = threadIdx.x < 2 * TL;
    if (f64) {
      const bool gauge = kz == 0 && i0 + l == 0;  // the (0, 0) mode's row 0: phi_0 = 0
      FF v{0.0f, 0.0f};
      split(hy);
      if (sweeper) tdma_fwd_ff<8>(d, 2 * TL, F2 + l, 0, TL, ROWS64, 0, hy, gauge, v);
      __syncthreads();
      stage64(a.fac64, hy, ny);
      landed();
      split(ny - hy);
      if (sweeper) tdma_fwd_ff<8>(d, 2 * TL, F2 + l, hy, TL, ROWS64, hy, ny, gauge, v);
      __syncthreads();
      stage64(a.fac64 + plane, hy, ny);
      landed();
      split(ny - hy);
      if (sweeper) tdma_bwd_ff<8>(d, 2 * TL, F2 + l, hy, TL, hy, ny - 2, v);
      __syncthreads();
      stage64(a.fac64 + plane, 0, hy);
      landed();
      split(hy);
      if (sweeper) tdma_bwd_ff<8>(d, 2 * TL, F2 + l, 0, TL, 0, min(hy - 1, ny - 2), v);
    } else if (sweeper) {
      tdma_line32_ip<8>(d, 2 * TL, IP + l, TL, ROWS, ny);
    }
    __syncthreads();
    for (int q = threadIdx.x; q < ny * dq; q += blockDim.x) {
      const int j = q / dq, r = q - j * dq;
      reinterpret_cast<float4*>(a.spec + row0 + (long)j * nx)[r] = reinterpret_cast<const float4*>(D + (size_t)j * TL)[r];
    }
  }
};

// inverse z transform of the mixed form (complex-to-real, FP32): pass 1 stores phi1 (FP32);
// pass 2 (ACC) adds its result to phi1 in FP64 and writes phi
template <bool ACC>
struct IfftzMK {
  struct Args {
    const float2* spec;
    const float2* twz;
    float* phi1;
    double* phi;
    int nx, ny, nz, pz, TX;
  };
  static constexpr int kThreads = 256;
  static constexpr int kMinBlocks = 4;
  static __device__ __forceinline__ void run(const Args& a, const dim3 bid_, const dim3) {
    const int nx = a.nx, ny = a.ny, nz = a.nz, TX = a.TX;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nseq = TX >> 1;
    float2* A = reinterpret_cast<float2*>(smem_raw);
    float2* B = A + nseq * nz;
    const int i0 = bid_.x * TX;
    const int j = bid_.y;
    const int nh = nz >> 1;
    const long pl = (long)ny * nx;
    // ACC: the tile of phi1 this block adds to ([nz][TX] floats after A, B) is copied in at once
    // (cp.async), so that the output loop does not wait on a global load per element
    float* P1 = reinterpret_cast<float*>(B + nseq * nz);
    if (ACC) {
      if ((TX & 3) == 0) {
        const int pr = TX >> 2;  // 16-byte pieces per row
        for (int q = threadIdx.x; q < nz * pr; q += blockDim.x) {
          const int k = q / pr, r = q - k * pr;
          cp_async16(reinterpret_cast<float4*>(P1 + k * TX) + r,
                     reinterpret_cast<const float4*>(a.phi1 + k * pl + (long)j * nx + i0) + r);
        }
        cp_async_commit();
      } else {
        for (int q = threadIdx.x; q < nz * TX; q += blockDim.x)
          P1[q] = a.phi1[(q / TX) * pl + (long)j * nx + i0 + q % TX];
      }
    }
    // spectrum loads in groups of four per thread, all issued before any is used
    constexpr int G = 4;
    const int nq = nseq * (nh + 1);
    for (int q0 = threadIdx.x; q0 < nq; q0 += G * blockDim.x) {
      float2 xa[G], xb[G];
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const int q = q0 + g * blockDim.x;
        if (q < nq) {
          const int c = q % nseq, m = q / nseq;
          const long o = ((long)m * ny + j) * nx + i0 + 2 * c;
          xa[g] = a.spec[o];
          xb[g] = a.spec[o + 1];
        }
      }
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const int q = q0 + g * blockDim.x;
        if (q < nq) {
          const int c = q % nseq, m = q / nseq;
          if (m == 0 || m == nh) {
            xa[g].y = 0.0f;
            xb[g].y = 0.0f;
          }
          A[c * nz + m] = make_float2(xa[g].x - xb[g].y, xa[g].y + xb[g].x);
          if (m > 0 && m < nh) A[c * nz + nz - m] = make_float2(xa[g].x + xb[g].y, xb[g].x - xa[g].y);
        }
      }
    }
    if (ACC) cp_async_wait<0>();
    __syncthreads();
    const float2* R = stockham<1, float2>(A, B, nz, a.pz, nseq, a.twz);
    for (int q = threadIdx.x; q < TX * nz; q += blockDim.x) {
      const int il = q % TX, k = q / TX;
      const float2 t = R[(il >> 1) * nz + k];
      const float val = (il & 1) ? t.y : t.x;
      const long cc = k * pl + (long)j * nx + i0 + il;
      if (ACC) a.phi[cc] = f2d(P1[q]) + f2d(val);
      else a.phi1[cc] = val;
    }
  }
};

// ------------------------------------------------------------------------------------------
// projection u = u* - s G phi; p += phi (if update_p).  One thread per (i, j) of kZ consecutive
// z-planes, j = 0..ny.
// ------------------------------------------------------------------------------------------
// Dyn: sx, sz, s, beta_p from device memory, else from the arguments; KM: the Kim-Moin pressure
// update (compiled only into the variants that use it)
template <bool Dyn, bool KM>
struct ProjectK {
  struct Args {
    double* u;
    double* v;
    double* w;
    double* p;
    const double* phi;
    const double* gc;
    int nx;
    int ny;
    int nz;
    const StepK* sk;  // sx, sz, s and the Kim-Moin beta_p (0: p += phi)
    double sx, sz, s, beta_p;  // the same as arguments
    int update_p;
    int bl;
    double idx2, idz2;
  };
  static constexpr int kThreads = 128;
  static constexpr int kMinBlocks = KM ? 8 : 12;  // the Kim-Moin update reads six more neighbours
  static constexpr int kZ = 4;  // z planes per thread (nz is a multiple of 8)
  static Args make(double* u, double* v, double* w, double* p, const double* phi, const double* gc, int nx, int ny, int nz, const StepK* sk, const StepK& kc, int update_p, int bl, double idx2, double idz2) { return Args{u, v, w, p, phi, gc, nx, ny, nz, sk, kc.sx, kc.sz, kc.s, kc.beta_p, update_p, bl, idx2, idz2}; }
  static __device__ __forceinline__ void run(const Args& a_, const dim3 bid_, const dim3 gdim_) {
    double* __restrict__ u = a_.u;
    double* __restrict__ v = a_.v;
    double* __restrict__ w = a_.w;
    double* __restrict__ p = a_.p;
    const double* __restrict__ phi = a_.phi;
    const double* __restrict__ gc = a_.gc;
    int nx = a_.nx;
    int ny = a_.ny;
    int nz = a_.nz;
    const double sx = Dyn ? a_.sk->sx : a_.sx;
    const double sz = Dyn ? a_.sk->sz : a_.sz;
    int update_p = a_.update_p;
    const double s = Dyn ? a_.sk->s : a_.s;
    const double beta_p = Dyn ? a_.sk->beta_p : a_.beta_p;
    int bl = a_.bl;

  const long plane = (long)nx * (ny + 1);
  const long q = (long)bid_.x * blockDim.x + threadIdx.x;
  if (q >= plane) return;
  const int j = (int)(q / nx);
  const int i = (int)(q - (long)j * nx);
  if (j >= ny) return;  // the top wall row of v: nothing to update
  const int im = (i == 0) ? nx - 1 : i - 1;
  const long pl = (long)ny * nx, vpl = (long)(ny + 1) * nx;
  const long row = (long)j * nx;
  const double sv = j >= 1 ? s * __ldg(gc + GC_IHC * (ny + 1) + j) : 0.0;  // v: s / hc_j
  // kZ consecutive z planes per thread: phi of the plane below carries over to the w update
  const int k0 = bid_.y * kZ;
  double fprev = __ldg(phi + (k0 == 0 ? nz - 1 : k0 - 1) * pl + row + i);
#pragma unroll 1
  for (int kk = 0; kk < kZ; ++kk) {
    const int k = k0 + kk;
    const long cc = k * pl + row + i;
    const double f0 = __ldg(phi + cc);
    if (!(bl && i == 0)) u[cc] -= sx * (f0 - __ldg(phi + k * pl + row + im));  // inflow face fixed
    w[cc] -= sz * (f0 - fprev);
    if (j >= 1) v[k * vpl + row + i] -= sv * (f0 - __ldg(phi + cc - nx));
    if (update_p) {
      double dp = f0;
      if (KM && beta_p != 0.0) {
        // Kim-Moin: p += phi - beta_k (D G phi), with G phi = 0 on the walls (PA_0 = PC_{ny-1} = 0)
        // and, with inflow / outflow, on the x = 0 and x = Lx faces
        const long rk = k * pl + row;
        double lx;
        if (bl) {
          const double ge = (i + 1 < nx) ? __ldg(phi + rk + i + 1) - f0 : 0.0;
          const double gw = (i > 0) ? f0 - __ldg(phi + rk + i - 1) : 0.0;
          lx = (ge - gw) * a_.idx2;
        } else {
          const int ip = (i + 1 == nx) ? 0 : i + 1;
          lx = ((__ldg(phi + rk + ip) - f0) - (f0 - __ldg(phi + rk + im))) * a_.idx2;
        }
        const double ly = (j > 0 ? __ldg(gc + GC_PA * (ny + 1) + j) * (__ldg(phi + cc - nx) - f0) : 0.0) +
                          (j + 1 < ny ? __ldg(gc + GC_PC * (ny + 1) + j) * (__ldg(phi + cc + nx) - f0) : 0.0);
        const int kp = (k + 1 == nz) ? 0 : k + 1;
        const double lz = ((__ldg(phi + kp * pl + row + i) - f0) - (f0 - fprev)) * a_.idz2;
        dp = f0 - beta_p * (lx + ly + lz);
      }
      p[cc] += dp;
    }
    fprev = f0;
  }

  }
};

// ------------------------------------------------------------------------------------------
// cosine transform along x (inflow / outflow): DCT-II  X_l = sum_i x_i cos(pi l (2i+1) / (2N)) of
// each complex row (real and imaginary parts independently), by one complex FFT of length N
// (Makhoul 1980): v = (x_0, x_2, ..., x_3, x_1), V = FFT(v); with V_a, V_b the transforms of
// the real and imaginary parts of v (separated through V_{N-l}), X_l = Re(w_l V_a) + i Re(w_l V_b),
// w_l = exp(-i pi l / (2N)).  Inverse (unnormalised, N times the DCT-III inverse):
// V_l = conj(w_l) (X_l - i X_{N-l}) (X_N = 0), v = IFFT(V), x_{2n} = v_n, x_{2n+1} = v_{N-1-n}.
// twd holds w_l for l < N and then w_l / 2: the forward kernel takes the halved entries, which
// absorb the 1/2 of the real / imaginary separation exactly (a power of two).
// ------------------------------------------------------------------------------------------
template <typename C>
__global__ void __launch_bounds__(256) dctx_fwd_kernel(C* __restrict__ spec, const C* __restrict__ twx,
                                                       const C* __restrict__ twd, long nrows, int nx, int px,
                                                       int R) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* A = reinterpret_cast<C*>(smem_raw);
  C* B = A + R * nx;
  const long row0 = (long)blockIdx.x * R;
  const int nr = (int)min((long)R, nrows - row0);
  C* g = spec + row0 * nx;
  for (int q = threadIdx.x; q < R * nx; q += blockDim.x) {
    const int rr = q / nx, i = q - rr * nx;
    const int dst = (i & 1) ? nx - 1 - (i >> 1) : (i >> 1);
    A[rr * nx + dst] = rr < nr ? g[q] : Cplx<C>::mk(0, 0);
  }
  __syncthreads();
  const C* V = stockham<-1, C>(A, B, nx, px, R, twx);
  for (int q = threadIdx.x; q < nr * nx; q += blockDim.x) {
    const int rr = q / nx, l = q - rr * nx;
    const C vl = V[rr * nx + l];
    const C vn = V[rr * nx + (l == 0 ? 0 : nx - l)];
    const C w = __ldg(twd + nx + l);  // w_l / 2
    using R_ = typename Cplx<C>::R;
    const R_ ax = vl.x + vn.x, ay = vl.y - vn.y;
    const R_ bx = vl.y + vn.y, by = vn.x - vl.x;
    g[q] = Cplx<C>::mk(fmaT(w.x, ax, -w.y * ay), fmaT(w.x, bx, -w.y * by));
  }
}

template <typename C>
__global__ void __launch_bounds__(256) dctx_inv_kernel(C* __restrict__ spec, const C* __restrict__ twx,
                                                       const C* __restrict__ twd, long nrows, int nx, int px,
                                                       int R) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* A = reinterpret_cast<C*>(smem_raw);
  C* B = A + R * nx;
  const long row0 = (long)blockIdx.x * R;
  const int nr = (int)min((long)R, nrows - row0);
  C* g = spec + row0 * nx;
  for (int q = threadIdx.x; q < R * nx; q += blockDim.x) {
    const int rr = q / nx, l = q - rr * nx;
    C v = Cplx<C>::mk(0, 0);
    if (rr < nr) {
      const C xl = g[q];
      const C xn = l == 0 ? Cplx<C>::mk(0, 0) : g[rr * nx + nx - l];
      const C w = __ldg(twd + l);
      const auto ax = xl.x + xn.y, ay = xl.y - xn.x;  // X_l - i X_{N-l}
      v = Cplx<C>::mk(fmaT(w.x, ax, w.y * ay), fmaT(w.x, ay, -w.y * ax));  // conj(w) (..)
    }
    A[q] = v;
  }
  __syncthreads();
  const C* X = stockham<1, C>(A, B, nx, px, R, twx);
  for (int q = threadIdx.x; q < nr * nx; q += blockDim.x) {
    const int rr = q / nx, i = q - rr * nx;
    const int src = (i & 1) ? nx - 1 - (i >> 1) : (i >> 1);
    g[q] = X[rr * nx + src];
  }
}

// ------------------------------------------------------------------------------------------
// convective outflow dF/dt + U_c dF/dx = 0 on the outflow planes: one upwind step of
// alpha_k dt; the interior neighbour is the last u face (distance dx) or the last v, w centre
// (distance dx/2).  Writes the new planes and their increments.
// ------------------------------------------------------------------------------------------
__global__ void outflow_kernel(const double* __restrict__ u, const double* __restrict__ v,
                               const double* __restrict__ w, double* __restrict__ u_out, double* __restrict__ v_out,
                               double* __restrict__ w_out, double* __restrict__ du, double* __restrict__ dv,
                               double* __restrict__ dw, int nx, int ny, int nz, const StepK* __restrict__ sk) {
  const double cu = sk->cu, cv = sk->cv;
  const long nu = (long)nz * ny, nv = (long)nz * (ny + 1);
  for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < 2 * nu + nv; q += (long)gridDim.x * blockDim.x) {
    if (q < nu) {
      const double old = u_out[q];
      const double nb = __ldg(u + q * nx + nx - 1);  // plane index q = k * ny + j
      const double nw = old - cu * (old - nb);
      du[q] = nw - old;
      u_out[q] = nw;
    } else if (q < nu + nv) {
      const long e = q - nu;
      const int j = (int)(e % (ny + 1));
      const double old = v_out[e];
      double nw = 0.0;
      if (j > 0 && j < ny) nw = old - cv * (old - __ldg(v + e * nx + nx - 1));
      dv[e] = nw - old;
      v_out[e] = nw;
    } else {
      const long e = q - nu - nv;
      const double old = w_out[e];
      const double nw = old - cv * (old - __ldg(w + e * nx + nx - 1));
      dw[e] = nw - old;
      w_out[e] = nw;
    }
  }
}

// ------------------------------------------------------------------------------------------
// outflow mass-flux correction: u_out += (Q_in - Q_out) / (Ly Lz) with Q = sum u dy_j dz over the
// inflow face (face 0 of u) and the outflow plane.  One block, fixed reduction order.
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) flux_correct_kernel(const double* __restrict__ u, double* __restrict__ u_out,
                                                            const double* __restrict__ gc, int nx, int ny, int nz,
                                                            double dz_over_area, double* __restrict__ flux) {
  __shared__ double red[1024];
  const double* dy = gc + GC_DY * (ny + 1);
  const long n = (long)nz * ny;
  double acc = 0.0;
  for (long q = threadIdx.x; q < n; q += blockDim.x) {
    const int j = (int)(q % ny);
    acc += (__ldg(u + q * nx) - u_out[q]) * __ldg(dy + j);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s2 = blockDim.x / 2; s2 > 0; s2 >>= 1) {
    if (threadIdx.x < s2) red[threadIdx.x] += red[threadIdx.x + s2];
    __syncthreads();
  }
  const double corr = red[0] * dz_over_area;
  for (long q = threadIdx.x; q < n; q += blockDim.x) u_out[q] += corr;
  if (threadIdx.x == 0 && flux) flux[1] = corr;
}

// ------------------------------------------------------------------------------------------
// convective rate max over cells of |u| (1/dx) + |v_c| (1/dy_j) + |w| (1/dz) (u, w on the cell's
// lower faces, v_c the mean of its two y faces), the measure of the fixed-CFL time step.  The
// value of a cell that can be the maximum is computed with its products and sums rounded one by
// one (no contraction), so the maximum equals the plain definition.  Values are >= 0, so their
// bit patterns order like the values and one atomicMax per block on the bits combines the blocks
// in any order.  A non-finite value stores the bits of a NaN (above every finite value).
//
// Screening: the FP64 pipe is the scarce unit, so each cell first gets an upper bound of its
// value on the integer and FP32 pipes, from the high words of the doubles (every magnitude
// truncated to 20 fraction bits as a float, a lower bound within 2^-20; magnitudes below 2^-126
// as 0, above 2^128 or non-finite as inf).  The bound adds the slack of those truncations and of
// the float and double roundings with a margin (a factor 1 + 2^-14 and 1e-30).  A cell whose bound
// is below an exact value already found (the running maximum of the block) cannot be the maximum
// and skips the exact evaluation; a warp evaluates exactly only when one of its lanes needs it.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ float trunc_mag(unsigned hi) {  // |x| from the high word, truncated
  const unsigned h = hi & 0x7FFFFFFFu;
  unsigned b = (h - 0x38000000u) << 3;  // binary64 exponent e -> binary32 exponent e - 896
  b = h < 0x38100000u ? 0u : b;         // |x| < 2^-126
  b = h >= 0x47F00000u ? 0x7F800000u : b;  // |x| >= 2^128, inf, NaN
  return __uint_as_float(b);
}

__global__ void __launch_bounds__(128) rate_kernel(const double* __restrict__ u, const double* __restrict__ v,
                                                   const double* __restrict__ w, const double* __restrict__ gc,
                                                   int nx, int ny, int nz, double ix, double iz,
                                                   unsigned long long* __restrict__ out) {
  // ix = 1/dx, iz = 1/dz and the rows 1/dy_j (GC_IDY) are rounded on the host
  __shared__ unsigned long long s_max;  // bits of the block's running maximum
  if (threadIdx.x == 0) s_max = 0ull;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float ixf = trunc_mag((unsigned)__double2hiint(ix)), izf = trunc_mag((unsigned)__double2hiint(iz));
  double m = 0.0;
  float mf = 0.0f;  // a float <= m
  bool bad = false;
  for (int row = blockIdx.x; row < ny * nz; row += gridDim.x) {
    const int k = row / ny, j = row - k * ny;
    const double iy = __ldg(gc + GC_IDY * (ny + 1) + j);
    const float iyf = trunc_mag((unsigned)__double2hiint(iy));
    const long c0 = ((long)k * ny + j) * nx;
    const long v0 = ((long)k * (ny + 1) + j) * nx;
    const unsigned long long bm = *(volatile unsigned long long*)&s_max;
    if (bm > (unsigned long long)__double_as_longlong(m)) {
      m = __longlong_as_double((long long)bm);
      mf = __double2float_rd(m);
    }
    for (int i0 = warp * 32; i0 < nx; i0 += blockDim.x) {
      const int i = i0 + lane;
      const bool in = i < nx;
      double du = 0.0, dw = 0.0, dv0 = 0.0, dv1 = 0.0;
      if (in) {
        du = __ldg(u + c0 + i);
        dw = __ldg(w + c0 + i);
        dv0 = __ldg(v + v0 + i);
        dv1 = __ldg(v + v0 + nx + i);
      }
      const unsigned h0 = (unsigned)__double2hiint(dv0), h1 = (unsigned)__double2hiint(dv1);
      const float f0 = __uint_as_float(__float_as_uint(trunc_mag(h0)) | (h0 & 0x80000000u));
      const float f1 = __uint_as_float(__float_as_uint(trunc_mag(h1)) | (h1 & 0x80000000u));
      const float avh = fabsf(f0 + f1) + 0x1p-18f * (fabsf(f0) + fabsf(f1));
      const float rh = (trunc_mag((unsigned)__double2hiint(du)) * ixf + 0.5f * avh * iyf +
                        trunc_mag((unsigned)__double2hiint(dw)) * izf) * (1.0f + 0x1p-14f) + 1e-30f;
      const bool cand = in && !(rh < mf);
      if (__any_sync(NS_FULL_MASK, cand)) {
        if (cand) {
          const double au = fabs(du), aw = fabs(dw);
          const double av = fabs(__dmul_rn(0.5, __dadd_rn(dv0, dv1)));
          const double r = __dadd_rn(__dadd_rn(__dmul_rn(au, ix), __dmul_rn(av, iy)), __dmul_rn(aw, iz));
          bad |= !(r <= 1.7976931348623157e308);
          m = fmax(m, r);
        }
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(NS_FULL_MASK, m, o));
        mf = __double2float_rd(m);
        if (lane == 0) atomicMax(&s_max, (unsigned long long)__double_as_longlong(m));
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    m = fmax(m, __shfl_xor_sync(NS_FULL_MASK, m, o));
    bad |= __shfl_xor_sync(NS_FULL_MASK, (int)bad, o) != 0;
  }
  __shared__ double sm[4];
  __shared__ int sb[4];
  if (lane == 0) {
    sm[warp] = m;
    sb[warp] = bad;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < (int)(blockDim.x >> 5); ++q) {
      m = fmax(m, sm[q]);
      bad |= sb[q] != 0;
    }
    atomicMax(out, bad ? 0x7FF8000000000000ull : (unsigned long long)__double_as_longlong(m));
  }
}

// ------------------------------------------------------------------------------------------
// factor table of the y systems: per (kx, kz, j): (1/pivot_j, c_j/pivot_j).  Init only.
// The mixed form (fac32 != null) also gets the factors rounded to float and one flag per mode:
// FP32 y solves where kz > 0 and the Skeel condition number of the mode's matrix A,
// kappa = || |A^-1| |A| 1 ||_inf, is at most kappa_max.  -A is an M-matrix (a_j, c_j >= 0 and
// a diagonal larger by lam), so |A^-1| |A| 1 = y with -A y = |A| 1, |A| 1 = 2 (a_j + c_j) + lam,
// found by one more solve with the FP64 factors (scratch: the FP64 spectrum, idle at init).  The
// kz = 0 modes (the gauge among them) and the ill-conditioned lowest modes keep FP64 arithmetic.
// ------------------------------------------------------------------------------------------
__global__ void pois_factor_kernel(double2* __restrict__ fac, const double* __restrict__ gc,
                                   const double* __restrict__ lamx, const double* __restrict__ lamz, int nx, int ny,
                                   int nzh, float* __restrict__ fac32, unsigned char* __restrict__ mode,
                                   double* __restrict__ scratch, double kappa_max) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int kz = blockIdx.y;
  if (i >= nx || kz >= nzh) return;
  const double* pa = gc + GC_PA * (ny + 1);
  const double* pc = gc + GC_PC * (ny + 1);
  const double lam = lamx[i] + lamz[kz];
  const bool gauge = (i == 0 && kz == 0);
  double cprev = 0.0;
  for (int j = 0; j < ny; ++j) {
    double a = pa[j], c = pc[j];
    double b = -(a + c) - lam;
    if (gauge && j == 0) {
      a = 0.0;
      b = 1.0;
      c = 0.0;
    }
    const double piv = b - a * cprev;
    const double ip = 1.0 / piv;
    cprev = c * ip;
    // two planes of one double each: 1/pivot (forward sweep) and c/pivot (back sweep)
    double* f = reinterpret_cast<double*>(fac);
    const long q = ((long)kz * ny + j) * nx + i;
    f[q] = ip;
    f[(long)nzh * ny * nx + q] = cprev;
    if (fac32) {
      fac32[q] = (float)ip;
      fac32[(long)nzh * ny * nx + q] = (float)cprev;
    }
  }
  if (!fac32) return;
  bool fp32 = false;
  if (kz > 0) {
    const double* f = reinterpret_cast<const double*>(fac);
    double prev = 0.0;
    for (int j = 0; j < ny; ++j) {  // A y' = -|A| 1, y = -y'
      const long q = ((long)kz * ny + j) * nx + i;
      prev = (-(2.0 * (pa[j] + pc[j]) + lam) - pa[j] * prev) * f[q];
      scratch[q] = prev;
    }
    double kappa = fabs(prev);
    for (int j = ny - 2; j >= 0; --j) {
      const long q = ((long)kz * ny + j) * nx + i;
      prev = scratch[q] - f[(long)nzh * ny * nx + q] * prev;
      kappa = fmax(kappa, fabs(prev));
    }
    fp32 = kappa <= kappa_max;
  }
  mode[(long)kz * nx + i] = fp32 ? 1 : 0;
}

}  // namespace

cudaError_t poisson_set_attributes() {
  set_smem_limit<DivzK>(200 * 1024);
  set_smem_limit<DivzMK<false>>(200 * 1024);
  set_smem_limit<DivzMK<true>>(200 * 1024);
  set_smem_limit<IfftzMK<false>>(200 * 1024);
  set_smem_limit<IfftzMK<true>>(200 * 1024);
  set_smem_limit<IfftzK>(200 * 1024);
  set_smem_limit<FftxK<-1>>(200 * 1024);
  set_smem_limit<FftxK<1>>(200 * 1024);
  set_smem_limit<FftxPK<-1>>(200 * 1024);
  set_smem_limit<FftxPK<1>>(200 * 1024);
  set_smem_limit<TdmaSK>(NS_SMEM_MAX);
  cudaFuncSetAttribute(dctx_fwd_kernel<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(dctx_inv_kernel<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  return cudaGetLastError();
}

cudaError_t launch_convective_rate(ns_ctx* c) {
  cudaError_t e = cudaMemsetAsync(c->rate, 0, sizeof(unsigned long long), c->launch);
  if (e != cudaSuccess) return e;
  const int rows = c->cfg.ny * c->cfg.nz;
  const int blocks = rows < 16 * c->num_sms ? rows : 16 * c->num_sms;
  rate_kernel<<<blocks, 128, 0, c->launch>>>(c->f.u, c->f.v, c->f.w, c->gc, c->cfg.nx, c->cfg.ny, c->cfg.nz,
                                             1.0 / c->dx, 1.0 / c->dz, c->rate);
  return cudaGetLastError();
}

size_t pois_staged_smem(int ny) { return TdmaSK::smem_bytes(ny); }
int pois_staged_tile() { return TdmaSK::TL; }

cudaError_t launch_pois_factor(ns_ctx* c, const double* lamx, const double* lamz) {
  dim3 grid((c->cfg.nx + 127) / 128, c->nzh);
  pois_factor_kernel<<<grid, 128, 0, c->launch>>>(c->pois, c->gc, lamx, lamz, c->cfg.nx, c->cfg.ny, c->nzh,
                                                  c->pois32 ? c->pois_f32 : nullptr, c->pois_mode,
                                                  reinterpret_cast<double*>(c->spec), NS_POIS_FP32_KAPPA);
  return cudaGetLastError();
}

static int z_tile(int nz) {
  // complex sequences of length nz: keep 2 * (TX/2) * nz * 16 B <= 64 KB
  int tx = 16;
  while (tx > 2 && (size_t)tx * nz * 16 > 64 * 1024) tx >>= 1;
  return tx;
}

namespace {
struct PoisShape {
  int nx, ny, nz, pz, px, TX, R, TXm;
  size_t smz, smx;
  long nrows;
  unsigned bx;
};
PoisShape pois_shape(const ns_ctx* c) {
  PoisShape q;
  q.nx = c->cfg.nx;
  q.ny = c->cfg.ny;
  q.nz = c->cfg.nz;
  q.pz = fft_plan(q.nz);
  q.px = fft_plan(q.nx);
  q.TX = z_tile(q.nz);
  while (q.nx % q.TX) q.TX >>= 1;  // TX divides nx (nx is a multiple of 8)
  q.smz = (size_t)q.TX * q.nz * sizeof(double2);  // two buffers of TX/2 sequences
  // the FP32 z transforms of the mixed form (complex64): TX nz 8 bytes <= 32 KB, but at least 8
  // columns while that stays within 160 KB; 4-column tiles of long lines leave those kernels far
  // from their bounds (2048x288x1024 divergence + z FFT 15.9 -> 8.4 ms at 8 columns; wider tiles
  // are slower at every size measured)
  q.TXm = 16;
  while (q.TXm > 2 && (size_t)q.TXm * q.nz * 8 > 32 * 1024) q.TXm >>= 1;
  if (q.TXm < 8 && (size_t)8 * q.nz * 8 <= 160 * 1024) q.TXm = 8;
  while (q.nx % q.TXm) q.TXm >>= 1;
  q.nrows = (long)c->nzh * q.ny;
  q.R = 1;
  while (q.R < 16 && (size_t)2 * q.R * 2 * q.nx * sizeof(double2) <= 64 * 1024) q.R <<= 1;
  q.smx = (size_t)2 * q.R * q.nx * sizeof(double2);
  q.bx = (unsigned)((q.nrows + q.R - 1) / q.R);
  return q;
}
// the mixed form's FP32 pipeline: spectrum (complex64) over the dead increments r_u, r_v; phi1 in
// r_w; the FP64 right-hand side bs in the FP64 spectrum block
float2* sp32(const ns_ctx* c) { return reinterpret_cast<float2*>(c->ru); }
float* phi1(const ns_ctx* c) { return reinterpret_cast<float*>(c->rw); }
double* bs64(const ns_ctx* c) { return reinterpret_cast<double*>(c->spec); }

template <bool RES>
cudaError_t emit_divzm(LaunchSink& s, int k) {
  ns_ctx* c = s.c;
  const PoisShape q = pois_shape(c);
  typename DivzMK<RES>::Args a;
  a.u = c->f.u;
  a.v = c->f.v;
  a.w = c->f.w;
  a.gc = c->gc;
  a.twz = c->twz32;
  a.spec = sp32(c);
  a.bs = bs64(c);
  a.phi1 = phi1(c);
  a.nx = q.nx;
  a.ny = q.ny;
  a.nz = q.nz;
  a.pz = q.pz;
  a.TX = q.TX;
  a.bl = c->bl;
  a.idx = 1.0 / c->dx;
  a.idz = 1.0 / c->dz;
  a.idx2 = 1.0 / (c->dx * c->dx);
  a.idz2 = 1.0 / (c->dz * c->dz);
  a.inv_nxnz = 1.0 / ((double)q.nx * q.nz);
  a.sk = c->stepk + stepk_index(k);
  a.u_out = c->bl ? c->f.u_out : nullptr;
  a.TX = q.TXm;
  return emit<DivzMK<RES>>(s, a, dim3(q.nx / q.TXm, q.ny), dim3(256), (size_t)q.TXm * q.nz * sizeof(float2));
}

cudaError_t emit_xm(LaunchSink& s, bool fwd) {
  ns_ctx* c = s.c;
  const PoisShape q = pois_shape(c);
  if (c->bl) {
    if (fwd)
      dctx_fwd_kernel<float2><<<q.bx, 256, q.smx / 2, c->launch>>>(sp32(c), c->twx32, c->twd32, q.nrows, q.nx, q.px, q.R);
    else
      dctx_inv_kernel<float2><<<q.bx, 256, q.smx / 2, c->launch>>>(sp32(c), c->twx32, c->twd32, q.nrows, q.nx, q.px, q.R);
    return cudaGetLastError();
  }
  if (s.plan) {  // batched ensembles: many small instances fill the GPU with one batch per block
    if (fwd)
      return emit<FftxK<-1, float2>>(s, FftxK<-1, float2>::make(sp32(c), c->twx32, q.nrows, q.nx, q.px, q.R, 1.0f),
                                     dim3(q.bx), dim3(256), q.smx / 2);
    return emit<FftxK<1, float2>>(s, FftxK<1, float2>::make(sp32(c), c->twx32, q.nrows, q.nx, q.px, q.R, 1.0f),
                                  dim3(q.bx), dim3(256), q.smx / 2);
  }
  // single instance: persistent, double-buffered: R rows per batch with 4 buffers of R nx float2
  // in shared memory
  int R = 1;
  while (R < 4 && (size_t)4 * 2 * R * q.nx * sizeof(float2) <= 64 * 1024) R <<= 1;
  const long nbatch = (q.nrows + R - 1) / R;
  const size_t smem = (size_t)4 * R * q.nx * sizeof(float2);
  int bps = 1;
  const cudaError_t oe = fwd ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, single_kernel<FftxPK<-1>>, 256, smem)
                             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, single_kernel<FftxPK<1>>, 256, smem);
  if (oe != cudaSuccess) return oe;
  const long blocks = std::min(nbatch, (long)std::max(bps, 1) * c->num_sms);
  if (fwd)
    return emit<FftxPK<-1>>(s, FftxPK<-1>::Args{sp32(c), c->twx32, q.nrows, q.nx, q.px, R, nbatch}, dim3((unsigned)blocks),
                            dim3(256), smem);
  return emit<FftxPK<1>>(s, FftxPK<1>::Args{sp32(c), c->twx32, q.nrows, q.nx, q.px, R, nbatch}, dim3((unsigned)blocks),
                         dim3(256), smem);
}

cudaError_t emit_tdmam(LaunchSink& s) {
  ns_ctx* c = s.c;
  const PoisShape q = pois_shape(c);
  if (c->pois_tiles)  // staged: the FP64 tiles, then the FP32 ones, in one launch
    return emit<TdmaSK>(s,
                        TdmaSK::Args{sp32(c), reinterpret_cast<const double*>(c->pois), c->pois_f32, c->pois_rows32,
                                     c->pois_tiles, c->ntile64, q.nx, q.ny, c->nzh},
                        dim3((unsigned)(c->ntile64 + c->ntile32)), dim3(TdmaSK::kThreads), TdmaSK::smem_bytes(q.ny));
  return emit<TdmaMK>(s, TdmaMK::Args{sp32(c), c->pois, c->gc, q.nx, q.ny, c->nzh, c->pois_f32, c->pois_pa32, c->pois_mode},
                      dim3((2 * q.nx + 127) / 128, c->nzh), dim3(128), 0);
}

template <bool ACC>
cudaError_t emit_ifftzm(LaunchSink& s) {
  ns_ctx* c = s.c;
  const PoisShape q = pois_shape(c);
  return emit<IfftzMK<ACC>>(s, typename IfftzMK<ACC>::Args{sp32(c), c->twz32, phi1(c), c->phi, q.nx, q.ny, q.nz, q.pz,
                                                           q.TXm},
                            dim3(q.nx / q.TXm, q.ny), dim3(256),
                            (size_t)q.TXm * q.nz * (sizeof(float2) + (ACC ? sizeof(float) : 0)));
}

void single_kernel_dct_fwd(ns_ctx* c, unsigned bx, size_t smx, long nrows, int nx, int px, int R) {
  dctx_fwd_kernel<double2><<<bx, 256, smx, c->launch>>>(c->spec, c->twx, c->twd, nrows, nx, px, R);
}
void single_kernel_dct_inv(ns_ctx* c, unsigned bx, size_t smx, long nrows, int nx, int px, int R) {
  dctx_inv_kernel<double2><<<bx, 256, smx, c->launch>>>(c->spec, c->twx, c->twd, nrows, nx, px, R);
}
}  // namespace

// A5: divergence of u* scaled by 1/(alpha_k dt) (1 if k < 0) + forward real FFT along z
cudaError_t stage_pois_divz(LaunchSink& s, int k) {
  ns_ctx* c = s.c;
  if (c->pois32) return emit_divzm<false>(s, k);
  const PoisShape q = pois_shape(c);
  // 1/(alpha_k dt) of the right-hand side and 1/(nx nz) of the inverse transforms, applied once
  // (StepK::pscale)
  return emit<DivzK>(s, DivzK::make(c->f.u, c->f.v, c->f.w, c->gc, c->twz, c->spec, q.nx, q.ny, q.nz, q.pz, q.TX,
                                    1.0 / c->dx, 1.0 / c->dz, c->stepk + stepk_index(k),
                                    c->bl ? c->f.u_out : nullptr),
                     dim3(q.nx / q.TX, q.ny), dim3(256), q.smz);
}

// A6: forward complex FFT along x (periodic) or DCT-II (inflow / outflow; single instance only)
cudaError_t stage_pois_x_fwd(LaunchSink& s, int) {
  ns_ctx* c = s.c;
  if (c->pois32) return emit_xm(s, true);
  const PoisShape q = pois_shape(c);
  if (c->bl) {
    single_kernel_dct_fwd(c, q.bx, q.smx, q.nrows, q.nx, q.px, q.R);
    return cudaGetLastError();
  }
  return emit<FftxK<-1>>(s, FftxK<-1>::make(c->spec, c->twx, q.nrows, q.nx, q.px, q.R, 1.0), dim3(q.bx), dim3(256),
                         q.smx);
}

// A7: complex tridiagonal solve along y per (kx, kz)
cudaError_t stage_pois_tdma(LaunchSink& s, int) {
  ns_ctx* c = s.c;
  if (c->pois32) return emit_tdmam(s);
  const PoisShape q = pois_shape(c);
  return emit<TdmaK>(s, TdmaK::make(c->spec, c->pois, c->gc, q.nx, q.ny, c->nzh), dim3((2 * q.nx + 127) / 128, c->nzh),
                     dim3(128), 0);
}

// A8: inverse complex FFT along x (the 1/(nx nz) was applied to the right-hand side)
cudaError_t stage_pois_x_inv(LaunchSink& s, int) {
  ns_ctx* c = s.c;
  if (c->pois32) return emit_xm(s, false);
  const PoisShape q = pois_shape(c);
  if (c->bl) {
    single_kernel_dct_inv(c, q.bx, q.smx, q.nrows, q.nx, q.px, q.R);
    return cudaGetLastError();
  }
  return emit<FftxK<1>>(s, FftxK<1>::make(c->spec, c->twx, q.nrows, q.nx, q.px, q.R, 1.0), dim3(q.bx), dim3(256),
                        q.smx);
}

// A9: inverse real FFT along z -> phi
cudaError_t stage_pois_ifftz(LaunchSink& s, int) {
  ns_ctx* c = s.c;
  if (c->pois32) return emit_ifftzm<false>(s);
  const PoisShape q = pois_shape(c);
  return emit<IfftzK>(s, IfftzK::make(c->spec, c->twz, c->phi, q.nx, q.ny, q.nz, q.pz, q.TX, 1.0),
                      dim3(q.nx / q.TX, q.ny), dim3(256), q.smz);
}

// A9b (mixed form only): the FP64 residual of phi1 and the second FP32 solve, phi = phi1 + phi2
cudaError_t stage_pois_refine(LaunchSink& s, int k) {
  if (!s.c->pois32) return cudaSuccess;
  cudaError_t e;
  if ((e = emit_divzm<true>(s, k)) != cudaSuccess || (e = emit_xm(s, true)) != cudaSuccess ||
      (e = emit_tdmam(s)) != cudaSuccess || (e = emit_xm(s, false)) != cudaSuccess)
    return e;
  return emit_ifftzm<true>(s);
}

template <bool Dyn, bool KM>
cudaError_t emit_project(LaunchSink& s, int q, int k) {
  ns_ctx* c = s.c;
  const int nx = c->cfg.nx, ny = c->cfg.ny, nz = c->cfg.nz;
  const long plane = (long)nx * (ny + 1);
  dim3 grid((unsigned)((plane + 127) / 128), nz / ProjectK<Dyn, KM>::kZ);
  return emit<ProjectK<Dyn, KM>>(s, ProjectK<Dyn, KM>::make(c->f.u, c->f.v, c->f.w, c->f.p, c->phi, c->gc, nx, ny, nz,
                                                            c->stepk + q, c->stepk_h[q], k >= 0 ? 1 : 0, c->bl,
                                                            1.0 / (c->dx * c->dx), 1.0 / (c->dz * c->dz)),
                                 grid, dim3(128), 0);
}

// A10: projection u = u* - alpha_k dt G phi, p += phi (or the Kim-Moin form)
cudaError_t stage_project(LaunchSink& s, int k) {
  ns_ctx* c = s.c;
  const int q = stepk_index(k);
  const bool km = c->cfg.pressure_update == NS_PRESSURE_KIM_MOIN;
  if (c->dyn_consts) return km ? emit_project<true, true>(s, q, k) : emit_project<true, false>(s, q, k);
  return km ? emit_project<false, true>(s, q, k) : emit_project<false, false>(s, q, k);
}

#define NS_SINGLE_LAUNCH(name, stage)   \
  cudaError_t name(ns_ctx* c, int k) {  \
    LaunchSink s{c, nullptr};           \
    return stage(s, k);                 \
  }
NS_SINGLE_LAUNCH(launch_pois_divz, stage_pois_divz)
NS_SINGLE_LAUNCH(launch_pois_fftx_fwd, stage_pois_x_fwd)
NS_SINGLE_LAUNCH(launch_pois_tdma, stage_pois_tdma)
NS_SINGLE_LAUNCH(launch_pois_fftx_inv, stage_pois_x_inv)
NS_SINGLE_LAUNCH(launch_pois_ifftz, stage_pois_ifftz)
NS_SINGLE_LAUNCH(launch_pois_refine, stage_pois_refine)
NS_SINGLE_LAUNCH(launch_project, stage_project)
#undef NS_SINGLE_LAUNCH

cudaError_t launch_poisson(ns_ctx* c, int k) {
  cudaError_t e;
  if ((e = launch_pois_divz(c, k)) != cudaSuccess) return e;
  if ((e = launch_pois_fftx_fwd(c, k)) != cudaSuccess) return e;
  if ((e = launch_pois_tdma(c, k)) != cudaSuccess) return e;
  if ((e = launch_pois_fftx_inv(c, k)) != cudaSuccess) return e;
  if ((e = launch_pois_ifftz(c, k)) != cudaSuccess) return e;
  return launch_pois_refine(c, k);
}

cudaError_t launch_outflow(ns_ctx* c, int k) {
  if (!c->bl) return cudaSuccess;
  const int nx = c->cfg.nx, ny = c->cfg.ny, nz = c->cfg.nz;
  const long n = 2L * nz * ny + (long)nz * (ny + 1);
  const unsigned blocks = (unsigned)min((n + 255) / 256, 4096L);
  outflow_kernel<<<blocks, 256, 0, c->launch>>>(c->f.u, c->f.v, c->f.w, c->f.u_out, c->f.v_out, c->f.w_out,
                                                c->dout[0], c->dout[1], c->dout[2], nx, ny, nz, c->stepk + k);
  return cudaGetLastError();
}

cudaError_t launch_flux_correct(ns_ctx* c, int) {
  if (!c->bl) return cudaSuccess;
  const int ny = c->cfg.ny;
  const double area = (c->yf[ny] - c->yf[0]) * c->cfg.lz;
  flux_correct_kernel<<<1, 1024, 0, c->launch>>>(c->f.u, c->f.u_out, c->gc, c->cfg.nx, ny, c->cfg.nz,
                                                 c->dz / area, c->flux);
  return cudaGetLastError();
}
