// Internal declarations shared by the CUDA translation units of the library.
#pragma once
#include <cmath>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <utility>
#include <algorithm>
#include <vector>

#include "../../include/ns.h"

// FFT plan of a length N = 2^a 3^b: a | (b << 8), or -1 for any other N.
inline __host__ __device__ int fft_plan(int N) {
  if (N < 1) return -1;
  int a = 0, b = 0;
  while (N % 2 == 0) N /= 2, ++a;
  while (N % 3 == 0) N /= 3, ++b;
  return N == 1 ? (a | (b << 8)) : -1;
}

// Doubles in the twiddle table of a length-N FFT (fft_twiddles): six per entry, N entries.
inline size_t fft_twiddle_doubles(int N) { return 6 * (size_t)N; }

// Twiddles of the DIT stages of the shared-memory FFT in FMA form (Goedecker's tangent
// factorisation), one entry of six doubles per (stage, k), at index Ns + k, where Ns is the
// length of the sub-transforms the stage combines and k < Ns.  The stage order is a radix-2
// stage (Ns = 1, no twiddles) when a is odd, a/2 radix-4 stages, then b radix-3 stages; the index
// ranges [Ns, 2 Ns) of the stages are disjoint and end below 2N/3.
//   radix 4, th = 2 pi k / (4 Ns): {tan th, cos th}, {tan 2th, cos 2th}, {tan 3th, cos 3th / cos th}
//   radix 3, th = 2 pi k / (3 Ns): {tan th, cos th}, {tan 2th, cos 2th / cos th},
//                                  {cos th / 2, (sqrt 3 / 2) cos th}
// out has room for fft_twiddle_doubles(N); unused entries are zero.
inline void fft_twiddles(int N, double* out) {
  const double PI = 3.14159265358979323846;
  const double S3 = 0.86602540378443864676;
  for (size_t q = 0; q < fft_twiddle_doubles(N); ++q) out[q] = 0.0;
  const int plan = fft_plan(N);
  if (plan < 0) return;
  const int a = plan & 0xff, b = plan >> 8;
  int Ns = (a & 1) ? 2 : 1;
  for (int s = 0; s < (a >> 1); ++s, Ns *= 4)
    for (int k = 0; k < Ns && Ns > 1; ++k) {
      const double th = 2.0 * PI * k / (4.0 * Ns);
      const double c1 = std::cos(th), c2 = std::cos(2.0 * th), c3 = std::cos(3.0 * th);
      double* e = out + 6 * (size_t)(Ns + k);
      e[0] = std::tan(th);
      e[1] = c1;
      e[2] = std::tan(2.0 * th);
      e[3] = c2;
      e[4] = std::tan(3.0 * th);
      e[5] = c3 / c1;
    }
  for (int s = 0; s < b; ++s, Ns *= 3)
    for (int k = 0; k < Ns && Ns > 1; ++k) {
      const double th = 2.0 * PI * k / (3.0 * Ns);
      const double c1 = std::cos(th), c2 = std::cos(2.0 * th);
      double* e = out + 6 * (size_t)(Ns + k);
      e[0] = std::tan(th);
      e[1] = c1;
      e[2] = std::tan(2.0 * th);
      e[3] = c2 / c1;
      e[4] = 0.5 * c1;
      e[5] = S3 * c1;
    }
}

// Partition shapes the x solver is built for: P lanes (a power of two <= 32) of M rows, with
// M <= 16 from {1, 2, 3, 4, 6, 8, 9, 12, 16} (rows in registers) or, at P = 32, the long-line
// shapes M in {24, 32, 48, 64, 96, 128} (lines staged in shared memory; nx up to 4096).
inline bool x_partition_ok(int P, int M) {
  if (P < 1 || P > 32 || (P & (P - 1)) != 0) return false;
  switch (M) {
    case 1: case 2: case 3: case 4: case 6: case 8: case 9: case 12: case 16: return true;
    case 24: case 32: case 48: case 64: case 96: case 128: return P == 32;
    default: return false;
  }
}

// (P, M) shapes built for the partitioned y and z lines of the mixed form (AdiLinePK): n = P M
// rows, P partitions of M rows held in registers by a block of 32 lines x P.
inline bool line_part_ok(int P, int M) {
  if (P == 8) return M == 4 || M == 6 || M == 8 || M == 12 || M == 16 || M == 24 || M == 32;
  if (P == 16) return M == 18 || M == 32;
  if (P == 32) return M == 32;
  return false;
}
inline int line_partition(int n) {
  for (int P = 8; P <= 32; P <<= 1)
    if (n % P == 0 && line_part_ok(P, n / P)) return P;
  return 0;
}

// Default partition count of an x line of nx rows: the largest admissible P with at least 8 rows
// per partition, else the smallest admissible P; 0 if none is admissible.
inline int x_default_partition(int nx) {
  for (int P = 32; P >= 1; P >>= 1)
    if (nx % P == 0 && nx / P >= 8 && x_partition_ok(P, nx / P)) return P;
  for (int P = 1; P <= 32; P <<= 1)
    if (nx % P == 0 && x_partition_ok(P, nx / P)) return P;
  return 0;
}

#define NS_FULL_MASK 0xffffffffu

// ---------------------------------------------------------------------------------------------
// Grid coefficient block (device, double): NS_GC_COUNT arrays of (ny + 1) entries each.
//   DY, IDY    : cell height dy_j = yf_{j+1} - yf_j and its inverse (j < ny)
//   HC, IHC    : centre spacing across face j, hc_j = yc_j - yc_{j-1}, and inverse (1 <= j < ny)
//   WLO, WHI   : linear-interpolation weights of centres j-1 and j at face j (1 <= j < ny)
//   AC, CC     : y second-derivative weights of the lower / upper neighbour at centre j
//                (three-point non-uniform formula, exact for quadratics; the wall neighbour
//                 value is 0; CC = 0 at a stress-free top)
//   AF, CF     : the same weights at interior face j (1 <= j < ny)
//   PA, PC     : Poisson y rows 1/(dy_j hc_j) and 1/(dy_j hc_{j+1}) (zero at the boundaries)
// ---------------------------------------------------------------------------------------------
enum { GC_DY = 0, GC_IDY, GC_HC, GC_IHC, GC_WLO, GC_WHI, GC_AC, GC_CC, GC_AF, GC_CF, GC_PA, GC_PC,
       NS_GC_COUNT };

// Per-(sub-step, j) assembly coefficients of the tiled RHS (double, RT_COUNT rows of ny + 1),
// every factor pre-multiplied by dt: with cl = dt alpha_k / Re,
//   AC/CC/DC : cl A_j, cl C_j, -cl (2/dx^2 + 2/dz^2 + A_j + C_j) at centres (AC, CC of GC_*)
//   AF/CF/DF : the same at interior faces (AF, CF of GC_*)
//   CGY      : -dt alpha_k / hc_j (pressure gradient at face j)
//   QIHC     : cn / (4 hc_j), with cn = -dt gamma_k
//   RHO      : WHI / WLO of interior face j (the y-face fluxes are formed as
//              (f_{j-1} + RHO f_j)(g + g'), i.e. divided by WLO_j; zero off the interior faces)
//   HYM, HYP : -cn WLO_j / (2 dy_j) and cn WLO_{j+1} / (2 dy_j) at centre j: the weights of those
//              fluxes on the faces below and above (WLO zero at the walls)
//   HXW, HZW : cn WLO_j / (2 dx) and cn WLO_j / (2 dz) at interior face j: their weights in the
//              x and z differences of v
enum { RT_AC = 0, RT_CC, RT_DC, RT_AF, RT_CF, RT_DF, RT_CGY, RT_QIHC, RT_HYM, RT_HYP, RT_HXW, RT_HZW, RT_RHO,
       RT_COUNT };

// Constants of the tiled RHS in StepK::kd / kf: quarter and half inverse spacings in x and z times
// the convection weight cn = -dt gamma_k (the RHS forms and stores N pre-multiplied by cn), cn
// itself, the weight zeta_k / gamma_(k-1) of the stored N of the previous sub-step, the pressure-
// gradient and viscous weights -dt alpha_k / dx, -dt alpha_k / dz, dt alpha_k / (Re dx^2),
// dt alpha_k / (Re dz^2), and the body force dt alpha_k fx.
enum { RK_QIDX, RK_QIDZ, RK_HIDX, RK_HIDZ, RK_CN, RK_CP, RK_CGX, RK_CGZ, RK_CX, RK_CZ, RK_CB };

// RK3 constants (Sec. 2.2): gamma, zeta, alpha = gamma + zeta.
static const double NS_GAMMA[3] = {8.0 / 15.0, 5.0 / 12.0, 3.0 / 4.0};
static const double NS_ZETA[3] = {0.0, -17.0 / 60.0, -5.0 / 12.0};
static const double NS_ALPHA[3] = {8.0 / 15.0, 2.0 / 15.0, 1.0 / 3.0};

// ---------------------------------------------------------------------------------------------
// Partitioned x-line solver tables (Sec. 3.2), one per sub-step, element type T.
// P partitions of M rows; L = log2(P) reduction levels (0 for PDD).
//   [0 .. 5MP)         : per (field f, row e, partition r) at (f*M + e)*P + r, fields
//                        INV (1/pivot), AINV (a/pivot), CP (c/pivot) of the block Thomas
//                        factorisation of A~, and the spikes V, W (Eq. blockAY)
//   [5MP .. 5MP+4P)    : inverse of the final 2x2 diagonal block of interface r, [4][P]
//   then L levels of ML [4][P] and L levels of MU [4][P]: block eliminators of the reduced
//   system (block parallel cyclic reduction across partitions, precomputed because the
//   matrix is the same for every line)
// ---------------------------------------------------------------------------------------------
enum { XT_INV = 0, XT_AINV, XT_CP, XT_V, XT_W, XT_NF };
__host__ __device__ inline size_t xtab_count(int M, int P, int L) {
  return (size_t)XT_NF * M * P + 4 * (size_t)P + 8 * (size_t)L * P;
}

struct ns_layout {
  size_t off[32];
  size_t total;
};

enum {
  LB_RU = 0, LB_RV, LB_RW, LB_NU, LB_NV, LB_NW, LB_PHI, LB_SPEC, LB_POIS, LB_GC, LB_XTAB, LB_YTAB,
  LB_ZTAB, LB_TWZ, LB_TWX, LB_LAMX, LB_LAMZ, LB_RTAB, LB_DOUT, LB_TWD, LB_RCY, LB_STEPK, LB_PTAB, LB_TW32, LB_DT,
  LB_POIS32, LB_COUNT
};

// dt-dependent constants of one RK3 sub-step (entries 0..2) and of the projection of an initial
// field (entry 3).  They live in device memory, so a new dt reaches every kernel of a captured
// step without capturing it again.
struct StepK {
  double dt;          // the time step
  double kd[11];      // tiled RHS constants in double (RhsTiledK)
  float kf[12];       // the same rounded to float (11 used)
  double pscale;      // divergence scale 1 / (alpha_k dt nx nz) (1 / (nx nz) for entry 3)
  double sx, sz, s;   // projection: alpha_k dt / dx, alpha_k dt / dz, alpha_k dt
  double beta_p;      // Kim-Moin beta_k (0 with the plain pressure update)
  double cu, cv;      // convective outflow: alpha_k dt U_c / dx and / (dx / 2)
  double xcf[3];      // outflow increment weights of the x sweep (u, v, w): r, 2r, 2r, r = beta_k / dx^2
  float xcff[4];      // the same in float (3 used)
  int L;              // reduction levels of the x solve (0: PDD)
  int Ly, Lz;         // the same for the partitioned y and z lines of the mixed form
  int xhalf[2];       // x tables of class 0 (u) / 1 (v, w): 1 if every spike v^(r)_e of the back
                      // half of a partition and w^(r)_e of the front half is below the truncation
                      // tolerance (x_half_tol), so each row takes one correction only
};
constexpr int NS_STEPK = 4;

inline size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// Control block of the fixed-CFL steps whose dt is set on the device (k_dt.cu): the host writes
// cfl, dt (the current one), count = status = 0 before a run of at most NS_DTLOG steps; each step
// logs the dt it used.  status: 0, 1 (a non-finite convective rate) or 2 (a zero rate) at step
// fail_step, which then keeps the previous dt.
constexpr int NS_DTLOG = 1024;
struct DtCtl {
  double cfl;
  double dt;
  unsigned count, status, fail_step, pad;
  double dts[NS_DTLOG];
};

struct ns_ctx {
  ns_config cfg;
  std::vector<double> yf;
  ns_fields f;
  cudaStream_t stream;      // caller's stream
  cudaStream_t launch;      // where stage launches go (caller's stream, or the capture stream)
  cudaStream_t cap_stream;  // private stream used for graph capture
  void* ws;
  size_t ws_bytes;
  bool own_ws;
  ns_layout lay;
  int es;                   // bytes per element of r / N (8 FP64, 4 mixed)
  int nzh;                  // nz/2 + 1
  double dx, dz;
  // device pointers (into ws)
  void *ru, *rv, *rw, *nu, *nv, *nw;
  double* phi;
  double2* spec;
  double2* pois;
  double* gc;
  void* xtab[3][2];         // x-solver tables per sub-step: [0] u-class, [1] v/w-class (same when
                            // periodic; differ at the inflow / outflow rows otherwise)
  void* ytab[3][2];
  void* ztab[3];
  // partitioned y and z lines of the mixed form (0: thread per line): P per direction, the
  // levels per sub-step, and the tables [k][0 y centres, 1 y faces, 2 z]
  int yP = 0, zP = 0;
  int yL[3] = {0, 0, 0}, zL[3] = {0, 0, 0};
  void* ptab[3][3] = {};
  double ypdd_drop = 0.0, zpdd_drop = 0.0;
  double2* twz;
  double2* twx;
  double* rtab[3];
  float* rtabf[3];          // float copies of rtab for the FP32 form
  int bl;                   // inflow / convective outflow in x
  double* dout[3];          // outflow-plane increments of the current sub-step (u, v, w)
  double2* twd;             // exp(-i pi l / (2 nx)), l < nx, then the same halved: x cosine transform twiddles
  // the mixed form's Poisson solve: FP32 transforms (twiddles rounded to float) and one FP64
  // refinement (k_poisson.cu); off for FP64 contexts
  bool pois32 = false;
  float2 *twz32 = nullptr, *twx32 = nullptr, *twd32 = nullptr;
  // its y solves: the FP64 factors rounded to float (two planes; the staged form reads only the
  // first), a_j in float, and one flag per (kz, kx) mode, 1 where the solve runs in FP32
  // (pois_factor_kernel)
  float* pois_f32 = nullptr;
  float* pois_pa32 = nullptr;
  unsigned char* pois_mode = nullptr;
  // the staged y solve's tiles of pois_staged_tile() kx (nx a multiple of it, a tile within
  // shared memory): the ntile64 tiles holding a mode that takes FP64, then the ntile32 others;
  // null: the register form
  int* pois_tiles = nullptr;
  int ntile32 = 0, ntile64 = 0;
  // the staged y solve's rows (a_j, c_j, -(a_j + c_j), a_j - (float)a_j) in float: the FP32
  // sweeps form c/pivot from them, the FP64 tiles take a_j as a float-float pair
  float4* pois_rows32 = nullptr;
  double* flux;             // [0]: inflow flux, [1]: last outflow correction (diagnostics)
  unsigned long long* rate; // bits of the convective rate of ns_convective_rate (in the flux block)
  std::vector<double> gc_h; // host copy of the grid coefficients (tables are rebuilt when dt changes)
  double* rcy;              // recycling inflow: sample heights, plane means, gamma (k_recycle.cu)
  StepK* stepk;             // device: dt-dependent constants per sub-step (NS_STEPK entries)
  StepK stepk_h[NS_STEPK];  // host image of stepk
  // ns_set_dt stages the rebuilt tables in pinned host memory (a mirror of the workspace bytes
  // [pin_lo, pin_hi)) and copies the written ranges asynchronously
  char* pin = nullptr;
  size_t pin_lo = 0, pin_hi = 0;
  bool staging = false;
  bool dyn_consts = false;  // set by ns_set_dt: kernels read the sub-step constants from stepk
  bool dry = false;         // table builders update the host state only (upload_raw copies nothing)
  // device-side dt update of the fixed-CFL steps: control block, FP64 scratch of the table
  // builders, and the doubles reserved per x table (dt_xs) and per line table (dt_ls)
  DtCtl* dtctl = nullptr;
  double* dtscr = nullptr;
  size_t dt_xs = 0, dt_ls = 0;
  std::vector<std::pair<size_t, size_t>> dirty;  // (workspace offset, bytes) written while staging
  int num_sms;
  int rhs_bps[4];           // resident blocks per SM of the tiled RHS (FP64, FP64 dyn, FP32, FP32 dyn)
  // partitioned x solver
  int P, M, L[3];
  int part_req;             // NS_PART_AUTO / PPT / PDD
  int part_mode;            // resolved: NS_PART_PPT or NS_PART_PDD
  double pdd_drop;
  size_t xtab_stride;       // elements reserved per sub-step
  // graph
  cudaGraph_t graph;
  cudaGraphExec_t gexec;
  bool have_graph;
  // profiled graph: the same launches with an event recorded before each kernel and after the
  // last one
  cudaGraph_t pgraph;
  cudaGraphExec_t pgexec;
  bool have_pgraph;
  cudaEvent_t pev[64];
  int npev;
  // fixed-CFL graph: convective rate, dt update, then the step; the tables sub-step 0's RHS does not
  // read are built on side_stream beside it (fork / join events)
  cudaStream_t side_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaGraph_t cgraph;
  cudaGraphExec_t cgexec;
  bool have_cgraph = false;
  std::string err;
};

// ---------------------------------------------------------------------------------------------
// FP64 <-> FP32 conversions on the integer pipe (IEEE 754 binary64 / binary32 field layouts).
// The mixed form converts every state value it reads; the hardware conversion occupies the
// FP64 pipe, which is the scarce unit here.  d2f rounds to nearest even; results below the
// smallest normal float flush to +-0 and overflow gives +-inf (state values are finite and far
// from both limits).  f2d is exact for normal floats and zero.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ float d2f_rn(double x) {
  const unsigned hi = (unsigned)__double2hiint(x);
  const unsigned lo = (unsigned)__double2loint(x);
  const unsigned sign = hi & 0x80000000u;
  const unsigned e = (hi >> 20) & 0x7FFu;                    // biased binary64 exponent
  const unsigned mant = ((hi & 0xFFFFFu) << 3) | (lo >> 29);  // top 23 fraction bits
  const unsigned rem = lo & 0x1FFFFFFFu;                      // 29 dropped bits
  unsigned bits = ((e - 896u) << 23) | mant;                  // binary32 exponent = e - 1023 + 127
  bits += (unsigned)(rem > 0x10000000u) | ((unsigned)(rem == 0x10000000u) & (mant & 1u));
  bits = (e <= 896u) ? 0u : ((e >= 1151u) ? 0x7F800000u : bits);
  return __uint_as_float(sign | bits);
}

__device__ __forceinline__ double f2d(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned sign = b & 0x80000000u, e = (b >> 23) & 0xFFu, m = b & 0x7FFFFFu;
  const unsigned hi = (e == 0u) ? sign : (sign | ((e + 896u) << 20) | (m >> 3));
  const unsigned lo = (e == 0u) ? 0u : (m << 29);
  return __hiloint2double((int)hi, (int)lo);
}

// value of a double in the arithmetic type T of a kernel
template <typename T>
__device__ __forceinline__ T from_double(double x) {
  if constexpr (sizeof(T) == 4) return d2f_rn(x);
  else return (T)x;
}

// ---------------------------------------------------------------------------------------------
// Kernels are written as functors K with `Args`, `kThreads` / `kMinBlocks` (launch bounds) and
// `static __device__ void run(const Args&, dim3 block, dim3 grid)` (block / grid replace
// blockIdx / gridDim).  single_kernel<K> runs one instance.  batched_kernel<K> runs many: the
// blocks of every instance are numbered consecutively (first[i] = index of instance i's first
// block, first[n] = total) and a persistent grid walks them; each item decodes its instance by
// binary search, rebuilds its local block index and runs the same body with that instance's
// arguments.  One launch per stage and variant serves the whole ensemble.
// ---------------------------------------------------------------------------------------------
struct BatchMap {
  const int* first;   // n + 1 prefix offsets
  const uint3* grid;  // per-instance grid shape
  int n;
  int total;
};

template <typename K>
__global__ void __launch_bounds__(K::kThreads, K::kMinBlocks) single_kernel(const __grid_constant__ typename K::Args a) {
  K::run(a, blockIdx, gridDim);
}

template <typename K>
__global__ void __launch_bounds__(K::kThreads, K::kMinBlocks) batched_kernel(const typename K::Args* __restrict__ args,
                                                              const BatchMap m) {
  for (int item = blockIdx.x; item < m.total; item += gridDim.x) {
    int lo = 0, hi = m.n;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (__ldg(m.first + mid) <= item) lo = mid; else hi = mid;
    }
    const uint3 g = m.grid[lo];
    const int local = item - __ldg(m.first + lo);
    const dim3 b(local % g.x, (local / g.x) % g.y, local / (g.x * g.y));
    K::run(args[lo], b, dim3(g.x, g.y, g.z));
    __syncthreads();  // shared memory of this item is reused by the next
  }
}

// Dynamic shared-memory limit of both launch forms of functor K.
template <typename K>
cudaError_t set_smem_limit(int bytes) {
  cudaError_t e = cudaFuncSetAttribute(single_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(batched_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

// ---------------------------------------------------------------------------------------------
// Launch sink.  Every stage is written once as `stage(LaunchSink&, substep)` and emits its kernel
// with emit<K>(sink, args, grid, block, smem): a single-instance sink launches at once on the
// context's stream; a batch sink hands the launch to a planner that groups the instances of a
// stage by functor type K and by the launch's place in the instance's sequence for that stage
// (instances of different shapes may emit different sequences, e.g. the y solve of the mixed
// form), and later launches the groups in the order of those places, each as one persistent
// batched_kernel<K>.
// ---------------------------------------------------------------------------------------------
struct BatchGroup {
  const void* key;                      // identifies K
  int ord;                              // place of the launch in each instance's sequence
  size_t arg_size;
  std::vector<unsigned char> args;      // packed K::Args, one per instance of the group
  std::vector<int> first;               // block prefix, first[0] = 0
  std::vector<uint3> grid;              // per-instance grid
  dim3 block;
  size_t smem;                          // largest dynamic shared memory of the group
  cudaError_t (*enqueue)(const void* dargs, const BatchMap& m, unsigned grid, dim3 block, size_t smem,
                         cudaStream_t s);
  int (*blocks_per_sm)(int threads, size_t smem);
};

struct BatchPlanner {
  std::vector<BatchGroup> groups;
  int ord = 0;  // place of the next launch in the current instance's sequence
  void next_instance() { ord = 0; }
  // groups in launch order: by place, then by first appearance
  void order() {
    std::stable_sort(groups.begin(), groups.end(),
                     [](const BatchGroup& x, const BatchGroup& y) { return x.ord < y.ord; });
  }
  template <typename K>
  static cudaError_t enqueue_k(const void* dargs, const BatchMap& m, unsigned grid, dim3 block, size_t smem,
                               cudaStream_t s) {
    batched_kernel<K><<<grid, block, smem, s>>>((const typename K::Args*)dargs, m);
    return cudaGetLastError();
  }
  template <typename K>
  static int bps_k(int threads, size_t smem) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batched_kernel<K>, threads, smem) != cudaSuccess) n = 1;
    return n > 0 ? n : 1;
  }
  template <typename K>
  cudaError_t collect(const typename K::Args& a, dim3 grid, dim3 block, size_t smem) {
    static const char key = 0;
    BatchGroup* g = nullptr;
    for (auto& q : groups)
      if (q.key == &key && q.ord == ord) g = &q;
    if (!g) {
      groups.emplace_back();
      g = &groups.back();
      g->key = &key;
      g->ord = ord;
      g->arg_size = sizeof(typename K::Args);
      g->first.push_back(0);
      g->block = block;
      g->smem = 0;
      g->enqueue = &enqueue_k<K>;
      g->blocks_per_sm = &bps_k<K>;
    }
    const unsigned char* p = reinterpret_cast<const unsigned char*>(&a);
    g->args.insert(g->args.end(), p, p + sizeof(a));
    g->grid.push_back(make_uint3(grid.x, grid.y, grid.z));
    g->first.push_back(g->first.back() + (int)(grid.x * grid.y * grid.z));
    if (smem > g->smem) g->smem = smem;
    ++ord;
    return cudaSuccess;
  }
};

struct LaunchSink {
  ns_ctx* c;            // the instance (its stream is used in single mode)
  BatchPlanner* plan;   // non-null: collect instead of launching
};

template <typename K>
cudaError_t emit(LaunchSink& s, const typename K::Args& a, dim3 grid, dim3 block, size_t smem);

template <typename K>
cudaError_t emit(LaunchSink& s, const typename K::Args& a, dim3 grid, dim3 block, size_t smem) {
  if (s.plan) return s.plan->collect<K>(a, grid, block, smem);
  single_kernel<K><<<grid, block, smem, s.c->launch>>>(a);
  return cudaGetLastError();
}

// Stage functions (emit one kernel through the sink) ...
cudaError_t stage_rhs(LaunchSink& s, int k);
cudaError_t stage_adi_x(LaunchSink& s, int k);
cudaError_t stage_adi_y(LaunchSink& s, int k);
cudaError_t stage_adi_z(LaunchSink& s, int k);
cudaError_t stage_pois_divz(LaunchSink& s, int k);
cudaError_t stage_pois_x_fwd(LaunchSink& s, int k);
cudaError_t stage_pois_tdma(LaunchSink& s, int k);
cudaError_t stage_pois_x_inv(LaunchSink& s, int k);
cudaError_t stage_pois_ifftz(LaunchSink& s, int k);
cudaError_t stage_pois_refine(LaunchSink& s, int k);  // mixed form: FP64 residual, second FP32 solve
cudaError_t stage_project(LaunchSink& s, int k);

// ... and their single-instance launchers (enqueue on ctx->launch; return the launch error).
cudaError_t launch_rhs(ns_ctx* c, int k);
cudaError_t rhs_set_attributes(int* bps);  // once per device, outside any capture
cudaError_t launch_adi_x(ns_ctx* c, int k);
// ns_autotune; lines = false keeps the default y and z line shapes (batched instances share them)
ns_status autotune_ctx(ns_ctx* c, bool lines);
cudaError_t adi_set_attributes();  // once per device, outside any capture
cudaError_t launch_adi_y(ns_ctx* c, int k);
cudaError_t launch_adi_z(ns_ctx* c, int k);
cudaError_t launch_poisson(ns_ctx* c, int k);   // the five kernels below, in order
cudaError_t launch_pois_divz(ns_ctx* c, int k);
cudaError_t launch_pois_fftx_fwd(ns_ctx* c, int k);   // x FFT (periodic) or DCT-II (inflow / outflow)
cudaError_t launch_pois_tdma(ns_ctx* c, int k);
cudaError_t launch_pois_fftx_inv(ns_ctx* c, int k);
cudaError_t launch_pois_ifftz(ns_ctx* c, int k);
cudaError_t launch_pois_refine(ns_ctx* c, int k);
cudaError_t launch_project(ns_ctx* c, int k);
cudaError_t launch_outflow(ns_ctx* c, int k);        // convective outflow update + increments
cudaError_t launch_flux_correct(ns_ctx* c, int k);   // outflow volume flux := inflow flux
cudaError_t launch_pois_factor(ns_ctx* c, const double* lamx, const double* lamz);
cudaError_t launch_convective_rate(ns_ctx* c);  // max-reduction into c->rate (zeroed first)
// dt-dependent tables (k_dt.cu).  build_dt_tables: RHS rows, ADI y and z factors;
// build_x_tables: x-solver and partitioned-line tables (modes chosen by the PDD drop) and the
// sub-step constants.  launch_dt_update: the same tables on the device from dt = cfl / rate.
ns_status build_dt_tables(ns_ctx* c);
ns_status build_x_tables(ns_ctx* c);
cudaError_t launch_dt_update(ns_ctx* c, int part);
size_t dt_scratch_doubles(int nz, size_t xs, size_t ls);  // doubles of the dtscr block
// Host -> workspace copy of a table: to the pinned mirror while c->staging (flush_staging
// copies the recorded ranges asynchronously), nothing while c->dry, else a copy and a sync.
cudaError_t upload_raw(ns_ctx* c, void* dst, const void* src, size_t bytes);
cudaError_t flush_staging(ns_ctx* c);
inline int stepk_index(int k) { return k < 0 ? 3 : k; }
cudaError_t launch_recycle(ns_ctx* c, int k);    // recycled inflow planes (sub-step 0, if enabled)
size_t recycle_block_doubles(int ny);
cudaError_t recycle_upload_grid(ns_ctx* c);
// the grid part of a recycling block for faces yf[0..ny] (host; the rest zero)
void recycle_grid_host(const double* yf, int ny, double* h);
// Recycling from a gathered recycle plane (y slabs): g holds the whole domain's samples (row j of
// u at g + uoff[j], of w at g + woff[j], face f of v at g + voff[f], nz each); rcy is a recycling
// block of the whole grid (ny rows); the inflow rows written are the rows local rows of u (face 0
// of each), v_in (rows + 1 faces) and w_in held here, local row 0 being row jg0 of the domain.
cudaError_t launch_recycle_gathered(const double* g, const long* uoff, const long* woff, const long* voff, double* rcy,
                                    int ny, int nz, double delta_in, double u_inf, double* u, double* v_in,
                                    double* w_in, int nx, int rows, int jg0, cudaStream_t st);
cudaError_t poisson_set_attributes();  // once per process and device, outside any capture

// Sets the message ns_last_error(NULL) returns on this thread.
void ns_set_thread_error(const char* msg);

// Grid coefficient block (GC_* layout, NS_GC_COUNT arrays of ny + 1) of cfg, on the host.
std::vector<double> grid_coefficients_host(const ns_config* cfg);

// Host-side table builders (ns_tables.cpp-style code lives in ns_api.cu).
size_t adi_y_tab_count(int ny);
size_t adi_z_tab_count(int nz);

// Entries of a z-sweep table (dt_ztab): the Sherman-Morrison Thomas factors INV, AINV, CP and the
// vector Q (nz each), fac, bg, then the factorised circulant form: lambda, 1/alpha, use (1 or 0),
// K, lambda^1 .. lambda^NS_ZF_KMAX.
constexpr int NS_ZF_KMAX = 8;
inline size_t ztab_entries(int nz) { return 4 * (size_t)nz + 2 + 4 + NS_ZF_KMAX; }

// The mixed form solves a Poisson y system in FP32 arithmetic when kz > 0 and its Skeel condition
// number is at most this: the FP32 Thomas error then stays near the FP32 transforms' own rounding
// (a few 1e-7 of the line on the stretched channel and boundary-layer grids), which the FP64
// refinement absorbs like theirs.
constexpr double NS_POIS_FP32_KAPPA = 4096.0;
// bytes of the mixed form's FP32 y-solve block: two float factor planes, a_j, the mode flags
inline size_t pois32_bytes(size_t nx, size_t ny, size_t nzh) {
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  return al(2 * nzh * ny * nx * 4) + al(ny * 4) + al(nzh * nx) + al(nzh * (nx / 8 + 1) * 4) + al(ny * 16);
}
// largest dynamic shared memory of one block (227 KB)
constexpr int NS_SMEM_MAX = 227 * 1024;
// shared memory and tile width (kx) of the staged Poisson y solve of the mixed form (k_poisson.cu)
size_t pois_staged_smem(int ny);
int pois_staged_tile();
