// ns_poisson_solve_static: the pressure Poisson solve without a context and without any device
// allocation.  Its scratch (spectral buffer, y factor table, grid coefficients, FFT twiddles,
// modified wavenumbers) lives in one file-scope __device__ array of NS_STATIC_SCRATCH_BYTES that
// every GPU loading the library holds until the process exits.
//
// Some callers cannot call cudaMalloc: plugins inside a host framework that owns all device
// memory through its own pool allocator, and fixed-latency loops that must not allocate after
// start-up (an allocation can synchronise the device and take unbounded time).  They pass only
// their inputs (u, v, w) and output (phi).  The solve is the FP64 one.
//
// The kernels are the library's own Poisson kernels; only where their scratch and tables live
// differs.  Every call rewrites each scratch region it reads before reading it, so the contents
// left by an earlier call never matter.  Calls that overlap on the GPU (for example on two
// streams) share the one array and race.
#include <cmath>
#include <mutex>
#include <string>

#include "ns_internal.cuh"

namespace {

constexpr int kMaxDevices = 64;
static __device__ __align__(256) unsigned char g_ns_static_scratch[NS_STATIC_SCRATCH_BYTES];

std::mutex g_mu;
void* g_scratch[kMaxDevices] = {};  // device address of g_ns_static_scratch, per device

// host staging for the small tables (static: no allocation at call time); guarded by g_mu
double h_gc[NS_GC_COUNT * 1025];
double h_twz[6 * 4096];
double h_twx[6 * 4096];
double h_lamx[4096];
double h_lamz[2049];
StepK h_stepk[NS_STEPK];


struct Regions {
  size_t spec, pois, gc, twz, twx, lamx, lamz, stepk, total;
};

Regions regions(int nx, int ny, int nz) {
  const size_t nzh = nz / 2 + 1;
  Regions r;
  size_t o = 0;
  r.spec = o;
  o += al256(nzh * ny * nx * 16);
  r.pois = o;
  o += al256(nzh * ny * nx * 16);
  r.gc = o;
  o += al256((size_t)NS_GC_COUNT * (ny + 1) * 8);
  r.twz = o;
  o += al256(fft_twiddle_doubles(nz) * 8);
  r.twx = o;
  o += al256(fft_twiddle_doubles(nx) * 8);
  r.lamx = o;
  o += al256((size_t)nx * 8);
  r.lamz = o;
  o += al256(nzh * 8);
  r.stepk = o;
  o += al256(NS_STEPK * sizeof(StepK));
  r.total = o;
  return r;
}

ns_status fail(ns_status s, const std::string& m) {
  ns_set_thread_error(m.c_str());
  return s;
}

}  // namespace

extern "C" ns_status ns_poisson_solve_static(const ns_config* cfg, const double* u, const double* v,
                                             const double* w, double* phi, int substep, void* cuda_stream) {
  ns_set_thread_error("");
  if (!cfg || !cfg->yf || !u || !v || !w || !phi) return fail(NS_ERR_ARG, "NULL argument");
  const int nx = cfg->nx, ny = cfg->ny, nz = cfg->nz;
  if (fft_plan(nx) < 0 || nx % 8 || nx < 8 || nx > 4096 || fft_plan(nz) < 0 || nz % 8 || nz < 8 || nz > 4096 ||
      ny < 4 || ny > 1024)
    return fail(NS_ERR_SIZE, "nx, nz must be 2^a 3^b (a >= 3) in [8, 4096] and ny in [4, 1024]");
  if (cfg->bc_x != 0) return fail(NS_ERR_UNSUPPORTED, "only periodic x is built");
  if (cfg->precision != NS_FP64)
    return fail(cfg->precision == NS_MIXED ? NS_ERR_UNSUPPORTED : NS_ERR_ARG,
                "the allocation-free solve runs in FP64 only: precision must be NS_FP64");
  for (const void* q : {(const void*)u, (const void*)v, (const void*)w, (const void*)phi})
    if ((size_t)q % 256) return fail(NS_ERR_ARG, "u, v, w and phi must be 256-byte aligned");
  if (substep < -1 || substep > 2) return fail(NS_ERR_ARG, "substep must be -1, 0, 1 or 2");
  if (!(cfg->lx > 0) || !(cfg->lz > 0) || (substep >= 0 && !(cfg->dt > 0)))
    return fail(NS_ERR_ARG, "lx, lz (and dt for substep >= 0) must be positive");
  for (int j = 0; j < ny; ++j)
    if (!(cfg->yf[j + 1] > cfg->yf[j])) return fail(NS_ERR_ARG, "yf must be strictly increasing");
  const Regions R = regions(nx, ny, nz);
  if (R.total > (size_t)NS_STATIC_SCRATCH_BYTES)
    return fail(NS_ERR_SIZE, "grid needs " + std::to_string(R.total) + " scratch bytes; the static scratch holds " +
                                 std::to_string((size_t)NS_STATIC_SCRATCH_BYTES) + " (use ns_init for larger grids)");

  std::lock_guard<std::mutex> lock(g_mu);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(NS_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(NS_ERR_ARG, "device index out of range");
  if (!g_scratch[dev]) {
    // set-up, once per device, with that device current: the host-side name of the array is
    // only a stand-in, the kernels need its device address
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_ns_static_scratch);
    if (e != cudaSuccess) return fail(NS_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    if ((e = poisson_set_attributes()) != cudaSuccess)
      return fail(NS_ERR_CUDA, std::string("kernel attributes: ") + cudaGetErrorString(e));
    g_scratch[dev] = p;
  }
  char* base = (char*)g_scratch[dev];

  // grid coefficients (same definitions as the context path)
  const int G = ny + 1;
  for (int q = 0; q < NS_GC_COUNT * G; ++q) h_gc[q] = 0.0;
  auto GC = [&](int f, int j) -> double& { return h_gc[f * G + j]; };
  const double* yf = cfg->yf;
  auto yc = [&](int j) { return 0.5 * (yf[j] + yf[j + 1]); };
  for (int j = 0; j < ny; ++j) {
    GC(GC_DY, j) = yf[j + 1] - yf[j];
    GC(GC_IDY, j) = 1.0 / (yf[j + 1] - yf[j]);
  }
  for (int j = 1; j < ny; ++j) {
    const double hc = yc(j) - yc(j - 1);
    GC(GC_HC, j) = hc;
    GC(GC_IHC, j) = 1.0 / hc;
  }
  for (int j = 1; j < ny; ++j) GC(GC_PA, j) = 1.0 / ((yf[j + 1] - yf[j]) * (yc(j) - yc(j - 1)));
  for (int j = 0; j + 1 < ny; ++j) GC(GC_PC, j) = 1.0 / ((yf[j + 1] - yf[j]) * (yc(j + 1) - yc(j)));
  const double PI = 3.14159265358979323846;
  const double dx = cfg->lx / nx, dz = cfg->lz / nz;
  fft_twiddles(nz, h_twz);
  fft_twiddles(nx, h_twx);
  for (int q = 0; q < nx; ++q) {
    const int qq = q <= nx - q ? q : nx - q;
    h_lamx[q] = (2.0 / (dx * dx)) * (1.0 - std::cos(2.0 * PI * qq / nx));
  }
  for (int q = 0; q <= nz / 2; ++q) h_lamz[q] = (2.0 / (dz * dz)) * (1.0 - std::cos(2.0 * PI * q / nz));

  // divergence scale of the requested sub-step (the only dt-dependent constant of the solve)
  for (int q = 0; q < NS_STEPK; ++q) h_stepk[q] = StepK{};
  h_stepk[stepk_index(substep)].pscale =
      ((substep >= 0) ? 1.0 / (NS_ALPHA[substep] * cfg->dt) : 1.0) / ((double)nx * nz);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const struct {
    size_t off;
    const void* src;
    size_t bytes;
  } up[] = {{R.gc, h_gc, (size_t)NS_GC_COUNT * G * 8}, {R.twz, h_twz, fft_twiddle_doubles(nz) * 8},
            {R.twx, h_twx, fft_twiddle_doubles(nx) * 8},           {R.lamx, h_lamx, (size_t)nx * 8},
            {R.lamz, h_lamz, (size_t)(nz / 2 + 1) * 8}, {R.stepk, h_stepk, sizeof(h_stepk)}};
  for (const auto& q : up)
    if ((e = cudaMemcpyAsync(base + q.off, q.src, q.bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess)
      return fail(NS_ERR_CUDA, std::string("table upload: ") + cudaGetErrorString(e));
  // the pageable host tables are reused by the next call: wait until the copies have read them
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess)
    return fail(NS_ERR_CUDA, std::string("table upload: ") + cudaGetErrorString(e));

  ns_ctx c{};  // value-initialised: every member not set below is zero
  c.cfg = *cfg;
  c.bl = 0;
  c.launch = st;
  c.stream = st;
  c.nzh = nz / 2 + 1;
  c.dx = dx;
  c.dz = dz;
  c.f.u = const_cast<double*>(u);
  c.f.v = const_cast<double*>(v);
  c.f.w = const_cast<double*>(w);
  c.f.p = nullptr;
  c.phi = phi;
  c.spec = (double2*)(base + R.spec);
  c.pois = (double2*)(base + R.pois);
  c.gc = (double*)(base + R.gc);
  c.twz = (double2*)(base + R.twz);
  c.twx = (double2*)(base + R.twx);
  c.stepk = (StepK*)(base + R.stepk);
  if ((e = launch_pois_factor(&c, (const double*)(base + R.lamx), (const double*)(base + R.lamz))) != cudaSuccess)
    return fail(NS_ERR_CUDA, std::string("factor table: ") + cudaGetErrorString(e));
  if ((e = launch_poisson(&c, substep)) != cudaSuccess)
    return fail(NS_ERR_CUDA, std::string("poisson: ") + cudaGetErrorString(e));
  return NS_OK;
}
