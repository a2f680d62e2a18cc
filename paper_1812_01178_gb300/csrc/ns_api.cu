// C ABI entry points, workspace layout, coefficient tables and graph capture.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "ns_internal.cuh"

namespace {

thread_local std::string g_init_error;


// Returns "" if the configuration is valid, else a message; *kind receives the status to report.
std::string check_cfg(const ns_config* c, ns_status* kind = nullptr) {
  ns_status dummy;
  ns_status& k = kind ? *kind : dummy;
  k = NS_ERR_ARG;
  if (!c) return "cfg is NULL";
  if (!c->yf) return "cfg->yf is NULL";
  if (c->bc_x != 0 && c->bc_x != 1) return "bc_x must be 0 or 1";
  if (c->bc_ytop != 0 && c->bc_ytop != 1) return "bc_ytop must be 0 or 1";
  if (c->precision != NS_FP64 && c->precision != NS_MIXED) return "precision must be NS_FP64 or NS_MIXED";
  if (c->pressure_update != NS_PRESSURE_DELTA && c->pressure_update != NS_PRESSURE_KIM_MOIN)
    return "pressure_update must be NS_PRESSURE_DELTA or NS_PRESSURE_KIM_MOIN";
  if (c->recycle_i != 0) {
    if (c->bc_x != 1) return "recycling needs inflow / outflow in x (bc_x = 1)";
    if (c->recycle_i < 1 || c->recycle_i >= c->nx) return "recycle_i must be in [1, nx - 1]";
    if (!(c->delta_in > 0.0) || !std::isfinite(c->delta_in)) return "delta_in must be positive and finite";
  }
  k = NS_ERR_SIZE;
  if (fft_plan(c->nx) < 0 || c->nx % 8 || c->nx < 8 || c->nx > 4096)
    return "nx must be 2^a 3^b with a >= 3, in [8, 4096]";
  if (fft_plan(c->nz) < 0 || c->nz % 8 || c->nz < 8 || c->nz > 4096)
    return "nz must be 2^a 3^b with a >= 3, in [8, 4096]";
  if (x_default_partition(c->nx) == 0) return "nx has no partition shape of the x solver (P <= 32 lanes, M rows)";
  if (c->ny < 4 || c->ny > 1024) return "ny must be in [4, 1024]";
  k = NS_ERR_ARG;
  if (!(c->lx > 0) || !(c->lz > 0) || !(c->dt > 0)) return "lx, lz and dt must be positive";
  for (int j = 0; j < c->ny; ++j)
    if (!(c->yf[j + 1] > c->yf[j])) return "yf must be strictly increasing";
  return "";
}

int ilog2i(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

// Partitioned y / z lines are used by the mixed form when x is a multiple of 32 (one block holds
// 32 lines) and the line length has a built shape.
int line_P(const ns_config* c, int n) {
  if (c->precision != NS_MIXED || c->nx % 32 != 0) return 0;
  return line_partition(n);
}

// floats of one partitioned-line table (the larger of the y and z shapes, PPT levels included)
size_t line_table_floats(const ns_config* c) {
  size_t m = 0;
  const int py = line_P(c, c->ny), pz = line_P(c, c->nz);
  if (py) m = std::max(m, xtab_count(c->ny / py, py, ilog2i(py)));
  if (pz) m = std::max(m, xtab_count(c->nz / pz, pz, ilog2i(pz)));
  return m;
}

// elements reserved per x-solver table: any admissible P <= 32 (L <= 5 levels)
size_t x_table_elems(const ns_config* c) { return 5 * (size_t)c->nx + 4 * 32 + 8 * 5 * 32; }

ns_layout make_layout(const ns_config* c) {
  ns_layout L;
  memset(&L, 0, sizeof(L));
  const size_t es = c->precision == NS_MIXED ? 4 : 8;
  const size_t nx = c->nx, ny = c->ny, nz = c->nz, nzh = nz / 2 + 1;
  const size_t cells = nx * ny * nz, vcells = nx * (ny + 1) * nz;
  size_t sz[LB_COUNT];
  sz[LB_RU] = cells * es;
  sz[LB_RV] = vcells * es;
  sz[LB_RW] = cells * es;
  sz[LB_NU] = cells * es;
  sz[LB_NV] = vcells * es;
  sz[LB_NW] = cells * es;
  sz[LB_PHI] = cells * 8;
  sz[LB_SPEC] = nzh * ny * nx * 16;
  sz[LB_POIS] = nzh * ny * nx * 16;
  sz[LB_GC] = NS_GC_COUNT * (ny + 1) * 8;
  sz[LB_XTAB] = 6 * al256(x_table_elems(c) * es);
  sz[LB_YTAB] = 6 * al256(3 * ny * es);
  sz[LB_ZTAB] = 3 * al256(ztab_entries(nz) * es);
  sz[LB_TWZ] = fft_twiddle_doubles((int)nz) * 8;
  sz[LB_TWX] = fft_twiddle_doubles((int)nx) * 8;
  sz[LB_LAMX] = nx * 8;
  sz[LB_LAMZ] = nzh * 8;
  sz[LB_RTAB] = 3 * al256((size_t)RT_COUNT * (ny + 1) * 8) + 3 * al256((size_t)RT_COUNT * (ny + 1) * 4);
  sz[LB_DOUT] = 3 * al256((ny + 1) * nz * 8) + 256;
  sz[LB_TWD] = nx * 32;
  sz[LB_RCY] = recycle_block_doubles((int)ny) * 8;
  sz[LB_STEPK] = NS_STEPK * sizeof(StepK);
  sz[LB_PTAB] = 9 * al256(line_table_floats(c) * 4);
  sz[LB_TW32] = c->precision == NS_MIXED ? al256(fft_twiddle_doubles((int)nz) * 4) + al256(fft_twiddle_doubles((int)nx) * 4) +
                                               al256(nx * 16)
                                         : 0;
  sz[LB_DT] = al256(sizeof(DtCtl)) + 8 * dt_scratch_doubles((int)nz, x_table_elems(c), line_table_floats(c));
  sz[LB_POIS32] = c->precision == NS_MIXED ? pois32_bytes(nx, ny, nzh) : 0;
  size_t o = 0;
  for (int b = 0; b < LB_COUNT; ++b) {
    L.off[b] = o;
    o += al256(sz[b]);
  }
  L.total = o;
  return L;
}

// Tile list of the mixed form's staged Poisson y solve, from the mode flags pois_factor_kernel
// wrote: tiles of pois_staged_tile() kx holding a mode that takes FP64 first, then the tiles whose
// modes all take FP32.  The register form stays (pois_tiles = null) when nx is not a multiple of
// the tile width or a tile does not fit in shared memory.
ns_status build_pois_tiles(ns_ctx* c) {
  const int nx = c->cfg.nx, ny = c->cfg.ny, nzh = c->nzh, TL = pois_staged_tile();
  if (nx % TL != 0 || pois_staged_smem(ny) > (size_t)NS_SMEM_MAX) {
    c->pois_tiles = nullptr;
    return NS_OK;
  }
  std::vector<unsigned char> mode((size_t)nzh * nx);
  if (cudaMemcpy(mode.data(), c->pois_mode, mode.size(), cudaMemcpyDeviceToHost) != cudaSuccess) return NS_ERR_CUDA;
  std::vector<int> t64, t32;
  const int ntx = nx / TL;
  for (int kz = 0; kz < nzh; ++kz)
    for (int t = 0; t < ntx; ++t) {
      bool all = true;
      for (int l = 0; l < TL; ++l) all = all && mode[(size_t)kz * nx + t * TL + l];
      (all ? t32 : t64).push_back(kz * ntx + t);
    }
  c->ntile64 = (int)t64.size();
  c->ntile32 = (int)t32.size();
  t64.insert(t64.end(), t32.begin(), t32.end());
  if (upload_raw(c, c->pois_tiles, t64.data(), t64.size() * sizeof(int)) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return NS_ERR_CUDA;
  return NS_OK;
}

cudaError_t upload_d(ns_ctx* c, void* dst, const std::vector<double>& src) {
  return upload_raw(c, dst, src.data(), src.size() * 8);
}

void drop_graph(ns_ctx* c) {
  if (c->have_graph) {
    cudaGraphExecDestroy(c->gexec);
    cudaGraphDestroy(c->graph);
    c->have_graph = false;
  }
  if (c->have_pgraph) {
    cudaGraphExecDestroy(c->pgexec);
    cudaGraphDestroy(c->pgraph);
    c->have_pgraph = false;
  }
  if (c->have_cgraph) {
    cudaGraphExecDestroy(c->cgexec);
    cudaGraphDestroy(c->cgraph);
    c->have_cgraph = false;
  }
}

ns_status fail(ns_ctx* c, ns_status s, const std::string& msg) {
  c->err = msg;
  return s;
}

ns_status cuda_fail(ns_ctx* c, cudaError_t e, const char* where) {
  c->err = std::string(where) + ": " + cudaGetErrorString(e);
  return NS_ERR_CUDA;
}

bool capturing(ns_ctx* c) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(c->launch, &st);
  return st != cudaStreamCaptureStatusNone;
}

// The kernels of one sub-step, in launch order (one launch each).
struct Stage {
  const char* name;
  cudaError_t (*fn)(ns_ctx*, int);
};
const Stage STAGES[] = {
    {"recycle", launch_recycle},              // inflow planes from the recycle plane (sub-step 0 only)
    {"rhs", launch_rhs},                      // A1
    {"outflow", launch_outflow},              // A10 (convective outflow; inflow / outflow only)
    {"adi_x", launch_adi_x},                  // A2
    {"adi_y", launch_adi_y},                  // A3
    {"adi_z", launch_adi_z},                  // A4
    {"flux_correct", launch_flux_correct},    // A10 (outflow mass flux; inflow / outflow only)
    {"poisson_div_fftz", launch_pois_divz},   // A5
    {"poisson_x_fwd", launch_pois_fftx_fwd},  // A6 (FFT, or DCT-II for inflow / outflow)
    {"poisson_tdma_y", launch_pois_tdma},     // A7
    {"poisson_x_inv", launch_pois_fftx_inv},  // A8
    {"poisson_ifftz", launch_pois_ifftz},     // A9
    {"poisson_refine", launch_pois_refine},   // A5-A9 again on the FP64 residual (mixed form only)
    {"project", launch_project},              // A10
};
const int NSTAGES = (int)(sizeof(STAGES) / sizeof(STAGES[0]));

// join: an event the x sweep waits for (the side branch of the fixed-CFL dt update)
ns_status run_substep(ns_ctx* c, int k, cudaEvent_t* ev = nullptr, cudaEvent_t join = nullptr) {
  for (int q = 0; q < NSTAGES; ++q) {
    if (ev) cudaEventRecordWithFlags(ev[q], c->launch, cudaEventRecordExternal);
    if (join && STAGES[q].fn == launch_adi_x) {
      cudaError_t e = cudaStreamWaitEvent(c->launch, join, 0);
      if (e != cudaSuccess) return cuda_fail(c, e, "join");
    }
    cudaError_t e = STAGES[q].fn(c, k);
    if (e != cudaSuccess) return cuda_fail(c, e, STAGES[q].name);
  }
  return NS_OK;
}

// Capture the three sub-steps of one time step into a graph (optionally with event nodes) and
// instantiate it.  With cfl the step is preceded by the convective rate and the device-side dt
// update: its first part on the step's stream, the rest on a side branch that the x sweep of
// sub-step 0 joins.
ns_status capture_step(ns_ctx* c, bool profiled, cudaGraph_t* graph, cudaGraphExec_t* exec, bool cfl = false) {
  c->launch = c->cap_stream;
  cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    c->launch = c->stream;
    return cuda_fail(c, e, "begin capture");
  }
  ns_status s = NS_OK;
  if (cfl) {
    if ((e = launch_convective_rate(c)) == cudaSuccess && (e = launch_dt_update(c, 0)) == cudaSuccess &&
        (e = cudaEventRecord(c->ev_fork, c->cap_stream)) == cudaSuccess &&
        (e = cudaStreamWaitEvent(c->side_stream, c->ev_fork, 0)) == cudaSuccess) {
      c->launch = c->side_stream;
      e = launch_dt_update(c, 1);
      c->launch = c->cap_stream;
      if (e == cudaSuccess) e = cudaEventRecord(c->ev_join, c->side_stream);
    }
    if (e != cudaSuccess) s = cuda_fail(c, e, "dt update");
  }
  for (int k = 0; k < 3 && s == NS_OK; ++k)
    s = run_substep(c, k, profiled ? c->pev + k * NSTAGES : nullptr, cfl && k == 0 ? c->ev_join : nullptr);
  if (s == NS_OK && profiled) cudaEventRecordWithFlags(c->pev[3 * NSTAGES], c->cap_stream, cudaEventRecordExternal);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(c->cap_stream, &g);
  c->launch = c->stream;
  if (s != NS_OK) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "end capture");
  if ((e = cudaGraphInstantiate(exec, g, 0)) != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_fail(c, e, "graph instantiate");
  }
  *graph = g;
  return NS_OK;
}

}  // namespace

void ns_set_thread_error(const char* msg) { g_init_error = msg ? msg : ""; }

// Grid coefficient block (layout of GC_*) of a configuration, on the host.
std::vector<double> grid_coefficients_host(const ns_config* cfg) {
  const int ny = cfg->ny;
  const double* yf = cfg->yf;
  std::vector<double> yc(ny), dy(ny);
  for (int j = 0; j < ny; ++j) {
    yc[j] = 0.5 * (yf[j] + yf[j + 1]);
    dy[j] = yf[j + 1] - yf[j];
  }
  const int G = ny + 1;
  std::vector<double> gc((size_t)NS_GC_COUNT * G, 0.0);
  auto GCv = [&](int f, int j) -> double& { return gc[(size_t)f * G + j]; };
  for (int j = 0; j < ny; ++j) {
    GCv(GC_DY, j) = dy[j];
    GCv(GC_IDY, j) = 1.0 / dy[j];
  }
  for (int j = 1; j < ny; ++j) {
    const double hc = yc[j] - yc[j - 1];
    GCv(GC_HC, j) = hc;
    GCv(GC_IHC, j) = 1.0 / hc;
    const double whi = (yf[j] - yc[j - 1]) / hc;
    GCv(GC_WHI, j) = whi;
    GCv(GC_WLO, j) = 1.0 - whi;
  }
  for (int j = 0; j < ny; ++j) {
    const double hm = j == 0 ? yc[0] - yf[0] : yc[j] - yc[j - 1];
    const double hp = j == ny - 1 ? yf[ny] - yc[ny - 1] : yc[j + 1] - yc[j];
    GCv(GC_AC, j) = 2.0 / (hm * (hm + hp));
    GCv(GC_CC, j) = (j == ny - 1 && cfg->bc_ytop == 1) ? 0.0 : 2.0 / (hp * (hm + hp));
  }
  for (int j = 1; j < ny; ++j) {
    const double hm = dy[j - 1], hp = dy[j];
    GCv(GC_AF, j) = 2.0 / (hm * (hm + hp));
    GCv(GC_CF, j) = 2.0 / (hp * (hm + hp));
  }
  for (int j = 1; j < ny; ++j) GCv(GC_PA, j) = 1.0 / (dy[j] * (yc[j] - yc[j - 1]));
  for (int j = 0; j + 1 < ny; ++j) GCv(GC_PC, j) = 1.0 / (dy[j] * (yc[j + 1] - yc[j]));
  return gc;
}


extern "C" {

size_t ns_workspace_bytes(const ns_config* cfg) {
  if (!check_cfg(cfg).empty()) return 0;
  return make_layout(cfg).total;
}

ns_status ns_init(ns_ctx** out, const ns_config* cfg, const ns_fields* fields, void* workspace, size_t ws_bytes,
                  void* cuda_stream) {
  g_init_error.clear();
  if (!out) {
    g_init_error = "out is NULL";
    return NS_ERR_ARG;
  }
  *out = nullptr;
  ns_status kind = NS_OK;
  const std::string msg = check_cfg(cfg, &kind);
  if (!msg.empty()) {
    g_init_error = msg;
    return kind;
  }
  if (!fields || !fields->u || !fields->v || !fields->w || !fields->p) {
    g_init_error = "fields or a field pointer is NULL";
    return NS_ERR_ARG;
  }
  if (cfg->bc_x == 1 && (!fields->u_out || !fields->v_in || !fields->v_out || !fields->w_in || !fields->w_out)) {
    g_init_error = "inflow / outflow in x needs the five boundary planes in fields";
    return NS_ERR_ARG;
  }
  const void* ptrs[4] = {fields->u, fields->v, fields->w, fields->p};
  for (const void* p : ptrs)
    if ((uintptr_t)p % 256 != 0) {
      g_init_error = "field pointers must be 256-byte aligned";
      return NS_ERR_ARG;
    }
  ns_ctx* c = new (std::nothrow) ns_ctx();
  if (!c) {
    g_init_error = "out of host memory";
    return NS_ERR_ARG;
  }
  c->cfg = *cfg;
  c->bl = cfg->bc_x == 1;
  c->yf.assign(cfg->yf, cfg->yf + cfg->ny + 1);
  c->cfg.yf = c->yf.data();
  c->f = *fields;
  c->stream = (cudaStream_t)cuda_stream;
  c->launch = c->stream;
  c->es = cfg->precision == NS_MIXED ? 4 : 8;
  c->nzh = cfg->nz / 2 + 1;
  c->dx = cfg->lx / cfg->nx;
  c->dz = cfg->lz / cfg->nz;
  c->lay = make_layout(cfg);
  c->have_graph = false;
  c->have_pgraph = false;
  c->npev = 0;
  cudaError_t e;
  if (workspace) {
    if (ws_bytes < c->lay.total || (uintptr_t)workspace % 256 != 0) {
      g_init_error = "workspace too small or not 256-byte aligned";
      delete c;
      return NS_ERR_ARG;
    }
    c->ws = workspace;
    c->own_ws = false;
  } else {
    if ((e = cudaMalloc(&c->ws, c->lay.total)) != cudaSuccess) {
      g_init_error = std::string("cudaMalloc workspace: ") + cudaGetErrorString(e);
      delete c;
      return NS_ERR_CUDA;
    }
    c->own_ws = true;
  }
  c->ws_bytes = c->lay.total;
  if ((e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking)) != cudaSuccess) {
    g_init_error = std::string("stream create: ") + cudaGetErrorString(e);
    if (c->own_ws) cudaFree(c->ws);
    delete c;
    return NS_ERR_CUDA;
  }
  char* base = (char*)c->ws;
  c->ru = base + c->lay.off[LB_RU];
  c->rv = base + c->lay.off[LB_RV];
  c->rw = base + c->lay.off[LB_RW];
  c->nu = base + c->lay.off[LB_NU];
  c->nv = base + c->lay.off[LB_NV];
  c->nw = base + c->lay.off[LB_NW];
  c->phi = (double*)(base + c->lay.off[LB_PHI]);
  c->spec = (double2*)(base + c->lay.off[LB_SPEC]);
  c->pois = (double2*)(base + c->lay.off[LB_POIS]);
  c->gc = (double*)(base + c->lay.off[LB_GC]);
  const int nx = cfg->nx, ny = cfg->ny, nz = cfg->nz;
  c->xtab_stride = x_table_elems(cfg);
  for (int k = 0; k < 3; ++k) {
    for (int cls = 0; cls < 2; ++cls)
      c->xtab[k][cls] = base + c->lay.off[LB_XTAB] + (2 * k + cls) * al256(c->xtab_stride * c->es);
    for (int q = 0; q < 2; ++q) c->ytab[k][q] = base + c->lay.off[LB_YTAB] + (2 * k + q) * al256(3 * ny * c->es);
    c->ztab[k] = base + c->lay.off[LB_ZTAB] + k * al256(ztab_entries(nz) * c->es);
  }
  c->twz = (double2*)(base + c->lay.off[LB_TWZ]);
  c->twx = (double2*)(base + c->lay.off[LB_TWX]);
  double* lamx_d = (double*)(base + c->lay.off[LB_LAMX]);
  for (int q = 0; q < 3; ++q) c->dout[q] = (double*)(base + c->lay.off[LB_DOUT] + q * al256((size_t)(ny + 1) * nz * 8));
  c->flux = (double*)(base + c->lay.off[LB_DOUT] + 3 * al256((size_t)(ny + 1) * nz * 8));
  c->rate = (unsigned long long*)(c->flux + 4);
  c->rcy = (double*)(base + c->lay.off[LB_RCY]);
  c->stepk = (StepK*)(base + c->lay.off[LB_STEPK]);
  c->dtctl = (DtCtl*)(base + c->lay.off[LB_DT]);
  c->dtscr = (double*)(base + c->lay.off[LB_DT] + al256(sizeof(DtCtl)));
  c->dt_xs = x_table_elems(cfg);
  c->dt_ls = line_table_floats(cfg);
  c->yP = line_P(cfg, cfg->ny);
  c->zP = line_P(cfg, cfg->nz);
  for (int k = 0; k < 3; ++k)
    for (int q = 0; q < 3; ++q)
      c->ptab[k][q] = base + c->lay.off[LB_PTAB] + (3 * k + q) * al256(line_table_floats(cfg) * 4);
  c->twd = (double2*)(base + c->lay.off[LB_TWD]);
  c->pois32 = cfg->precision == NS_MIXED;
  if (c->pois32) {
    char* t32 = base + c->lay.off[LB_TW32];
    c->twz32 = (float2*)t32;
    c->twx32 = (float2*)(t32 + al256(fft_twiddle_doubles(nz) * 4));
    c->twd32 = (float2*)(t32 + al256(fft_twiddle_doubles(nz) * 4) + al256(fft_twiddle_doubles(nx) * 4));
    char* p32 = base + c->lay.off[LB_POIS32];
    const size_t planes = al256(2 * (size_t)c->nzh * ny * nx * 4);
    c->pois_f32 = (float*)p32;
    c->pois_pa32 = (float*)(p32 + planes);
    c->pois_mode = (unsigned char*)(p32 + planes + al256((size_t)ny * 4));
    c->pois_tiles = (int*)(p32 + planes + al256((size_t)ny * 4) + al256((size_t)c->nzh * nx));
    c->pois_rows32 = (float4*)(p32 + planes + al256((size_t)ny * 4) + al256((size_t)c->nzh * nx) +
                               al256((size_t)c->nzh * (nx / 8 + 1) * 4));
  }
  double* lamz_d = (double*)(base + c->lay.off[LB_LAMZ]);

  // ---------------- grid coefficients (Sec. 2.1 / 2.2 readings)
  const std::vector<double>& yf = c->yf;
  std::vector<double> yc(ny), dy(ny);
  for (int j = 0; j < ny; ++j) {
    yc[j] = 0.5 * (yf[j] + yf[j + 1]);
    dy[j] = yf[j + 1] - yf[j];
  }
  const int G = ny + 1;
  std::vector<double> gc = grid_coefficients_host(&c->cfg);
  auto GCv = [&](int f, int j) -> double& { return gc[(size_t)f * G + j]; };
  ns_status st = NS_OK;
  c->gc_h = gc;
  if (c->cfg.recycle_i && recycle_upload_grid(c) != cudaSuccess) st = NS_ERR_CUDA;
  if (upload_d(c, c->gc, gc) != cudaSuccess) st = NS_ERR_CUDA;

  // ---------------- RHS assembly coefficients per sub-step (tiled kernel)
  {
    int dev = 0;
    cudaGetDevice(&dev);
    c->num_sms = 152;
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev);
    for (int& b : c->rhs_bps) b = 1;
  }
  if (st == NS_OK) st = build_dt_tables(c);
  // ---------------- x partitioned solver: default P
  c->part_req = NS_PART_AUTO;
  {
    // default: partitions of about 8 rows (at most 32 per line, one per lane)
    const int P = x_default_partition(nx);
    c->P = P > 0 ? P : 1;
    c->M = nx / c->P;
    if (st == NS_OK && P == 0) {
      st = NS_ERR_SIZE;
      c->err = "nx has no partition shape of the x solver";
    }
  }
  if (st == NS_OK) st = build_x_tables(c);
  // ---------------- FFT twiddles, modified wavenumbers, Poisson y factors
  if (st == NS_OK) {
    const double PI = 3.14159265358979323846;
    std::vector<double> tw(fft_twiddle_doubles(nz)), tx(fft_twiddle_doubles(nx));
    fft_twiddles(nz, tw.data());
    fft_twiddles(nx, tx.data());
    if (upload_d(c, c->twz, tw) != cudaSuccess) st = NS_ERR_CUDA;
    if (upload_d(c, c->twx, tx) != cudaSuccess) st = NS_ERR_CUDA;
    std::vector<double> lx(nx), lz(c->nzh);
    for (int q = 0; q < nx; ++q) {
      if (c->bl) {  // DCT-II modes (zero gradient at x = 0 and x = Lx)
        lx[q] = (2.0 / (c->dx * c->dx)) * (1.0 - std::cos(PI * q / nx));
      } else {
        const int qq = q <= nx - q ? q : nx - q;
        lx[q] = (2.0 / (c->dx * c->dx)) * (1.0 - std::cos(2.0 * PI * qq / nx));
      }
    }
    std::vector<double> td(4 * nx);  // w_l, then w_l / 2 (exact) for the forward transform
    for (int q = 0; q < nx; ++q) {
      td[2 * q] = std::cos(PI * q / (2.0 * nx));
      td[2 * q + 1] = -std::sin(PI * q / (2.0 * nx));
      td[2 * (nx + q)] = 0.5 * td[2 * q];
      td[2 * (nx + q) + 1] = 0.5 * td[2 * q + 1];
    }
    if (upload_d(c, c->twd, td) != cudaSuccess) st = NS_ERR_CUDA;
    if (c->pois32) {  // the same tables rounded to float for the FP32 transforms of the mixed form
      const std::vector<float> fz(tw.begin(), tw.end()), fx(tx.begin(), tx.end()), fd(td.begin(), td.end());
      const std::vector<float> pa32(gc.begin() + (size_t)GC_PA * G, gc.begin() + (size_t)GC_PA * G + ny);
      std::vector<float> rows32(4 * (size_t)ny, 0.0f);  // (a_j, c_j, -(a_j + c_j), a_j - (float)a_j)
      for (int j = 0; j < ny; ++j) {
        const double aj = gc[(size_t)GC_PA * G + j], cj = gc[(size_t)GC_PC * G + j];
        rows32[4 * j] = (float)aj;
        rows32[4 * j + 1] = (float)cj;
        rows32[4 * j + 2] = (float)(-(aj + cj));
        rows32[4 * j + 3] = (float)(aj - (double)(float)aj);
      }
      if (upload_raw(c, c->pois_rows32, rows32.data(), rows32.size() * 4) != cudaSuccess ||
          upload_raw(c, c->twz32, fz.data(), fz.size() * 4) != cudaSuccess ||
          upload_raw(c, c->twx32, fx.data(), fx.size() * 4) != cudaSuccess ||
          upload_raw(c, c->twd32, fd.data(), fd.size() * 4) != cudaSuccess ||
          upload_raw(c, c->pois_pa32, pa32.data(), pa32.size() * 4) != cudaSuccess)
        st = NS_ERR_CUDA;
    }
    for (int q = 0; q < c->nzh; ++q) lz[q] = (2.0 / (c->dz * c->dz)) * (1.0 - std::cos(2.0 * PI * q / nz));
    if (upload_d(c, lamx_d, lx) != cudaSuccess) st = NS_ERR_CUDA;
    if (upload_d(c, lamz_d, lz) != cudaSuccess) st = NS_ERR_CUDA;
    if (st == NS_OK && poisson_set_attributes() != cudaSuccess) st = NS_ERR_CUDA;
    if (st == NS_OK && rhs_set_attributes(c->rhs_bps) != cudaSuccess) st = NS_ERR_CUDA;
    if (st == NS_OK && adi_set_attributes() != cudaSuccess) st = NS_ERR_CUDA;
    if (st == NS_OK && launch_pois_factor(c, lamx_d, lamz_d) != cudaSuccess) st = NS_ERR_CUDA;
    if (st == NS_OK && cudaStreamSynchronize(c->stream) != cudaSuccess) st = NS_ERR_CUDA;
    if (st == NS_OK && c->pois32) st = build_pois_tiles(c);
  }
  // N_prev starts at zero (sub-step 0 does not read it; zero keeps it finite)
  if (st == NS_OK) {
    for (int b = LB_NU; b <= LB_NW; ++b)
      if (cudaMemsetAsync(base + c->lay.off[b], 0, c->lay.off[b + 1] - c->lay.off[b], c->stream) != cudaSuccess)
        st = NS_ERR_CUDA;
    if (cudaMemsetAsync(base + c->lay.off[LB_DOUT], 0, c->lay.off[LB_DOUT + 1] - c->lay.off[LB_DOUT], c->stream) !=
        cudaSuccess)
      st = NS_ERR_CUDA;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) st = NS_ERR_CUDA;
  }
  if (st != NS_OK) {
    g_init_error = c->err.empty() ? std::string("init failed: ") + cudaGetErrorString(cudaGetLastError()) : c->err;
    cudaStreamDestroy(c->cap_stream);
    if (c->own_ws) cudaFree(c->ws);
    delete c;
    return st;
  }
  *out = c;
  return NS_OK;
}

ns_status ns_rhs(ns_ctx* c, int k) {
  if (!c) return NS_ERR_ARG;
  if (k < 0 || k > 2) return fail(c, NS_ERR_ARG, "substep must be 0, 1 or 2");
  cudaError_t e = launch_rhs(c, k);
  return e == cudaSuccess ? NS_OK : cuda_fail(c, e, "rhs");
}

ns_status ns_adi_sweep(ns_ctx* c, int dir, int k) {
  if (!c) return NS_ERR_ARG;
  if (k < 0 || k > 2) return fail(c, NS_ERR_ARG, "substep must be 0, 1 or 2");
  cudaError_t e;
  switch (dir) {
    case 0: e = launch_adi_x(c, k); break;
    case 1: e = launch_adi_y(c, k); break;
    case 2: e = launch_adi_z(c, k); break;
    default: return fail(c, NS_ERR_ARG, "dir must be 0, 1 or 2");
  }
  return e == cudaSuccess ? NS_OK : cuda_fail(c, e, "adi");
}

ns_status ns_poisson_solve(ns_ctx* c, int k) {
  if (!c) return NS_ERR_ARG;
  if (k < -1 || k > 2) return fail(c, NS_ERR_ARG, "substep must be -1, 0, 1 or 2");
  cudaError_t e = launch_poisson(c, k);
  return e == cudaSuccess ? NS_OK : cuda_fail(c, e, "poisson");
}

ns_status ns_project(ns_ctx* c, int k) {
  if (!c) return NS_ERR_ARG;
  if (k < -1 || k > 2) return fail(c, NS_ERR_ARG, "substep must be -1, 0, 1 or 2");
  cudaError_t e = launch_project(c, k);
  return e == cudaSuccess ? NS_OK : cuda_fail(c, e, "project");
}

ns_status ns_substep(ns_ctx* c, int k) {
  if (!c) return NS_ERR_ARG;
  if (k < 0 || k > 2) return fail(c, NS_ERR_ARG, "substep must be 0, 1 or 2");
  return run_substep(c, k);
}

ns_status ns_make_divergence_free(ns_ctx* c) {
  if (!c) return NS_ERR_ARG;
  if (c->bl) {
    cudaError_t e = launch_flux_correct(c, -1);
    if (e != cudaSuccess) return cuda_fail(c, e, "flux_correct");
  }
  ns_status s = ns_poisson_solve(c, -1);
  if (s != NS_OK) return s;
  return ns_project(c, -1);
}

ns_status ns_step(ns_ctx* c, int nsteps) {
  if (!c) return NS_ERR_ARG;
  if (nsteps < 0) return fail(c, NS_ERR_ARG, "nsteps must be >= 0");
  if (nsteps == 0) return NS_OK;
  if (capturing(c)) return fail(c, NS_ERR_STATE, "ns_step called while its stream is being captured");
  if (!c->have_graph) {
    ns_status s = capture_step(c, false, &c->graph, &c->gexec);
    if (s != NS_OK) return s;
    c->have_graph = true;
  }
  cudaError_t e;
  for (int s = 0; s < nsteps; ++s)
    if ((e = cudaGraphLaunch(c->gexec, c->stream)) != cudaSuccess) return cuda_fail(c, e, "graph launch");
  return NS_OK;
}

int ns_launches_per_step(ns_ctx* c) {
  if (!c) return -1;
  if (capturing(c)) {
    fail(c, NS_ERR_STATE, "ns_launches_per_step during capture");
    return -1;
  }
  if (!c->have_graph) {
    if (capture_step(c, false, &c->graph, &c->gexec) != NS_OK) return -1;
    c->have_graph = true;
  }
  size_t n = 0;
  if (cudaGraphGetNodes(c->graph, nullptr, &n) != cudaSuccess) {
    fail(c, NS_ERR_CUDA, "graph nodes");
    return -1;
  }
  std::vector<cudaGraphNode_t> nodes(n);
  if (n && cudaGraphGetNodes(c->graph, nodes.data(), &n) != cudaSuccess) {
    fail(c, NS_ERR_CUDA, "graph nodes");
    return -1;
  }
  int k = 0;
  for (size_t q = 0; q < n; ++q) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nodes[q], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
  }
  return k;
}

ns_status ns_convective_rate(ns_ctx* c, double* rate) {
  if (!c || !rate) return NS_ERR_ARG;
  if (capturing(c)) return fail(c, NS_ERR_STATE, "ns_convective_rate during capture");
  cudaError_t e = launch_convective_rate(c);
  if (e != cudaSuccess) return cuda_fail(c, e, "convective rate");
  unsigned long long bits = 0;
  if ((e = cudaMemcpyAsync(&bits, c->rate, sizeof(bits), cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "convective rate read");
  double r;
  memcpy(&r, &bits, sizeof(r));
  if (!std::isfinite(r)) return fail(c, NS_ERR_STATE, "the velocity field holds a non-finite value");
  *rate = r;
  return NS_OK;
}

ns_status ns_set_dt(ns_ctx* c, double dt) {
  if (!c) return NS_ERR_ARG;
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(c, NS_ERR_ARG, "dt must be positive and finite");
  if (capturing(c)) return fail(c, NS_ERR_STATE, "ns_set_dt during capture");
  // the staging mirror may still feed copies of the previous call
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return fail(c, NS_ERR_CUDA, "sync");
  if (!c->pin) {
    // workspace bytes of the dt tables and the step constants
    c->pin_lo = c->lay.off[LB_XTAB];
    c->pin_hi = c->lay.off[LB_DT];  // through LB_PTAB
    if (cudaMallocHost(&c->pin, c->pin_hi - c->pin_lo) != cudaSuccess) {
      c->pin = nullptr;
      return fail(c, NS_ERR_CUDA, "pinned staging buffer");
    }
  }
  const double old = c->cfg.dt;
  c->cfg.dt = dt;
  c->staging = true;
  c->dirty.clear();
  ns_status s = build_dt_tables(c);
  if (s == NS_OK) s = build_x_tables(c);
  c->staging = false;
  if (s != NS_OK) {
    c->dirty.clear();
    c->cfg.dt = old;
    build_dt_tables(c);
    build_x_tables(c);
    return fail(c, s, "rebuilding the dt tables failed");
  }
  // from now on every kernel reads the sub-step constants from the workspace, so the step graph,
  // captured once more here, stays valid across later changes of dt
  if (!c->dyn_consts) {
    c->dyn_consts = true;
    drop_graph(c);
  }
  cudaError_t e = flush_staging(c);
  if (e != cudaSuccess) return cuda_fail(c, e, "dt table copies");
  return NS_OK;
}

ns_status ns_step_cfl(ns_ctx* c, int nsteps, double cfl, double* dts) {
  if (!c) return NS_ERR_ARG;
  if (nsteps < 0) return fail(c, NS_ERR_ARG, "nsteps must be >= 0");
  if (!(cfl > 0.0) || !std::isfinite(cfl)) return fail(c, NS_ERR_ARG, "cfl must be positive and finite");
  if (capturing(c)) return fail(c, NS_ERR_STATE, "ns_step_cfl during capture");
  if (nsteps == 0) return NS_OK;
  // every kernel reads the sub-step constants from the workspace, where the dt update writes them
  if (!c->dyn_consts) {
    c->dyn_consts = true;
    drop_graph(c);
  }
  if (!c->side_stream) {
    cudaError_t e0 = cudaStreamCreateWithFlags(&c->side_stream, cudaStreamNonBlocking);
    if (e0 == cudaSuccess) e0 = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
    if (e0 == cudaSuccess) e0 = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
    if (e0 != cudaSuccess) return cuda_fail(c, e0, "side stream");
  }
  if (!c->have_cgraph) {
    ns_status s = capture_step(c, false, &c->cgraph, &c->cgexec, true);
    if (s != NS_OK) return s;
    c->have_cgraph = true;
  }
  // runs of at most NS_DTLOG steps: reset the control block, launch, read the log back
  const size_t head = offsetof(DtCtl, dts);
  std::vector<char> hbuf(sizeof(DtCtl));
  DtCtl* h = reinterpret_cast<DtCtl*>(hbuf.data());
  cudaError_t e;
  ns_status st = NS_OK;
  for (int done = 0; done < nsteps && st == NS_OK;) {
    const int n = std::min(nsteps - done, NS_DTLOG);
    memset(h, 0, head);
    h->cfl = cfl;
    h->dt = c->cfg.dt;
    if ((e = cudaMemcpyAsync(c->dtctl, h, head, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess)
      return cuda_fail(c, e, "dt control block");
    for (int q = 0; q < n; ++q)
      if ((e = cudaGraphLaunch(c->cgexec, c->stream)) != cudaSuccess) return cuda_fail(c, e, "graph launch");
    if ((e = cudaMemcpyAsync(h, c->dtctl, head + (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, c->stream)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
      return cuda_fail(c, e, "dt log");
    if (dts) memcpy(dts + done, h->dts, (size_t)n * sizeof(double));
    c->cfg.dt = h->dt;
    if (h->status)
      st = fail(c, NS_ERR_STATE,
                std::string(h->status == 1 ? "the velocity field holds a non-finite value"
                                           : "fluid at rest: no convective time step") +
                    " (step " + std::to_string(done + (int)h->fail_step) + " kept the previous dt)");
    done += n;
  }
  // the host image of the tables (modes, levels, sub-step constants) at the last dt; the device
  // already holds the same bytes
  c->dry = true;
  ns_status r = build_dt_tables(c);
  if (r == NS_OK) r = build_x_tables(c);
  c->dry = false;
  if (st == NS_OK && r != NS_OK) st = fail(c, r, "host image of the dt tables");
  return st;
}

// Stages that launch nothing in this configuration (the boundary-plane stages of periodic x).
bool stage_idle(const ns_ctx* c, int q) {
  if (STAGES[q].fn == launch_recycle) return !c->cfg.recycle_i;
  if (STAGES[q].fn == launch_pois_refine) return !c->pois32;
  return !c->bl && (STAGES[q].fn == launch_outflow || STAGES[q].fn == launch_flux_correct);
}

ns_status ns_step_profiled(ns_ctx* c, int nsteps, float* kernel_ms, int nk) {
  if (!c || !kernel_ms) return NS_ERR_ARG;
  if (nk < NSTAGES) return fail(c, NS_ERR_ARG, "kernel_ms needs ns_kernel_count() entries");
  if (nsteps < 0) return fail(c, NS_ERR_ARG, "nsteps must be >= 0");
  if (capturing(c)) return fail(c, NS_ERR_STATE, "ns_step_profiled during capture");
  for (int q = 0; q < NSTAGES; ++q) kernel_ms[q] = 0.0f;
  cudaError_t e;
  if (!c->have_pgraph) {
    if (c->npev == 0) {
      for (int q = 0; q <= 3 * NSTAGES; ++q)
        if ((e = cudaEventCreate(&c->pev[q])) != cudaSuccess) return cuda_fail(c, e, "event create");
      c->npev = 3 * NSTAGES + 1;
    }
    ns_status s = capture_step(c, true, &c->pgraph, &c->pgexec);
    if (s != NS_OK) return s;
    c->have_pgraph = true;
  }
  for (int s = 0; s < nsteps; ++s) {
    if ((e = cudaGraphLaunch(c->pgexec, c->stream)) != cudaSuccess) return cuda_fail(c, e, "graph launch");
    if ((e = cudaEventSynchronize(c->pev[3 * NSTAGES])) != cudaSuccess) return cuda_fail(c, e, "profiled step");
    for (int q = 0; q < 3 * NSTAGES; ++q) {
      float ms = 0.0f;
      if ((e = cudaEventElapsedTime(&ms, c->pev[q], c->pev[q + 1])) != cudaSuccess)
        return cuda_fail(c, e, "event time");
      kernel_ms[q % NSTAGES] += ms;
    }
  }
  for (int q = 0; q < NSTAGES; ++q)
    if (stage_idle(c, q)) kernel_ms[q] = 0.0f;
  return NS_OK;
}

int ns_kernel_count(void) { return NSTAGES; }

const char* ns_kernel_name(int idx) { return (idx >= 0 && idx < NSTAGES) ? STAGES[idx].name : ""; }

ns_status ns_step_host(ns_ctx* c, double* u, double* v, double* w, double* p, int nsteps) {
  if (!c || !u || !v || !w || !p) return NS_ERR_ARG;
  const size_t nx = c->cfg.nx, ny = c->cfg.ny, nz = c->cfg.nz;
  const size_t bc = nx * ny * nz * 8, bv = nx * (ny + 1) * nz * 8;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(c->f.u, u, bc, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(c->f.v, v, bv, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(c->f.w, w, bc, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(c->f.p, p, bc, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "h2d");
  ns_status s = ns_step(c, nsteps);
  if (s != NS_OK) return s;
  if ((e = cudaMemcpyAsync(u, c->f.u, bc, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(v, c->f.v, bv, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(w, c->f.w, bc, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(p, c->f.p, bc, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "d2h");
  return ns_sync(c);
}

// y (dir 1) or z (dir 2) lines of the mixed form: P = 0 solves them whole (one thread per line),
// else P must be the partition count line_partition(n) the line kernels are built for.
static ns_status set_line_partition(ns_ctx* c, int dir, int P, int mode) {
  if (c->cfg.precision != NS_MIXED || c->cfg.nx % 32 != 0)
    return fail(c, NS_ERR_UNSUPPORTED, "y and z lines are partitioned only in the mixed form with nx % 32 == 0");
  const int n = dir == 1 ? c->cfg.ny : c->cfg.nz;
  if (P != 0 && P != line_partition(n)) return fail(c, NS_ERR_ARG, "invalid line partition count");
  if (mode != NS_PART_AUTO) return fail(c, NS_ERR_ARG, "y and z lines take NS_PART_AUTO");
  if (capturing(c)) return fail(c, NS_ERR_STATE, "ns_set_partition during capture");
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return fail(c, NS_ERR_CUDA, "sync");
  int& slot = dir == 1 ? c->yP : c->zP;
  const int old = slot;
  slot = P;
  ns_status s = build_x_tables(c);
  if (s != NS_OK) {
    slot = old;
    build_x_tables(c);
    return fail(c, s, "rebuilding line tables failed");
  }
  drop_graph(c);
  return NS_OK;
}

ns_status ns_set_partition(ns_ctx* c, int dir, int P, int mode) {
  if (!c) return NS_ERR_ARG;
  if (dir == 1 || dir == 2) return set_line_partition(c, dir, P, mode);
  if (dir != 0) return fail(c, NS_ERR_ARG, "dir must be 0, 1 or 2");
  const int nx = c->cfg.nx;
  if (P < 1 || P > 32 || nx % P != 0 || !x_partition_ok(P, nx / P))
    return fail(c, NS_ERR_ARG, "invalid partition count");
  if (mode != NS_PART_AUTO && mode != NS_PART_PPT && mode != NS_PART_PDD)
    return fail(c, NS_ERR_ARG, "invalid partition mode");
  if (capturing(c)) return fail(c, NS_ERR_STATE, "ns_set_partition during capture");
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return fail(c, NS_ERR_CUDA, "sync");
  const int oldP = c->P, oldM = c->M, oldreq = c->part_req;
  c->P = P;
  c->M = nx / P;
  c->part_req = mode;
  ns_status s = build_x_tables(c);
  if (s != NS_OK) {
    c->P = oldP;
    c->M = oldM;
    c->part_req = oldreq;
    build_x_tables(c);
    return fail(c, s, "rebuilding x tables failed");
  }
  drop_graph(c);
  return NS_OK;
}

ns_status ns_get_partition(ns_ctx* c, int dir, int* P, int* mode, double* dropped) {
  if (!c) return NS_ERR_ARG;
  if (dir == 1 || dir == 2) {
    const int lp = dir == 1 ? c->yP : c->zP;
    const int L = dir == 1 ? c->yL[0] : c->zL[0];
    if (P) *P = lp;
    if (mode) *mode = lp && L == 0 ? NS_PART_PDD : NS_PART_PPT;
    if (dropped) *dropped = lp ? (dir == 1 ? c->ypdd_drop : c->zpdd_drop) : 0.0;
    return NS_OK;
  }
  if (dir != 0) return fail(c, NS_ERR_ARG, "dir must be 0, 1 or 2");
  if (P) *P = c->P;
  if (mode) *mode = c->part_mode;
  if (dropped) *dropped = c->pdd_drop;
  return NS_OK;
}

extern "C++" {
// mean time of five launches of one sweep (after one untimed launch), in ms; < 0 on a failure
static float time_sweep(ns_ctx* c, int dir, cudaEvent_t e0, cudaEvent_t e1) {
  LaunchSink s{c, nullptr};
  auto one = [&](int k) {
    return dir == 0 ? stage_adi_x(s, k) : (dir == 1 ? stage_adi_y(s, k) : stage_adi_z(s, k));
  };
  if (one(0) != cudaSuccess) return -1.0f;
  cudaEventRecord(e0, c->stream);
  for (int it = 0; it < 5; ++it)
    if (one(it % 3) != cudaSuccess) return -1.0f;
  cudaEventRecord(e1, c->stream);
  cudaEventSynchronize(e1);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  return cudaGetLastError() == cudaSuccess ? ms / 5 : -1.0f;
}

// The x partitioning (every admissible P, automatic mode and forced PPT); with lines, also the y
// and z lines of the mixed form (partitioned or whole).  Each candidate's sweep is timed on the
// context's stream; the fastest stays installed.  The timed sweeps overwrite r and, in z, the
// velocity (u* = u + delta): both are saved first and restored afterwards.
ns_status autotune_ctx(ns_ctx* c, bool lines) {
  if (!c) return NS_ERR_ARG;
  if (capturing(c)) return fail(c, NS_ERR_STATE, "ns_autotune during capture");
  const int nx = c->cfg.nx;
  const bool tune_lines = lines && c->cfg.precision == NS_MIXED && nx % 32 == 0;
  const size_t rbytes = c->lay.off[LB_NU] - c->lay.off[LB_RU];
  const size_t cells = (size_t)nx * c->cfg.ny * c->cfg.nz, vcells = (size_t)nx * (c->cfg.ny + 1) * c->cfg.nz;
  const size_t fbytes = tune_lines ? (2 * cells + vcells) * 8 : 0;
  char* save = nullptr;
  cudaError_t e = cudaMalloc((void**)&save, rbytes + fbytes);
  if (e != cudaSuccess) return cuda_fail(c, e, "autotune scratch");
  cudaMemcpyAsync(save, c->ru, rbytes, cudaMemcpyDeviceToDevice, c->stream);
  if (tune_lines) {
    cudaMemcpyAsync(save + rbytes, c->f.u, cells * 8, cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(save + rbytes + cells * 8, c->f.v, vcells * 8, cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(save + rbytes + (cells + vcells) * 8, c->f.w, cells * 8, cudaMemcpyDeviceToDevice, c->stream);
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int bestP = c->P, bestMode = c->part_req;
  float best = 1e30f;
  for (int P = 1; P <= 32; P <<= 1) {
    if (nx % P || !x_partition_ok(P, nx / P)) continue;
    for (int mode : {NS_PART_AUTO, NS_PART_PPT}) {
      if (ns_set_partition(c, 0, P, mode) != NS_OK) continue;
      if (mode == NS_PART_PPT && c->part_mode != NS_PART_PPT) continue;
      const float ms = time_sweep(c, 0, e0, e1);
      if (ms >= 0 && ms < best) {
        best = ms;
        bestP = P;
        bestMode = mode;
      }
    }
  }
  ns_status st = ns_set_partition(c, 0, bestP, bestMode);
  for (int dir = 1; dir <= 2 && tune_lines && st == NS_OK; ++dir) {
    const int Pl = line_partition(dir == 1 ? c->cfg.ny : c->cfg.nz);
    if (!Pl) continue;
    int bestL = dir == 1 ? c->yP : c->zP;
    float bl = 1e30f;
    for (int P : {Pl, 0}) {
      if (ns_set_partition(c, dir, P, NS_PART_AUTO) != NS_OK) continue;
      const float ms = time_sweep(c, dir, e0, e1);
      if (ms >= 0 && ms < bl) {
        bl = ms;
        bestL = P;
      }
    }
    st = ns_set_partition(c, dir, bestL, NS_PART_AUTO);
  }
  cudaMemcpyAsync(c->ru, save, rbytes, cudaMemcpyDeviceToDevice, c->stream);
  if (tune_lines) {
    cudaMemcpyAsync(c->f.u, save + rbytes, cells * 8, cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(c->f.v, save + rbytes + cells * 8, vcells * 8, cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(c->f.w, save + rbytes + (cells + vcells) * 8, cells * 8, cudaMemcpyDeviceToDevice, c->stream);
  }
  cudaStreamSynchronize(c->stream);
  cudaFree(save);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}

}  // extern "C++"

ns_status ns_autotune(ns_ctx* c) { return autotune_ctx(c, true); }

ns_status ns_get_buffer(ns_ctx* c, int which, void** ptr, size_t* bytes) {
  if (!c || !ptr) return NS_ERR_ARG;
  static const int map[8] = {LB_RU, LB_RV, LB_RW, LB_NU, LB_NV, LB_NW, LB_PHI, LB_SPEC};
  if (which < 0 || which > 8) return fail(c, NS_ERR_ARG, "unknown buffer");
  const size_t nx = c->cfg.nx, ny = c->cfg.ny, nz = c->cfg.nz;
  if (which == NS_BUF_POIS_MODE) {
    if (!c->pois32) return fail(c, NS_ERR_UNSUPPORTED, "the Poisson mode flags exist only in the mixed form");
    *ptr = c->pois_mode;
    if (bytes) *bytes = (size_t)c->nzh * nx;
    return NS_OK;
  }
  const int b = map[which];
  size_t n;
  switch (which) {
    case NS_BUF_RV:
    case NS_BUF_NV: n = nx * (ny + 1) * nz * c->es; break;
    case NS_BUF_PHI: n = nx * ny * nz * 8; break;
    case NS_BUF_SPEC: n = (size_t)c->nzh * ny * nx * 16; break;
    default: n = nx * ny * nz * c->es;
  }
  *ptr = (char*)c->ws + c->lay.off[b];
  if (bytes) *bytes = n;
  return NS_OK;
}

ns_status ns_sync(ns_ctx* c) {
  if (!c) return NS_ERR_ARG;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "stream");
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "async");
  return NS_OK;
}

const char* ns_last_error(ns_ctx* c) {
  if (!c) return g_init_error.c_str();
  return c->err.c_str();
}

void ns_destroy(ns_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  drop_graph(c);
  for (int q = 0; q < c->npev; ++q) cudaEventDestroy(c->pev[q]);
  cudaStreamDestroy(c->cap_stream);
  if (c->side_stream) cudaStreamDestroy(c->side_stream);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->pin) cudaFreeHost(c->pin);
  if (c->own_ws) cudaFree(c->ws);
  delete c;
}

}  // extern "C"
