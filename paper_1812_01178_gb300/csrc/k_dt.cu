// The tables that depend on dt, built on the host (ns_init, ns_set_dt) and on the device (the
// fixed-CFL step graph: convective rate -> dt = cfl / rate -> every table -> the step, with no
// host round trip).  Both builders run the same functions (dt_tables.cuh), and this translation
// unit is compiled without floating-point contraction on either side (nvcc -fmad=false, host
// -ffp-contract=off), so they round every operation alike and give bitwise equal tables.
#include <algorithm>
#include <cstring>
#include <vector>

#include "dt_tables.cuh"

namespace {

__host__ __device__ int ilog2c(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

DtSpec dt_spec(const ns_ctx* c, bool device) {
  DtSpec s;
  s.nx = c->cfg.nx;
  s.ny = c->cfg.ny;
  s.nz = c->cfg.nz;
  s.es = c->es;
  s.bl = c->bl;
  s.P = c->P;
  s.M = c->M;
  s.yP = c->yP;
  s.zP = c->zP;
  s.part_req = c->part_req;
  s.kim_moin = c->cfg.pressure_update == NS_PRESSURE_KIM_MOIN;
  s.dt = c->cfg.dt;
  s.re = c->cfg.re;
  s.dx = c->dx;
  s.dz = c->dz;
  s.fx = c->cfg.fx;
  s.u_conv = c->cfg.u_conv;
  s.gc = device ? c->gc : c->gc_h.data();
  return s;
}

// a double table in the context's element type
cudaError_t upload_tab(ns_ctx* c, void* dst, const double* src, size_t n) {
  if (c->es == 8) return upload_raw(c, dst, src, n * 8);
  std::vector<float> f(src, src + n);
  return upload_raw(c, dst, f.data(), n * 4);
}

// the partitioned-line directions of the mixed form: q = 0 y centres, 1 y faces, 2 z
struct LineDir {
  int n, P;
  bool cyclic;
};
LineDir line_dir(const DtSpec& s, int q) {
  return q < 2 ? LineDir{s.ny, s.yP, false} : LineDir{s.nz, s.zP, true};
}

// Partitioned y and z line tables of the mixed form for every sub-step.  PDD per direction when the
// coupling it drops stays below the FP32 tolerance for every sub-step, else PPT.
ns_status build_line_tables(ns_ctx* c, const DtSpec& s) {
  if (!c->yP && !c->zP) return NS_OK;
  std::vector<double> t[3][3];
  double drop[2] = {0.0, 0.0};  // y, z
  for (int k = 0; k < 3; ++k)
    for (int q = 0; q < 3; ++q) {
      const LineDir d = line_dir(s, q);
      if (!d.P) continue;
      t[k][q].assign(xtab_count(d.n / d.P, d.P, ilog2c(d.P)), 0.0);
      auto row = [&](int i, double& a, double& b, double& cc) { line_row(s, k, q, i, a, b, cc); };
      for (int r = 0; r < d.P; ++r) xtab_phase1_part(d.n, d.P, r, d.cyclic, row, t[k][q].data());
      double& dq = drop[q < 2 ? 0 : 1];
      dq = std::fmax(dq, xtab_drop(d.n, d.P, d.cyclic, t[k][q].data()));
    }
  c->ypdd_drop = drop[0];
  c->zpdd_drop = drop[1];
  std::vector<double> scr(xtab_scratch_doubles(32));
  for (int k = 0; k < 3; ++k)
    for (int q = 0; q < 3; ++q) {
      const LineDir d = line_dir(s, q);
      if (!d.P) continue;
      const int mode = drop[q < 2 ? 0 : 1] <= pdd_tol(4) ? NS_PART_PDD : NS_PART_PPT;
      const int L = xtab_phase2(d.n, d.P, d.cyclic, mode, t[k][q].data(), scr.data());
      if (upload_tab(c, c->ptab[k][q], t[k][q].data(), xtab_count(d.n / d.P, d.P, L)) != cudaSuccess)
        return NS_ERR_CUDA;
      if (q == 0) c->yL[k] = L;
      if (q == 2) c->zL[k] = L;
    }
  return NS_OK;
}

// ---------------------------------------------------------------------------------------------
// device builder
// ---------------------------------------------------------------------------------------------
struct DtDev {
  DtSpec s;  // dt is replaced by cfl / rate
  const unsigned long long* rate;
  DtCtl* ctl;
  StepK* stepk;
  double* rtab[3];
  float* rtabf[3];
  void* ytab[3][2];
  void* ztab[3];
  void* xtab[3][2];
  void* ptab[3][3];
  double* scr;  // 6 x tables of xs doubles, 9 line tables of ls, 3 z scratch of 4 nz
  size_t xs, ls;
};

__device__ __forceinline__ double* scr_x(const DtDev& a, int tab) { return a.scr + (size_t)tab * a.xs; }
__device__ __forceinline__ double* scr_line(const DtDev& a, int tab) {
  return a.scr + 6 * a.xs + (size_t)tab * a.ls;
}
__device__ __forceinline__ double* scr_z(const DtDev& a, int k) {
  return a.scr + 6 * a.xs + 9 * a.ls + (size_t)k * 4 * a.s.nz;
}

// dt = cfl / rate, as the host computes it from the rate ns_convective_rate reads; false for a
// rate that is not positive and finite
__device__ __forceinline__ bool dt_of_rate(const DtDev& a, double* dt, double* rate) {
  const double r = __longlong_as_double((long long)*a.rate);
  *rate = r;
  if (!isfinite(r) || !(r > 0.0)) return false;
  *dt = a.ctl->cfl / r;
  return true;
}

// Phase 1: tasks [t0, t1) of: the sub-step constants, the RHS rows (the tables the RHS of sub-step
// 0 reads), then the y and z factors and phase 1 of every partition of the x and line tables.  One
// task per thread, or with per_warp one per warp (lane 0): the long serial tasks then run side by
// side on separate FP64 units instead of one after another in a diverged warp.
__global__ void __launch_bounds__(128) dt_phase1_kernel(const __grid_constant__ DtDev a, int t0, int t1,
                                                        int per_warp) {
  double dt, rate;
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (per_warp && (g & 31)) return;
  int t = t0 + (per_warp ? g >> 5 : g);
  if (t >= t1 || !dt_of_rate(a, &dt, &rate)) return;
  DtSpec s = a.s;
  s.dt = dt;
  if (t < NS_STEPK) {
    StepK sk;
    dt_stepk(s, t, sk);
    a.stepk[t] = sk;  // the levels follow in phase 2
    return;
  }
  t -= NS_STEPK;
  const int G = s.ny + 1;
  if (t < 3 * G) {
    const int k = t / G;
    dt_rtab_row(s, k, t - k * G, a.rtab[k], a.rtabf[k]);
    return;
  }
  t -= 3 * G;
  if (t < 6) {
    dt_ytab(s, t >> 1, t & 1, a.ytab[t >> 1][t & 1]);
    return;
  }
  t -= 6;
  if (t < 3) {
    dt_ztab(s, t, a.ztab[t], scr_z(a, t));
    return;
  }
  t -= 3;
  if (t < 6 * s.P) {
    const int tab = t / s.P, r = t - tab * s.P, k = tab >> 1, cls = tab & 1;
    auto row = [&](int i, double& ra, double& rb, double& rc) { x_row(s, k, cls, i, ra, rb, rc); };
    xtab_phase1_part(s.nx, s.P, r, !s.bl, row, scr_x(a, tab));
    return;
  }
  t -= 6 * s.P;
  for (int q = 0; q < 3; ++q) {
    const int P = q < 2 ? s.yP : s.zP, n = q < 2 ? s.ny : s.nz;
    if (!P) continue;
    if (t < 3 * P) {
      const int k = t / P, r = t - k * P;
      auto row = [&](int i, double& ra, double& rb, double& rc) { line_row(s, k, q, i, ra, rb, rc); };
      xtab_phase1_part(n, P, r, q == 2, row, scr_line(a, 3 * k + q));
      return;
    }
    t -= 3 * P;
  }
}

__device__ int dt_x_mode(const DtDev& a) {
  const DtSpec& s = a.s;
  double drop = 0.0;
  for (int tab = 0; tab < 6; ++tab) drop = fmax(drop, xtab_drop(s.nx, s.P, !s.bl, scr_x(a, tab)));
  if (s.part_req != NS_PART_AUTO) return s.part_req;
  return drop <= pdd_tol(s.es) ? NS_PART_PDD : NS_PART_PPT;
}
__device__ int dt_line_mode(const DtDev& a, bool z) {
  const DtSpec& s = a.s;
  const int P = z ? s.zP : s.yP, n = z ? s.nz : s.ny;
  double drop = 0.0;
  for (int k = 0; k < 3; ++k)
    for (int q = z ? 2 : 0; q < (z ? 3 : 2); ++q) drop = fmax(drop, xtab_drop(n, P, z, scr_line(a, 3 * k + q)));
  return drop <= pdd_tol(4) ? NS_PART_PDD : NS_PART_PPT;
}

// Phase 2: blocks 0..5 the x tables (k, cls), 6..14 the line tables (k, q): the mode from the PDD
// drop of every table of the direction, the reduced system (one thread per partition, a barrier
// between the levels of block cyclic reduction), and the copy in the element type; block 15 the
// levels of the sub-step constants and the dt log.
__global__ void __launch_bounds__(128) dt_phase2_kernel(const __grid_constant__ DtDev a) {
  __shared__ M2 sb[6 * 32];
  __shared__ int sh_mode;
  double dt, rate;
  const bool ok = dt_of_rate(a, &dt, &rate);
  const DtSpec& s = a.s;
  const int b = blockIdx.x;
  if (b == 15) {
    if (threadIdx.x != 0) return;
    DtCtl* ctl = a.ctl;
    const unsigned n = ctl->count;
    if (ok) {
      ctl->dt = dt;
      const int Lx = xtab_levels(s.P, dt_x_mode(a));
      const int Ly = s.yP ? xtab_levels(s.yP, dt_line_mode(a, false)) : 0;
      const int Lz = s.zP ? xtab_levels(s.zP, dt_line_mode(a, true)) : 0;
      for (int k = 0; k < 3; ++k) {
        a.stepk[k].L = Lx;
        a.stepk[k].Ly = Ly;
        a.stepk[k].Lz = Lz;
        for (int cls = 0; cls < 2; ++cls)
          a.stepk[k].xhalf[cls] = xtab_half(s.nx, s.P, scr_x(a, 2 * k + cls), x_half_tol(s.es));
      }
    } else if (ctl->status == 0) {
      ctl->status = isfinite(rate) ? 2u : 1u;
      ctl->fail_step = n;
    }
    if (n < (unsigned)NS_DTLOG) ctl->dts[n] = ctl->dt;
    ctl->count = n + 1;
    return;
  }
  if (!ok) return;
  int n, P, q = 0;
  double* t;
  void* dst;
  if (b < 6) {
    n = s.nx;
    P = s.P;
    t = scr_x(a, b);
    dst = a.xtab[b >> 1][b & 1];
  } else {
    const int tab = b - 6;
    q = tab % 3;
    P = q < 2 ? s.yP : s.zP;
    n = q < 2 ? s.ny : s.nz;
    if (!P) return;
    t = scr_line(a, tab);
    dst = a.ptab[tab / 3][q];
  }
  const bool cyclic = b < 6 ? !s.bl : q == 2;
  if (threadIdx.x == 0) sh_mode = b < 6 ? dt_x_mode(a) : dt_line_mode(a, q == 2);
  __syncthreads();
  const int mode = sh_mode, M = n / P, L = xtab_levels(P, mode), r = threadIdx.x;
  M2 *Lb = sb, *Db = sb + P, *Ub = sb + 2 * P, *nL = sb + 3 * P, *nD = sb + 4 * P, *nU = sb + 5 * P;
  if (r < P) xtab_p2_init(n, P, cyclic, mode, r, t, Lb, Db, Ub);
  __syncthreads();
  for (int lv = 0; lv < L; ++lv) {
    if (r < P) xtab_p2_level(M, P, L, lv, r, Lb, Db, Ub, nL, nD, nU, t);
    __syncthreads();
    M2* x;
    x = Lb, Lb = nL, nL = x;
    x = Db, Db = nD, nD = x;
    x = Ub, Ub = nU, nU = x;
  }
  if (r < P) xtab_p2_final(M, P, r, Db, t);
  __syncthreads();
  const int cnt = (int)xtab_count(M, P, L);
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) put_es(dst, (size_t)i, t[i], s.es);
}

}  // namespace

// ---------------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------------
cudaError_t upload_raw(ns_ctx* c, void* dst, const void* src, size_t bytes) {
  if (c->dry) return cudaSuccess;
  const size_t off = (size_t)((char*)dst - (char*)c->ws);
  if (c->staging && c->pin && off >= c->pin_lo && off + bytes <= c->pin_hi) {
    memcpy(c->pin + (off - c->pin_lo), src, bytes);
    c->dirty.emplace_back(off, bytes);
    return cudaSuccess;
  }
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return e;
}

// Asynchronous copies of the staged ranges (pinned source: nothing waits).
cudaError_t flush_staging(ns_ctx* c) {
  cudaError_t e = cudaSuccess;
  for (const auto& r : c->dirty)
    if (e == cudaSuccess)
      e = cudaMemcpyAsync((char*)c->ws + r.first, c->pin + (r.first - c->pin_lo), r.second, cudaMemcpyHostToDevice,
                          c->stream);
  c->dirty.clear();
  return e;
}

size_t dt_scratch_doubles(int nz, size_t xs, size_t ls) {
  return 6 * xs + 9 * ls + 12 * (size_t)nz;
}

// RHS rows (FP64 and an FP32 copy) and the ADI y and z factors of every sub-step.
ns_status build_dt_tables(ns_ctx* c) {
  const DtSpec s = dt_spec(c, false);
  const int ny = s.ny, nz = s.nz, G = ny + 1;
  char* base = (char*)c->ws;
  std::vector<double> rt((size_t)RT_COUNT * G);
  std::vector<float> rtf((size_t)RT_COUNT * G);
  ns_status st = NS_OK;
  for (int k = 0; k < 3 && st == NS_OK; ++k) {
    c->rtab[k] = (double*)(base + c->lay.off[LB_RTAB] + k * al256((size_t)RT_COUNT * G * 8));
    c->rtabf[k] = (float*)(base + c->lay.off[LB_RTAB] + 3 * al256((size_t)RT_COUNT * G * 8) +
                           k * al256((size_t)RT_COUNT * G * 4));
    for (int j = 0; j < G; ++j) dt_rtab_row(s, k, j, rt.data(), rtf.data());
    if (upload_raw(c, c->rtab[k], rt.data(), rt.size() * 8) != cudaSuccess ||
        upload_raw(c, c->rtabf[k], rtf.data(), rtf.size() * 4) != cudaSuccess)
      st = NS_ERR_CUDA;
  }
  std::vector<unsigned char> buf;
  std::vector<double> scr(4 * (size_t)nz);
  for (int k = 0; k < 3 && st == NS_OK; ++k) {
    for (int cls = 0; cls < 2 && st == NS_OK; ++cls) {
      const int n = cls == 0 ? ny : ny - 1;
      buf.assign(3 * (size_t)n * s.es, 0);
      dt_ytab(s, k, cls, buf.data());
      if (upload_raw(c, c->ytab[k][cls], buf.data(), buf.size()) != cudaSuccess) st = NS_ERR_CUDA;
    }
    buf.assign(ztab_entries(nz) * s.es, 0);
    dt_ztab(s, k, buf.data(), scr.data());
    if (st == NS_OK && upload_raw(c, c->ztab[k], buf.data(), buf.size()) != cudaSuccess) st = NS_ERR_CUDA;
  }
  if (st == NS_OK && !c->staging && !c->dry && cudaStreamSynchronize(c->stream) != cudaSuccess) st = NS_ERR_CUDA;
  return st;
}

// x-solver tables of every sub-step and line class with the context's P and requested mode (PDD
// when its dropped coupling is below the tolerance of the precision), the partitioned-line tables,
// and the sub-step constants.
ns_status build_x_tables(ns_ctx* c) {
  const DtSpec s = dt_spec(c, false);
  const int nx = s.nx, P = c->P, M = c->M;
  const bool cyclic = !c->bl;
  std::vector<double> t[3][2];
  double drop = 0.0;
  for (int k = 0; k < 3; ++k)
    for (int cls = 0; cls < 2; ++cls) {
      t[k][cls].assign(xtab_count(M, P, ilog2c(P)), 0.0);
      auto row = [&](int i, double& a, double& b, double& cc) { x_row(s, k, cls, i, a, b, cc); };
      for (int r = 0; r < P; ++r) xtab_phase1_part(nx, P, r, cyclic, row, t[k][cls].data());
      drop = std::fmax(drop, xtab_drop(nx, P, cyclic, t[k][cls].data()));
    }
  int half[3][2];
  for (int k = 0; k < 3; ++k)
    for (int cls = 0; cls < 2; ++cls) half[k][cls] = xtab_half(nx, P, t[k][cls].data(), x_half_tol(c->es));
  int mode = c->part_req;
  if (mode == NS_PART_AUTO) mode = drop <= pdd_tol(c->es) ? NS_PART_PDD : NS_PART_PPT;
  c->part_mode = mode;
  c->pdd_drop = drop;
  std::vector<double> scr(xtab_scratch_doubles(P));
  for (int k = 0; k < 3; ++k)
    for (int cls = 0; cls < 2; ++cls) {
      const int L = xtab_phase2(nx, P, cyclic, mode, t[k][cls].data(), scr.data());
      c->L[k] = L;
      const size_t n = xtab_count(M, P, L);
      if (n > c->xtab_stride) return NS_ERR_SIZE;
      if (upload_tab(c, c->xtab[k][cls], t[k][cls].data(), n) != cudaSuccess) return NS_ERR_CUDA;
    }
  const ns_status ls = build_line_tables(c, s);
  if (ls != NS_OK) return ls;
  for (int q = 0; q < NS_STEPK; ++q) {
    dt_stepk(s, q, c->stepk_h[q]);
    if (q < 3) {
      c->stepk_h[q].L = c->L[q];
      c->stepk_h[q].Ly = c->yL[q];
      c->stepk_h[q].Lz = c->zL[q];
      c->stepk_h[q].xhalf[0] = half[q][0];
      c->stepk_h[q].xhalf[1] = half[q][1];
    }
  }
  if (upload_raw(c, c->stepk, c->stepk_h, sizeof(c->stepk_h)) != cudaSuccess) return NS_ERR_CUDA;
  if (!c->staging && !c->dry && cudaStreamSynchronize(c->stream) != cudaSuccess) return NS_ERR_CUDA;
  return NS_OK;
}

// The device-side dt update on c->launch (capturable): from c->rate and c->dtctl->cfl it rewrites
// every dt-dependent table, as build_dt_tables and build_x_tables would.  part 0: the sub-step
// constants and RHS rows (what the RHS of sub-step 0 reads); part 1: everything else (ADI factors,
// x and line tables, levels, the dt log), which may run beside that RHS.
cudaError_t launch_dt_update(ns_ctx* c, int part) {
  DtDev a;
  a.s = dt_spec(c, true);
  a.rate = c->rate;
  a.ctl = c->dtctl;
  a.stepk = c->stepk;
  for (int k = 0; k < 3; ++k) {
    a.rtab[k] = c->rtab[k];
    a.rtabf[k] = c->rtabf[k];
    a.ztab[k] = c->ztab[k];
    for (int q = 0; q < 2; ++q) {
      a.ytab[k][q] = c->ytab[k][q];
      a.xtab[k][q] = c->xtab[k][q];
    }
    for (int q = 0; q < 3; ++q) a.ptab[k][q] = c->ptab[k][q];
  }
  a.scr = c->dtscr;
  a.xs = c->dt_xs;
  a.ls = c->dt_ls;
  const int quick = NS_STEPK + 3 * (a.s.ny + 1);
  const int tasks = quick + 6 + 3 + 6 * a.s.P + 6 * a.s.yP + 3 * a.s.zP;
  if (part == 0) {
    dt_phase1_kernel<<<(quick + 127) / 128, 128, 0, c->launch>>>(a, 0, quick, 0);
    return cudaGetLastError();
  }
  dt_phase1_kernel<<<(32 * (tasks - quick) + 127) / 128, 128, 0, c->launch>>>(a, quick, tasks, 1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  dt_phase2_kernel<<<16, 128, 0, c->launch>>>(a);
  return cudaGetLastError();
}
