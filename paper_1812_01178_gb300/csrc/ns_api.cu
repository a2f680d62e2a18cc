// C ABI entry points, workspace layout, coefficient tables and graph capture.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "ns_internal.cuh"

namespace {

thread_local std::string g_init_error;


size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

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
  sz[LB_XTAB] = 6 * al256((5 * nx + 4 * 32 + 8 * 5 * 32) * es);
  sz[LB_YTAB] = 6 * al256(3 * ny * es);
  sz[LB_ZTAB] = 3 * al256((4 * nz + 2) * es);
  sz[LB_TWZ] = fft_twiddle_doubles((int)nz) * 8;
  sz[LB_TWX] = fft_twiddle_doubles((int)nx) * 8;
  sz[LB_LAMX] = nx * 8;
  sz[LB_LAMZ] = nzh * 8;
  sz[LB_RTAB] = 3 * al256((size_t)RT_COUNT * (ny + 1) * 8) + 3 * al256((size_t)RT_COUNT * (ny + 1) * 4);
  sz[LB_DOUT] = 3 * al256((ny + 1) * nz * 8) + 256;
  sz[LB_TWD] = nx * 16;
  sz[LB_RCY] = recycle_block_doubles((int)ny) * 8;
  sz[LB_STEPK] = NS_STEPK * sizeof(StepK);
  sz[LB_PTAB] = 9 * al256(line_table_floats(c) * 4);
  size_t o = 0;
  for (int b = 0; b < LB_COUNT; ++b) {
    L.off[b] = o;
    o += al256(sz[b]);
  }
  L.total = o;
  return L;
}

// --------------------------------------------------------------------------------------------
// tridiagonal helpers (host, double)
// --------------------------------------------------------------------------------------------
// Thomas factors of rows (a, b, c), a[0] and c[n-1] ignored: inv = 1/pivot, ainv = a/pivot, cp = c/pivot.
void thomas_factors(const std::vector<double>& a, const std::vector<double>& b, const std::vector<double>& c,
                    std::vector<double>& inv, std::vector<double>& ainv, std::vector<double>& cp) {
  const size_t n = b.size();
  inv.assign(n, 0.0);
  ainv.assign(n, 0.0);
  cp.assign(n, 0.0);
  double cprev = 0.0;
  for (size_t j = 0; j < n; ++j) {
    const double aj = j > 0 ? a[j] : 0.0;
    const double cj = j + 1 < n ? c[j] : 0.0;
    const double piv = b[j] - aj * cprev;
    inv[j] = 1.0 / piv;
    ainv[j] = aj * inv[j];
    cp[j] = cj * inv[j];
    cprev = cp[j];
  }
}

std::vector<double> thomas_apply(const std::vector<double>& inv, const std::vector<double>& ainv,
                                 const std::vector<double>& cp, std::vector<double> d) {
  const size_t n = d.size();
  d[0] *= inv[0];
  for (size_t j = 1; j < n; ++j) d[j] = d[j] * inv[j] - ainv[j] * d[j - 1];
  for (size_t j = n - 1; j-- > 0;) d[j] -= cp[j] * d[j + 1];
  return d;
}

struct M2 {
  double a, b, c, d;  // [[a, b], [c, d]]
};
M2 mmul(M2 x, M2 y) {
  return {x.a * y.a + x.b * y.c, x.a * y.b + x.b * y.d, x.c * y.a + x.d * y.c, x.c * y.b + x.d * y.d};
}
M2 madd(M2 x, M2 y) { return {x.a + y.a, x.b + y.b, x.c + y.c, x.d + y.d}; }
M2 msub(M2 x, M2 y) { return {x.a - y.a, x.b - y.b, x.c - y.c, x.d - y.d}; }
M2 minv(M2 x) {
  const double det = x.a * x.d - x.b * x.c;
  return {x.d / det, -x.b / det, -x.c / det, x.a / det};
}
M2 mzero() { return {0, 0, 0, 0}; }

// Partitioned x solver tables (Sec. 3.2) for the rows (a, b, c) of one x-line of n = P*M rows,
// periodic (cyclic) or not.  mode: NS_PART_PDD or NS_PART_PPT.  Per partition r: the block
// Thomas factors of A~ (couplings to the neighbouring partitions cut), the spikes v^(r), w^(r)
// of Eq. (blockAY) (zero where no coupling was cut: the ends of a non-periodic line), and the
// 2x2-block reduced system Z of Eq. (Zpdd) over the interfaces (r, r+1):
//   L_r Y_{r-1} + D_r Y_r + U_r Y_{r+1} = (x~^(r)_m, x~^(r+1)_1),
//   D_r = [[1, w^(r)_m], [v^(r+1)_1, 1]], L_r = [[v^(r)_m, 0], [0, 0]], U_r = [[0, 0], [0, w^(r+1)_1]];
// a non-periodic line has P-1 interfaces and a decoupled identity row in slot P-1.  PDD keeps D_r;
// PPT eliminates L, U by block parallel cyclic reduction (multipliers stored per level).
// Returns the table, the number of reduction levels and the largest coupling PDD drops.
std::vector<double> build_xtab(const std::vector<double>& A, const std::vector<double>& Bv,
                               const std::vector<double>& Cv, int P, bool cyclic, int mode, int* levels,
                               double* dropped) {
  const int n = (int)Bv.size();
  const int M = n / P;
  int L = 0;
  while ((1 << L) < P) ++L;
  std::vector<double> inv(n), ainv(n), cp(n), sv(n, 0.0), sw(n, 0.0);
  for (int r = 0; r < P; ++r) {
    const int o = r * M;
    std::vector<double> a(A.begin() + o, A.begin() + o + M), b(Bv.begin() + o, Bv.begin() + o + M),
        c(Cv.begin() + o, Cv.begin() + o + M), i1, i2, i3;
    thomas_factors(a, b, c, i1, i2, i3);  // a[0], c[M-1] (the cut couplings) are ignored
    std::copy(i1.begin(), i1.end(), inv.begin() + o);
    std::copy(i2.begin(), i2.end(), ainv.begin() + o);
    std::copy(i3.begin(), i3.end(), cp.begin() + o);
    std::vector<double> e1(M, 0.0), em(M, 0.0);
    if (cyclic || r > 0) e1[0] = A[o];                 // a of the first row couples partition r-1
    if (cyclic || r < P - 1) em[M - 1] = Cv[o + M - 1];  // c of the last row couples partition r+1
    const std::vector<double> v1 = thomas_apply(i1, i2, i3, e1), w1 = thomas_apply(i1, i2, i3, em);
    std::copy(v1.begin(), v1.end(), sv.begin() + o);
    std::copy(w1.begin(), w1.end(), sw.begin() + o);
  }
  auto V = [&](int r, int e) { return sv[r * M + e]; };
  auto W = [&](int r, int e) { return sw[r * M + e]; };
  std::vector<M2> Lb(P), Db(P), Ub(P);
  double drop = 0.0;
  for (int r = 0; r < P; ++r) {
    const int rn = (r + 1) % P;
    if (!cyclic && r == P - 1) {
      Db[r] = {1.0, 0.0, 0.0, 1.0};
      Lb[r] = mzero();
      Ub[r] = mzero();
      continue;
    }
    Db[r] = {1.0, W(r, M - 1), V(rn, 0), 1.0};
    Lb[r] = {V(r, M - 1), 0.0, 0.0, 0.0};
    Ub[r] = {0.0, 0.0, 0.0, W(rn, 0)};
    drop = std::fmax(drop, std::fmax(std::fabs(Lb[r].a), std::fabs(Ub[r].d)));
  }
  *dropped = drop;
  std::vector<M2> MLs, MUs;  // per level, per r
  if (mode == NS_PART_PPT && P == 1) {
    // one partition: both couplings of the single interface point back at itself
    Db[0] = madd(Db[0], madd(Lb[0], Ub[0]));
  }
  if (mode == NS_PART_PPT) {
    for (int lv = 0, st = 1; lv < L; ++lv, st <<= 1) {
      std::vector<M2> nL(P), nD(P), nU(P);
      for (int r = 0; r < P; ++r) {
        const int rm = ((r - st) % P + P) % P, rp = (r + st) % P;
        M2 ml, mu;
        if (rm == rp) {
          ml = mmul(madd(Lb[r], Ub[r]), minv(Db[rm]));
          mu = mzero();
          nD[r] = msub(Db[r], mmul(ml, madd(Lb[rm], Ub[rm])));
          nL[r] = mzero();
          nU[r] = mzero();
        } else {
          ml = mmul(Lb[r], minv(Db[rm]));
          mu = mmul(Ub[r], minv(Db[rp]));
          nD[r] = msub(msub(Db[r], mmul(ml, Ub[rm])), mmul(mu, Lb[rp]));
          // new couplings at distance 2 st; when they coincide (4 st = P) the next level folds them
          nL[r] = msub(mzero(), mmul(ml, Lb[rm]));
          nU[r] = msub(mzero(), mmul(mu, Ub[rp]));
        }
        MLs.push_back(ml);
        MUs.push_back(mu);
      }
      Lb = nL;
      Db = nD;
      Ub = nU;
    }
  } else {
    L = 0;
  }
  std::vector<double> t(xtab_count(M, P, L), 0.0);
  for (int r = 0; r < P; ++r)
    for (int e = 0; e < M; ++e) {
      t[(XT_INV * M + e) * P + r] = inv[r * M + e];
      t[(XT_AINV * M + e) * P + r] = ainv[r * M + e];
      t[(XT_CP * M + e) * P + r] = cp[r * M + e];
      t[(XT_V * M + e) * P + r] = V(r, e);
      t[(XT_W * M + e) * P + r] = W(r, e);
    }
  const size_t d0 = (size_t)XT_NF * M * P;
  for (int r = 0; r < P; ++r) {
    const M2 di = minv(Db[r]);
    t[d0 + r] = di.a;
    t[d0 + P + r] = di.b;
    t[d0 + 2 * P + r] = di.c;
    t[d0 + 3 * P + r] = di.d;
  }
  const size_t m0 = d0 + 4 * (size_t)P, u0 = m0 + 4 * (size_t)L * P;
  for (int lv = 0; lv < L; ++lv)
    for (int r = 0; r < P; ++r) {
      const M2 ml = MLs[(size_t)lv * P + r], mu = MUs[(size_t)lv * P + r];
      t[m0 + (4 * lv + 0) * P + r] = ml.a;
      t[m0 + (4 * lv + 1) * P + r] = ml.b;
      t[m0 + (4 * lv + 2) * P + r] = ml.c;
      t[m0 + (4 * lv + 3) * P + r] = ml.d;
      t[u0 + (4 * lv + 0) * P + r] = mu.a;
      t[u0 + (4 * lv + 1) * P + r] = mu.b;
      t[u0 + (4 * lv + 2) * P + r] = mu.c;
      t[u0 + (4 * lv + 3) * P + r] = mu.d;
    }
  *levels = L;
  return t;
}

cudaError_t upload_d(ns_ctx* c, void* dst, const std::vector<double>& src);

// Copy a host table to the device in the context's element type (double or float).  Waits for
// the copy, so the host vector may be released afterwards.
// Host -> workspace copy of a table.  While c->staging, the bytes go to the pinned mirror and
// the range is recorded (flush_staging copies it); otherwise a copy followed by a stream sync.
cudaError_t upload_raw(ns_ctx* c, void* dst, const void* src, size_t bytes) {
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

cudaError_t upload(ns_ctx* c, void* dst, const std::vector<double>& src) {
  if (c->es == 8) return upload_d(c, dst, src);
  std::vector<float> f(src.begin(), src.end());
  return upload_raw(c, dst, f.data(), f.size() * 4);
}

cudaError_t upload_d(ns_ctx* c, void* dst, const std::vector<double>& src) {
  return upload_raw(c, dst, src.data(), src.size() * 8);
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

// The dt-dependent kernel constants of every sub-step (StepK) from cfg.dt and the x-solver levels.
cudaError_t upload_step_constants(ns_ctx* c) {
  const double dt = c->cfg.dt, nxz = (double)c->cfg.nx * c->cfg.nz;
  const double inv_re = c->cfg.re > 0 ? 1.0 / c->cfg.re : 0.0;
  for (int k = 0; k < 3; ++k) {
    StepK& sk = c->stepk_h[k];
    memset(&sk, 0, sizeof(sk));
    rhs_fill_step(c, k, sk);
    const double sc = NS_ALPHA[k] * dt;
    sk.dt = dt;
    sk.pscale = 1.0 / sc / nxz;
    sk.sx = sc / c->dx;
    sk.sz = sc / c->dz;
    sk.s = sc;
    sk.beta_p = c->cfg.pressure_update == NS_PRESSURE_KIM_MOIN ? sc * inv_re / 2.0 : 0.0;
    const double step = sc * c->cfg.u_conv;
    sk.cu = step / c->dx;
    sk.cv = step / (0.5 * c->dx);
    const double rx = NS_ALPHA[k] * dt * inv_re / 2.0 / (c->dx * c->dx);
    sk.xcf[0] = rx;  // u: the outflow face is the neighbour of the last unknown face
    sk.xcf[1] = 2.0 * rx;  // v, w: linear ghost 2 f_out - f_last
    sk.xcf[2] = 2.0 * rx;
    for (int q = 0; q < 3; ++q) sk.xcff[q] = (float)sk.xcf[q];
    sk.L = c->L[k];
    sk.Ly = c->yL[k];
    sk.Lz = c->zL[k];
  }
  StepK& s3 = c->stepk_h[3];  // projection of an initial field: scale 1
  memset(&s3, 0, sizeof(s3));
  s3.dt = dt;
  s3.pscale = 1.0 / nxz;
  s3.sx = 1.0 / c->dx;
  s3.sz = 1.0 / c->dz;
  s3.s = 1.0;
  return upload_raw(c, c->stepk, c->stepk_h, sizeof(c->stepk_h));
}

double beta_of(const ns_ctx* c, int k) {
  const double inv_re = c->cfg.re > 0 ? 1.0 / c->cfg.re : 0.0;
  return NS_ALPHA[k] * c->cfg.dt * inv_re / 2.0;
}

// Rows of (I - beta_k delta_xx) on one x-line (Sec. 2.2) for the u lines (cls 0) and the v, w
// lines (cls 1).  Periodic: every row (-r, 1 + 2r, -r), cyclic.  Inflow / outflow: the u line
// holds faces 0..nx-1 with face 0 fixed (identity row) and the outflow face as the neighbour of
// the last row (its increment enters the right-hand side); v, w lines are cell centres whose
// first and last rows see linear ghosts of the boundary faces: b = 1 + 3r there.
void x_rows(const ns_ctx* c, int k, int cls, std::vector<double>& a, std::vector<double>& b,
            std::vector<double>& cc) {
  const int nx = c->cfg.nx;
  const double r = beta_of(c, k) / (c->dx * c->dx);
  a.assign(nx, -r);
  b.assign(nx, 1.0 + 2.0 * r);
  cc.assign(nx, -r);
  if (!c->bl) return;
  a[0] = 0.0;
  cc[nx - 1] = 0.0;
  if (cls == 0) {
    b[0] = 1.0;
    cc[0] = 0.0;
  } else {
    b[0] = 1.0 + 3.0 * r;
    b[nx - 1] = 1.0 + 3.0 * r;
  }
}

// Tables of the partitioned y and z lines of the mixed form (AdiLinePK), every sub-step: the rows
// of the thread-per-line solvers, split into P partitions by build_xtab.  y centres (u, w) and y
// faces (v, with the wall row 0 as an identity row) are not periodic; z is.  PDD when the
// coupling it drops stays below the FP32 tolerance for every sub-step of the direction, else PPT.
ns_status build_line_tables(ns_ctx* c) {
  if (!c->yP && !c->zP) return NS_OK;
  const int ny = c->cfg.ny, nz = c->cfg.nz, G = ny + 1;
  auto GCv = [&](int f, int j) -> double { return c->gc_h[(size_t)f * G + j]; };
  const double tol = 1e-8;
  std::vector<double> tabs[3][3][2];
  int levs[3][3][2];
  double ydrop = 0.0, zdrop = 0.0;
  for (int k = 0; k < 3; ++k) {
    const double beta = beta_of(c, k);
    if (c->yP) {
      std::vector<double> a(ny), b(ny), cc(ny);
      for (int j = 0; j < ny; ++j) {
        a[j] = -beta * GCv(GC_AC, j);
        cc[j] = -beta * GCv(GC_CC, j);
        b[j] = 1.0 + beta * (GCv(GC_AC, j) + GCv(GC_CC, j));
      }
      double d0, d1;
      tabs[k][0][0] = build_xtab(a, b, cc, c->yP, false, NS_PART_PDD, &levs[k][0][0], &d0);
      tabs[k][0][1] = build_xtab(a, b, cc, c->yP, false, NS_PART_PPT, &levs[k][0][1], &d1);
      ydrop = std::fmax(ydrop, d0);
      a.assign(ny, 0.0);
      b.assign(ny, 1.0);
      cc.assign(ny, 0.0);
      for (int j = 1; j < ny; ++j) {
        a[j] = -beta * GCv(GC_AF, j);
        cc[j] = -beta * GCv(GC_CF, j);
        b[j] = 1.0 + beta * (GCv(GC_AF, j) + GCv(GC_CF, j));
      }
      a[1] = 0.0;  // row 0 is the wall (v = 0, identity row)
      tabs[k][1][0] = build_xtab(a, b, cc, c->yP, false, NS_PART_PDD, &levs[k][1][0], &d0);
      tabs[k][1][1] = build_xtab(a, b, cc, c->yP, false, NS_PART_PPT, &levs[k][1][1], &d1);
      ydrop = std::fmax(ydrop, d0);
    }
    if (c->zP) {
      const double r = beta / (c->dz * c->dz);
      std::vector<double> a(nz, -r), b(nz, 1.0 + 2.0 * r), cc(nz, -r);
      double d0, d1;
      tabs[k][2][0] = build_xtab(a, b, cc, c->zP, true, NS_PART_PDD, &levs[k][2][0], &d0);
      tabs[k][2][1] = build_xtab(a, b, cc, c->zP, true, NS_PART_PPT, &levs[k][2][1], &d1);
      zdrop = std::fmax(zdrop, d0);
    }
  }
  c->ypdd_drop = ydrop;
  c->zpdd_drop = zdrop;
  const int ysel = ydrop <= tol ? 0 : 1, zsel = zdrop <= tol ? 0 : 1;
  for (int k = 0; k < 3; ++k) {
    for (int q = 0; q < 3; ++q) {
      const bool on = q < 2 ? c->yP != 0 : c->zP != 0;
      if (!on) continue;
      const int sel = q < 2 ? ysel : zsel;
      if (upload(c, c->ptab[k][q], tabs[k][q][sel]) != cudaSuccess) return NS_ERR_CUDA;
    }
    c->yL[k] = c->yP ? levs[k][0][ysel] : 0;
    c->zL[k] = c->zP ? levs[k][2][zsel] : 0;
  }
  return NS_OK;
}

// x-solver tables for every sub-step and line class with the context's P and requested mode.
ns_status build_x_tables(ns_ctx* c) {
  const double tol = c->es == 8 ? 1e-15 : 1e-8;
  double drop_max = 0.0;
  std::vector<double> tabs[3][2][2];
  int levs[3][2];
  const bool cyclic = !c->bl;
  for (int k = 0; k < 3; ++k)
    for (int cls = 0; cls < 2; ++cls) {
      std::vector<double> a, b, cc;
      x_rows(c, k, cls, a, b, cc);
      double d0, d1;
      tabs[k][cls][0] = build_xtab(a, b, cc, c->P, cyclic, NS_PART_PDD, &levs[k][0], &d0);
      tabs[k][cls][1] = build_xtab(a, b, cc, c->P, cyclic, NS_PART_PPT, &levs[k][1], &d1);
      drop_max = std::fmax(drop_max, d0);
    }
  int mode = c->part_req;
  if (mode == NS_PART_AUTO) mode = drop_max <= tol ? NS_PART_PDD : NS_PART_PPT;
  c->part_mode = mode;
  c->pdd_drop = drop_max;
  const int sel = mode == NS_PART_PDD ? 0 : 1;
  for (int k = 0; k < 3; ++k) {
    c->L[k] = levs[k][sel];
    for (int cls = 0; cls < 2; ++cls) {
      if (tabs[k][cls][sel].size() > c->xtab_stride) return NS_ERR_SIZE;
      if (upload(c, c->xtab[k][cls], tabs[k][cls][sel]) != cudaSuccess) return NS_ERR_CUDA;
    }
  }
  const ns_status ls = build_line_tables(c);
  if (ls != NS_OK) return ls;
  if (upload_step_constants(c) != cudaSuccess) return NS_ERR_CUDA;
  if (!c->staging && cudaStreamSynchronize(c->stream) != cudaSuccess) return NS_ERR_CUDA;
  return NS_OK;
}

// Tables that depend on dt: the RHS rows pre-multiplied by the sub-step constants (FP64 and an
// FP32 copy) and the ADI y and z factors of every sub-step.  The x tables are build_x_tables.
ns_status build_dt_tables(ns_ctx* c) {
  const int ny = c->cfg.ny, nz = c->cfg.nz;
  const int G = ny + 1;
  char* base = (char*)c->ws;
  auto GCv = [&](int f, int j) -> double { return c->gc_h[(size_t)f * G + j]; };
  ns_status st = NS_OK;
  for (int k = 0; k < 3 && st == NS_OK; ++k) {
    c->rtab[k] = (double*)(base + c->lay.off[LB_RTAB] + k * al256((size_t)RT_COUNT * G * 8));
    const double inv_re = c->cfg.re > 0 ? 1.0 / c->cfg.re : 0.0;
    const double cl = c->cfg.dt * NS_ALPHA[k] * inv_re;
    const double dd = 2.0 / (c->dx * c->dx) + 2.0 / (c->dz * c->dz);
    std::vector<double> rt((size_t)RT_COUNT * G, 0.0);
    auto RT = [&](int f, int j) -> double& { return rt[(size_t)f * G + j]; };
    for (int j = 0; j < ny; ++j) {
      RT(RT_AC, j) = cl * GCv(GC_AC, j);
      RT(RT_CC, j) = cl * GCv(GC_CC, j);
      RT(RT_DC, j) = -cl * (dd + GCv(GC_AC, j) + GCv(GC_CC, j));
      RT(RT_HIDY, j) = 0.5 * GCv(GC_IDY, j);
    }
    for (int j = 1; j < ny; ++j) {
      RT(RT_AF, j) = cl * GCv(GC_AF, j);
      RT(RT_CF, j) = cl * GCv(GC_CF, j);
      RT(RT_DF, j) = -cl * (dd + GCv(GC_AF, j) + GCv(GC_CF, j));
      RT(RT_CGY, j) = -c->cfg.dt * NS_ALPHA[k] * GCv(GC_IHC, j);
      RT(RT_QIHC, j) = 0.25 * GCv(GC_IHC, j);
    }
    if (upload_d(c, c->rtab[k], rt) != cudaSuccess) st = NS_ERR_CUDA;
    c->rtabf[k] = (float*)(base + c->lay.off[LB_RTAB] + 3 * al256((size_t)RT_COUNT * G * 8) +
                           k * al256((size_t)RT_COUNT * G * 4));
    {
      std::vector<float> rf(rt.begin(), rt.end());
      if (upload_raw(c, c->rtabf[k], rf.data(), rf.size() * 4) != cudaSuccess) st = NS_ERR_CUDA;
    }
  }
  // ADI y and z factors per sub-step
  for (int k = 0; k < 3 && st == NS_OK; ++k) {
    const double beta = beta_of(c, k);
    {  // centres (u, w): rows j = 0..ny-1
      std::vector<double> a(ny), b(ny), cc(ny), inv, ainv, cp;
      for (int j = 0; j < ny; ++j) {
        a[j] = -beta * GCv(GC_AC, j);
        cc[j] = -beta * GCv(GC_CC, j);
        b[j] = 1.0 + beta * (GCv(GC_AC, j) + GCv(GC_CC, j));
      }
      thomas_factors(a, b, cc, inv, ainv, cp);
      std::vector<double> t;
      t.insert(t.end(), inv.begin(), inv.end());
      t.insert(t.end(), ainv.begin(), ainv.end());
      t.insert(t.end(), cp.begin(), cp.end());
      if (upload(c, c->ytab[k][0], t) != cudaSuccess) st = NS_ERR_CUDA;
    }
    {  // faces (v): rows j = 1..ny-1
      const int n = ny - 1;
      std::vector<double> a(n), b(n), cc(n), inv, ainv, cp;
      for (int q = 0; q < n; ++q) {
        const int j = q + 1;
        a[q] = -beta * GCv(GC_AF, j);
        cc[q] = -beta * GCv(GC_CF, j);
        b[q] = 1.0 + beta * (GCv(GC_AF, j) + GCv(GC_CF, j));
      }
      thomas_factors(a, b, cc, inv, ainv, cp);
      std::vector<double> t;
      t.insert(t.end(), inv.begin(), inv.end());
      t.insert(t.end(), ainv.begin(), ainv.end());
      t.insert(t.end(), cp.begin(), cp.end());
      if (upload(c, c->ytab[k][1], t) != cudaSuccess) st = NS_ERR_CUDA;
    }
    {  // z: cyclic rows (-r, 1 + 2r, -r) by Sherman-Morrison
      const double r = beta / (c->dz * c->dz);
      const double lo = -r, di = 1.0 + 2.0 * r, up = -r;
      const double gam = -di, alpha = up /* A[n-1][0] */, bet = lo /* A[0][n-1] */;
      std::vector<double> a(nz, lo), b(nz, di), cc(nz, up), inv, ainv, cp;
      b[0] = di - gam;
      b[nz - 1] = di - alpha * bet / gam;
      thomas_factors(a, b, cc, inv, ainv, cp);
      std::vector<double> s(nz, 0.0);
      s[0] = gam;
      s[nz - 1] = alpha;
      std::vector<double> q = thomas_apply(inv, ainv, cp, s);
      const double bg = bet / gam;
      const double fac = 1.0 / (1.0 + q[0] + bg * q[nz - 1]);
      std::vector<double> t;
      t.insert(t.end(), inv.begin(), inv.end());
      t.insert(t.end(), ainv.begin(), ainv.end());
      t.insert(t.end(), cp.begin(), cp.end());
      t.insert(t.end(), q.begin(), q.end());
      t.push_back(fac);
      t.push_back(bg);
      if (upload(c, c->ztab[k], t) != cudaSuccess) st = NS_ERR_CUDA;
    }
  }
  if (st == NS_OK && !c->staging && cudaStreamSynchronize(c->stream) != cudaSuccess) st = NS_ERR_CUDA;
  return st;
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
    {"project", launch_project},              // A10
};
const int NSTAGES = (int)(sizeof(STAGES) / sizeof(STAGES[0]));

ns_status run_substep(ns_ctx* c, int k, cudaEvent_t* ev = nullptr) {
  for (int q = 0; q < NSTAGES; ++q) {
    if (ev) cudaEventRecordWithFlags(ev[q], c->launch, cudaEventRecordExternal);
    cudaError_t e = STAGES[q].fn(c, k);
    if (e != cudaSuccess) return cuda_fail(c, e, STAGES[q].name);
  }
  return NS_OK;
}

// Capture the three sub-steps of one time step into a graph (optionally with event nodes) and
// instantiate it.
ns_status capture_step(ns_ctx* c, bool profiled, cudaGraph_t* graph, cudaGraphExec_t* exec) {
  c->launch = c->cap_stream;
  cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    c->launch = c->stream;
    return cuda_fail(c, e, "begin capture");
  }
  ns_status s = NS_OK;
  for (int k = 0; k < 3 && s == NS_OK; ++k) s = run_substep(c, k, profiled ? c->pev + k * NSTAGES : nullptr);
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
  c->xtab_stride = (5 * (size_t)nx + 4 * 32 + 8 * 5 * 32);
  for (int k = 0; k < 3; ++k) {
    for (int cls = 0; cls < 2; ++cls)
      c->xtab[k][cls] = base + c->lay.off[LB_XTAB] + (2 * k + cls) * al256(c->xtab_stride * c->es);
    for (int q = 0; q < 2; ++q) c->ytab[k][q] = base + c->lay.off[LB_YTAB] + (2 * k + q) * al256(3 * ny * c->es);
    c->ztab[k] = base + c->lay.off[LB_ZTAB] + k * al256((4 * nz + 2) * c->es);
  }
  c->twz = (double2*)(base + c->lay.off[LB_TWZ]);
  c->twx = (double2*)(base + c->lay.off[LB_TWX]);
  double* lamx_d = (double*)(base + c->lay.off[LB_LAMX]);
  for (int q = 0; q < 3; ++q) c->dout[q] = (double*)(base + c->lay.off[LB_DOUT] + q * al256((size_t)(ny + 1) * nz * 8));
  c->flux = (double*)(base + c->lay.off[LB_DOUT] + 3 * al256((size_t)(ny + 1) * nz * 8));
  c->rate = (unsigned long long*)(c->flux + 4);
  c->rcy = (double*)(base + c->lay.off[LB_RCY]);
  c->stepk = (StepK*)(base + c->lay.off[LB_STEPK]);
  c->yP = line_P(cfg, cfg->ny);
  c->zP = line_P(cfg, cfg->nz);
  for (int k = 0; k < 3; ++k)
    for (int q = 0; q < 3; ++q)
      c->ptab[k][q] = base + c->lay.off[LB_PTAB] + (3 * k + q) * al256(line_table_floats(cfg) * 4);
  c->twd = (double2*)(base + c->lay.off[LB_TWD]);
  double* lamz_d = (double*)(base + c->lay.off[LB_LAMZ]);

  // ---------------- grid coefficients (Sec. 2.1 / 2.2 readings)
  const std::vector<double>& yf = c->yf;
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
    c->rhs_bps[0] = c->rhs_bps[1] = 1;
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
    std::vector<double> td(2 * nx);
    for (int q = 0; q < nx; ++q) {
      td[2 * q] = std::cos(PI * q / (2.0 * nx));
      td[2 * q + 1] = -std::sin(PI * q / (2.0 * nx));
    }
    if (upload_d(c, c->twd, td) != cudaSuccess) st = NS_ERR_CUDA;
    for (int q = 0; q < c->nzh; ++q) lz[q] = (2.0 / (c->dz * c->dz)) * (1.0 - std::cos(2.0 * PI * q / nz));
    if (upload_d(c, lamx_d, lx) != cudaSuccess) st = NS_ERR_CUDA;
    if (upload_d(c, lamz_d, lz) != cudaSuccess) st = NS_ERR_CUDA;
    if (st == NS_OK && poisson_set_attributes() != cudaSuccess) st = NS_ERR_CUDA;
    if (st == NS_OK && rhs_set_attributes(&c->rhs_bps[0], &c->rhs_bps[1]) != cudaSuccess) st = NS_ERR_CUDA;
    if (st == NS_OK && adi_set_attributes() != cudaSuccess) st = NS_ERR_CUDA;
    if (st == NS_OK && launch_pois_factor(c, lamx_d, lamz_d) != cudaSuccess) st = NS_ERR_CUDA;
    if (st == NS_OK && cudaStreamSynchronize(c->stream) != cudaSuccess) st = NS_ERR_CUDA;
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
    c->pin_hi = c->lay.total;  // through LB_PTAB, the last block
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
  for (int n = 0; n < nsteps; ++n) {
    double rate = 0.0;
    ns_status s = ns_convective_rate(c, &rate);
    if (s != NS_OK) return s;
    if (!(rate > 0.0)) return fail(c, NS_ERR_STATE, "fluid at rest: no convective time step");
    const double dt = cfl / rate;
    if (dt != c->cfg.dt && (s = ns_set_dt(c, dt)) != NS_OK) return s;
    if (dts) dts[n] = dt;
    if ((s = ns_step(c, 1)) != NS_OK) return s;
  }
  return NS_OK;
}

// Stages that launch nothing in this configuration (the boundary-plane stages of periodic x).
bool stage_idle(const ns_ctx* c, int q) {
  if (STAGES[q].fn == launch_recycle) return !c->cfg.recycle_i;
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

ns_status ns_set_partition(ns_ctx* c, int dir, int P, int mode) {
  if (!c) return NS_ERR_ARG;
  if (dir != 0) return fail(c, NS_ERR_UNSUPPORTED, "only dir 0 (x) is partitioned");
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
  if (dir != 0) return fail(c, NS_ERR_UNSUPPORTED, "only dir 0 (x) is partitioned");
  if (P) *P = c->P;
  if (mode) *mode = c->part_mode;
  if (dropped) *dropped = c->pdd_drop;
  return NS_OK;
}

ns_status ns_autotune(ns_ctx* c) {
  if (!c) return NS_ERR_ARG;
  if (capturing(c)) return fail(c, NS_ERR_STATE, "ns_autotune during capture");
  const int nx = c->cfg.nx;
  // The timed sweeps overwrite r: keep a copy and restore it afterwards.
  const size_t rbytes = c->lay.off[LB_NU] - c->lay.off[LB_RU];
  void* save = nullptr;
  cudaError_t e = cudaMalloc(&save, rbytes);
  if (e != cudaSuccess) return cuda_fail(c, e, "autotune scratch");
  cudaMemcpyAsync(save, c->ru, rbytes, cudaMemcpyDeviceToDevice, c->stream);
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
      launch_adi_x(c, 0);
      cudaEventRecord(e0, c->stream);
      for (int it = 0; it < 5; ++it) launch_adi_x(c, it % 3);
      cudaEventRecord(e1, c->stream);
      cudaEventSynchronize(e1);
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (cudaGetLastError() == cudaSuccess && ms < best) {
        best = ms;
        bestP = P;
        bestMode = mode;
      }
    }
  }
  cudaMemcpyAsync(c->ru, save, rbytes, cudaMemcpyDeviceToDevice, c->stream);
  cudaStreamSynchronize(c->stream);
  cudaFree(save);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ns_set_partition(c, 0, bestP, bestMode);
}

ns_status ns_get_buffer(ns_ctx* c, int which, void** ptr, size_t* bytes) {
  if (!c || !ptr) return NS_ERR_ARG;
  static const int map[8] = {LB_RU, LB_RV, LB_RW, LB_NU, LB_NV, LB_NW, LB_PHI, LB_SPEC};
  if (which < 0 || which > 7) return fail(c, NS_ERR_ARG, "unknown buffer");
  const int b = map[which];
  const size_t nx = c->cfg.nx, ny = c->cfg.ny, nz = c->cfg.nz;
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
  if (c->pin) cudaFreeHost(c->pin);
  if (c->own_ws) cudaFree(c->ws);
  delete c;
}

}  // extern "C"
