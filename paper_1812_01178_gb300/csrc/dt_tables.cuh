// The tables and constants that depend on the time step (ADI factors, PDD/PPT tables, RHS rows,
// sub-step constants), written once for both builders: the host (ns_init, ns_set_dt) and the
// device (dt_phase1_kernel and dt_phase2_kernel in the fixed-CFL step graph, k_dt.cu).  Every
// function here is a task on one table or row that a host loop or a device thread runs; all
// arithmetic is FP64 and the tables are stored in the context's element type (double, or float
// for the mixed form).
#pragma once

#include <string.h>

#include "ns_internal.cuh"

#define NS_HD __host__ __device__ inline

// RK3 constants (the same values as NS_GAMMA, NS_ZETA, NS_ALPHA, usable in device code)
NS_HD double rk_gamma(int k) { return k == 0 ? 8.0 / 15.0 : (k == 1 ? 5.0 / 12.0 : 3.0 / 4.0); }
NS_HD double rk_zeta(int k) { return k == 0 ? 0.0 : (k == 1 ? -17.0 / 60.0 : -5.0 / 12.0); }
NS_HD double rk_alpha(int k) { return k == 0 ? 8.0 / 15.0 : (k == 1 ? 2.0 / 15.0 : 1.0 / 3.0); }

// Everything the dt-dependent tables depend on (plain values; gc is host or device memory).
struct DtSpec {
  int nx, ny, nz;
  int es;        // 8 (FP64) or 4 (mixed)
  int bl;        // inflow / outflow in x
  int P, M;      // x partitions
  int yP, zP;    // partitioned y / z lines of the mixed form (0: none)
  int part_req;  // NS_PART_AUTO / PPT / PDD for the x solver
  int kim_moin;
  double dt, re, dx, dz, fx, u_conv;
  const double* gc;  // NS_GC_COUNT rows of ny + 1
};

NS_HD double spec_inv_re(const DtSpec& s) { return s.re > 0 ? 1.0 / s.re : 0.0; }
NS_HD double spec_beta(const DtSpec& s, int k) { return rk_alpha(k) * s.dt * spec_inv_re(s) / 2.0; }
NS_HD double spec_gc(const DtSpec& s, int f, int j) { return s.gc[(size_t)f * (s.ny + 1) + j]; }

template <typename T>
NS_HD void put(void* base, size_t q, double x) {
  static_cast<T*>(base)[q] = (T)x;
}
NS_HD void put_es(void* base, size_t q, double x, int es) {
  if (es == 8) put<double>(base, q, x);
  else put<float>(base, q, x);
}

// ---------------------------------------------------------------------------------------------
// sub-step constants (StepK) of entry q: sub-steps 0..2, and 3 for the projection of an initial
// field; the levels L, Ly, Lz are set after the modes are chosen
// ---------------------------------------------------------------------------------------------
NS_HD void dt_stepk(const DtSpec& s, int q, StepK& sk) {
  memset(&sk, 0, sizeof(sk));
  const double nxz = (double)s.nx * s.nz;
  sk.dt = s.dt;
  if (q == 3) {
    sk.pscale = 1.0 / nxz;
    sk.sx = 1.0 / s.dx;
    sk.sz = 1.0 / s.dz;
    sk.s = 1.0;
    return;
  }
  const int k = q;
  const double dt = s.dt, gam = rk_gamma(k), zet = rk_zeta(k), alp = rk_alpha(k);
  const double idx = 1.0 / s.dx, idz = 1.0 / s.dz, idx2 = idx * idx, idz2 = idz * idz;
  const double inv_re = spec_inv_re(s);
  // tiled RHS constants, each rounded to double and to float as the expressions would be in that
  // type (products of the double inputs rounded once; cx, cz formed in the type itself).  The
  // convection N is formed and stored pre-multiplied by cn = -dt gamma_k (its difference weights
  // carry cn), so the weight of the stored N of sub-step k-1 is cp = zeta_k / gamma_(k-1).
  const double cn = -dt * gam;
  const double d[11] = {0.25 * idx * cn, 0.25 * idz * cn, 0.5 * idx * cn, 0.5 * idz * cn, cn,
                        k > 0 ? zet / rk_gamma(k - 1) : 0.0, -dt * alp * idx, -dt * alp * idz, 0.0, 0.0,
                        dt * alp * s.fx};
  const double cl = dt * alp * inv_re;
  for (int i = 0; i < 11; ++i) {
    sk.kd[i] = d[i];
    sk.kf[i] = (float)d[i];
  }
  sk.kd[RK_CX] = cl * idx2;
  sk.kd[RK_CZ] = cl * idz2;
  const float clf = (float)cl;
  sk.kf[RK_CX] = clf * (float)idx2;
  sk.kf[RK_CZ] = clf * (float)idz2;
  const double sc = alp * dt;
  sk.pscale = 1.0 / sc / nxz;
  sk.sx = sc / s.dx;
  sk.sz = sc / s.dz;
  sk.s = sc;
  sk.beta_p = s.kim_moin ? sc * inv_re / 2.0 : 0.0;
  const double step = sc * s.u_conv;
  sk.cu = step / s.dx;
  sk.cv = step / (0.5 * s.dx);
  const double rx = alp * dt * inv_re / 2.0 / (s.dx * s.dx);
  sk.xcf[0] = rx;        // u: the outflow face is the neighbour of the last unknown face
  sk.xcf[1] = 2.0 * rx;  // v, w: linear ghost 2 f_out - f_last
  sk.xcf[2] = 2.0 * rx;
  for (int i = 0; i < 3; ++i) sk.xcff[i] = (float)sk.xcf[i];
}

// ---------------------------------------------------------------------------------------------
// RHS rows of sub-step k, row j (0..ny) of every RT_* field: pre-multiplied by the sub-step
// constants, zero where a field is not defined (double and float copies)
// ---------------------------------------------------------------------------------------------
NS_HD void dt_rtab_row(const DtSpec& s, int k, int j, double* rt, float* rtf) {
  const int ny = s.ny, G = ny + 1;
  const double cl = s.dt * rk_alpha(k) * spec_inv_re(s);
  const double dd = 2.0 / (s.dx * s.dx) + 2.0 / (s.dz * s.dz);
  const double cn = -s.dt * rk_gamma(k);  // the convection weight
  // interpolation weight of the lower centre at face jf, zero at the walls
  auto wlo = [&](int jf) { return (jf >= 1 && jf < ny) ? spec_gc(s, GC_WLO, jf) : 0.0; };
  double v[RT_COUNT];
  for (int f = 0; f < RT_COUNT; ++f) v[f] = 0.0;
  if (j < ny) {
    v[RT_AC] = cl * spec_gc(s, GC_AC, j);
    v[RT_CC] = cl * spec_gc(s, GC_CC, j);
    v[RT_DC] = -cl * (dd + spec_gc(s, GC_AC, j) + spec_gc(s, GC_CC, j));
    const double hidy = 0.5 * spec_gc(s, GC_IDY, j) * cn;
    v[RT_HYM] = -hidy * wlo(j);
    v[RT_HYP] = hidy * wlo(j + 1);
  }
  if (j >= 1 && j < ny) {
    v[RT_AF] = cl * spec_gc(s, GC_AF, j);
    v[RT_CF] = cl * spec_gc(s, GC_CF, j);
    v[RT_DF] = -cl * (dd + spec_gc(s, GC_AF, j) + spec_gc(s, GC_CF, j));
    v[RT_CGY] = -s.dt * rk_alpha(k) * spec_gc(s, GC_IHC, j);
    v[RT_QIHC] = 0.25 * spec_gc(s, GC_IHC, j) * cn;
    v[RT_HXW] = 0.5 / s.dx * cn * wlo(j);
    v[RT_HZW] = 0.5 / s.dz * cn * wlo(j);
    v[RT_RHO] = spec_gc(s, GC_WHI, j) / spec_gc(s, GC_WLO, j);
  }
  for (int f = 0; f < RT_COUNT; ++f) {
    rt[(size_t)f * G + j] = v[f];
    rtf[(size_t)f * G + j] = (float)v[f];
  }
}

// ---------------------------------------------------------------------------------------------
// Thomas factors of rows (a, b, c) given by a functor row(i, a, b, c), i < n; a_0 and c_{n-1} are
// ignored: inv = 1/pivot, ainv = a/pivot, cp = c/pivot, written as double through put(idx, x)
// ---------------------------------------------------------------------------------------------
template <typename Row, typename P0, typename P1, typename P2>
NS_HD void thomas_factors_f(int n, Row row, P0 put_inv, P1 put_ainv, P2 put_cp, double* inv_out = nullptr,
                            double* ainv_out = nullptr, double* cp_out = nullptr) {
  double cprev = 0.0;
  for (int j = 0; j < n; ++j) {
    double a, b, c;
    row(j, a, b, c);
    const double aj = j > 0 ? a : 0.0;
    const double cj = j + 1 < n ? c : 0.0;
    const double piv = b - aj * cprev;
    const double inv = 1.0 / piv;
    const double ainv = aj * inv;
    const double cp = cj * inv;
    put_inv(j, inv);
    put_ainv(j, ainv);
    put_cp(j, cp);
    if (inv_out) {
      inv_out[j] = inv;
      ainv_out[j] = ainv;
      cp_out[j] = cp;
    }
    cprev = cp;
  }
}

// y factors of sub-step k: cls 0 centres (u, w; rows j = 0..ny-1), cls 1 faces (v; rows
// j = 1..ny-1); out holds [inv, ainv, cp] of n rows in the element type
NS_HD void dt_ytab(const DtSpec& s, int k, int cls, void* out) {
  const double beta = spec_beta(s, k);
  const int n = cls == 0 ? s.ny : s.ny - 1;
  auto row = [&](int q, double& a, double& b, double& c) {
    const int j = cls == 0 ? q : q + 1;
    const double A = spec_gc(s, cls == 0 ? GC_AC : GC_AF, j), C = spec_gc(s, cls == 0 ? GC_CC : GC_CF, j);
    a = -beta * A;
    c = -beta * C;
    b = 1.0 + beta * (A + C);
  };
  const int es = s.es;
  auto p0 = [&](int j, double x) { put_es(out, (size_t)j, x, es); };
  auto p1 = [&](int j, double x) { put_es(out, (size_t)n + j, x, es); };
  auto p2 = [&](int j, double x) { put_es(out, 2 * (size_t)n + j, x, es); };
  thomas_factors_f(n, row, p0, p1, p2);
}

// z factors of sub-step k: cyclic rows (-r, 1 + 2r, -r) by Sherman-Morrison: the factors of the
// modified matrix, the vector q = A'^{-1} (gamma, 0, .., alpha), and fac, bg; scratch: 4 nz doubles
NS_HD void dt_ztab(const DtSpec& s, int k, void* out, double* scratch) {
  const int nz = s.nz, es = s.es;
  const double r = spec_beta(s, k) / (s.dz * s.dz);
  const double lo = -r, di = 1.0 + 2.0 * r, up = -r;
  const double gam = -di, alpha = up /* A[n-1][0] */, bet = lo /* A[0][n-1] */;
  auto row = [&](int j, double& a, double& b, double& c) {
    a = lo;
    c = up;
    b = di;
    if (j == 0) b = di - gam;
    if (j == nz - 1) b = di - alpha * bet / gam;
  };
  double* inv = scratch;
  double* ainv = scratch + nz;
  double* cp = scratch + 2 * nz;
  double* q = scratch + 3 * nz;
  auto p0 = [&](int j, double x) { put_es(out, (size_t)j, x, es); };
  auto p1 = [&](int j, double x) { put_es(out, (size_t)nz + j, x, es); };
  auto p2 = [&](int j, double x) { put_es(out, 2 * (size_t)nz + j, x, es); };
  thomas_factors_f(nz, row, p0, p1, p2, inv, ainv, cp);
  // q = A'^{-1} s, s = (gamma, 0, .., 0, alpha): the forward and backward sweeps carry the previous
  // value in a register and prefetch the factors in chunks of 8 (the same operations as a sweep
  // over a stored vector)
  auto sv = [&](int j) { return j == nz - 1 ? alpha : (j == 0 ? gam : 0.0); };
  double qv = sv(0) * inv[0];
  q[0] = qv;
  for (int j0 = 1; j0 < nz; j0 += 8) {
    double iv[8], ai[8];
    for (int u = 0; u < 8; ++u)
      if (j0 + u < nz) {
        iv[u] = inv[j0 + u];
        ai[u] = ainv[j0 + u];
      }
    for (int u = 0; u < 8; ++u)
      if (j0 + u < nz) {
        qv = sv(j0 + u) * iv[u] - ai[u] * qv;
        q[j0 + u] = qv;
      }
  }
  for (int j1 = nz - 1; j1 > 0; j1 -= 8) {  // rows j1-1 down to j1-8
    double cv[8], qo[8];
    for (int u = 0; u < 8; ++u)
      if (j1 - 1 - u >= 0) {
        cv[u] = cp[j1 - 1 - u];
        qo[u] = q[j1 - 1 - u];
      }
    for (int u = 0; u < 8; ++u)
      if (j1 - 1 - u >= 0) {
        qv = qo[u] - cv[u] * qv;
        q[j1 - 1 - u] = qv;
      }
  }
  const double bg = bet / gam;
  const double fac = 1.0 / (1.0 + q[0] + bg * q[nz - 1]);
  for (int j = 0; j < nz; ++j) put_es(out, 3 * (size_t)nz + j, q[j], es);
  put_es(out, 4 * (size_t)nz, fac, es);
  put_es(out, 4 * (size_t)nz + 1, bg, es);
  // The same rows are circulant (uniform, periodic z) and factor exactly as
  //   A = alpha (I - lam S)(I - lam S^-1),  S the cyclic shift, (S x)_j = x_{j-1},
  // with lam = 2r / (1 + 2r + sqrt(1 + 4r)) (the root below 1 of lam + 1/lam = (1 + 2r) / r) and
  // alpha = r / lam, so A x = d is two first-order cyclic recurrences (t_j = d_j + lam t_{j-1},
  // then x_j = t_j + lam x_{j+1}, x = result / alpha).  Each starts from its periodic sum,
  // t_0 = sum_k lam^k d_{-k}, truncated after the K terms with lam^(K+1) > 1e-17 (the spike
  // truncation tolerance of the x solve).  use = 0 (the Thomas path) in the float table, or when
  // K exceeds NS_ZF_KMAX or the line.
  const double lam = 2.0 * r / (1.0 + 2.0 * r + sqrt(1.0 + 4.0 * r));
  const double ialpha = r > 0.0 ? lam / r : 1.0;
  int K = 0;
  double pw = lam;  // lam^(K+1)
  while (pw > 1e-17 && K <= NS_ZF_KMAX) {
    ++K;
    pw *= lam;
  }
  const bool use = es == 8 && K <= NS_ZF_KMAX && K + 1 < nz;
  const size_t z0 = 4 * (size_t)nz + 2;
  put_es(out, z0, lam, es);
  put_es(out, z0 + 1, ialpha, es);
  put_es(out, z0 + 2, use ? 1.0 : 0.0, es);
  put_es(out, z0 + 3, (double)(use ? K : 0), es);
  double lk = lam;
  for (int q = 0; q < NS_ZF_KMAX; ++q) {
    put_es(out, z0 + 4 + q, use && q < K ? lk : 0.0, es);
    lk *= lam;
  }
}

// ---------------------------------------------------------------------------------------------
// Partitioned-line tables (Sec. 3.2) of n = P M rows in the x-solver layout (xtab_count), built
// in double in t[], in two phases:
//   phase 1 (one partition r): the block Thomas factors of A~ (couplings to the neighbouring
//            partitions cut) and the spikes v^(r), w^(r) of Eq. (blockAY) (zero where no coupling
//            was cut: the ends of a non-periodic line); xtab_drop gives the largest coupling PDD
//            drops;
//   phase 2: the 2x2-block reduced system Z of Eq. (Zpdd) over the interfaces (r, r+1),
//              L_r Y_{r-1} + D_r Y_r + U_r Y_{r+1} = (x~^(r)_m, x~^(r+1)_1),
//              D_r = [[1, w^(r)_m], [v^(r+1)_1, 1]], L_r = [[v^(r)_m, 0], [0, 0]],
//              U_r = [[0, 0], [0, w^(r+1)_1]],
//            a non-periodic line has P-1 interfaces and a decoupled identity row in slot P-1;
//            PDD keeps D_r, PPT eliminates L, U by block parallel cyclic reduction (multipliers
//            per level); writes D^-1 and the multipliers and returns the number of levels.
// ---------------------------------------------------------------------------------------------
struct M2 {
  double a, b, c, d;  // [[a, b], [c, d]]
};
NS_HD M2 mmul(M2 x, M2 y) {
  return {x.a * y.a + x.b * y.c, x.a * y.b + x.b * y.d, x.c * y.a + x.d * y.c, x.c * y.b + x.d * y.d};
}
NS_HD M2 madd(M2 x, M2 y) { return {x.a + y.a, x.b + y.b, x.c + y.c, x.d + y.d}; }
NS_HD M2 msub(M2 x, M2 y) { return {x.a - y.a, x.b - y.b, x.c - y.c, x.d - y.d}; }
NS_HD M2 minv(M2 x) {
  const double id = 1.0 / (x.a * x.d - x.b * x.c);
  return {x.d * id, -x.b * id, -x.c * id, x.a * id};
}
NS_HD M2 mzero() { return {0, 0, 0, 0}; }

template <typename Row>
NS_HD void xtab_phase1_part(int n, int P, int r, bool cyclic, Row row, double* t) {
  const int M = n / P;
  double* INV = t + (size_t)XT_INV * M * P;
  double* AINV = t + (size_t)XT_AINV * M * P;
  double* CP = t + (size_t)XT_CP * M * P;
  double* SV = t + (size_t)XT_V * M * P;
  double* SW = t + (size_t)XT_W * M * P;
  const int o = r * M;
  auto prow = [&](int e, double& a, double& b, double& c) { row(o + e, a, b, c); };
  auto pi = [&](int e, double x) { INV[(size_t)e * P + r] = x; };
  auto pa = [&](int e, double x) { AINV[(size_t)e * P + r] = x; };
  auto pc = [&](int e, double x) { CP[(size_t)e * P + r] = x; };
  thomas_factors_f(M, prow, pi, pa, pc);  // a of the first row, c of the last (the cut couplings) ignored
  double a0, b0, c0, am, bm, cm;
  row(o, a0, b0, c0);
  row(o + M - 1, am, bm, cm);
  // v = A~^-1 (a_first e_1), w = A~^-1 (c_last e_M), in place in the spike rows
  for (int e = 0; e < M; ++e) {
    SV[(size_t)e * P + r] = 0.0;
    SW[(size_t)e * P + r] = 0.0;
  }
  if (cyclic || r > 0) SV[r] = a0;                            // a of the first row couples partition r-1
  if (cyclic || r < P - 1) SW[(size_t)(M - 1) * P + r] = cm;  // c of the last row couples partition r+1
  double* spk[2] = {SV, SW};
  for (int q = 0; q < 2; ++q) {
    double* d = spk[q];
    d[r] *= INV[r];
    for (int e = 1; e < M; ++e)
      d[(size_t)e * P + r] =
          d[(size_t)e * P + r] * INV[(size_t)e * P + r] - AINV[(size_t)e * P + r] * d[(size_t)(e - 1) * P + r];
    for (int e = M - 1; e-- > 0;) d[(size_t)e * P + r] -= CP[(size_t)e * P + r] * d[(size_t)(e + 1) * P + r];
  }
}

// the largest coupling PDD drops: |v^(r)_m| and |w^(r+1)_1| over the interfaces
NS_HD double xtab_drop(int n, int P, bool cyclic, const double* t) {
  const int M = n / P;
  const double* SV = t + (size_t)XT_V * M * P;
  const double* SW = t + (size_t)XT_W * M * P;
  double drop = 0.0;
  for (int r = 0; r < P; ++r) {
    if (!cyclic && r == P - 1) continue;
    const int rn = (r + 1) % P;
    drop = fmax(drop, fmax(fabs(SV[(size_t)(M - 1) * P + r]), fabs(SW[rn])));
  }
  return drop;
}

// Spike truncation of the x solve: the spikes decay geometrically away from the partition end
// they start from (by about r = beta / dx^2 per row here), so the back half of v^(r) and the front
// half of w^(r) are often below any effect on the solution.  1 if, for every partition, |v_e| and
// |w_{M-1-e}| are at most tol for e >= M/2 (M even, M >= 2); the correction x_e -= v_e x_m^(r-1) +
// w_e x_1^(r+1) then keeps one term per row.  tol: 1e-17 in FP64 (a hundredth of the coupling PDD
// may drop, below the rounding of the solve itself), 1e-9 in FP32.
NS_HD double x_half_tol(int es) { return es == 8 ? 1e-17 : 1e-9; }
NS_HD int xtab_half(int n, int P, const double* t, double tol) {
  const int M = n / P;
  if (M < 2 || (M & 1)) return 0;
  const double* SV = t + (size_t)XT_V * M * P;
  const double* SW = t + (size_t)XT_W * M * P;
  for (int e = M / 2; e < M; ++e)
    for (int r = 0; r < P; ++r)
      if (!(fabs(SV[(size_t)e * P + r]) <= tol) || !(fabs(SW[(size_t)(M - 1 - e) * P + r]) <= tol)) return 0;
  return 1;
}

// Phase 2 in three steps, each over the partitions r independently (a device block runs them
// with one thread per r and a barrier between levels): the blocks of interface r, one level of
// block cyclic reduction, and the final inverse diagonal block.
NS_HD void xtab_p2_init(int n, int P, bool cyclic, int mode, int r, const double* t, M2* Lb, M2* Db, M2* Ub) {
  const int M = n / P;
  const double* SV = t + (size_t)XT_V * M * P;
  const double* SW = t + (size_t)XT_W * M * P;
  const int rn = (r + 1) % P;
  if (!cyclic && r == P - 1) {
    Db[r] = {1.0, 0.0, 0.0, 1.0};
    Lb[r] = mzero();
    Ub[r] = mzero();
  } else {
    Db[r] = {1.0, SW[(size_t)(M - 1) * P + r], SV[rn], 1.0};
    Lb[r] = {SV[(size_t)(M - 1) * P + r], 0.0, 0.0, 0.0};
    Ub[r] = {0.0, 0.0, 0.0, SW[rn]};
  }
  // one periodic partition: both couplings of the single interface point back at itself
  if (mode == NS_PART_PPT && P == 1) Db[0] = madd(Db[0], madd(Lb[0], Ub[0]));
}

// level lv (stride st = 2^lv) for partition r: multipliers into t, the new blocks into nL, nD, nU
NS_HD void xtab_p2_level(int M, int P, int L, int lv, int r, const M2* Lb, const M2* Db, const M2* Ub, M2* nL,
                         M2* nD, M2* nU, double* t) {
  const int st = 1 << lv;
  const size_t m0 = (size_t)XT_NF * M * P + 4 * (size_t)P, u0 = m0 + 4 * (size_t)L * P;
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
  t[m0 + (4 * lv + 0) * (size_t)P + r] = ml.a;
  t[m0 + (4 * lv + 1) * (size_t)P + r] = ml.b;
  t[m0 + (4 * lv + 2) * (size_t)P + r] = ml.c;
  t[m0 + (4 * lv + 3) * (size_t)P + r] = ml.d;
  t[u0 + (4 * lv + 0) * (size_t)P + r] = mu.a;
  t[u0 + (4 * lv + 1) * (size_t)P + r] = mu.b;
  t[u0 + (4 * lv + 2) * (size_t)P + r] = mu.c;
  t[u0 + (4 * lv + 3) * (size_t)P + r] = mu.d;
}

NS_HD void xtab_p2_final(int M, int P, int r, const M2* Db, double* t) {
  const size_t d0 = (size_t)XT_NF * M * P;
  const M2 di = minv(Db[r]);
  t[d0 + r] = di.a;
  t[d0 + P + r] = di.b;
  t[d0 + 2 * (size_t)P + r] = di.c;
  t[d0 + 3 * (size_t)P + r] = di.d;
}

NS_HD int xtab_levels(int P, int mode) {
  int L = 0;
  while ((1 << L) < P) ++L;
  return mode == NS_PART_PPT ? L : 0;
}

// All of phase 2 in sequence (the host form); scratch: xtab_scratch_doubles(P).  Returns L.
NS_HD int xtab_phase2(int n, int P, bool cyclic, int mode, double* t, double* scratch) {
  const int M = n / P, L = xtab_levels(P, mode);
  M2* b0 = reinterpret_cast<M2*>(scratch);
  M2 *Lb = b0, *Db = b0 + P, *Ub = b0 + 2 * P, *nL = b0 + 3 * P, *nD = b0 + 4 * P, *nU = b0 + 5 * P;
  for (int r = 0; r < P; ++r) xtab_p2_init(n, P, cyclic, mode, r, t, Lb, Db, Ub);
  for (int lv = 0; lv < L; ++lv) {
    for (int r = 0; r < P; ++r) xtab_p2_level(M, P, L, lv, r, Lb, Db, Ub, nL, nD, nU, t);
    M2* x;
    x = Lb, Lb = nL, nL = x;
    x = Db, Db = nD, nD = x;
    x = Ub, Ub = nU, nU = x;
  }
  for (int r = 0; r < P; ++r) xtab_p2_final(M, P, r, Db, t);
  return L;
}

// rows of (I - beta_k delta_xx) on one x-line (Sec. 2.2) for the u lines (cls 0) and the v, w
// lines (cls 1).  Periodic: every row (-r, 1 + 2r, -r), cyclic.  Inflow / outflow: the u line holds
// faces 0..nx-1 with face 0 fixed (identity row) and the outflow face as the neighbour of the last
// row (its increment enters the right-hand side); v, w lines are cell centres whose first and last
// rows see linear ghosts of the boundary faces: b = 1 + 3r there.
NS_HD void x_row(const DtSpec& s, int k, int cls, int i, double& a, double& b, double& c) {
  const int nx = s.nx;
  const double r = spec_beta(s, k) / (s.dx * s.dx);
  a = -r;
  b = 1.0 + 2.0 * r;
  c = -r;
  if (!s.bl) return;
  if (i == 0) a = 0.0;
  if (i == nx - 1) c = 0.0;
  if (cls == 0) {
    if (i == 0) {
      b = 1.0;
      c = 0.0;
    }
  } else if (i == 0 || i == nx - 1) {
    b = 1.0 + 3.0 * r;
  }
}

// rows of the partitioned y / z lines of the mixed form: q = 0 y centres (u, w), q = 1 y faces (v;
// the wall row 0 as an identity row), q = 2 z (cyclic)
NS_HD void line_row(const DtSpec& s, int k, int q, int i, double& a, double& b, double& c) {
  const double beta = spec_beta(s, k);
  if (q == 2) {
    const double r = beta / (s.dz * s.dz);
    a = -r;
    c = -r;
    b = 1.0 + 2.0 * r;
    return;
  }
  if (q == 1 && i == 0) {
    a = 0.0;
    b = 1.0;
    c = 0.0;
    return;
  }
  const double A = spec_gc(s, q == 0 ? GC_AC : GC_AF, i), C = spec_gc(s, q == 0 ? GC_CC : GC_CF, i);
  a = (q == 1 && i == 1) ? 0.0 : -beta * A;  // row 1 of the faces: its wall neighbour is row 0
  c = -beta * C;
  b = 1.0 + beta * (A + C);
}

// doubles of the phase-2 scratch of a line table, and the PDD tolerances
NS_HD size_t xtab_scratch_doubles(int P) { return 24 * (size_t)P; }
NS_HD double pdd_tol(int es) { return es == 8 ? 1e-15 : 1e-8; }
