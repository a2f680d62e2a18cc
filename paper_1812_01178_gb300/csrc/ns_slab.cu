// y-slab decomposition of the time step (Sec. 3.2, "Domain decomposition using parallel
// algorithms", and Algorithm 1): the domain is cut into p slabs of whole x-z planes, slab r holding
// the cell rows [j0, j1) of y.  Everything along x and z (RHS, x and z sweeps, x and z
// transforms, projection) is local to a slab; the two solves along y are split across slabs with
// the partitioned tridiagonal algorithms of Sec. 3.2 (inflow / convective outflow in x adds one
// all-gather of each slab's share of the outflow flux correction):
//   * the y sweep of the ADI factorisation by PDD (one exchange of the end values x~_1, x~_m with
//     the two neighbouring slabs, Algorithm 1) where the coupling PDD drops is negligible, else
//     by PPT (all-gather of the end values, every slab solving the whole reduced system);
//   * the Poisson y solve of every (kx, kz) line by PPT (all-gather of the end values).
// Each slab is an ordinary context (ns_init) on its sub-grid with one halo row on each side that
// has a neighbour; the stages that are local in y run on that context unchanged, and their halo
// rows' outputs are never used.  The slab kernels below replace the y solves.
//
// Data moves between slabs only through exchange buffers: for each exchange, a slab writes its
// send buffer and reads the p-slot receive buffer, slot s holding slab s's send buffer.  Who moves
// the bytes is the caller's business: device copies between slabs on one GPU, NCCL point-to-point
// or all-gather between GPUs.  ns_slab_slots tells which slots a slab reads.
//
// Per-line data of the reduced systems: the end values h of the partitions' local solutions and
// two rows of the reduced system's inverse (PPT) or of its 2x2 block-diagonal part (PDD), see
// split_line.  Every line of the y sweep has the same matrix, so its tables are 1-D; the Poisson
// lines have one matrix per (kx, kz), tabulated once (the operator does not change).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "ns_internal.cuh"

struct ns_slab {
  ns_ctx* c = nullptr;       // context of the sub-grid (halo rows included)
  ns_config gcfg{};          // the whole domain
  std::vector<double> gyf;
  int p = 1, r = 0, j0 = 0, j1 = 0, hb = 0, ha = 0, nyl = 0, nyv = 0;
  int ymode = NS_PART_PPT;   // y sweep: NS_PART_PDD or NS_PART_PPT
  double ydrop = 0.0;        // largest coupling PDD drops in the y sweep (all sub-steps, both classes)
  int Q = 0;                 // unknowns of the reduced system, 2 (p - 1)
  int ym[2] = {0, 0};        // y-sweep unknowns of this slab: [0] centres (u, w), [1] faces (v)
  int yjo[2] = {0, 0};       // sub-grid row of the first unknown
  double* ytab[3][2] = {};   // per sub-step and class: a, 1/pivot, c/pivot, v, w (m each), clo, chi (Q each)
  double* pfinv = nullptr;   // Poisson: 1/pivot, c/pivot, spikes v, w: (nzh, nyl, nx) each
  double* pfcp = nullptr;
  double* pv = nullptr;
  double* pw = nullptr;
  double* pcoef = nullptr;   // (nzh, nx, 2, Q): rows clo, chi of every line
  char* send[NS_XCH_COUNT] = {};
  char* recv[NS_XCH_COUNT] = {};
  size_t slot[NS_XCH_COUNT] = {};
  // recycling inflow: a recycling block of the whole grid and, per row / face of the whole
  // domain, where its samples sit in the gathered RCY buffer (u, w rows; v faces)
  double* rcy = nullptr;
  long* rcy_off = nullptr;  // uoff[ny], woff[ny], voff[ny + 1]
  void* ws = nullptr;
  bool own_ws = false;
  std::string err;
};

namespace {

// rows of slab r of p: as even as possible
void slab_rows(int ny, int p, int r, int* j0, int* j1) {
  *j0 = (int)(((long)r * ny) / p);
  *j1 = (int)(((long)(r + 1) * ny) / p);
}

std::string check_slab(const ns_config* cfg, int p, int r) {
  if (!cfg || !cfg->yf) return "cfg or cfg->yf is NULL";
  if (p < 1 || p > 64) return "p must be in [1, 64]";
  if (r < 0 || r >= p) return "r must be in [0, p)";
  if (cfg->precision != NS_FP64) return "slabs are built for NS_FP64";
  if (cfg->recycle_i != 0) {
    if (cfg->bc_x != 1) return "recycling needs inflow / outflow in x (bc_x = 1)";
    if (cfg->recycle_i < 1 || cfg->recycle_i >= cfg->nx) return "recycle_i must be in [1, nx - 1]";
    if (!(cfg->delta_in > 0.0) || !std::isfinite(cfg->delta_in)) return "delta_in must be positive and finite";
  }
  if (cfg->ny < 3 * p) return "every slab needs at least 3 rows (ny >= 3 p)";
  return "";
}

// most rows of any slab
int rows_max(int ny, int p) { return (ny + p - 1) / p; }

// the sub-grid of slab r: its rows plus one halo row on each side that has a neighbour
void sub_config(const ns_config* g, int p, int r, std::vector<double>& yf, ns_config* out, int* hb, int* ha) {
  int j0, j1;
  slab_rows(g->ny, p, r, &j0, &j1);
  *hb = r > 0 ? 1 : 0;
  *ha = r < p - 1 ? 1 : 0;
  yf.assign(g->yf + (j0 - *hb), g->yf + (j1 + *ha) + 1);
  *out = *g;
  out->ny = (j1 - j0) + *hb + *ha;
  out->yf = yf.data();
  out->bc_ytop = r == p - 1 ? g->bc_ytop : 0;
  out->recycle_i = 0;  // the slab recycles from the gathered plane of the whole domain
}

size_t slot_bytes(const ns_config* g, int p, int xch) {
  const size_t plane = (size_t)g->nz * g->nx * 8, nzh = g->nz / 2 + 1;
  switch (xch) {
    case NS_XCH_RCY:  // u and w samples of the slab's rows, v of its faces (rows_max + 1 slots)
      return g->recycle_i ? al256((3 * (size_t)rows_max(g->ny, p) + 1) * g->nz * 8) : 0;
    case NS_XCH_HALO: return al256(2 * 4 * plane);
    case NS_XCH_ADIY: return al256(2 * 3 * plane);
    case NS_XCH_VSTAR: return al256(plane);
    case NS_XCH_POIS: return al256(2 * nzh * g->nx * 16);
    case NS_XCH_PHI: return al256(2 * plane);  // part 0: row j0 (to slab r-1), part 1: row j1-1 (to r+1)
    case NS_XCH_FLUX: return 256;  // one double: this slab's share of Q_in - Q_out
    default: return 0;
  }
}

// slab bytes beyond the sub-grid context's workspace
size_t extra_bytes(const ns_config* g, int p, int r) {
  int j0, j1;
  slab_rows(g->ny, p, r, &j0, &j1);
  const size_t nyl = j1 - j0, nzh = g->nz / 2 + 1, Q = 2 * (size_t)(p - 1);
  size_t b = 0;
  b += 6 * al256((5 * (nyl + 1) + 2 * Q) * 8);                      // y-sweep tables
  b += 4 * al256(nzh * nyl * g->nx * 8) + al256(nzh * g->nx * 2 * Q * 8 + 8);  // Poisson tables
  for (int x = 0; x < NS_XCH_COUNT; ++x) b += (1 + (size_t)p) * slot_bytes(g, p, x);
  if (g->recycle_i) b += al256(recycle_block_doubles(g->ny) * 8) + al256((3 * (size_t)g->ny + 1) * 8);
  return b;
}

// the Thomas algorithm for one block of rows (a, b, c), a[0] and c[m-1] ignored
void thomas_h(const double* a, const double* b, const double* c, const double* d, double* x, int m,
              std::vector<double>& cp) {
  cp.resize(m);
  double piv = b[0];
  cp[0] = c[0] / piv;
  x[0] = d[0] / piv;
  for (int j = 1; j < m; ++j) {
    piv = b[j] - a[j] * cp[j - 1];
    cp[j] = c[j] / piv;
    x[j] = (d[j] - a[j] * x[j - 1]) / piv;
  }
  for (int j = m - 2; j >= 0; --j) x[j] -= cp[j] * x[j + 1];
}

// inverse of the n x n row-major matrix A by Gauss-Jordan elimination with partial pivoting
bool invert_h(std::vector<double> A, int n, std::vector<double>& inv) {
  inv.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1.0;
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int i = col + 1; i < n; ++i)
      if (std::fabs(A[(size_t)i * n + col]) > std::fabs(A[(size_t)piv * n + col])) piv = i;
    if (A[(size_t)piv * n + col] == 0.0) return false;
    if (piv != col)
      for (int q = 0; q < n; ++q) {
        std::swap(A[(size_t)piv * n + q], A[(size_t)col * n + q]);
        std::swap(inv[(size_t)piv * n + q], inv[(size_t)col * n + q]);
      }
    const double s = 1.0 / A[(size_t)col * n + col];
    for (int q = 0; q < n; ++q) {
      A[(size_t)col * n + q] *= s;
      inv[(size_t)col * n + q] *= s;
    }
    for (int i = 0; i < n; ++i) {
      if (i == col) continue;
      const double f = A[(size_t)i * n + col];
      if (f == 0.0) continue;
      for (int q = 0; q < n; ++q) {
        A[(size_t)i * n + q] -= f * A[(size_t)col * n + q];
        inv[(size_t)i * n + q] -= f * inv[(size_t)col * n + q];
      }
    }
  }
  return true;
}

// One tridiagonal line of N unknowns (rows a, b, c) split into the blocks [lo[s], hi[s]) of the
// p slabs (Sec. 3.2, Eq. (smidentity): A = A~ + V E^T).  For slab r it returns the Thomas factors
// of its block of A~ (a, 1/pivot, c/pivot), its spikes v = A~_r^-1 a_first e_1 and
// w = A~_r^-1 c_last e_m (Eq. (blockAY)), and two rows of the inverse of the reduced system
// Z y = h on the unknowns y = (x^(0)_m, x^(1)_1, x^(1)_m, x^(2)_1, ...):
//   y[2t]   + v^(t)_m y[2t-2]   + w^(t)_m y[2t+1]   = x~^(t)_m    = h[2t]
//   y[2t+1] + v^(t+1)_1 y[2t]   + w^(t+1)_1 y[2t+3] = x~^(t+1)_1  = h[2t+1]
// clo = the row of x^(r-1)_m, chi = the row of x^(r+1)_1 (zero where there is no neighbour), so
// that the solution of the slab is x = x~ - v (clo . h) - w (chi . h).  PPT: rows of Z^-1 (exact).
// PDD: rows of the inverse of Z's 2x2 diagonal blocks (Eq. (Zpdd)), which drop v^(t)_m and
// w^(t+1)_1; drop returns the largest of those.
struct SplitOut {
  std::vector<double> a, ip, cp, v, w, clo, chi;
  double drop = 0.0;
  bool ok = true;
};

void split_line(const double* a, const double* b, const double* c, const std::vector<int>& lo,
                const std::vector<int>& hi, int r, bool pdd, SplitOut& o, std::vector<double>& scr) {
  const int p = (int)lo.size(), Q = 2 * (p - 1);
  std::vector<double> v1(p, 0.0), vm(p, 0.0), w1(p, 0.0), wm(p, 0.0);
  std::vector<double> e, x;
  for (int s = 0; s < p; ++s) {
    const int m = hi[s] - lo[s];
    const double* as = a + lo[s];
    const double* bs = b + lo[s];
    const double* cs = c + lo[s];
    e.assign(m, 0.0);
    x.assign(m, 0.0);
    if (s > 0) {  // coupling of the first row to the last unknown of slab s-1
      e[0] = as[0];
      thomas_h(as, bs, cs, e.data(), x.data(), m, scr);
      v1[s] = x[0];
      vm[s] = x[m - 1];
      if (s == r) o.v = x;
      e[0] = 0.0;
    }
    if (s < p - 1) {  // coupling of the last row to the first unknown of slab s+1
      e[m - 1] = cs[m - 1];
      thomas_h(as, bs, cs, e.data(), x.data(), m, scr);
      w1[s] = x[0];
      wm[s] = x[m - 1];
      if (s == r) o.w = x;
    }
    if (s == r) {
      o.a.assign(as, as + m);
      o.a[0] = 0.0;  // the coupling to the slab below is cut
      o.ip.resize(m);
      o.cp.resize(m);
      double cprev = 0.0;
      for (int j = 0; j < m; ++j) {
        const double piv = bs[j] - o.a[j] * cprev;
        o.ip[j] = 1.0 / piv;
        cprev = (j + 1 < m ? cs[j] : 0.0) * o.ip[j];
        o.cp[j] = cprev;
      }
      if (o.v.empty()) o.v.assign(m, 0.0);
      if (o.w.empty()) o.w.assign(m, 0.0);
    }
  }
  o.clo.assign(Q, 0.0);
  o.chi.assign(Q, 0.0);
  o.drop = 0.0;
  for (int t = 0; t + 1 < p; ++t) {
    if (t >= 1) o.drop = std::max(o.drop, std::fabs(vm[t]));
    if (t + 2 <= p - 1) o.drop = std::max(o.drop, std::fabs(w1[t + 1]));
  }
  if (Q == 0) return;
  if (pdd) {
    if (r >= 1) {
      const int t = r - 1;
      const double det = 1.0 - wm[t] * v1[t + 1];
      o.clo[2 * t] = 1.0 / det;
      o.clo[2 * t + 1] = -wm[t] / det;
    }
    if (r <= p - 2) {
      const int t = r;
      const double det = 1.0 - wm[t] * v1[t + 1];
      o.chi[2 * t] = -v1[t + 1] / det;
      o.chi[2 * t + 1] = 1.0 / det;
    }
    return;
  }
  std::vector<double> Z((size_t)Q * Q, 0.0), Zi;
  for (int t = 0; t + 1 < p; ++t) {
    Z[(size_t)(2 * t) * Q + 2 * t] = 1.0;
    if (t >= 1) Z[(size_t)(2 * t) * Q + 2 * t - 2] = vm[t];
    Z[(size_t)(2 * t) * Q + 2 * t + 1] = wm[t];
    Z[(size_t)(2 * t + 1) * Q + 2 * t + 1] = 1.0;
    Z[(size_t)(2 * t + 1) * Q + 2 * t] = v1[t + 1];
    if (t + 2 <= p - 1) Z[(size_t)(2 * t + 1) * Q + 2 * t + 3] = w1[t + 1];
  }
  if (!invert_h(Z, Q, Zi)) {
    o.ok = false;
    return;
  }
  if (r >= 1)
    for (int q = 0; q < Q; ++q) o.clo[q] = Zi[(size_t)(2 * (r - 1)) * Q + q];
  if (r <= p - 2)
    for (int q = 0; q < Q; ++q) o.chi[q] = Zi[(size_t)(2 * r + 1) * Q + q];
}

// ---------------------------------------------------------------------------------------------
// kernels (one thread per line; the y solves of a slab are short and few)
// ---------------------------------------------------------------------------------------------
struct YArgs {
  double* r[3];      // increments of u, v, w on the sub-grid
  int rows[3];       // rows per (x, z) column of each (ny_v, ny_v + 1, ny_v)
  int nx, nz;
  int jo[2], m[2];   // first unknown's sub-grid row, unknowns: [0] centres, [1] faces
  const double* tab[2];
  int Q;
  double* send;      // ends [end][comp][k][i]
  double* own;       // this slab's receive slot
  const double* recv;
  size_t slot;       // doubles per slot
  int qlo, qhi;      // entries of h this slab reads
};

// the line of component comp (u, w: the centre class; v: the face class); the argument arrays are
// selected with constant indices, so the kernel arguments stay in the constant bank
struct YLine {
  double* line;
  const double* T;
  int m;
};
__device__ __forceinline__ YLine y_line(const YArgs& a, int comp, int k, int i) {
  const bool f = comp == 1;
  double* r = comp == 0 ? a.r[0] : (f ? a.r[1] : a.r[2]);
  const int rows = f ? a.rows[1] : a.rows[0];
  const int jo = f ? a.jo[1] : a.jo[0];
  return YLine{r + ((long)k * rows + jo) * a.nx + i, f ? a.tab[1] : a.tab[0], f ? a.m[1] : a.m[0]};
}

__global__ void __launch_bounds__(128) slab_ysweep_local(const YArgs a) {
  const int comp = blockIdx.z, k = blockIdx.y, i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.nx) return;
  const YLine L = y_line(a, comp, k, i);
  const int m = L.m;
  const double* T = L.T;
  const double *A = T, *IP = T + m, *CP = T + 2 * m;
  double* line = L.line;
  const long s = a.nx;
  // rows fetched U at a time ahead of the recurrence (their latency overlaps it)
  constexpr int U = 4;
  double prev = 0.0;
  for (int j0 = 0; j0 < m; j0 += U) {
    double dv[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (j0 + u < m) dv[u] = line[(long)(j0 + u) * s];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (j0 + u < m) {
        prev = (dv[u] - __ldg(A + j0 + u) * prev) * __ldg(IP + j0 + u);
        line[(long)(j0 + u) * s] = prev;
      }
  }
  double x = prev;
  for (int j1 = m - 2; j1 >= 0; j1 -= U) {
    double dv[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (j1 - u >= 0) dv[u] = line[(long)(j1 - u) * s];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (j1 - u >= 0) {
        x = dv[u] - __ldg(CP + j1 - u) * x;
        line[(long)(j1 - u) * s] = x;
      }
  }
  const long plane = (long)a.nz * a.nx, o = (long)k * a.nx + i;
  const double x1 = line[0], xm = line[(long)(m - 1) * s];
  a.send[(0 * 3 + comp) * plane + o] = x1;
  a.send[(1 * 3 + comp) * plane + o] = xm;
  a.own[(0 * 3 + comp) * plane + o] = x1;
  a.own[(1 * 3 + comp) * plane + o] = xm;
}

__global__ void __launch_bounds__(128) slab_ysweep_correct(const YArgs a) {
  const int comp = blockIdx.z, k = blockIdx.y, i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.nx) return;
  const YLine L = y_line(a, comp, k, i);
  const int m = L.m;
  const double* T = L.T;
  const double *V = T + 3 * m, *W = T + 4 * m, *CLO = T + 5 * m, *CHI = CLO + a.Q;
  const long plane = (long)a.nz * a.nx, o = (long)k * a.nx + i;
  // h[2t] = x~^(t)_m (slot t, end 1), h[2t+1] = x~^(t+1)_1 (slot t + 1, end 0)
  double ylo = 0.0, yhi = 0.0;
  for (int q = a.qlo; q < a.qhi; ++q) {
    const int t = q >> 1;
    const double h = (q & 1) ? a.recv[(size_t)(t + 1) * a.slot + (0 * 3 + comp) * plane + o]
                             : a.recv[(size_t)t * a.slot + (1 * 3 + comp) * plane + o];
    ylo = fma(CLO[q], h, ylo);
    yhi = fma(CHI[q], h, yhi);
  }
  double* line = L.line;
  const long s = a.nx;
  for (int j = 0; j < m; ++j) line[j * s] -= V[j] * ylo + W[j] * yhi;
}

struct PArgs {
  double* spec;      // complex spectrum of the sub-grid, [kz][row][kx], as doubles
  const double* pa;  // Poisson sub-diagonal of the sub-grid rows
  int nx, nyv, nzh, jo, m;
  const double *finv, *fcp, *pv, *pw, *coef;
  int Q;
  bool gauge;        // this slab holds row 0 of the (0, 0) line: phi_0 = 0
  double* send;      // ends [end][kz][kx] complex, as doubles
  double* own;
  const double* recv;
  size_t slot;       // doubles per slot
};

// two threads per (kx, kz) line: real and imaginary parts share the real matrix
__global__ void __launch_bounds__(128) slab_pois_local(const PArgs a) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = t >> 1, part = t & 1, kz = blockIdx.y;
  if (i >= a.nx) return;
  const long sd = 2L * a.nx;
  double* d = a.spec + 2 * (((long)kz * a.nyv + a.jo) * a.nx + i) + part;
  const double* F = a.finv + (long)kz * a.m * a.nx + i;
  const double* C = a.fcp + (long)kz * a.m * a.nx + i;
  const bool g = a.gauge && i == 0 && kz == 0;
  constexpr int U = 4;  // rows fetched U at a time ahead of the recurrence
  const int m = a.m;
  double prev = 0.0;
  for (int j0 = 0; j0 < m; j0 += U) {
    double dv[U], fv[U], av[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (j0 + u < m) {
        dv[u] = d[(long)(j0 + u) * sd];
        fv[u] = __ldg(F + (long)(j0 + u) * a.nx);
        av[u] = (j0 + u) ? __ldg(a.pa + j0 + u) : 0.0;
      }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (j0 + u < m) {
        const double dj = (g && j0 + u == 0) ? 0.0 : dv[u];
        prev = (dj - av[u] * prev) * fv[u];
        d[(long)(j0 + u) * sd] = prev;
      }
  }
  double x = prev;
  for (int j1 = m - 2; j1 >= 0; j1 -= U) {
    double dv[U], cv[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (j1 - u >= 0) {
        dv[u] = d[(long)(j1 - u) * sd];
        cv[u] = __ldg(C + (long)(j1 - u) * a.nx);
      }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (j1 - u >= 0) {
        x = dv[u] - cv[u] * x;
        d[(long)(j1 - u) * sd] = x;
      }
  }
  const long o0 = 2 * (((long)0 * a.nzh + kz) * a.nx + i) + part;
  const long o1 = 2 * (((long)1 * a.nzh + kz) * a.nx + i) + part;
  const double x1 = d[0], xm = d[(long)(a.m - 1) * sd];
  a.send[o0] = x1;
  a.send[o1] = xm;
  a.own[o0] = x1;
  a.own[o1] = xm;
}

__global__ void __launch_bounds__(128) slab_pois_correct(const PArgs a) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = t >> 1, part = t & 1, kz = blockIdx.y;
  if (i >= a.nx) return;
  const double* CLO = a.coef + ((long)kz * a.nx + i) * 2 * a.Q;
  const double* CHI = CLO + a.Q;
  double ylo = 0.0, yhi = 0.0;
  for (int q = 0; q < a.Q; ++q) {
    const int tt = q >> 1;
    const long o = (q & 1) ? (size_t)(tt + 1) * a.slot + 2 * (((long)0 * a.nzh + kz) * a.nx + i) + part
                           : (size_t)tt * a.slot + 2 * (((long)1 * a.nzh + kz) * a.nx + i) + part;
    const double h = a.recv[o];
    ylo = fma(CLO[q], h, ylo);
    yhi = fma(CHI[q], h, yhi);
  }
  const long sd = 2L * a.nx;
  double* d = a.spec + 2 * (((long)kz * a.nyv + a.jo) * a.nx + i) + part;
  const double* V = a.pv + (long)kz * a.m * a.nx + i;
  const double* W = a.pw + (long)kz * a.m * a.nx + i;
  for (int j = 0; j < a.m; ++j) d[j * sd] -= V[(long)j * a.nx] * ylo + W[(long)j * a.nx] * yhi;
}

// Outflow mass-flux correction across slabs (inflow / outflow x): each slab sums
// (u_in - u_out) dy_j over its own rows (one block, fixed order) into its FLUX send buffer and its
// own slot; after the all-gather every slab adds the p shares in slab order and shifts u_out by
// the same amount on all its rows (halo rows too: they mirror the neighbours' own rows).
__global__ void __launch_bounds__(1024) slab_flux_partial(const double* __restrict__ u, const double* __restrict__ u_out,
                                                          const double* __restrict__ gc, int nx, int nyv, int nz,
                                                          int jo, int m, double* send, double* own) {
  __shared__ double red[1024];
  const double* dy = gc + GC_DY * (nyv + 1);
  const long n = (long)nz * m;
  double acc = 0.0;
  for (long q = threadIdx.x; q < n; q += blockDim.x) {
    const int j = jo + (int)(q % m);
    const long pq = (q / m) * nyv + j;  // plane index k * rows + j
    acc += (__ldg(u + pq * nx) - u_out[pq]) * __ldg(dy + j);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s2 = blockDim.x / 2; s2 > 0; s2 >>= 1) {
    if (threadIdx.x < s2) red[threadIdx.x] += red[threadIdx.x + s2];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *send = red[0];
    *own = red[0];
  }
}

__global__ void slab_flux_apply(double* __restrict__ u_out, long n, const double* __restrict__ recv, size_t slot, int p,
                                double dz_over_area) {
  double tot = 0.0;
  for (int q = 0; q < p; ++q) tot += recv[(size_t)q * slot];
  const double corr = tot * dz_over_area;
  for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) u_out[q] += corr;
}

ns_status slab_fail(ns_slab* s, ns_status st, const std::string& m) {
  if (s) s->err = m;
  ns_set_thread_error(m.c_str());
  return st;
}

ns_status cuda_fail(ns_slab* s, const char* what, cudaError_t e) {
  return slab_fail(s, NS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// one row (centre row or face row jrow of a field with `rows` rows per column) to / from a
// contiguous nz x nx block
cudaError_t copy_row_out(const double* f, int rows, int jrow, int nx, int nz, double* dst, cudaStream_t st) {
  return cudaMemcpy2DAsync(dst, nx * 8, f + (size_t)jrow * nx, (size_t)rows * nx * 8, nx * 8, nz,
                           cudaMemcpyDeviceToDevice, st);
}
cudaError_t copy_row_in(double* f, int rows, int jrow, int nx, int nz, const double* src, cudaStream_t st) {
  return cudaMemcpy2DAsync(f + (size_t)jrow * nx, (size_t)rows * nx * 8, src, nx * 8, nx * 8, nz,
                           cudaMemcpyDeviceToDevice, st);
}

// Recycle-plane samples of this slab's rows for the RCY all-gather: u on face ir of rows
// j0 .. j1-1, w and v averaged over the centres ir-1 and ir (rows j0 .. j1-1; faces j0 .. j1-1,
// and face ny on the last slab), written [row][k] into the send buffer and the slab's own slot.
__global__ void slab_rcy_pack(const double* __restrict__ u, const double* __restrict__ v,
                              const double* __restrict__ w, int nx, int nyv, int nz, int hb, int nyl, int nface,
                              int ir, long rm, double* __restrict__ send, double* __restrict__ own) {
  const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int jl = (int)(q / nz), k = (int)(q - (long)jl * nz);
  if (jl >= nface) return;
  const long o = (long)jl * nz + k;
  if (jl < nyl) {
    const long c = ((long)k * nyv + hb + jl) * nx;
    const double ur = u[c + ir], wr = 0.5 * (w[c + ir - 1] + w[c + ir]);
    send[o] = ur;
    own[o] = ur;
    send[rm * nz + o] = wr;
    own[rm * nz + o] = wr;
  }
  const long cv = ((long)k * (nyv + 1) + hb + jl) * nx;
  const double vr = 0.5 * (v[cv + ir - 1] + v[cv + ir]);
  send[2 * rm * nz + o] = vr;
  own[2 * rm * nz + o] = vr;
}

cudaError_t pack_rcy(ns_slab* s) {
  if (!s->gcfg.recycle_i) return cudaSuccess;
  ns_ctx* c = s->c;
  const int nz = c->cfg.nz, nface = s->nyl + (s->r == s->p - 1 ? 1 : 0);
  const long n = (long)nface * nz;
  slab_rcy_pack<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(
      c->f.u, c->f.v, c->f.w, c->cfg.nx, s->nyv, nz, s->hb, s->nyl, nface, s->gcfg.recycle_i,
      rows_max(s->gcfg.ny, s->p), (double*)s->send[NS_XCH_RCY],
      (double*)(s->recv[NS_XCH_RCY] + (size_t)s->r * s->slot[NS_XCH_RCY]));
  return cudaGetLastError();
}

// halo send buffer: part 0 (to slab r-1) = u, w, p of row j0 and v of face j0; part 1 (to slab
// r+1) = u, w, p of row j1-1 and v of face j1-1
cudaError_t pack_halo(ns_slab* s) {
  ns_ctx* c = s->c;
  const int nx = c->cfg.nx, nz = c->cfg.nz, ny = s->nyv;
  const size_t plane = (size_t)nz * nx;
  double* buf = (double*)s->send[NS_XCH_HALO];
  cudaError_t e = cudaSuccess;
  for (int part = 0; part < 2; ++part) {
    if ((part == 0 && s->r == 0) || (part == 1 && s->r == s->p - 1)) continue;
    const int jr = part == 0 ? s->hb : s->hb + s->nyl - 1;
    double* b = buf + part * 4 * plane;
    if ((e = copy_row_out(c->f.u, ny, jr, nx, nz, b, c->stream)) != cudaSuccess) return e;
    if ((e = copy_row_out(c->f.w, ny, jr, nx, nz, b + plane, c->stream)) != cudaSuccess) return e;
    if ((e = copy_row_out(c->f.p, ny, jr, nx, nz, b + 2 * plane, c->stream)) != cudaSuccess) return e;
    if ((e = copy_row_out(c->f.v, ny + 1, jr, nx, nz, b + 3 * plane, c->stream)) != cudaSuccess) return e;
  }
  return e;
}

cudaError_t unpack_halo(ns_slab* s) {
  ns_ctx* c = s->c;
  const int nx = c->cfg.nx, nz = c->cfg.nz, ny = s->nyv;
  const size_t plane = (size_t)nz * nx, sl = s->slot[NS_XCH_HALO] / 8;
  const double* rb = (const double*)s->recv[NS_XCH_HALO];
  cudaError_t e = cudaSuccess;
  for (int side = 0; side < 2; ++side) {
    if ((side == 0 && s->r == 0) || (side == 1 && s->r == s->p - 1)) continue;
    // below: slab r-1's part 1 into row / face 0; above: slab r+1's part 0 into row / face hb + nyl
    const double* b = side == 0 ? rb + (size_t)(s->r - 1) * sl + 4 * plane : rb + (size_t)(s->r + 1) * sl;
    const int jr = side == 0 ? 0 : s->hb + s->nyl;
    if ((e = copy_row_in(c->f.u, ny, jr, nx, nz, b, c->stream)) != cudaSuccess) return e;
    if ((e = copy_row_in(c->f.w, ny, jr, nx, nz, b + plane, c->stream)) != cudaSuccess) return e;
    if ((e = copy_row_in(c->f.p, ny, jr, nx, nz, b + 2 * plane, c->stream)) != cudaSuccess) return e;
    if ((e = copy_row_in(c->f.v, ny + 1, jr, nx, nz, b + 3 * plane, c->stream)) != cudaSuccess) return e;
  }
  return e;
}

YArgs y_args(ns_slab* s, int k) {
  ns_ctx* c = s->c;
  YArgs a{};
  a.r[0] = (double*)c->ru;
  a.r[1] = (double*)c->rv;
  a.r[2] = (double*)c->rw;
  a.rows[0] = a.rows[2] = s->nyv;
  a.rows[1] = s->nyv + 1;
  a.nx = c->cfg.nx;
  a.nz = c->cfg.nz;
  for (int q = 0; q < 2; ++q) {
    a.jo[q] = s->yjo[q];
    a.m[q] = s->ym[q];
    a.tab[q] = s->ytab[k][q];
  }
  a.Q = s->Q;
  a.send = (double*)s->send[NS_XCH_ADIY];
  a.slot = s->slot[NS_XCH_ADIY] / 8;
  a.recv = (const double*)s->recv[NS_XCH_ADIY];
  a.own = (double*)s->recv[NS_XCH_ADIY] + (size_t)s->r * a.slot;
  // PDD reads the neighbours' ends only; PPT every slab's
  if (s->ymode == NS_PART_PDD) {
    a.qlo = std::max(0, 2 * s->r - 2);
    a.qhi = std::min(s->Q, 2 * s->r + 2);
  } else {
    a.qlo = 0;
    a.qhi = s->Q;
  }
  return a;
}

PArgs p_args(ns_slab* s) {
  ns_ctx* c = s->c;
  PArgs a{};
  a.spec = (double*)c->spec;
  a.pa = c->gc + GC_PA * (s->nyv + 1) + s->hb;
  a.nx = c->cfg.nx;
  a.nyv = s->nyv;
  a.nzh = c->nzh;
  a.jo = s->hb;
  a.m = s->nyl;
  a.finv = s->pfinv;
  a.fcp = s->pfcp;
  a.pv = s->pv;
  a.pw = s->pw;
  a.coef = s->pcoef;
  a.Q = s->Q;
  a.gauge = s->r == 0;
  a.send = (double*)s->send[NS_XCH_POIS];
  a.slot = s->slot[NS_XCH_POIS] / 8;
  a.recv = (const double*)s->recv[NS_XCH_POIS];
  a.own = (double*)s->recv[NS_XCH_POIS] + (size_t)s->r * a.slot;
  return a;
}

// y-sweep and Poisson tables of slab s (host, once)
ns_status build_slab_tables(ns_slab* s, char* base) {
  const ns_config* g = &s->gcfg;
  const int ny = g->ny, nx = g->nx, nz = g->nz, nzh = nz / 2 + 1, p = s->p, Q = s->Q;
  std::vector<double> gc = grid_coefficients_host(g);
  auto GC = [&](int f, int j) { return gc[(size_t)f * (ny + 1) + j]; };
  std::vector<int> clo(p), chi(p), flo(p), fhi(p);
  for (int q = 0; q < p; ++q) {
    slab_rows(ny, p, q, &clo[q], &chi[q]);
    flo[q] = std::max(clo[q], 1) - 1;  // face unknowns are faces 1..ny-1, index f - 1
    fhi[q] = chi[q] - 1;
  }
  std::vector<double> scr;
  // y sweep: (I - beta_k delta_yy) per sub-step and class (rows of Sec. 2.2's factor along y:
  // centres for u and w, the interior faces 1 .. ny-1 for v)
  const double inv_re = g->re > 0 ? 1.0 / g->re : 0.0;
  auto yrows = [&](int k, int cl, std::vector<double>& a, std::vector<double>& b, std::vector<double>& cc) {
    const double beta = NS_ALPHA[k] * g->dt * inv_re / 2.0;
    const int n = cl ? ny - 1 : ny;
    a.resize(n);
    b.resize(n);
    cc.resize(n);
    for (int q = 0; q < n; ++q) {
      const int j = cl ? q + 1 : q;
      const double A = GC(cl ? GC_AF : GC_AC, j), C = GC(cl ? GC_CF : GC_CC, j);
      a[q] = -beta * A;
      cc[q] = -beta * C;
      b[q] = 1.0 + beta * (A + C);
    }
  };
  // the coupling PDD would drop, largest over every sub-step, class and slab boundary
  double drop = 0.0;
  for (int k = 0; k < 3; ++k)
    for (int cl = 0; cl < 2; ++cl) {
      std::vector<double> a, b, cc;
      yrows(k, cl, a, b, cc);
      SplitOut o;
      split_line(a.data(), b.data(), cc.data(), cl ? flo : clo, cl ? fhi : chi, s->r, false, o, scr);
      drop = std::max(drop, o.drop);
    }
  s->ydrop = drop;
  if (s->ymode == NS_PART_AUTO) s->ymode = drop <= 1e-15 ? NS_PART_PDD : NS_PART_PPT;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* q = base + off;
    off += al256(bytes);
    return q;
  };
  for (int k = 0; k < 3; ++k) {
    for (int cl = 0; cl < 2; ++cl) {
      std::vector<double> a, b, cc;
      yrows(k, cl, a, b, cc);
      SplitOut o;
      split_line(a.data(), b.data(), cc.data(), cl ? flo : clo, cl ? fhi : chi, s->r, s->ymode == NS_PART_PDD, o,
                 scr);
      if (!o.ok) return slab_fail(s, NS_ERR_STATE, "singular reduced system of the y sweep");
      const int m = (int)o.a.size();
      std::vector<double> t;
      for (auto* vec : {&o.a, &o.ip, &o.cp, &o.v, &o.w}) t.insert(t.end(), vec->begin(), vec->end());
      t.insert(t.end(), o.clo.begin(), o.clo.end());
      t.insert(t.end(), o.chi.begin(), o.chi.end());
      double* dtab = (double*)take((5 * (s->nyl + 1) + 2 * Q) * 8);
      cudaError_t e = cudaMemcpy(dtab, t.data(), t.size() * 8, cudaMemcpyHostToDevice);
      if (e != cudaSuccess) return cuda_fail(s, "slab y tables", e);
      s->ytab[k][cl] = dtab;
      s->ym[cl] = m;
    }
  }
  s->yjo[0] = s->hb;
  s->yjo[1] = s->hb + (s->j0 == 0 ? 1 : 0);
  // Poisson: one tridiagonal system per (kx, kz) in y, zero normal gradient at both ends, the
  // (0, 0) line gauged by phi_0 = 0; modified wavenumbers as the context's
  const size_t pl = (size_t)nzh * s->nyl * nx;
  std::vector<double> hf(pl), hc(pl), hv(pl), hw(pl), hco((size_t)nzh * nx * 2 * Q);
  const double PI = 3.14159265358979323846;
  const double dx = g->lx / nx, dz = g->lz / nz;
  std::vector<double> a(ny), b(ny), cc(ny);
  for (int kz = 0; kz < nzh; ++kz)
    for (int i = 0; i < nx; ++i) {
      // periodic x: the DFT's wavenumbers; inflow / outflow: the cosine transform's (DCT-II)
      const int ii = i <= nx - i ? i : nx - i;
      const double lamx = g->bc_x == 1 ? (2.0 / (dx * dx)) * (1.0 - std::cos(PI * i / nx))
                                       : (2.0 / (dx * dx)) * (1.0 - std::cos(2.0 * PI * ii / nx));
      const double lam = lamx + (2.0 / (dz * dz)) * (1.0 - std::cos(2.0 * PI * kz / nz));
      for (int j = 0; j < ny; ++j) {
        a[j] = GC(GC_PA, j);
        cc[j] = GC(GC_PC, j);
        b[j] = -(a[j] + cc[j]) - lam;
      }
      if (i == 0 && kz == 0) {
        a[0] = 0.0;
        b[0] = 1.0;
        cc[0] = 0.0;
      }
      SplitOut o;
      split_line(a.data(), b.data(), cc.data(), clo, chi, s->r, false, o, scr);
      if (!o.ok) return slab_fail(s, NS_ERR_STATE, "singular reduced system of the Poisson y solve");
      for (int j = 0; j < s->nyl; ++j) {
        const size_t q = ((size_t)kz * s->nyl + j) * nx + i;
        hf[q] = o.ip[j];
        hc[q] = o.cp[j];
        hv[q] = o.v[j];
        hw[q] = o.w[j];
      }
      for (int q = 0; q < Q; ++q) {
        hco[(((size_t)kz * nx + i) * 2 + 0) * Q + q] = o.clo[q];
        hco[(((size_t)kz * nx + i) * 2 + 1) * Q + q] = o.chi[q];
      }
    }
  s->pfinv = (double*)take(pl * 8);
  s->pfcp = (double*)take(pl * 8);
  s->pv = (double*)take(pl * 8);
  s->pw = (double*)take(pl * 8);
  s->pcoef = (double*)take(hco.size() * 8 + 8);
  const std::pair<double*, const std::vector<double>*> up[] = {
      {s->pfinv, &hf}, {s->pfcp, &hc}, {s->pv, &hv}, {s->pw, &hw}, {s->pcoef, &hco}};
  for (const auto& q : up)
    if (!q.second->empty()) {
      cudaError_t e = cudaMemcpy(q.first, q.second->data(), q.second->size() * 8, cudaMemcpyHostToDevice);
      if (e != cudaSuccess) return cuda_fail(s, "slab Poisson tables", e);
    }
  if (g->recycle_i) {  // recycling block of the whole grid, sample offsets in the gathered buffer
    std::vector<double> hr(recycle_block_doubles(ny));
    recycle_grid_host(s->gyf.data(), ny, hr.data());
    s->rcy = (double*)take(hr.size() * 8);
    const long sd = (long)(slot_bytes(g, p, NS_XCH_RCY) / 8), rm = rows_max(ny, p);
    std::vector<long> off(3 * (size_t)ny + 1);
    for (int q = 0; q < p; ++q) {
      for (int j = clo[q]; j < chi[q]; ++j) {
        off[j] = q * sd + (long)(j - clo[q]) * nz;               // u
        off[ny + j] = q * sd + (rm + j - clo[q]) * (long)nz;     // w
        off[2 * ny + j] = q * sd + (2 * rm + j - clo[q]) * (long)nz;  // v, face j
      }
    }
    off[3 * ny] = (p - 1) * sd + (2 * rm + ny - clo[p - 1]) * (long)nz;  // v, the top face
    s->rcy_off = (long*)take(off.size() * 8);
    cudaError_t e = cudaMemcpy(s->rcy, hr.data(), hr.size() * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(s->rcy_off, off.data(), off.size() * 8, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(s, "slab recycling tables", e);
  }
  for (int x = 0; x < NS_XCH_COUNT; ++x) {
    s->slot[x] = slot_bytes(g, p, x);
    s->send[x] = take(s->slot[x]);
    s->recv[x] = take((size_t)p * s->slot[x]);
    cudaError_t e = cudaMemset(s->recv[x], 0, (size_t)p * s->slot[x]);
    if (e != cudaSuccess) return cuda_fail(s, "slab exchange buffers", e);
  }
  return NS_OK;
}

}  // namespace

extern "C" {

ns_status ns_slab_rows(int ny, int p, int r, int* j0, int* j1) {
  if (!j0 || !j1 || p < 1 || r < 0 || r >= p || ny < 1) return NS_ERR_ARG;
  slab_rows(ny, p, r, j0, j1);
  return NS_OK;
}

size_t ns_slab_slot_bytes(const ns_config* cfg, int p, int xch) {
  if (!check_slab(cfg, p, 0).empty() || xch < 0 || xch >= NS_XCH_COUNT) return 0;
  return slot_bytes(cfg, p, xch);
}

ns_status ns_slab_slots(int p, int r, int xch, int ymode, int* lo, int* hi) {
  if (!lo || !hi || p < 1 || r < 0 || r >= p) return NS_ERR_ARG;
  const int below = std::max(0, r - 1), above = std::min(p - 1, r + 1);
  switch (xch) {
    case NS_XCH_HALO: *lo = below, *hi = above; break;
    case NS_XCH_ADIY:
      if (ymode == NS_PART_PDD) *lo = below, *hi = above;
      else if (ymode == NS_PART_PPT) *lo = 0, *hi = p - 1;
      else return NS_ERR_ARG;
      break;
    case NS_XCH_VSTAR: *lo = r, *hi = above; break;
    case NS_XCH_POIS: *lo = 0, *hi = p - 1; break;
    case NS_XCH_PHI: *lo = below, *hi = above; break;
    case NS_XCH_FLUX: *lo = 0, *hi = p - 1; break;
    case NS_XCH_RCY: *lo = 0, *hi = p - 1; break;
    default: return NS_ERR_ARG;
  }
  return NS_OK;
}

ns_status ns_slab_solve_line_host(int n, const double* a, const double* b, const double* c, const double* d, int p,
                                  int mode, double* x, double* dropped) {
  if (!a || !b || !c || !d || !x || p < 1 || n < 2 * p || (mode != NS_PART_PPT && mode != NS_PART_PDD))
    return NS_ERR_ARG;
  std::vector<int> lo(p), hi(p);
  for (int q = 0; q < p; ++q) slab_rows(n, p, q, &lo[q], &hi[q]);
  std::vector<double> scr, h(2 * (size_t)(p - 1), 0.0);
  std::vector<SplitOut> tab(p);
  // each slab's tables, and its block solve x~ (the slab kernels' forward and back sweeps)
  for (int r = 0; r < p; ++r) {
    split_line(a, b, c, lo, hi, r, mode == NS_PART_PDD, tab[r], scr);
    if (!tab[r].ok) return NS_ERR_STATE;
    const SplitOut& o = tab[r];
    const int m = hi[r] - lo[r];
    double prev = 0.0;
    for (int j = 0; j < m; ++j) {
      prev = (d[lo[r] + j] - o.a[j] * prev) * o.ip[j];
      x[lo[r] + j] = prev;
    }
    for (int j = m - 2; j >= 0; --j) x[lo[r] + j] -= o.cp[j] * x[lo[r] + j + 1];
  }
  // the gathered end values h[2t] = x~^(t)_m, h[2t+1] = x~^(t+1)_1, then each slab's correction
  for (int t = 0; t + 1 < p; ++t) {
    h[2 * t] = x[hi[t] - 1];
    h[2 * t + 1] = x[lo[t + 1]];
  }
  for (int r = 0; r < p; ++r) {
    const SplitOut& o = tab[r];
    double ylo = 0.0, yhi = 0.0;
    for (size_t q = 0; q < h.size(); ++q) {
      ylo += o.clo[q] * h[q];
      yhi += o.chi[q] * h[q];
    }
    for (int j = 0; j < hi[r] - lo[r]; ++j) x[lo[r] + j] -= o.v[j] * ylo + o.w[j] * yhi;
  }
  if (dropped) *dropped = tab[0].drop;
  return NS_OK;
}

size_t ns_slab_workspace_bytes(const ns_config* cfg, int p, int r) {
  if (!check_slab(cfg, p, r).empty()) return 0;
  std::vector<double> yf;
  ns_config sub;
  int hb, ha;
  sub_config(cfg, p, r, yf, &sub, &hb, &ha);
  const size_t w = ns_workspace_bytes(&sub);
  if (w == 0) return 0;
  return al256(w) + extra_bytes(cfg, p, r);
}

ns_status ns_slab_init(ns_slab** out, const ns_config* cfg, int p, int r, int ymode, const ns_fields* local,
                       void* workspace, size_t ws_bytes, void* cuda_stream) {
  ns_set_thread_error("");
  if (!out) return slab_fail(nullptr, NS_ERR_ARG, "out is NULL");
  *out = nullptr;
  const std::string m = check_slab(cfg, p, r);
  if (!m.empty()) return slab_fail(nullptr, NS_ERR_ARG, m);
  if (ymode != NS_PART_AUTO && ymode != NS_PART_PPT && ymode != NS_PART_PDD)
    return slab_fail(nullptr, NS_ERR_ARG, "ymode must be NS_PART_AUTO, NS_PART_PPT or NS_PART_PDD");
  const size_t need = ns_slab_workspace_bytes(cfg, p, r);
  if (need == 0) return slab_fail(nullptr, NS_ERR_SIZE, "grid size outside the supported range");
  ns_slab* s = new (std::nothrow) ns_slab();
  if (!s) return slab_fail(nullptr, NS_ERR_ARG, "out of host memory");
  s->gcfg = *cfg;
  s->gyf.assign(cfg->yf, cfg->yf + cfg->ny + 1);
  s->gcfg.yf = s->gyf.data();
  s->p = p;
  s->r = r;
  s->Q = 2 * (p - 1);
  slab_rows(cfg->ny, p, r, &s->j0, &s->j1);
  s->nyl = s->j1 - s->j0;
  s->ymode = ymode;
  std::vector<double> yf;
  ns_config sub;
  sub_config(cfg, p, r, yf, &sub, &s->hb, &s->ha);
  s->nyv = sub.ny;
  if (workspace) {
    if (ws_bytes < need || (uintptr_t)workspace % 256) {
      delete s;
      return slab_fail(nullptr, NS_ERR_ARG, "workspace too small or not 256-byte aligned");
    }
    s->ws = workspace;
  } else {
    cudaError_t e = cudaMalloc(&s->ws, need);
    if (e != cudaSuccess) {
      delete s;
      return slab_fail(nullptr, NS_ERR_CUDA, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    s->own_ws = true;
  }
  const size_t wctx = al256(ns_workspace_bytes(&sub));
  ns_status st = ns_init(&s->c, &sub, local, s->ws, wctx, cuda_stream);
  if (st != NS_OK) {
    const std::string msg = ns_last_error(nullptr);
    if (s->own_ws) cudaFree(s->ws);
    delete s;
    return slab_fail(nullptr, st, "sub-grid context: " + msg);
  }
  st = build_slab_tables(s, (char*)s->ws + wctx);
  if (st != NS_OK) {
    const std::string msg = s->err;
    ns_slab_destroy(s);
    return slab_fail(nullptr, st, msg);
  }
  *out = s;
  return NS_OK;
}

ns_status ns_slab_phase(ns_slab* s, int phase, int k) {
  if (!s) return slab_fail(nullptr, NS_ERR_ARG, "slab is NULL");
  if (k < 0 || k > 2) return slab_fail(s, NS_ERR_ARG, "substep must be 0, 1 or 2");
  ns_ctx* c = s->c;
  const int nx = c->cfg.nx, nz = c->cfg.nz;
  const dim3 ygrid((nx + 127) / 128, nz, 3), pgrid((2 * nx + 127) / 128, c->nzh);
  cudaError_t e = cudaSuccess;
  switch (phase) {
    case NS_SLAB_PACK:
      if ((e = pack_halo(s)) != cudaSuccess) break;
      e = pack_rcy(s);
      break;
    case NS_SLAB_RHS:
      if ((e = unpack_halo(s)) != cudaSuccess) break;
      if (k == 0 && s->gcfg.recycle_i) {  // inflow planes of every row held here, from the whole plane
        const int ny = s->gcfg.ny;
        e = launch_recycle_gathered((const double*)s->recv[NS_XCH_RCY], s->rcy_off, s->rcy_off + ny,
                                    s->rcy_off + 2 * ny, s->rcy, ny, nz, s->gcfg.delta_in, s->gcfg.u_conv, c->f.u,
                                    c->f.v_in, c->f.w_in, nx, s->nyv, s->j0 - s->hb, c->stream);
        if (e != cudaSuccess) break;
      }
      if ((e = launch_rhs(c, k)) != cudaSuccess) break;
      if ((e = launch_outflow(c, k)) != cudaSuccess) break;  // inflow / outflow only
      if ((e = launch_adi_x(c, k)) != cudaSuccess) break;
      slab_ysweep_local<<<ygrid, 128, 0, c->stream>>>(y_args(s, k));
      e = cudaGetLastError();
      break;
    case NS_SLAB_ADIZ:
      slab_ysweep_correct<<<ygrid, 128, 0, c->stream>>>(y_args(s, k));
      if ((e = cudaGetLastError()) != cudaSuccess) break;
      if ((e = launch_adi_z(c, k)) != cudaSuccess) break;
      if (s->r > 0 &&  // v* on face j0, which slab r-1 reads for the divergence of its top row
          (e = copy_row_out(c->f.v, s->nyv + 1, s->hb, nx, nz, (double*)s->send[NS_XCH_VSTAR], c->stream)) !=
              cudaSuccess)
        break;
      if (c->bl) {  // this slab's share of the inflow - outflow volume flux
        slab_flux_partial<<<1, 1024, 0, c->stream>>>(c->f.u, c->f.u_out, c->gc, nx, s->nyv, nz, s->hb, s->nyl,
                                                     (double*)s->send[NS_XCH_FLUX],
                                                     (double*)(s->recv[NS_XCH_FLUX] + (size_t)s->r * s->slot[NS_XCH_FLUX]));
        e = cudaGetLastError();
      }
      break;
    case NS_SLAB_POIS:
      if (c->bl) {  // u_out shifted so that the outflow flux equals the inflow flux (every slab alike)
        const double area = (s->gyf[s->gcfg.ny] - s->gyf[0]) * s->gcfg.lz;
        slab_flux_apply<<<64, 256, 0, c->stream>>>(c->f.u_out, (long)nz * s->nyv, (const double*)s->recv[NS_XCH_FLUX],
                                                   s->slot[NS_XCH_FLUX] / 8, s->p, c->dz / area);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
      }
      if (s->r < s->p - 1 &&
          (e = copy_row_in(c->f.v, s->nyv + 1, s->hb + s->nyl, nx, nz,
                           (const double*)(s->recv[NS_XCH_VSTAR] + (size_t)(s->r + 1) * s->slot[NS_XCH_VSTAR]),
                           c->stream)) != cudaSuccess)
        break;
      if ((e = launch_pois_divz(c, k)) != cudaSuccess) break;
      if ((e = launch_pois_fftx_fwd(c, k)) != cudaSuccess) break;
      slab_pois_local<<<pgrid, 128, 0, c->stream>>>(p_args(s));
      e = cudaGetLastError();
      break;
    case NS_SLAB_PHI:
      slab_pois_correct<<<pgrid, 128, 0, c->stream>>>(p_args(s));
      if ((e = cudaGetLastError()) != cudaSuccess) break;
      if ((e = launch_pois_fftx_inv(c, k)) != cudaSuccess) break;
      if ((e = launch_pois_ifftz(c, k)) != cudaSuccess) break;
      // phi of row j1-1, which slab r+1 reads for the gradient at its face j1, and of row j0, which
      // slab r-1 reads for the Laplacian of phi at its row j0-1 (the Kim-Moin pressure update)
      if (s->r < s->p - 1 &&
          (e = copy_row_out(c->phi, s->nyv, s->hb + s->nyl - 1, nx, nz,
                            (double*)s->send[NS_XCH_PHI] + (size_t)nz * nx, c->stream)) != cudaSuccess)
        break;
      if (s->r > 0) e = copy_row_out(c->phi, s->nyv, s->hb, nx, nz, (double*)s->send[NS_XCH_PHI], c->stream);
      break;
    case NS_SLAB_PROJECT: {
      const size_t sl = s->slot[NS_XCH_PHI] / 8, plane = (size_t)nz * nx;
      const double* rb = (const double*)s->recv[NS_XCH_PHI];
      if (s->r > 0 &&  // halo row below: slab r-1's row j0-1
          (e = copy_row_in(c->phi, s->nyv, 0, nx, nz, rb + (size_t)(s->r - 1) * sl + plane, c->stream)) != cudaSuccess)
        break;
      if (s->r < s->p - 1 &&  // halo row above: slab r+1's row j1
          (e = copy_row_in(c->phi, s->nyv, s->hb + s->nyl, nx, nz, rb + (size_t)(s->r + 1) * sl, c->stream)) !=
              cudaSuccess)
        break;
      if ((e = launch_project(c, k)) != cudaSuccess) break;
      if ((e = pack_halo(s)) != cudaSuccess) break;
      if (k == 2) e = pack_rcy(s);  // the recycle plane the next step's sub-step 0 reads
      break;
    }
    default:
      return slab_fail(s, NS_ERR_ARG, "unknown phase");
  }
  if (e != cudaSuccess) return cuda_fail(s, "slab phase", e);
  return NS_OK;
}

ns_status ns_slab_buffers(ns_slab* s, int xch, void** send, void** recv, size_t* slot) {
  if (!s || !send || !recv || !slot || xch < 0 || xch >= NS_XCH_COUNT) return NS_ERR_ARG;
  *send = s->send[xch];
  *recv = s->recv[xch];
  *slot = s->slot[xch];
  return NS_OK;
}

ns_status ns_slab_mode(ns_slab* s, int* ymode, double* ydrop) {
  if (!s || !ymode || !ydrop) return NS_ERR_ARG;
  *ymode = s->ymode;
  *ydrop = s->ydrop;
  return NS_OK;
}

ns_ctx* ns_slab_context(ns_slab* s) { return s ? s->c : nullptr; }

ns_status ns_slab_sync(ns_slab* s) {
  if (!s) return NS_ERR_ARG;
  const ns_status st = ns_sync(s->c);
  if (st != NS_OK) s->err = ns_last_error(s->c);
  return st;
}

const char* ns_slab_last_error(ns_slab* s) { return s ? s->err.c_str() : ns_last_error(nullptr); }

void ns_slab_destroy(ns_slab* s) {
  if (!s) return;
  if (s->c) ns_destroy(s->c);
  if (s->own_ws && s->ws) cudaFree(s->ws);
  delete s;
}

}  // extern "C"
