// Recycling inflow (Sec. 2.1: turbulent inflow by the rescaling method of Lund, Wu & Squires,
// J. Comput. Phys. 140, 1998).  Once per time step, before the RHS of sub-step 0:
//   1. spanwise means U (centres), V (faces), W (centres) of the recycle plane, the u face i_r,
//      with v and w averaged from the centres i_r - 1 and i_r (one block per row, fixed order);
//   2. delta_rec, the first height where U reaches 0.99 U_inf (linear between centres), and
//      gamma = (delta_rec / delta_in)^(1/8), the ratio of the inlet to the recycle friction
//      velocity under the 1/5 power law;
//   3. the inflow planes: each row at height y takes the plane's mean and fluctuation at
//      y gamma (inner, same y+) and y delta_rec / delta_in (outer, same y / delta) by linear
//      interpolation (wall value 0 for u and w below the first centre, top value held above),
//      inner mean gamma U, outer gamma U + (1 - gamma) U_inf, mean V unscaled, mean W zero,
//      fluctuations times gamma, blended with Lund's weight
//      W(eta) = (1 + tanh(4 (eta - 0.2) / (0.6 eta + 0.2)) / tanh 4) / 2 (1 above eta = 1).
// Writes u on face 0, v_in and w_in.  The recycle plane comes from the fields (one context) or
// from samples gathered from every y slab (ns_slab.cu: each slab packs its own rows, an all-gather
// gives every slab the whole plane, and every slab writes the inflow rows it holds); the
// arithmetic is the same either way.
#include "ns_internal.cuh"

namespace {

// rcy block: ys[ny+1] = (0 at the wall, yc_0 .. yc_{ny-1}), yf[ny+1], U[ny], V[ny+1], W[ny],
// {gamma, r = delta_rec / delta_in}
struct RcyView {
  const double* ys;
  const double* yf;
  double* U;
  double* V;
  double* W;
  double* sc;
};
__host__ __device__ inline RcyView rcy_view(double* b, int ny) {
  RcyView v;
  v.ys = b;
  v.yf = b + ny + 1;
  v.U = b + 2 * ny + 2;
  v.V = v.U + ny;
  v.W = v.V + ny + 1;
  v.sc = v.W + ny;
  return v;
}

// Samples of the recycle plane, rows and faces of the whole domain: u on face i_r, v and w
// averaged over the centres i_r - 1 and i_r.  From the fields, or (g set) from a gathered buffer
// where row j's nz samples start at uoff[j] (u), woff[j] (w) and face f's at voff[f] (v).
struct RcySrc {
  const double* u;
  const double* v;
  const double* w;
  int nx, ny, ir;
  const double* g;
  const long* uoff;
  const long* woff;
  const long* voff;
  __device__ __forceinline__ double ur(int j, int k) const {
    if (g) return g[__ldg(uoff + j) + k];
    return __ldg(u + ((long)k * ny + j) * nx + ir);
  }
  __device__ __forceinline__ double wr(int j, int k) const {
    if (g) return g[__ldg(woff + j) + k];
    const long c = ((long)k * ny + j) * nx;
    return 0.5 * (__ldg(w + c + ir - 1) + __ldg(w + c + ir));
  }
  __device__ __forceinline__ double vr(int f, int k) const {
    if (g) return g[__ldg(voff + f) + k];
    const long c = ((long)k * (ny + 1) + f) * nx;
    return 0.5 * (__ldg(v + c + ir - 1) + __ldg(v + c + ir));
  }
};

// Where the inflow planes go: rows rows of cells (and rows + 1 faces) of the arrays held here,
// local row 0 being row jg0 of the whole domain (one context: rows = ny, jg0 = 0).
struct RcyDst {
  double* u;     // u on face 0 of every local row: u[(k rows + jl) nx]
  double* v_in;  // [k (rows + 1) + fl]
  double* w_in;  // [k rows + jl]
  int nx, rows, jg0;
};

__global__ void __launch_bounds__(256) recycle_means_kernel(const RcySrc src, double* rcy, int ny, int nz) {
  const int j = blockIdx.x;  // 0..ny
  const RcyView R = rcy_view(rcy, ny);
  __shared__ double red[3][256];
  double su = 0.0, sv = 0.0, sw = 0.0;
  for (int k = threadIdx.x; k < nz; k += blockDim.x) {
    sv += src.vr(j, k);
    if (j < ny) {
      su += src.ur(j, k);
      sw += src.wr(j, k);
    }
  }
  red[0][threadIdx.x] = su;
  red[1][threadIdx.x] = sv;
  red[2][threadIdx.x] = sw;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int q = 0; q < 3; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    R.V[j] = red[1][0] / nz;
    if (j < ny) {
      R.U[j] = red[0][0] / nz;
      R.W[j] = red[2][0] / nz;
    }
  }
}

__global__ void recycle_scalars_kernel(double* rcy, int ny, double delta_in, double u_inf) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const RcyView R = rcy_view(rcy, ny);
  const double target = 0.99 * u_inf;
  const double* yc = R.ys + 1;
  double d = yc[ny - 1];
  for (int j = 0; j < ny; ++j)
    if (R.U[j] >= target) {
      d = (j == 0) ? yc[0] * target / R.U[0]
                   : yc[j - 1] + (target - R.U[j - 1]) * (yc[j] - yc[j - 1]) / (R.U[j] - R.U[j - 1]);
      break;
    }
  R.sc[0] = pow(d / delta_in, 0.125);
  R.sc[1] = d / delta_in;
}

// Linear interpolation at height y over n points ys (increasing) with values f(q), end values
// held outside; f is a functor of the point index.
template <typename F>
__device__ __forceinline__ double interp(double y, const double* ys, int n, F f) {
  if (y <= ys[0]) return f(0);
  if (y >= ys[n - 1]) return f(n - 1);
  int lo = 0, hi = n - 1;  // ys[lo] < y < ys[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (ys[mid] <= y) lo = mid;
    else hi = mid;
  }
  const double s = (f(hi) - f(lo)) / (ys[hi] - ys[lo]);
  return s * (y - ys[lo]) + f(lo);
}

__device__ __forceinline__ double lund_weight(double eta) {
  if (eta > 1.0) return 1.0;
  return 0.5 * (1.0 + tanh(4.0 * (eta - 0.2) / (0.6 * eta + 0.2)) / tanh(4.0));
}

__global__ void __launch_bounds__(128) recycle_apply_kernel(const RcySrc src, const RcyDst dst, const double* rcy,
                                                            int ny, double delta_in, double u_inf) {
  const int jl = blockIdx.x * blockDim.x + threadIdx.x;  // local row / face 0..rows
  const int k = blockIdx.y;
  if (jl > dst.rows) return;
  const int j = dst.jg0 + jl;  // row / face of the whole domain
  const RcyView R = rcy_view(const_cast<double*>(rcy), ny);
  const double gam = R.sc[0], r = R.sc[1];
  if (jl < dst.rows) {
    // centre samples with the wall point (y = 0, value 0) in front: sample q is centre q - 1
    const double y = R.ys[j + 1];
    const double yi = gam * y, yo = r * y;
    auto Uc = [&](int q) { return q == 0 ? 0.0 : R.U[q - 1]; };
    auto up = [&](int q) { return q == 0 ? 0.0 : src.ur(q - 1, k) - R.U[q - 1]; };
    auto wp = [&](int q) { return q == 0 ? 0.0 : src.wr(q - 1, k) - R.W[q - 1]; };
    const double W = lund_weight(y / delta_in);
    const double Ui = gam * interp(yi, R.ys, ny + 1, Uc);
    const double Uo = gam * interp(yo, R.ys, ny + 1, Uc) + (1.0 - gam) * u_inf;
    const double ui = gam * interp(yi, R.ys, ny + 1, up), uo = gam * interp(yo, R.ys, ny + 1, up);
    dst.u[((long)k * dst.rows + jl) * dst.nx] = (1.0 - W) * (Ui + ui) + W * (Uo + uo);
    const double wi = gam * interp(yi, R.ys, ny + 1, wp), wo = gam * interp(yo, R.ys, ny + 1, wp);
    dst.w_in[(long)k * dst.rows + jl] = (1.0 - W) * wi + W * wo;
  }
  {
    double val = 0.0;
    if (j > 0 && j < ny) {
      const double y = R.yf[j];
      const double yi = gam * y, yo = r * y;
      auto Vf = [&](int q) { return R.V[q]; };
      auto vp = [&](int q) { return src.vr(q, k) - R.V[q]; };
      const double W = lund_weight(y / delta_in);
      const double Vi = interp(yi, R.yf, ny + 1, Vf), Vo = interp(yo, R.yf, ny + 1, Vf);
      const double vi = gam * interp(yi, R.yf, ny + 1, vp), vo = gam * interp(yo, R.yf, ny + 1, vp);
      val = (1.0 - W) * (Vi + vi) + W * (Vo + vo);
    }
    dst.v_in[(long)k * (dst.rows + 1) + jl] = val;
  }
}

}  // namespace

size_t recycle_block_doubles(int ny) { return 5 * (size_t)ny + 4 + 2; }

void recycle_grid_host(const double* yf, int ny, double* h) {
  for (size_t q = 0; q < recycle_block_doubles(ny); ++q) h[q] = 0.0;
  h[0] = yf[0];
  for (int j = 0; j < ny; ++j) h[1 + j] = 0.5 * (yf[j] + yf[j + 1]);
  for (int j = 0; j <= ny; ++j) h[ny + 1 + j] = yf[j];
}

cudaError_t recycle_upload_grid(ns_ctx* c) {
  const int ny = c->cfg.ny;
  std::vector<double> h(recycle_block_doubles(ny));
  recycle_grid_host(c->yf.data(), ny, h.data());
  cudaError_t e = cudaMemcpyAsync(c->rcy, h.data(), h.size() * 8, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return e;
}

namespace {
cudaError_t recycle_run(const RcySrc& src, const RcyDst& dst, double* rcy, int ny, int nz, double delta_in,
                        double u_inf, cudaStream_t st) {
  recycle_means_kernel<<<ny + 1, 256, 0, st>>>(src, rcy, ny, nz);
  recycle_scalars_kernel<<<1, 32, 0, st>>>(rcy, ny, delta_in, u_inf);
  recycle_apply_kernel<<<dim3((dst.rows + 1 + 127) / 128, nz), 128, 0, st>>>(src, dst, rcy, ny, delta_in, u_inf);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_recycle(ns_ctx* c, int k) {
  if (k != 0 || !c->cfg.recycle_i) return cudaSuccess;
  const int nx = c->cfg.nx, ny = c->cfg.ny, nz = c->cfg.nz;
  const RcySrc src{c->f.u, c->f.v, c->f.w, nx, ny, c->cfg.recycle_i, nullptr, nullptr, nullptr, nullptr};
  const RcyDst dst{c->f.u, c->f.v_in, c->f.w_in, nx, ny, 0};
  return recycle_run(src, dst, c->rcy, ny, nz, c->cfg.delta_in, c->cfg.u_conv, c->launch);
}

cudaError_t launch_recycle_gathered(const double* g, const long* uoff, const long* woff, const long* voff, double* rcy,
                                    int ny, int nz, double delta_in, double u_inf, double* u, double* v_in,
                                    double* w_in, int nx, int rows, int jg0, cudaStream_t st) {
  const RcySrc src{nullptr, nullptr, nullptr, nx, ny, 0, g, uoff, woff, voff};
  const RcyDst dst{u, v_in, w_in, nx, rows, jg0};
  return recycle_run(src, dst, rcy, ny, nz, delta_in, u_inf, st);
}
