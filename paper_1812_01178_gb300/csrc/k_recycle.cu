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
// Writes u on face 0, v_in and w_in.
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

__global__ void __launch_bounds__(256) recycle_means_kernel(const double* __restrict__ u, const double* __restrict__ v,
                                                            const double* __restrict__ w, double* rcy, int nx,
                                                            int ny, int nz, int ir) {
  const int j = blockIdx.x;  // 0..ny
  const RcyView R = rcy_view(rcy, ny);
  __shared__ double red[3][256];
  double su = 0.0, sv = 0.0, sw = 0.0;
  for (int k = threadIdx.x; k < nz; k += blockDim.x) {
    const long fv = ((long)k * (ny + 1) + j) * nx;
    sv += 0.5 * (__ldg(v + fv + ir - 1) + __ldg(v + fv + ir));
    if (j < ny) {
      const long c = ((long)k * ny + j) * nx;
      su += __ldg(u + c + ir);
      sw += 0.5 * (__ldg(w + c + ir - 1) + __ldg(w + c + ir));
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

__global__ void __launch_bounds__(128) recycle_apply_kernel(double* __restrict__ u, const double* __restrict__ v,
                                                            const double* __restrict__ w, double* __restrict__ v_in,
                                                            double* __restrict__ w_in, const double* rcy, int nx,
                                                            int ny, int nz, int ir, double delta_in, double u_inf) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;  // 0..ny
  const int k = blockIdx.y;
  if (j > ny) return;
  const RcyView R = rcy_view(const_cast<double*>(rcy), ny);
  const double gam = R.sc[0], r = R.sc[1];
  if (j < ny) {
    // centre samples with the wall point (y = 0, value 0) in front: sample q is centre q - 1
    const double y = R.ys[j + 1];
    const double yi = gam * y, yo = r * y;
    const long row = (long)k * ny * nx;
    auto Uc = [&](int q) { return q == 0 ? 0.0 : R.U[q - 1]; };
    auto up = [&](int q) { return q == 0 ? 0.0 : __ldg(u + row + (long)(q - 1) * nx + ir) - R.U[q - 1]; };
    auto wp = [&](int q) {
      if (q == 0) return 0.0;
      const long c = row + (long)(q - 1) * nx;
      return 0.5 * (__ldg(w + c + ir - 1) + __ldg(w + c + ir)) - R.W[q - 1];
    };
    const double W = lund_weight(y / delta_in);
    const double Ui = gam * interp(yi, R.ys, ny + 1, Uc);
    const double Uo = gam * interp(yo, R.ys, ny + 1, Uc) + (1.0 - gam) * u_inf;
    const double ui = gam * interp(yi, R.ys, ny + 1, up), uo = gam * interp(yo, R.ys, ny + 1, up);
    u[row + (long)j * nx] = (1.0 - W) * (Ui + ui) + W * (Uo + uo);
    const double wi = gam * interp(yi, R.ys, ny + 1, wp), wo = gam * interp(yo, R.ys, ny + 1, wp);
    w_in[(long)k * ny + j] = (1.0 - W) * wi + W * wo;
  }
  {
    double val = 0.0;
    if (j > 0 && j < ny) {
      const double y = R.yf[j];
      const double yi = gam * y, yo = r * y;
      const long rowv = (long)k * (ny + 1) * nx;
      auto Vf = [&](int q) { return R.V[q]; };
      auto vp = [&](int q) {
        const long c = rowv + (long)q * nx;
        return 0.5 * (__ldg(v + c + ir - 1) + __ldg(v + c + ir)) - R.V[q];
      };
      const double W = lund_weight(y / delta_in);
      const double Vi = interp(yi, R.yf, ny + 1, Vf), Vo = interp(yo, R.yf, ny + 1, Vf);
      const double vi = gam * interp(yi, R.yf, ny + 1, vp), vo = gam * interp(yo, R.yf, ny + 1, vp);
      val = (1.0 - W) * (Vi + vi) + W * (Vo + vo);
    }
    v_in[(long)k * (ny + 1) + j] = val;
  }
}

}  // namespace

size_t recycle_block_doubles(int ny) { return 5 * (size_t)ny + 4 + 2; }

cudaError_t recycle_upload_grid(ns_ctx* c) {
  const int ny = c->cfg.ny;
  std::vector<double> h(recycle_block_doubles(ny), 0.0);
  h[0] = c->yf[0];
  for (int j = 0; j < ny; ++j) h[1 + j] = 0.5 * (c->yf[j] + c->yf[j + 1]);
  for (int j = 0; j <= ny; ++j) h[ny + 1 + j] = c->yf[j];
  cudaError_t e = cudaMemcpyAsync(c->rcy, h.data(), h.size() * 8, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return e;
}

cudaError_t launch_recycle(ns_ctx* c, int k) {
  if (k != 0 || !c->cfg.recycle_i) return cudaSuccess;
  const int nx = c->cfg.nx, ny = c->cfg.ny, nz = c->cfg.nz, ir = c->cfg.recycle_i;
  recycle_means_kernel<<<ny + 1, 256, 0, c->launch>>>(c->f.u, c->f.v, c->f.w, c->rcy, nx, ny, nz, ir);
  recycle_scalars_kernel<<<1, 32, 0, c->launch>>>(c->rcy, ny, c->cfg.delta_in, c->cfg.u_conv);
  recycle_apply_kernel<<<dim3((ny + 1 + 127) / 128, nz), 128, 0, c->launch>>>(
      c->f.u, c->f.v, c->f.w, c->f.v_in, c->f.w_in, c->rcy, nx, ny, nz, ir, c->cfg.delta_in, c->cfg.u_conv);
  return cudaGetLastError();
}
