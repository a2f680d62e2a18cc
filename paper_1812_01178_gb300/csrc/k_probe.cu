// ns_fp64_fma_probe: the FP64 FMA throughput of the GPU, measured, as the denominator of the
// FP64-ALU roofline of the solver's kernels (a measurement aid; the paper has no counterpart).
//
// Every thread runs kChains independent chains x <- x * b + c of n_iter dependent FMAs each, so
// the FP64 pipe always has independent work to issue; b and c are kernel arguments, so nothing
// folds at compile time.  One launch performs n_blocks * 256 * kChains * n_iter FMAs
// (2 flops each).  The sum of the chains is stored so that none of them is dead code.
#include "ns_internal.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) fp64_fma_probe_kernel(double* __restrict__ out, int n_iter,
                                                                   double b, double c) {
  double x[kChains];
#pragma unroll
  for (int q = 0; q < kChains; ++q) x[q] = 1e-3 * (double)(threadIdx.x + q);
  for (int it = 0; it < n_iter; ++it) {
#pragma unroll
    for (int q = 0; q < kChains; ++q) x[q] = fma(x[q], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < kChains; ++q) s += x[q];
  out[(size_t)blockIdx.x * kThreads + threadIdx.x] = s;
}

}  // namespace

extern "C" ns_status ns_fp64_fma_probe(double* out, int n_blocks, int n_iter, void* cuda_stream) {
  ns_set_thread_error("");
  if (!out || n_blocks < 1 || n_iter < 1) {
    ns_set_thread_error("ns_fp64_fma_probe: out must be non-NULL, n_blocks and n_iter positive");
    return NS_ERR_ARG;
  }
  // b slightly below 1 and c small keep every chain bounded (x tends to c / (1 - b))
  fp64_fma_probe_kernel<<<n_blocks, kThreads, 0, (cudaStream_t)cuda_stream>>>(out, n_iter, 1.0 - 1.0 / 1024.0,
                                                                             1e-6);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    ns_set_thread_error(cudaGetErrorString(e));
    return NS_ERR_CUDA;
  }
  return NS_OK;
}
