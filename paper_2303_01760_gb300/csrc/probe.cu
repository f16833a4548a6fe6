// Measurement and self-check entry points (no paper passage): the FP64 FMA
// throughput that bounds the weight solves, measured on the device the
// library runs on, and an elementwise evaluator of the hand-written math
// helpers of the weight and MLP kernels, so that they can be checked against
// IEEE results and their stated error bounds.
#include <algorithm>

#include "common.cuh"
#include "gelu.cuh"
#include "rbf_kernels.cuh"

namespace {

__device__ double g_fma_sink;

// CH independent FMA chains per thread, so that the FP64 pipe, not the
// dependency latency, bounds the issue rate.  The values stay bounded
// (|a| < 1) and are kept alive by a store that never happens at run time.
template <int CH>
__global__ void __launch_bounds__(256) k_fp64_fma(int iters, double a, double b) {
  double x[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) x[c] = 1e-3 * (threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < CH; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < CH; ++c) s += x[c];
  if (s == -1.0) g_fma_sink = s;
}

// The same with every operand in registers (a per-chain multiplier and a
// per-thread addend), as the FMAs of the weight and apply kernels have them.
template <int CH>
__global__ void __launch_bounds__(256) k_fp64_fma_reg(int iters, double a, double b) {
  double x[CH], m[CH];
  const double z = b * (1.0 + 1e-3 * threadIdx.x);
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    x[c] = 1e-3 * (threadIdx.x + c);
    m[c] = a - 1e-9 * c;
  }
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < CH; ++c) x[c] = fma(x[c], m[c], z);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < CH; ++c) s += x[c];
  if (s == -1.0) g_fma_sink = s;
}

__global__ void k_eval(int fn, const double* __restrict__ x, double* __restrict__ y, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = x[i];
    double r = 0.0;
    switch (fn) {
      case HSM_HELPER_RECIP: r = hsm::recip(v); break;
      case HSM_HELPER_SQRT_NR1: r = hsm::sqrt_nr1(v); break;
      case HSM_HELPER_SQRT_GS: r = hsm::sqrt_gs(v); break;
      case HSM_HELPER_ERF_AS: r = (double)erf_as((float)v); break;
      default: r = (double)gelu((float)v); break;
    }
    y[i] = r;
  }
}

hsm_status fail_cuda(cudaError_t e, const char* what) {
  hsm::set_global_error(std::string(what) + ": " + cudaGetErrorName(e));
  return HSM_ECUDA;
}

}  // namespace

extern "C" hsm_status hsm_probe_fp64_peak(double* gflops, float* ms, void* cuda_stream) {
  if (!gflops) {
    hsm::set_global_error("gflops is NULL");
    return HSM_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  // shapes: (chains per thread, blocks of 256 threads per SM)
  struct Shape {
    void (*fn)(int, double, double);
    int chains, bps;
  };
  const Shape shapes[] = {{k_fp64_fma<8>, 8, 8},      {k_fp64_fma<16>, 16, 4},     {k_fp64_fma<4>, 4, 8},
                          {k_fp64_fma<16>, 16, 8},    {k_fp64_fma_reg<8>, 8, 8},   {k_fp64_fma_reg<16>, 16, 4},
                          {k_fp64_fma_reg<4>, 4, 8},  {k_fp64_fma_reg<8>, 8, 4},   {k_fp64_fma_reg<32>, 32, 2}};
  const int threads = 256, iters = 4096;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  double best_rate = 0.0;
  float best_ms = 0.f;
  for (const Shape& sh : shapes) {
    const int blocks = hsm::num_sms() * sh.bps;
    const double flops = 2.0 * sh.chains * (double)iters * threads * blocks;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
      if ((e = cudaEventRecord(e0, s)) != cudaSuccess) break;
      sh.fn<<<blocks, threads, 0, s>>>(iters, 0.9999999, 1e-9);
      if ((e = cudaGetLastError()) != cudaSuccess) break;
      if ((e = cudaEventRecord(e1, s)) != cudaSuccess) break;
      if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
      float t = 0.f;
      if ((e = cudaEventElapsedTime(&t, e0, e1)) != cudaSuccess) break;
      const double rate = flops / (t * 1e-3) / 1e9;
      if (rep > 0 && rate > best_rate) {  // the first run of a shape warms up
        best_rate = rate;
        best_ms = t;
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return fail_cuda(e, "FP64 FMA probe");
  *gflops = best_rate;
  if (ms) *ms = best_ms;
  return HSM_OK;
}

extern "C" hsm_status hsm_eval_helper(int fn, const double* x, double* y, int64_t n, void* cuda_stream) {
  if (fn < HSM_HELPER_RECIP || fn > HSM_HELPER_GELU || n < 0 || (n > 0 && (!x || !y))) {
    hsm::set_global_error("hsm_eval_helper: unknown helper, negative n or NULL buffer");
    return HSM_EINVAL;
  }
  if (n == 0) return HSM_OK;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const int T = 256;
  const int grid = (int)std::min<int64_t>(hsm::ceil_div(n, T), (int64_t)hsm::num_sms() * 8);
  k_eval<<<grid, T, 0, s>>>(fn, x, y, n);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HSM_OK : fail_cuda(e, "hsm_eval_helper launch");
}
