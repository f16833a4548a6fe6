// Allocation-free entry point: RBF-FD weights (FP32 factorisation with FP64
// refinement, FP64 re-solve of the systems that do not converge) for
// stencils the caller already has, for callers that must not allocate device
// memory while they run -- for example a solver embedded in an application
// that hands all device memory to its own pool at start-up, or a real-time
// loop in which an allocation could stall or fail.  The caller passes inputs
// and outputs; the few scratch words this path needs (the list of systems
// that need the FP64 re-solve, its counter, a status word and the monomial and
// pair tables) live in one file-scope device array of fixed size below, so
// nothing is allocated.  The paper has no counterpart to this entry point.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace {

constexpr size_t kCtlBytes = 256;                                  // fail counter, status word
constexpr size_t kFailBytes = (size_t)HSM_NOALLOC_MAX_SYSTEMS * 4;  // int32 fail list
constexpr size_t kPairsBytes = ((size_t)hsm::kMaxStencil * (hsm::kMaxStencil - 1) / 2 * 2 + 255) / 256 * 256;
constexpr size_t kExpBytes = 256;
constexpr size_t kScratchBytes = kCtlBytes + kFailBytes + kPairsBytes + kExpBytes;

// Shared by every call on a device and kept until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once
// per device, with that device current).
cudaError_t scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

hsm_status fail_cuda(cudaError_t e, const char* what) {
  hsm::set_global_error(std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
  return HSM_ECUDA;
}

hsm_status fail(hsm_status s, const char* msg) {
  hsm::set_global_error(msg);
  return s;
}

int64_t binom(int a, int b) {
  int64_t r = 1;
  for (int i = 1; i <= b; ++i) r = r * (a - b + i) / i;
  return r;
}

// Sets kDevBounds in *flags when any of the `total` stencil entries lies
// outside [0, N).  Runs before the weight kernels, which gather coordinates
// and write node_status through these ids without checking them.
__global__ void k_check_ids(const int32_t* __restrict__ ids, int64_t total, int64_t N, unsigned* flags) {
  bool bad = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
    bad |= (uint64_t)(int64_t)__ldg(ids + i) >= (uint64_t)N;
  if (bad) atomicOr(flags, hsm::kDevBounds);
}

}  // namespace

extern "C" hsm_status hsm_rbf_weights_fp32r_noalloc(int dim, int aug_m, int stencil_n, unsigned op_mask,
                                                    const double* coords, int64_t n_nodes,
                                                    const int32_t* stencils, int64_t count, double* weights,
                                                    uint8_t* node_status, void* cuda_stream) {
  if (dim != 2 && dim != 3) return fail(HSM_EINVAL, "dim must be 2 or 3");
  if (aug_m < 1 || aug_m > 6) return fail(HSM_EINVAL, "aug_m must be in 1..6");
  if (op_mask == 0 || (op_mask & ~15u)) return fail(HSM_EINVAL, "op_mask must be a non-empty set of hsm_op");
  if (dim == 2 && (op_mask & HSM_DZ)) return fail(HSM_EINVAL, "HSM_DZ needs dim 3");
  const int n_mono = (int)binom(aug_m + dim, aug_m);
  if (stencil_n <= n_mono || stencil_n > hsm::kMaxStencil)
    return fail(HSM_EINVAL, "stencil_n must satisfy C(m+d,m) < n <= 128");
  if (n_nodes < 1 || n_nodes >= ((int64_t)1 << 31)) return fail(HSM_EINVAL, "n_nodes out of range");
  if (count < 0) return fail(HSM_EINVAL, "count must be >= 0");
  if (count > HSM_NOALLOC_MAX_SYSTEMS)
    return fail(HSM_EINVAL, "count exceeds HSM_NOALLOC_MAX_SYSTEMS (the fixed scratch of the allocation-free path)");
  if (!coords || !stencils || !weights) return fail(HSM_EINVAL, "coords, stencils and weights are required");
  if (count == 0) return HSM_OK;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  int nops = 0;
  for (int b = 0; b < 4; ++b) nops += (op_mask >> b) & 1;

  unsigned char* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) return fail_cuda(e, "cudaGetSymbolAddress");

  // both kernels must have a launch shape for these sizes: a system that the
  // FP32 pass cannot refine is re-solved by the FP64 kernel, whose shared
  // memory per system is larger for some (dim, m, n)
  {
    hsm::RbfExternal probe;
    probe.dim = dim;
    probe.n = stencil_n;
    probe.n_mono = n_mono;
    probe.nops = nops;
    for (bool r32 : {true, false}) {
      bool fits = false;
      if ((e = hsm::rbf_external_fits(probe, r32, &fits)) != cudaSuccess) return fail_cuda(e, "kernel shape");
      if (!fits)
        return fail(HSM_EINVAL, r32 ? "RBF-FD system too large for shared memory (FP32 refinement kernel)"
                                    : "RBF-FD system too large for shared memory (FP64 re-solve kernel)");
    }
  }
  int* fail_count = reinterpret_cast<int*>(base);
  unsigned* flags = reinterpret_cast<unsigned*>(base + 4);
  int32_t* fail_list = reinterpret_cast<int32_t*>(base + kCtlBytes);
  uint16_t* pairs = reinterpret_cast<uint16_t*>(base + kCtlBytes + kFailBytes);
  int8_t* exps = reinterpret_cast<int8_t*>(base + kCtlBytes + kFailBytes + kPairsBytes);

  // tables of this (dim, m, n); pageable sources are staged before the copy
  // call returns, so the host vectors may go out of scope afterwards
  std::vector<uint16_t> hp;
  for (int i = 0; i < stencil_n; ++i)
    for (int j = i + 1; j < stencil_n; ++j) hp.push_back((uint16_t)((i << 8) | j));
  std::vector<int8_t> he;
  for (int q = 0; q <= aug_m; ++q) {
    if (dim == 2) {
      for (int a = q; a >= 0; --a) {
        he.push_back((int8_t)a);
        he.push_back((int8_t)(q - a));
      }
    } else {
      for (int a = q; a >= 0; --a)
        for (int b = q - a; b >= 0; --b) {
          he.push_back((int8_t)a);
          he.push_back((int8_t)b);
          he.push_back((int8_t)(q - a - b));
        }
    }
  }
  if ((e = cudaMemcpyAsync(pairs, hp.data(), hp.size() * sizeof(uint16_t), cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return fail_cuda(e, "cudaMemcpyAsync(pairs)");
  if ((e = cudaMemcpyAsync(exps, he.data(), he.size(), cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return fail_cuda(e, "cudaMemcpyAsync(exponents)");
  // the scratch keeps the previous call's contents: clear what must start at zero
  if ((e = cudaMemsetAsync(base, 0, 8, s)) != cudaSuccess) return fail_cuda(e, "cudaMemsetAsync(scratch)");

  // every stencil id (centres included) must lie in [0, n_nodes) before any
  // kernel gathers through it; nothing is written to the outputs otherwise
  {
    const int64_t total = (int64_t)stencil_n * count;
    const int T = 256;
    const int grid = (int)std::min<int64_t>(hsm::ceil_div(total, T), (int64_t)hsm::num_sms() * 8);
    k_check_ids<<<grid, T, 0, s>>>(stencils, total, n_nodes, flags);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail_cuda(e, "stencil id check launch");
    unsigned fl0 = 0;
    if ((e = cudaMemcpyAsync(&fl0, flags, sizeof(unsigned), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
      return fail_cuda(e, "cudaMemcpyAsync(flags)");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail_cuda(e, "cudaStreamSynchronize");
    if (fl0 & hsm::kDevBounds) return fail(HSM_EBOUNDS, "a stencil id lies outside [0, n_nodes)");
  }
  if (node_status && (e = cudaMemsetAsync(node_status, HSM_NODE_OK, (size_t)n_nodes, s)) != cudaSuccess)
    return fail_cuda(e, "cudaMemsetAsync(node_status)");

  hsm::RbfExternal x;
  x.dim = dim;
  x.coords = coords;
  x.N = n_nodes;
  x.idx = stencils;
  x.G = count;
  x.n = stencil_n;
  x.n_mono = n_mono;
  x.op_mask = op_mask;
  x.nops = nops;
  x.mono_exp = exps;
  x.pairs = pairs;
  x.w = weights;
  x.flags = flags;
  x.fail_list = fail_list;
  x.fail_count = fail_count;
  x.stream = s;
  bool too_big = false;
  e = hsm::launch_rbf_external(x, true, nullptr, count, nullptr, 0, &too_big);
  if (e != cudaSuccess) return fail_cuda(e, "FP32 refinement launch");
  if (too_big) return fail(HSM_EINVAL, "RBF-FD system too large for shared memory");
  int fc = 0;
  if ((e = cudaMemcpyAsync(&fc, fail_count, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return fail_cuda(e, "cudaMemcpyAsync(fail count)");
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail_cuda(e, "cudaStreamSynchronize");
  if (fc > 0) {
    e = hsm::launch_rbf_external(x, false, fail_list, fc, node_status, HSM_NODE_REFINE_FP64, &too_big);
    if (e != cudaSuccess) return fail_cuda(e, "FP64 re-solve launch");
    // cannot happen after the shape check above; never return weights the
    // re-solve did not write as if they were valid
    if (too_big) return fail(HSM_EINVAL, "FP64 RBF-FD system too large for shared memory");
  }
  unsigned fl = 0;
  if ((e = cudaMemcpyAsync(&fl, flags, sizeof(unsigned), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return fail_cuda(e, "cudaMemcpyAsync(flags)");
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail_cuda(e, "cudaStreamSynchronize");
  if (fl & hsm::kDevSingular) return fail(HSM_ESINGULAR, "some stencils have singular weight systems");
  return HSM_OK;
}
