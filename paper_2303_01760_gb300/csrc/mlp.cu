// Learned RBF-FD weights: an MLP from the normalised offsets of a scattered
// stencil to its scaled operator weights, trained on this library's own FP64
// weights, and an exact FP64 projection of its output onto the monomial
// reproduction constraints (Eq. 1 enforced for every monomial of degree <= m),
// with the direct FP64 solve as fallback.  The paper has no learned part; this
// is the specification's predictor.
//
// Layers: Linear(2n -> H) GELU, (Linear(H -> H) GELU) x (L-1), Linear(H -> 3n),
// GELU(x) = x Phi(x).  Every dense layer of training is a BF16 tcgen05 GEMM
// with FP32 accumulation in tensor memory (mlp_tc.cu), bias and activation
// fused into its epilogue; the GEMMs of the backward pass read transposed
// copies that the forward pass and the loss write beside their outputs, so
// both operands are always K-major.  Master weights and Adam moments are
// FP32.  Dimensions are padded so every GEMM is a whole number of
// 128 x 64 x 64 tiles: inputs to a multiple of 64, hidden widths and outputs
// to multiples of 128, the batch to 128; the padded inputs, outputs and
// weights stay zero.
#include <cmath>
#include <vector>

#include <cuda_bf16.h>

#include "mlp.cuh"

struct hsm_mlp_s {
  hsm::Mlp m;
};

namespace hsm {
namespace {

constexpr int BM = 128;  // rows of a GEMM tile: the batch is padded to a multiple

// ---- small kernels ----------------------------------------------------------
__device__ __forceinline__ uint64_t mix64(uint64_t x) {
  // splitmix64 finaliser (Steele, Lea and Flood, 2014)
  x += 0x9e3779b97f4a7c15ull;
  x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
  x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
  return x ^ (x >> 31);
}

// Gathers rows of the dataset into padded bf16 inputs and fp32 targets.
// Row r of the batch takes sample idx = mix64(seed, step, r) % count, or r
// itself when seed == 0 (in order; rows beyond count are zero).
// Xt (optional): the transposed inputs [din][ldt].
__global__ void k_pack(const float* __restrict__ X, const float* __restrict__ Y, int64_t count, int n_in, int n_out,
                       int din, int dout, int64_t rows, uint64_t seed, int64_t step, int64_t base,
                       __nv_bfloat16* Xb, float* T, __nv_bfloat16* Xt = nullptr, int64_t ldt = 0) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
    int64_t src = -1;
    if (seed) src = (int64_t)(mix64(seed ^ mix64((uint64_t)step * 0x100000001b3ull + (uint64_t)r)) % (uint64_t)count);
    else if (base + r < count) src = base + r;
    for (int j = 0; j < din; ++j) {
      const __nv_bfloat16 v = __float2bfloat16(src >= 0 && j < n_in ? X[src * n_in + j] : 0.f);
      Xb[r * din + j] = v;
      if (Xt) Xt[(int64_t)j * ldt + r] = v;
    }
    if (T)
      for (int j = 0; j < dout; ++j) T[r * dout + j] = (src >= 0 && j < n_out && Y) ? Y[src * n_out + j] : 0.f;
  }
}

// dY = 2 (Y - T) / (rows_valid * n_out) on valid entries, 0 elsewhere; loss sum.
__global__ void k_mse(const float* __restrict__ Yo, const float* __restrict__ T, int64_t rows, int64_t valid,
                      int n_out, int dout, __nv_bfloat16* dY, __nv_bfloat16* dYt, int64_t ldt, double* loss) {
  double part = 0.0;
  const float scale = 2.0f / (float)((double)valid * n_out);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows * dout; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / dout;
    const int j = (int)(i - r * dout);
    float g = 0.f;
    if (r < valid && j < n_out) {
      const float d = Yo[i] - T[i];
      g = scale * d;
      part += (double)d * d;
    }
    dY[i] = __float2bfloat16(g);
    dYt[(int64_t)j * ldt + r] = __float2bfloat16(g);
  }
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, part);
}

// db[n] = sum_r dZ[r][n]
__global__ void k_colsum(const __nv_bfloat16* __restrict__ dZ, int64_t rows, int N, float* db) {
  const int n = blockIdx.x;
  float s = 0.f;
  for (int64_t r = threadIdx.x; r < rows; r += blockDim.x) s += __bfloat162float(dZ[r * N + n]);
  __shared__ float sh[32];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) t += sh[w];
    db[n] = t;
  }
}

// Adam (Kingma and Ba, 2015) on every master parameter; refreshes the bf16
// copies of the weight matrices.  Padded entries have zero gradient and stay 0.
__global__ void k_adam(float* p, float* m, float* v, const float* g, size_t n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// dst[c][r] = bf16(src[r][c]) for an R x C row-major matrix
__global__ void k_to_bf16_t(const float* __restrict__ src, __nv_bfloat16* dst, int R, int C) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)R * C;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = i / R, r = i - c * R;
    dst[i] = __float2bfloat16(src[r * C + c]);
  }
}

__global__ void k_to_bf16(const float* __restrict__ src, __nv_bfloat16* dst, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = __float2bfloat16(src[i]);
}

int rup(int a, int b) { return (a + b - 1) / b * b; }

hsm_status mlp_fail(Mlp& m, hsm_status s, const std::string& msg) {
  m.last_error = msg;
  set_global_error(msg);
  return s;
}

#define MLP_CUDA(call)                                                                                        \
  do {                                                                                                        \
    cudaError_t e_ = (call);                                                                                  \
    if (e_ != cudaSuccess)                                                                                    \
      return mlp_fail(m, e_ == cudaErrorMemoryAllocation ? HSM_ENOMEM : HSM_ECUDA,                             \
                      std::string(#call) + ": " + cudaGetErrorString(e_));                                    \
  } while (0)

hsm_status ensure_cap(Mlp& m, int64_t rows) {
  if (rows <= m.cap) return HSM_OK;
  cudaStream_t s = m.stream;
  dev_free(&m.X, s);
  for (auto& h : m.H) dev_free(&h, s);
  for (auto& z : m.Z) dev_free(&z, s);
  dev_free(&m.Yout, s);
  dev_free(&m.T, s);
  dev_free(&m.dA, s);
  dev_free(&m.dB, s);
  dev_free(&m.Xt, s);
  for (auto& h : m.Ht) dev_free(&h, s);
  dev_free(&m.dAt, s);
  dev_free(&m.dBt, s);
  int wmax = 0;
  for (int l = 0; l < m.nl; ++l) wmax = std::max(wmax, std::max(m.din[l], m.dout[l]));
  MLP_CUDA(dev_alloc(&m.X, (size_t)rows * m.din[0], s));
  m.H.assign(m.nl - 1, nullptr);
  m.Z.assign(m.nl - 1, nullptr);
  for (int l = 0; l < m.nl - 1; ++l) {
    MLP_CUDA(dev_alloc(&m.H[l], (size_t)rows * m.dout[l], s));
    MLP_CUDA(dev_alloc(&m.Z[l], (size_t)rows * m.dout[l], s));
  }
  MLP_CUDA(dev_alloc(&m.Yout, (size_t)rows * m.dout[m.nl - 1], s));
  MLP_CUDA(dev_alloc(&m.T, (size_t)rows * m.dout[m.nl - 1], s));
  MLP_CUDA(dev_alloc(&m.dA, (size_t)rows * wmax, s));
  MLP_CUDA(dev_alloc(&m.dB, (size_t)rows * wmax, s));
  MLP_CUDA(dev_alloc(&m.Xt, (size_t)rows * m.din[0], s));
  m.Ht.assign(m.nl - 1, nullptr);
  for (int l = 0; l < m.nl - 1; ++l) MLP_CUDA(dev_alloc(&m.Ht[l], (size_t)rows * m.dout[l], s));
  MLP_CUDA(dev_alloc(&m.dAt, (size_t)rows * wmax, s));
  MLP_CUDA(dev_alloc(&m.dBt, (size_t)rows * wmax, s));
  m.cap = rows;
  return HSM_OK;
}

hsm_status refresh_bf16(Mlp& m) {
  for (int l = 0; l < m.nl; ++l) {
    const size_t n = (size_t)m.dout[l] * m.din[l];
    k_to_bf16<<<(int)std::min<size_t>(ceil_div(n, 256), 4096), 256, 0, m.stream>>>(m.master + m.w_off[l],
                                                                                    m.wbf + m.wbf_off[l], n);
    k_to_bf16_t<<<(int)std::min<size_t>(ceil_div(n, 256), 4096), 256, 0, m.stream>>>(
        m.master + m.w_off[l], m.wbft + m.wbf_off[l], m.dout[l], m.din[l]);
  }
  MLP_CUDA(cudaGetLastError());
  return HSM_OK;
}

#define MLP_TRY(call)                                                      \
  do {                                                                     \
    const hsm_status s_ = (call);                                          \
    if (s_ != HSM_OK) return mlp_fail(m, s_, "tensor-core GEMM launch failed"); \
  } while (0)

// Forward pass of ``rows`` packed rows (m.X and m.Xt filled); output in
// m.Yout, hidden activations in m.H and (transposed) m.Ht.
hsm_status forward(Mlp& m, int64_t rows) {
  const __nv_bfloat16* in = m.X;
  for (int l = 0; l < m.nl; ++l) {
    MlpGemm g{};
    g.A = in;
    g.lda = m.din[l];
    g.B = m.wbf + m.wbf_off[l];
    g.ldb = m.din[l];
    g.M = (int)rows;
    g.N = m.dout[l];
    g.K = m.din[l];
    g.bias = m.master + m.b_off[l];
    if (l < m.nl - 1) {
      g.epi = MLP_EPI_BIAS_GELU;
      g.Ch = m.H[l];
      g.Zout = m.Z[l];
      g.Cht = m.Ht[l];
      g.ldt = m.cap;
      MLP_TRY(mlp_gemm_tc(m, g));
      in = m.H[l];
    } else {
      g.epi = MLP_EPI_BIAS;
      g.Cf = m.Yout;
      MLP_TRY(mlp_gemm_tc(m, g));
    }
  }
  return HSM_OK;
}

// Backward pass after forward(); gradients (fp32, padded layout) into m.grad.
// dW_l = dZ_l^T H_{l-1} reads the transposed gradient and activations (both
// [width][rows], K = rows); dZ_{l-1} = (dZ_l W_l) GELU'(Z_{l-1}) reads the
// transposed weights.
hsm_status backward(Mlp& m, int64_t rows, int64_t valid) {
  cudaStream_t s = m.stream;
  const int L = m.nl;
  MLP_CUDA(cudaMemsetAsync(m.loss, 0, sizeof(double), s));
  k_mse<<<(int)std::min<int64_t>(ceil_div(rows * m.dout[L - 1], 256), 2048), 256, 0, s>>>(
      m.Yout, m.T, rows, valid, m.n_out, m.dout[L - 1], m.dA, m.dAt, m.cap, m.loss);
  MLP_CUDA(cudaGetLastError());
  __nv_bfloat16 *dZ = m.dA, *dZt = m.dAt, *dnext = m.dB, *dnextt = m.dBt;
  for (int l = L - 1; l >= 0; --l) {
    MlpGemm gw{};
    gw.A = dZt;
    gw.lda = m.cap;
    gw.B = l == 0 ? m.Xt : m.Ht[l - 1];
    gw.ldb = m.cap;
    gw.M = m.dout[l];
    gw.N = m.din[l];
    gw.K = (int)rows;
    gw.epi = MLP_EPI_F32;
    gw.Cf = m.grad + m.w_off[l];
    MLP_TRY(mlp_gemm_tc(m, gw));
    k_colsum<<<m.dout[l], 256, 0, s>>>(dZ, rows, m.dout[l], m.grad + m.b_off[l]);
    MLP_CUDA(cudaGetLastError());
    if (l > 0) {
      MlpGemm gx{};
      gx.A = dZ;
      gx.lda = m.dout[l];
      gx.B = m.wbft + m.wbf_off[l];
      gx.ldb = m.dout[l];
      gx.M = (int)rows;
      gx.N = m.din[l];
      gx.K = m.dout[l];
      gx.epi = MLP_EPI_DGELU;
      gx.Zin = m.Z[l - 1];
      gx.Ch = dnext;
      gx.Cht = dnextt;
      gx.ldt = m.cap;
      MLP_TRY(mlp_gemm_tc(m, gx));
      std::swap(dZ, dnext);
      std::swap(dZt, dnextt);
    }
  }
  return HSM_OK;
}

#undef MLP_TRY

}  // namespace
}  // namespace hsm

using namespace hsm;

extern "C" {

hsm_status hsm_mlp_create(hsm_mlp* out, int n_in, int hidden, int layers, int n_out, uint64_t seed, void* stream) {
  if (!out) return set_error(nullptr, HSM_EINVAL, "out is NULL");
  *out = nullptr;
  if (n_in < 1 || n_in > 256 || n_out < 1 || n_out > 512 || hidden < 1 || hidden > 2048 || layers < 1 || layers > 8)
    return set_error(nullptr, HSM_EINVAL, "MLP sizes out of range");
  hsm_mlp h = new (std::nothrow) hsm_mlp_s();
  if (!h) return set_error(nullptr, HSM_ENOMEM, "host allocation failed");
  Mlp& m = h->m;
  m.n_in = n_in;
  m.hidden = hidden;
  m.layers = layers;
  m.n_out = n_out;
  m.nl = layers + 1;
  m.stream = (cudaStream_t)stream;
  const int hp = rup(hidden, 128);
  for (int l = 0; l < m.nl; ++l) {
    m.rin.push_back(l == 0 ? n_in : hidden);
    m.rout.push_back(l == m.nl - 1 ? n_out : hidden);
    m.din.push_back(l == 0 ? rup(n_in, 64) : hp);
    m.dout.push_back(l == m.nl - 1 ? rup(n_out, 128) : hp);
  }
  size_t off = 0, offb = 0;
  for (int l = 0; l < m.nl; ++l) {
    m.w_off.push_back(off);
    off += (size_t)m.dout[l] * m.din[l];
    m.b_off.push_back(off);
    off += m.dout[l];
    m.wbf_off.push_back(offb);
    offb += (size_t)m.dout[l] * m.din[l];
  }
  m.n_master = off;
  m.n_wbf = offb;
  cudaStream_t s = m.stream;
  auto fail = [&](const char* what) {
    hsm_mlp_destroy(h);
    return set_error(nullptr, HSM_ENOMEM, what);
  };
  if (dev_alloc(&m.master, m.n_master, s) || dev_alloc(&m.adam_m, m.n_master, s) ||
      dev_alloc(&m.adam_v, m.n_master, s) || dev_alloc(&m.grad, m.n_master, s) || dev_alloc(&m.wbf, m.n_wbf, s) ||
      dev_alloc(&m.wbft, m.n_wbf, s) || dev_alloc(&m.loss, 1, s) || dev_alloc(&m.tc_err, 1, s) ||
      cudaMemsetAsync(m.tc_err, 0, sizeof(unsigned), s))
    return fail("MLP allocation failed");
  // initialisation: uniform +-sqrt(6/fan_in)/2 on the real entries (seeded, on the host), zero bias
  std::vector<float> host(m.n_master, 0.f);
  uint64_t st = seed ? seed : 0x853c49e6748fea9bull;
  auto next = [&]() {
    st += 0x9e3779b97f4a7c15ull;
    uint64_t z = st;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
  };
  for (int l = 0; l < m.nl; ++l) {
    const double lim = std::sqrt(6.0 / m.rin[l]) * 0.5;
    for (int o = 0; o < m.rout[l]; ++o)
      for (int i = 0; i < m.rin[l]; ++i) host[m.w_off[l] + (size_t)o * m.din[l] + i] = (float)((2.0 * next() - 1.0) * lim);
  }
  if (cudaMemcpyAsync(m.master, host.data(), m.n_master * sizeof(float), cudaMemcpyHostToDevice, s) ||
      cudaMemsetAsync(m.adam_m, 0, m.n_master * sizeof(float), s) ||
      cudaMemsetAsync(m.adam_v, 0, m.n_master * sizeof(float), s) || cudaStreamSynchronize(s))
    return fail("MLP initialisation failed");
  if (refresh_bf16(m) != HSM_OK) return fail("MLP initialisation failed");
  *out = h;
  return HSM_OK;
}

hsm_status hsm_mlp_destroy(hsm_mlp h) {
  if (!h) return HSM_OK;
  Mlp& m = h->m;
  cudaStream_t s = m.stream;
  dev_free(&m.master, s);
  dev_free(&m.adam_m, s);
  dev_free(&m.adam_v, s);
  dev_free(&m.grad, s);
  dev_free(&m.wbf, s);
  dev_free(&m.wbft, s);
  dev_free(&m.loss, s);
  dev_free(&m.X, s);
  dev_free(&m.Xt, s);
  for (auto& x : m.H) dev_free(&x, s);
  for (auto& x : m.Ht) dev_free(&x, s);
  dev_free(&m.dAt, s);
  dev_free(&m.dBt, s);
  for (auto& x : m.Z) dev_free(&x, s);
  dev_free(&m.Yout, s);
  dev_free(&m.T, s);
  dev_free(&m.dA, s);
  dev_free(&m.dB, s);
  dev_free(&m.Xf, s);
  dev_free(&m.tc_err, s);
  cudaStreamSynchronize(s);
  delete h;
  return HSM_OK;
}

hsm_status hsm_mlp_param_count(hsm_mlp h, int64_t* count) {
  if (!h || !count) return set_error(nullptr, HSM_EINVAL, "mlp and count are required");
  const Mlp& m = h->m;
  int64_t c = 0;
  for (int l = 0; l < m.nl; ++l) c += (int64_t)m.rout[l] * m.rin[l] + m.rout[l];
  *count = c;
  return HSM_OK;
}

// packed (unpadded) host layout: per layer W [out][in] then b [out]
static hsm_status pack_io(hsm_mlp h, float* host, const float* host_in, const float* dev_src, bool to_device) {
  Mlp& m = h->m;
  std::vector<float> pad(m.n_master, 0.f);
  if (!to_device) MLP_CUDA(cudaMemcpyAsync(pad.data(), dev_src, m.n_master * sizeof(float), cudaMemcpyDeviceToHost, m.stream));
  MLP_CUDA(cudaStreamSynchronize(m.stream));
  size_t k = 0;
  for (int l = 0; l < m.nl; ++l) {
    for (int o = 0; o < m.rout[l]; ++o)
      for (int i = 0; i < m.rin[l]; ++i) {
        float& p = pad[m.w_off[l] + (size_t)o * m.din[l] + i];
        if (to_device) p = host_in[k++];
        else host[k++] = p;
      }
    for (int o = 0; o < m.rout[l]; ++o) {
      float& p = pad[m.b_off[l] + o];
      if (to_device) p = host_in[k++];
      else host[k++] = p;
    }
  }
  if (to_device) {
    MLP_CUDA(cudaMemcpyAsync(m.master, pad.data(), m.n_master * sizeof(float), cudaMemcpyHostToDevice, m.stream));
    MLP_CUDA(cudaStreamSynchronize(m.stream));
    return refresh_bf16(m);
  }
  return HSM_OK;
}

hsm_status hsm_mlp_get_params(hsm_mlp h, float* host, int64_t count) {
  int64_t c = 0;
  if (!h || !host) return set_error(nullptr, HSM_EINVAL, "mlp and host buffer are required");
  hsm_mlp_param_count(h, &c);
  if (count != c) return set_error(nullptr, HSM_EINVAL, "count must equal hsm_mlp_param_count");
  return pack_io(h, host, nullptr, h->m.master, false);
}

hsm_status hsm_mlp_set_params(hsm_mlp h, const float* host, int64_t count) {
  int64_t c = 0;
  if (!h || !host) return set_error(nullptr, HSM_EINVAL, "mlp and host buffer are required");
  hsm_mlp_param_count(h, &c);
  if (count != c) return set_error(nullptr, HSM_EINVAL, "count must equal hsm_mlp_param_count");
  h->m.t = 0;
  Mlp& m = h->m;
  MLP_CUDA(cudaMemsetAsync(m.adam_m, 0, m.n_master * sizeof(float), m.stream));
  MLP_CUDA(cudaMemsetAsync(m.adam_v, 0, m.n_master * sizeof(float), m.stream));
  return pack_io(h, nullptr, host, nullptr, true);
}

hsm_status hsm_mlp_grad(hsm_mlp h, const float* X, const float* Y, int64_t count, float* grads_host, float* loss) {
  if (!h || !X || !Y || count < 1) return set_error(nullptr, HSM_EINVAL, "mlp, X, Y and count >= 1 are required");
  Mlp& m = h->m;
  const int64_t rows = ceil_div(count, BM) * BM;
  hsm_status st = ensure_cap(m, rows);
  if (st != HSM_OK) return st;
  MLP_CUDA(cudaMemsetAsync(m.tc_err, 0, sizeof(unsigned), m.stream));
  k_pack<<<(int)std::min<int64_t>(ceil_div(rows, 256), 4096), 256, 0, m.stream>>>(
      X, Y, count, m.n_in, m.n_out, m.din[0], m.dout[m.nl - 1], rows, 0, 0, 0, m.X, m.T, m.Xt, m.cap);
  MLP_CUDA(cudaGetLastError());
  MLP_CUDA(cudaMemsetAsync(m.grad, 0, m.n_master * sizeof(float), m.stream));
  if ((st = forward(m, rows)) != HSM_OK) return st;
  if ((st = backward(m, rows, count)) != HSM_OK) return st;
  double l = 0.0;
  unsigned err = 0;
  MLP_CUDA(cudaMemcpyAsync(&l, m.loss, sizeof(double), cudaMemcpyDeviceToHost, m.stream));
  MLP_CUDA(cudaMemcpyAsync(&err, m.tc_err, sizeof(unsigned), cudaMemcpyDeviceToHost, m.stream));
  if (grads_host) {
    st = pack_io(h, grads_host, nullptr, m.grad, false);
    if (st != HSM_OK) return st;
  }
  MLP_CUDA(cudaStreamSynchronize(m.stream));
  if (err) return mlp_fail(m, HSM_ETIMEOUT, "a tensor-core GEMM timed out");
  if (loss) *loss = (float)(l / ((double)count * m.n_out));
  return HSM_OK;
}

hsm_status hsm_mlp_train(hsm_mlp h, const float* X, const float* Y, int64_t count, int steps, int batch, float lr,
                         uint64_t seed, float* loss_log) {
  if (!h || !X || !Y || count < 1 || steps < 0 || batch < 1 || !(lr > 0.f))
    return set_error(nullptr, HSM_EINVAL, "invalid training arguments");
  Mlp& m = h->m;
  const int64_t rows = ceil_div(batch, BM) * BM;
  hsm_status st = ensure_cap(m, rows);
  if (st != HSM_OK) return st;
  double* log_dev = nullptr;
  if (loss_log) MLP_CUDA(dev_alloc(&log_dev, std::max(steps, 1), m.stream));
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  MLP_CUDA(cudaMemsetAsync(m.tc_err, 0, sizeof(unsigned), m.stream));
  for (int it = 0; it < steps; ++it) {
    k_pack<<<(int)std::min<int64_t>(ceil_div(rows, 256), 4096), 256, 0, m.stream>>>(
        X, Y, count, m.n_in, m.n_out, m.din[0], m.dout[m.nl - 1], rows, seed ? seed : 1, m.t, 0, m.X, m.T, m.Xt,
        m.cap);
    if ((st = forward(m, rows)) != HSM_OK) break;
    if ((st = backward(m, rows, rows)) != HSM_OK) break;
    if (log_dev) MLP_CUDA(cudaMemcpyAsync(log_dev + it, m.loss, sizeof(double), cudaMemcpyDeviceToDevice, m.stream));
    m.t += 1;
    const float c1 = 1.f - std::pow(b1, (float)m.t), c2 = 1.f - std::pow(b2, (float)m.t);
    k_adam<<<(int)std::min<size_t>(ceil_div(m.n_master, 256), 4096), 256, 0, m.stream>>>(
        m.master, m.adam_m, m.adam_v, m.grad, m.n_master, lr, b1, b2, eps, c1, c2);
    MLP_CUDA(cudaGetLastError());
    if ((st = refresh_bf16(m)) != HSM_OK) break;
  }
  if (st == HSM_OK && log_dev) {
    std::vector<double> l(steps);
    MLP_CUDA(cudaMemcpyAsync(l.data(), log_dev, steps * sizeof(double), cudaMemcpyDeviceToHost, m.stream));
    MLP_CUDA(cudaStreamSynchronize(m.stream));
    for (int i = 0; i < steps; ++i) loss_log[i] = (float)(l[i] / ((double)rows * m.n_out));
  }
  dev_free(&log_dev, m.stream);
  if (st == HSM_OK) {
    unsigned err = 0;
    MLP_CUDA(cudaMemcpyAsync(&err, m.tc_err, sizeof(unsigned), cudaMemcpyDeviceToHost, m.stream));
    MLP_CUDA(cudaStreamSynchronize(m.stream));
    if (err) return mlp_fail(m, HSM_ETIMEOUT, "a tensor-core GEMM timed out");
  }
  return st;
}

hsm_status hsm_mlp_inject_fault(hsm_mlp h, int fault) {
  if (!h) return set_error(nullptr, HSM_EINVAL, "mlp is NULL");
  if (fault != HSM_FAULT_NONE && fault != HSM_FAULT_HOLD_MLP_LOADS)
    return set_error(nullptr, HSM_EINVAL, "unknown fault");
  h->m.fault_hold_loads = fault == HSM_FAULT_HOLD_MLP_LOADS;
  return HSM_OK;
}

hsm_status hsm_mlp_predict(hsm_mlp h, const float* X, int64_t count, float* Y) {
  if (!h || !X || !Y || count < 0) return set_error(nullptr, HSM_EINVAL, "mlp, X and Y are required");
  Mlp& m = h->m;
  if (mlp_forward_tc_supported(m)) {
    // fused tcgen05 forward pass: only the packed inputs live in global memory
    const int64_t chunk = 1 << 20;
    const int64_t rows = std::min<int64_t>(ceil_div(std::max<int64_t>(count, 1), BM) * BM, chunk);
    if (rows > m.capf) {
      dev_free(&m.Xf, m.stream);
      MLP_CUDA(dev_alloc(&m.Xf, (size_t)rows * m.din[0], m.stream));
      m.capf = rows;
    }
    // the timeout flag of the fused pass: cleared per call, so an expired
    // wait in one call does not fail the next
    if (m.tc_err) MLP_CUDA(cudaMemsetAsync(m.tc_err, 0, sizeof(unsigned), m.stream));
    for (int64_t b = 0; b < count; b += chunk) {
      const int64_t cnt = std::min(chunk, count - b);
      const int64_t r = ceil_div(cnt, BM) * BM;
      k_pack<<<(int)std::min<int64_t>(ceil_div(r, 256), 4096), 256, 0, m.stream>>>(
          X + b * m.n_in, nullptr, cnt, m.n_in, m.n_out, m.din[0], m.dout[m.nl - 1], r, 0, 0, 0, m.Xf, nullptr);
      MLP_CUDA(cudaGetLastError());
      const hsm_status st = mlp_forward_tc(m, m.Xf, cnt, Y + b * m.n_out, m.n_out);
      if (st != HSM_OK) return mlp_fail(m, st, "fused tensor-core forward pass failed to launch");
    }
    unsigned err = 0;
    MLP_CUDA(cudaMemcpyAsync(&err, m.tc_err, sizeof(unsigned), cudaMemcpyDeviceToHost, m.stream));
    MLP_CUDA(cudaStreamSynchronize(m.stream));
    if (err) return mlp_fail(m, HSM_ETIMEOUT, "fused tensor-core forward pass timed out");
    return HSM_OK;
  }
  const int64_t chunk = 1 << 18;
  const int64_t rows = std::min<int64_t>(ceil_div(std::max<int64_t>(count, 1), BM) * BM, chunk);
  hsm_status st = ensure_cap(m, rows);
  if (st != HSM_OK) return st;
  for (int64_t b = 0; b < count; b += chunk) {
    const int64_t cnt = std::min(chunk, count - b);
    const int64_t r = ceil_div(cnt, BM) * BM;
    k_pack<<<(int)std::min<int64_t>(ceil_div(r, 256), 4096), 256, 0, m.stream>>>(
        X + b * m.n_in, nullptr, cnt, m.n_in, m.n_out, m.din[0], m.dout[m.nl - 1], r, 0, 0, 0, m.X, nullptr);
    MLP_CUDA(cudaGetLastError());
    if ((st = forward(m, r)) != HSM_OK) return st;
    MLP_CUDA(cudaMemcpy2DAsync(Y + b * m.n_out, m.n_out * sizeof(float), m.Yout, m.dout[m.nl - 1] * sizeof(float),
                               m.n_out * sizeof(float), cnt, cudaMemcpyDeviceToDevice, m.stream));
  }
  return HSM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Learned weights for a plan: features -> MLP -> FP64 projection -> fallback
// ---------------------------------------------------------------------------
namespace hsm {
namespace {

// Features of one 2D stencil: the scale s = max |x_i - x_c| and the canonical
// frame Q (entry 1 onto +x, reflection putting entry 2 in the upper half
// plane) in FP64, then the rotated scaled offsets in FP32 -- they feed a bf16
// network.  Training data and inference use this one routine, so a stencil
// gets bit-identical features on both paths.  Returns inv = 1/s, the frame
// as (q00, q01, reflection sign).
template <int NN>
__device__ __forceinline__ void features2d(const double* __restrict__ coords, int64_t N,
                                           const int32_t* __restrict__ idx, int64_t G, int64_t pos, float* x,
                                           double& inv, double& q00, double& q01, double& sg) {
  const int32_t c = idx[pos];
  const double cx = coords[c], cy = coords[N + c];
  double ox[NN], oy[NN], s2 = 0.0;
#pragma unroll
  for (int j = 0; j < NN; ++j) {
    const int32_t id = idx[(int64_t)j * G + pos];
    ox[j] = coords[id] - cx;
    oy[j] = coords[N + id] - cy;
    s2 = fmax(s2, ox[j] * ox[j] + oy[j] * oy[j]);
  }
  inv = 1.0 / sqrt(s2);
  const double r1 = sqrt(ox[1] * ox[1] + oy[1] * oy[1]);
  q00 = ox[1] / r1;
  q01 = oy[1] / r1;
  sg = (q00 * oy[2] - q01 * ox[2]) < 0.0 ? -1.0 : 1.0;  // second row of Q is sg * (-q01, q00)
  const float f00 = (float)q00, f01 = (float)q01, fs = (float)sg, fi = (float)inv;
#pragma unroll
  for (int j = 0; j < NN; ++j) {
    const float a = (float)ox[j] * fi, b = (float)oy[j] * fi;
    x[2 * j] = fmaf(f00, a, f01 * b);
    x[2 * j + 1] = fs * fmaf(f00, b, -f01 * a);
  }
}

// Features of RBF-FD stencil positions (scaled offsets, node-major) and, when
// Ylab is given, the scaled FP64 weights as labels ([op][node]).
template <int DIM>
__global__ void k_features(const double* __restrict__ coords, int64_t N, const int32_t* __restrict__ idx, int64_t G,
                           int n, const int32_t* __restrict__ list, int64_t count, const double* __restrict__ w,
                           const int* __restrict__ op_kind, int nops, float* X, float* Ylab) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pos = list[t];
    const int32_t c = idx[pos];
    double s2 = 0.0;
    for (int j = 0; j < n; ++j) {
      const int32_t id = idx[(int64_t)j * G + pos];
      double r2 = 0.0;
      for (int k = 0; k < DIM; ++k) {
        const double o = coords[k * N + id] - coords[k * N + c];
        r2 += o * o;
      }
      s2 = fmax(s2, r2);
    }
    const double s = sqrt(s2);
    double inv = 1.0 / s;
    // canonical frame (2D): entry 1 onto +x, entry 2 into the upper half plane
    double q00 = 1.0, q01 = 0.0, q10 = 0.0, q11 = 1.0;
    if (DIM == 2 && n == 12) {
      double sg;
      features2d<12>(coords, N, idx, G, pos, X + t * (n * DIM), inv, q00, q01, sg);
      q10 = -sg * q01;
      q11 = sg * q00;
    } else {
      for (int j = 0; j < n; ++j) {
        const int32_t id = idx[(int64_t)j * G + pos];
        for (int k = 0; k < DIM; ++k)
          X[t * (n * DIM) + j * DIM + k] = (float)((coords[k * N + id] - coords[k * N + c]) * inv);
      }
    }
    if (Ylab) {
      for (int o = 0; o < nops; ++o) {
        const double sc = op_kind[o] == 3 ? s * s : s;
        for (int j = 0; j < n; ++j) Ylab[t * (n * nops) + o * n + j] = (float)(w[((int64_t)o * n + j) * G + pos] * sc);
      }
      if (DIM == 2 && nops >= 2 && op_kind[0] == 0 && op_kind[1] == 1)
        for (int j = 0; j < n; ++j) {
          float* yx = &Ylab[t * (n * nops) + j];
          float* yy = &Ylab[t * (n * nops) + n + j];
          const double a = w[(int64_t)j * G + pos] * s, b = w[((int64_t)n + j) * G + pos] * s;
          *yx = (float)(q00 * a + q01 * b);
          *yy = (float)(q10 * a + q11 * b);
        }
    }
  }
}

// Scale and canonical frame of one stencil's features: x = 1/s, (y, z) the
// first row of the rotation, w the reflection sign.
struct StencilFrame {
  double x, y, z, w;
};

template <int NN>
__global__ void k_features_infer2d(const double* __restrict__ coords, int64_t N, const int32_t* __restrict__ idx,
                                   int64_t G, const int32_t* __restrict__ list, int64_t count, float* X,
                                   StencilFrame* frame) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x) {
    double inv, q00, q01, sg;
    features2d<NN>(coords, N, idx, G, list[t], X + t * (2 * NN), inv, q00, q01, sg);
    frame[t] = StencilFrame{inv, q00, q01, sg};
  }
}

// FP64 projection w = w_hat + P (P^T P)^{-1} (l_p - P^T w_hat) in the scaled
// variable, per stencil and operator; accepts when the pre-projection
// relative residual is <= tau and the post-projection residual <= 1e-10.
// One thread per stencil; P^T P is factored by Cholesky.  Weights are written
// for every stencil; rejected ones are listed for the FP64 re-solve, which
// overwrites them.
// Specialised to 2D, m = 2 (basis 1, x, y, x^2, xy, y^2 in graded
// lexicographic order) so that every loop has compile-time bounds.
template <int NN>
__global__ void __launch_bounds__(128) k_project2d(const double* __restrict__ coords, int64_t N,
                                                   const int32_t* __restrict__ idx, int64_t G,
                                                   const int32_t* __restrict__ list, int64_t count,
                                                   const float* __restrict__ Yp, const StencilFrame* __restrict__ frame,
                                                   double tau, double* w, int32_t* fail_list, int* fail_count,
                                                   uint8_t* status, uint8_t* acc) {
  constexpr int MP = 6;
  // L p at the centre: d/dx -> (0,1,0,0,0,0), d/dy -> (0,0,1,0,0,0),
  // Laplacian -> (0,0,0,2,0,2)
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pos = list[t];
    const int32_t c = idx[pos];
    // scale and frame of the features the prediction was made from
    const StencilFrame fr = frame[t];
    const double inv = fr.x, q00 = fr.y, q01 = fr.z, q10 = -fr.w * fr.z, q11 = fr.w * fr.y;
    double pj[NN][MP - 1];  // x, y, x^2, xy, y^2 of every node
    const double cx = coords[c], cy = coords[N + c];
#pragma unroll
    for (int j = 0; j < NN; ++j) {
      const int32_t id = idx[(int64_t)j * G + pos];
      const double x = (coords[id] - cx) * inv, y = (coords[N + id] - cy) * inv;
      pj[j][0] = x;
      pj[j][1] = y;
      pj[j][2] = x * x;
      pj[j][3] = x * y;
      pj[j][4] = y * y;
    }
    // G = P^T P (lower triangle), P row j = (1, x, y, x^2, xy, y^2)
    double Lc[MP][MP];
    Lc[0][0] = (double)NN;
#pragma unroll
    for (int a = 1; a < MP; ++a) {
      double sa = 0.0;
#pragma unroll
      for (int j = 0; j < NN; ++j) sa += pj[j][a - 1];
      Lc[a][0] = sa;
#pragma unroll
      for (int b = 1; b <= a; ++b) {
        double v = 0.0;
#pragma unroll
        for (int j = 0; j < NN; ++j) v = fma(pj[j][a - 1], pj[j][b - 1], v);
        Lc[a][b] = v;
      }
    }
    bool accept = true;
    double rdiag[MP];
#pragma unroll
    for (int a = 0; a < MP; ++a) {  // Cholesky, lower triangle in place
      double d = Lc[a][a];
#pragma unroll
      for (int k = 0; k < a; ++k) d -= Lc[a][k] * Lc[a][k];
      if (!(d > 0.0)) accept = false;
      d = sqrt(fmax(d, 1e-300));
      Lc[a][a] = d;
      rdiag[a] = 1.0 / d;
#pragma unroll
      for (int b = a + 1; b < MP; ++b) {
        double v = Lc[b][a];
#pragma unroll
        for (int k = 0; k < a; ++k) v -= Lc[b][k] * Lc[a][k];
        Lc[b][a] = v * rdiag[a];
      }
    }
    const float* yrow = Yp + t * ((int64_t)NN * 3);
#pragma unroll 1
    for (int o = 0; o < 3; ++o) {
      double wh[NN];
#pragma unroll
      for (int j = 0; j < NN; ++j) {
        if (o < 2) {
          // Q^T per node: (a, b) canonical -> physical component o
          const double a = (double)yrow[j], b = (double)yrow[NN + j];
          wh[j] = o == 0 ? fma(q00, a, q10 * b) : fma(q01, a, q11 * b);
        } else {
          wh[j] = (double)yrow[2 * NN + j];
        }
      }
      // r = l_p - P^T w_hat
      double y[MP] = {0.0, o == 0 ? 1.0 : 0.0, o == 1 ? 1.0 : 0.0, o == 2 ? 2.0 : 0.0, 0.0, o == 2 ? 2.0 : 0.0};
#pragma unroll
      for (int j = 0; j < NN; ++j) {
        y[0] -= wh[j];
#pragma unroll
        for (int q = 1; q < MP; ++q) y[q] = fma(-pj[j][q - 1], wh[j], y[q]);
      }
      double rn = 0.0;
#pragma unroll
      for (int q = 0; q < MP; ++q) rn = fma(y[q], y[q], rn);
      const double lpn = o == 2 ? 8.0 : 1.0;  // |l_p|^2
      if (!(rn <= tau * tau * lpn)) accept = false;
#pragma unroll
      for (int a = 0; a < MP; ++a) {  // L z = r
        double v = y[a];
#pragma unroll
        for (int k = 0; k < a; ++k) v -= Lc[a][k] * y[k];
        y[a] = v * rdiag[a];
      }
#pragma unroll
      for (int a = MP - 1; a >= 0; --a) {  // L^T c = z
        double v = y[a];
#pragma unroll
        for (int k = a + 1; k < MP; ++k) v -= Lc[k][a] * y[k];
        y[a] = v * rdiag[a];
      }
      // w = w_hat + P c, then the post-projection residual P^T w - l_p
      double res[MP] = {0.0, o == 0 ? -1.0 : 0.0, o == 1 ? -1.0 : 0.0, o == 2 ? -2.0 : 0.0, 0.0, o == 2 ? -2.0 : 0.0};
      const double sc = o == 2 ? inv * inv : inv;
#pragma unroll
      for (int j = 0; j < NN; ++j) {
        double v = wh[j] + y[0];
#pragma unroll
        for (int q = 1; q < MP; ++q) v = fma(pj[j][q - 1], y[q], v);
        res[0] += v;
#pragma unroll
        for (int q = 1; q < MP; ++q) res[q] = fma(pj[j][q - 1], v, res[q]);
        w[((int64_t)o * NN + j) * G + pos] = v * sc;
      }
#pragma unroll
      for (int q = 0; q < MP; ++q)
        if (!(fabs(res[q]) <= 1e-10)) accept = false;
    }
    if (accept) {
      if (status) status[c] = HSM_NODE_OK;
    } else {
      const int slot = atomicAdd(fail_count, 1);
      fail_list[slot] = (int32_t)pos;
    }
    if (acc) acc[t] = accept ? 1 : 0;
  }
}

// Batch validation (a check the paper does not have): S stencils spread evenly
// over the learned list; their learned weights are saved, then solved
// directly in place, then compared.
__global__ void k_gate_sample(const int32_t* __restrict__ learn, int64_t lc, int S, const uint8_t* __restrict__ acc,
                              int32_t* sample_pos, uint8_t* sample_acc) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < S; i += gridDim.x * blockDim.x) {
    const int64_t t = (int64_t)i * lc / S;
    sample_pos[i] = learn[t];
    sample_acc[i] = acc[t];
  }
}

// The validation samples: S learned stencils spread evenly over the list.
__global__ void k_gate_pick(const int32_t* __restrict__ learn, int64_t lc, int S, int32_t* sample_pos) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < S; i += gridDim.x * blockDim.x)
    sample_pos[i] = learn[(int64_t)i * lc / S];
}

// Puts the samples' saved weights back (inverse of k_gate_gather) and marks
// their nodes as directly solved.
__global__ void k_gate_scatter(double* __restrict__ w, int64_t G, int width, int nops,
                               const int32_t* __restrict__ sample_pos, int S, const double* __restrict__ saved,
                               const int32_t* __restrict__ nodes, uint8_t* status) {
  const int64_t total = (int64_t)S * width * nops;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / ((int64_t)width * nops));
    const int64_t r = e - (int64_t)i * width * nops;
    w[r * G + sample_pos[i]] = saved[e];
    if (status && r == 0) status[nodes[sample_pos[i]]] = HSM_NODE_LEARNED_SOLVE;
  }
}

__global__ void k_gate_gather(const double* __restrict__ w, int64_t G, int width, int nops,
                              const int32_t* __restrict__ sample_pos, int S, double* saved) {
  const int64_t total = (int64_t)S * width * nops;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / ((int64_t)width * nops));
    const int64_t r = e - (int64_t)i * width * nops;  // o * width + j
    saved[e] = w[r * G + sample_pos[i]];
  }
}

// Mean over the accepted samples of max|w_learned - w_direct| / max|w_direct|
// (over all operators and stencil nodes), summed in a fixed order.
constexpr int kGateThreads = 256;

// Per-stencil out-of-distribution gate of the learned weights: a prediction
// whose relative pre-projection residual |P^T w_hat - l_p| / |l_p| exceeds
// this is re-solved directly.  The projection makes every accepted stencil
// exact on the monomials whatever its residual, so this gate only rejects
// gross outliers (the zero prediction, residual 1, projects to the
// minimum-norm consistent stencil and passes); accuracy against the direct
// solve is the batch validation's job.  The oracle states the same value.
constexpr double kTauOod = 1.5;
__global__ void __launch_bounds__(kGateThreads) k_gate_error(const double* __restrict__ w, int64_t G, int width,
                                                             int nops, const int32_t* __restrict__ sample_pos,
                                                             const uint8_t* __restrict__ sample_acc, int S,
                                                             const double* __restrict__ saved, double* out) {
  __shared__ double se[kGateThreads];
  __shared__ int sn[kGateThreads];
  double acc_e = 0.0;
  int acc_n = 0;
  for (int i = threadIdx.x; i < S; i += kGateThreads) {
    if (!sample_acc[i]) continue;
    double dmax = 0.0, wmax = 0.0;
    for (int r = 0; r < width * nops; ++r) {
      const double wd = w[(int64_t)r * G + sample_pos[i]];
      dmax = fmax(dmax, fabs(saved[(int64_t)i * width * nops + r] - wd));
      wmax = fmax(wmax, fabs(wd));
    }
    acc_e += wmax > 0.0 ? dmax / wmax : 0.0;
    ++acc_n;
  }
  se[threadIdx.x] = acc_e;
  sn[threadIdx.x] = acc_n;
  __syncthreads();
  for (int h = kGateThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      se[threadIdx.x] += se[threadIdx.x + h];
      sn[threadIdx.x] += sn[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = sn[0] > 0 ? se[0] / sn[0] : 0.0;
    out[1] = (double)sn[0];
  }
}

__global__ void k_mark_zero(const int32_t* __restrict__ list, int k, uint8_t* flag) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) flag[list[i]] = 0;
}

__global__ void k_boundary_key(const int32_t* __restrict__ nodes, const uint8_t* __restrict__ is_boundary, int64_t G,
                               uint8_t* key) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < G; p += (int64_t)gridDim.x * blockDim.x)
    key[p] = is_boundary && is_boundary[nodes[p]] ? 1 : 0;
}

// Positions of the RBF-FD group split into interior stencils (learned) and
// boundary ones (direct solve), both in ascending order, with their counts
// on the device.
cudaError_t learned_split(hsm_plan p, int32_t* learn_list, int* learn_count, int32_t* other_list, int* other_count,
                          cudaStream_t s) {
  const int64_t G = p->rbf.count;
  uint8_t* key = nullptr;
  int32_t* pos = nullptr;
  cudaError_t e = dev_alloc(&key, G, s);
  if (e == cudaSuccess) e = dev_alloc(&pos, G, s);
  if (e == cudaSuccess) {
    k_boundary_key<<<(int)std::min<int64_t>(ceil_div(G, 256), (int64_t)num_sms() * 8), 256, 0, s>>>(
        p->rbf.nodes, p->is_boundary, G, key);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = partition_indices(key, 0, G, learn_list, other_list, pos, learn_count, other_count, s, nullptr);
  dev_free(&key, s);
  dev_free(&pos, s);
  return e;
}

}  // namespace

hsm_status compute_rbf_weights_learned(hsm_plan p, uint8_t* status, int32_t* fail_list, int* fail_count,
                                       int64_t* gate_extra) {
  *gate_extra = 0;
  p->gate_error = -1.0;
  p->gate_failed = 0;
  p->gate_accepted = 0;
  Mlp& m = p->mlp->m;
  const int dim = p->dim, n = p->n;
  if (m.n_in != n * dim || m.n_out != n * p->nops)
    return set_error(p, HSM_EINVAL, "the attached predictor's sizes do not match the plan (2n inputs, nops*n outputs)");
  cudaStream_t s = p->stream;
  const int64_t G = p->rbf.count;
  if (G == 0) return HSM_OK;
  int32_t* learn = nullptr;
  int* lcount = nullptr;
  float *X = nullptr, *Y = nullptr;
  StencilFrame* frame = nullptr;
  int* kinds = nullptr;
  uint8_t* acc = nullptr;
  HSM_CUDA(p, dev_alloc(&learn, G, s));
  HSM_CUDA(p, dev_alloc(&lcount, 1, s));
  HSM_CUDA(p, cudaMemsetAsync(lcount, 0, sizeof(int), s));
  const int T = 256;
  const int grid = (int)std::min<int64_t>(ceil_div(G, T), (int64_t)num_sms() * 8);
  HSM_CUDA(p, learned_split(p, learn, lcount, fail_list, fail_count, s));
  int lc = 0;
  HSM_CUDA(p, cudaMemcpyAsync(&lc, lcount, sizeof(int), cudaMemcpyDeviceToHost, s));
  HSM_CUDA(p, cudaStreamSynchronize(s));
  if (lc > 0) {
    int kh[4] = {0, 0, 0, 0};
    int o = 0;
    for (int b = 0; b < 4; ++b)
      if (p->op_mask & (1u << b)) kh[o++] = b;
    HSM_CUDA(p, dev_alloc(&kinds, 4, s));
    HSM_CUDA(p, cudaMemcpyAsync(kinds, kh, sizeof(kh), cudaMemcpyHostToDevice, s));
    if (!(dim == 2 && n == 12 && p->n_mono == 6 && p->op_mask == (HSM_DX | HSM_DY | HSM_LAP)))
      return set_error(p, HSM_EINVAL, "learned weights support 2D m = 2, n = 12 plans with ops dx, dy, lap");
    const int width = n, nops = p->nops;
    // feature, output, frame and acceptance buffers for `rows` stencils
    // (first the validation samples alone, the whole batch only if it passes)
    int64_t cap = 0;
    auto reserve = [&](int64_t rows) -> hsm_status {
      if (rows <= cap) return HSM_OK;
      dev_free(&X, s);
      dev_free(&Y, s);
      dev_free(&frame, s);
      dev_free(&acc, s);
      HSM_CUDA(p, dev_alloc(&X, (size_t)rows * n * dim, s));
      HSM_CUDA(p, dev_alloc(&Y, (size_t)rows * n * nops, s));
      HSM_CUDA(p, dev_alloc(&frame, rows, s));
      HSM_CUDA(p, dev_alloc(&acc, rows, s));
      cap = rows;
      return HSM_OK;
    };
    // features, MLP and projection of the stencils in `list` (count of them)
    auto infer = [&](const int32_t* list, int64_t count, int32_t* flist, int* fcount, uint8_t* accs) -> hsm_status {
      const int gl = (int)std::min<int64_t>(ceil_div(count, T), (int64_t)num_sms() * 8);
      k_features_infer2d<12><<<gl, T, 0, s>>>(p->coords, p->N, p->rbf.idx, G, list, count, X, frame);
      HSM_CUDA(p, cudaGetLastError());
      cudaStream_t old = m.stream;
      m.stream = s;
      hsm_status st = hsm_mlp_predict(p->mlp, X, count, Y);
      m.stream = old;
      if (st != HSM_OK) return set_error(p, st, m.last_error);
      const int gp = (int)std::min<int64_t>(ceil_div(count, 128), (int64_t)num_sms() * 16);
      k_project2d<12><<<gp, 128, 0, s>>>(p->coords, p->N, p->rbf.idx, G, list, count, Y, frame, kTauOod,
                                         p->rbf.w64, flist, fcount, status, accs);
      HSM_CUDA(p, cudaGetLastError());
      p->launches += 4;
      return HSM_OK;
    };
    if (p->gate_samples > 0) {
      // Batch validation first, on S samples alone: their learned weights
      // against their direct solve.  A batch that fails it takes the direct
      // solve without the full inference; one that passes runs the full
      // inference and keeps the samples' direct weights.
      const int S = (int)std::min<int64_t>(lc, p->gate_samples);
      int32_t *spos = nullptr, *sfail = nullptr;
      int* sfc = nullptr;
      double *saved = nullptr, *gerr = nullptr;
      HSM_CUDA(p, dev_alloc(&spos, S, s));
      HSM_CUDA(p, dev_alloc(&sfail, S, s));
      HSM_CUDA(p, dev_alloc(&sfc, 1, s));
      HSM_CUDA(p, dev_alloc(&saved, (size_t)S * width * nops, s));
      HSM_CUDA(p, dev_alloc(&gerr, 2, s));
      HSM_CUDA(p, cudaMemsetAsync(sfc, 0, sizeof(int), s));
      k_gate_pick<<<(S + 255) / 256, 256, 0, s>>>(learn, lc, S, spos);
      HSM_CUDA(p, cudaGetLastError());
      hsm_status st = reserve(S);
      if (st != HSM_OK) return st;
      st = infer(spos, S, sfail, sfc, acc);
      if (st != HSM_OK) return st;
      const int gg = (int)std::min<int64_t>(ceil_div((int64_t)S * width * nops, 256), 1024);
      k_gate_gather<<<gg, 256, 0, s>>>(p->rbf.w64, G, width, nops, spos, S, saved);
      HSM_CUDA(p, cudaGetLastError());
      // the samples' direct solve, in place (their status: learned -> solve)
      st = compute_rbf_weights_fp64_marked(p, spos, S, status, HSM_NODE_LEARNED_SOLVE);
      if (st != HSM_OK) return st;
      k_gate_error<<<1, kGateThreads, 0, s>>>(p->rbf.w64, G, width, nops, spos, acc, S, saved, gerr);
      HSM_CUDA(p, cudaGetLastError());
      double gh[2] = {0.0, 0.0};
      HSM_CUDA(p, cudaMemcpyAsync(gh, gerr, sizeof(gh), cudaMemcpyDeviceToHost, s));
      HSM_CUDA(p, cudaStreamSynchronize(s));
      p->gate_error = gh[0];
      p->gate_failed = gh[0] > p->gate_tol ? 1 : 0;
      *gate_extra = (int64_t)gh[1];
      p->gate_accepted = (int64_t)gh[1];
      p->launches += 4;
      if (!p->gate_failed) {
        k_gate_gather<<<gg, 256, 0, s>>>(p->rbf.w64, G, width, nops, spos, S, saved);  // direct weights
        HSM_CUDA(p, cudaGetLastError());
        st = reserve(lc);
        if (st != HSM_OK) return st;
        st = infer(learn, lc, fail_list, fail_count, acc);
        if (st != HSM_OK) return st;
        k_gate_scatter<<<gg, 256, 0, s>>>(p->rbf.w64, G, width, nops, spos, S, saved, p->rbf.nodes, status);
        HSM_CUDA(p, cudaGetLastError());
        p->launches += 2;
      }
      dev_free(&spos, s);
      dev_free(&sfail, s);
      dev_free(&sfc, s);
      dev_free(&saved, s);
      dev_free(&gerr, s);
    } else {
      hsm_status st = reserve(lc);
      if (st != HSM_OK) return st;
      st = infer(learn, lc, fail_list, fail_count, acc);
      if (st != HSM_OK) return st;
    }
  }
  dev_free(&learn, s);
  dev_free(&lcount, s);
  dev_free(&X, s);
  dev_free(&Y, s);
  dev_free(&frame, s);
  dev_free(&kinds, s);
  dev_free(&acc, s);
  return HSM_OK;
}

}  // namespace hsm

extern "C" {

hsm_status hsm_mlp_attach(hsm_plan p, hsm_mlp h) {
  if (!p) return set_error(nullptr, HSM_EINVAL, "plan is NULL");
  p->mlp = h;
  return HSM_OK;
}

// Features and labels of the plan's interior RBF-FD stencils (training data).
hsm_status hsm_plan_learned_data(hsm_plan p, float* X, float* Y, int64_t* count) {
  if (!p || !count) return set_error(p, HSM_EINVAL, "plan and count are required");
  if (!p->stencils_built) return set_error(p, HSM_ESTATE, "hsm_plan_build_stencils must come first");
  cudaStream_t s = p->stream;
  const int64_t G = p->rbf.count;
  int32_t *learn = nullptr, *skip = nullptr;
  int* cnt = nullptr;
  HSM_CUDA(p, dev_alloc(&learn, G, s));
  HSM_CUDA(p, dev_alloc(&skip, G, s));
  HSM_CUDA(p, dev_alloc(&cnt, 2, s));
  HSM_CUDA(p, cudaMemsetAsync(cnt, 0, 2 * sizeof(int), s));
  if (G) {
    HSM_CUDA(p, learned_split(p, learn, cnt, skip, cnt + 1, s));
  }
  int lc[2] = {0, 0};
  HSM_CUDA(p, cudaMemcpyAsync(lc, cnt, sizeof(lc), cudaMemcpyDeviceToHost, s));
  HSM_CUDA(p, cudaStreamSynchronize(s));
  *count = lc[0];
  if (X && lc[0] > 0) {
    if (Y && !p->weights_built) return set_error(p, HSM_ESTATE, "labels need computed weights");
    int kh[4] = {0, 0, 0, 0};
    int o = 0;
    for (int b = 0; b < 4; ++b)
      if (p->op_mask & (1u << b)) kh[o++] = b;
    int* kinds = nullptr;
    HSM_CUDA(p, dev_alloc(&kinds, 4, s));
    HSM_CUDA(p, cudaMemcpyAsync(kinds, kh, sizeof(kh), cudaMemcpyHostToDevice, s));
    // ascending positions keep the data order deterministic
    int32_t* sorted = nullptr;
    uint8_t* flag = nullptr;
    HSM_CUDA(p, dev_alloc(&sorted, G, s));
    HSM_CUDA(p, dev_alloc(&flag, G, s));
    HSM_CUDA(p, cudaMemsetAsync(flag, 1, G, s));
    // mark boundary positions (listed in skip) with 0, then select the rest in order
    if (lc[1] > 0) k_mark_zero<<<(int)std::min<int64_t>(ceil_div(lc[1], 256), 1024), 256, 0, s>>>(skip, lc[1], flag);
    HSM_CUDA(p, select_indices(flag, 1, G, sorted, nullptr, cnt, s));
    const int gl = (int)std::min<int64_t>(ceil_div(lc[0], 256), (int64_t)num_sms() * 8);
    if (p->dim == 2)
      k_features<2><<<gl, 256, 0, s>>>(p->coords, p->N, p->rbf.idx, G, p->n, sorted, lc[0], p->rbf.w64, kinds,
                                         p->nops, X, Y);
    else
      k_features<3><<<gl, 256, 0, s>>>(p->coords, p->N, p->rbf.idx, G, p->n, sorted, lc[0], p->rbf.w64, kinds,
                                         p->nops, X, Y);
    HSM_CUDA(p, cudaGetLastError());
    dev_free(&sorted, s);
    dev_free(&flag, s);
    dev_free(&kinds, s);
  }
  dev_free(&learn, s);
  dev_free(&skip, s);
  dev_free(&cnt, s);
  HSM_CUDA(p, cudaStreamSynchronize(s));
  return HSM_OK;
}

}  // extern "C"
