// Learned weight predictor: the MLP state shared by mlp.cu (training,
// projection) and mlp_tc.cu (the tcgen05 training GEMMs and the fused
// tcgen05 forward pass).
#pragma once
#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "common.cuh"

namespace hsm {

struct Mlp {
  int n_in = 24, hidden = 256, layers = 3, n_out = 36;
  int nl = 4;                 // linear layers
  std::vector<int> din, dout;  // padded in/out width per layer
  std::vector<int> rin, rout;  // real widths
  float* master = nullptr;    // fp32 [sum W + b] padded layout
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  float* grad = nullptr;
  __nv_bfloat16* wbf = nullptr;  // bf16 copies of the weight matrices
  std::vector<size_t> w_off, b_off, wbf_off;
  size_t n_master = 0, n_wbf = 0;
  int64_t t = 0;               // Adam step counter
  int fault_hold_loads = 0;    // test hook: the next fused forward pass issues no loads
  cudaStream_t stream = nullptr;
  // activation workspace for a batch of up to cap rows
  int64_t cap = 0;
  __nv_bfloat16* X = nullptr;     // [cap][din0]
  std::vector<__nv_bfloat16*> H;  // per hidden layer [cap][dout]
  std::vector<float*> Z;          // pre-activations [cap][dout]
  float* Yout = nullptr;          // [cap][dout_last]
  float* T = nullptr;             // targets [cap][dout_last]
  __nv_bfloat16* dA = nullptr;    // [cap][max width]
  __nv_bfloat16* dB = nullptr;
  // transposed copies, [width][cap], so every training GEMM reads both
  // operands K-major: the inputs, the hidden activations, the gradients and
  // the bf16 weights ([din][dout] per layer, at wbf_off)
  __nv_bfloat16* Xt = nullptr;
  std::vector<__nv_bfloat16*> Ht;
  __nv_bfloat16* dAt = nullptr;
  __nv_bfloat16* dBt = nullptr;
  __nv_bfloat16* wbft = nullptr;
  double* loss = nullptr;         // device loss accumulator
  std::string last_error;
  // fused tcgen05 forward pass (mlp_tc.cu): packed inputs and error flag
  __nv_bfloat16* Xf = nullptr;    // [capf][din0]
  int64_t capf = 0;
  unsigned* tc_err = nullptr;
};

// Fused forward pass of every layer on the 5th-generation tensor cores
// (mlp_tc.cu).  X: bf16 [rows][din0] (padded inputs); writes Y[r * ldy + c]
// for c < n_out.  Returns false (and enqueues nothing) when the network's
// shape is not one the kernel handles.
bool mlp_forward_tc_supported(const Mlp& m);

// One training GEMM on the tensor cores (mlp_tc.cu): C[M x N] = A B^T with
// A bf16 [M][K] (row stride lda) and B bf16 [N][K] (row stride ldb), both
// K-major, M % 128 == K % 64 == N % 64 == 0; FP32 accumulation, then:
enum { MLP_EPI_BIAS_GELU = 0,  // Zout = C + bias, Ch = GELU(Zout) (and Cht = its transpose)
       MLP_EPI_BIAS = 1,       // Cf = C + bias
       MLP_EPI_DGELU = 2,      // Ch = C * GELU'(Zin) (and Cht = its transpose)
       MLP_EPI_F32 = 3 };      // Cf = C
struct MlpGemm {
  const __nv_bfloat16* A;
  const __nv_bfloat16* B;
  int64_t lda, ldb;
  int M, N, K, epi;
  const float* bias;
  const float* Zin;
  float* Cf;
  float* Zout;
  __nv_bfloat16* Ch;
  __nv_bfloat16* Cht;  // [N][ldt] or nullptr
  int64_t ldt;
};
hsm_status mlp_gemm_tc(Mlp& m, const MlpGemm& g);
hsm_status mlp_forward_tc(Mlp& m, const __nv_bfloat16* X, int64_t rows, float* Y, int ldy);

}  // namespace hsm

