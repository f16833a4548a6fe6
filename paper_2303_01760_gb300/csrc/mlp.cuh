// Learned weight predictor: the MLP state shared by mlp.cu (training, the
// mma.sync GEMMs, projection) and mlp_tc.cu (the fused tcgen05 forward pass).
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
hsm_status mlp_forward_tc(Mlp& m, const __nv_bfloat16* X, int64_t rows, float* Y, int ldy);

}  // namespace hsm

