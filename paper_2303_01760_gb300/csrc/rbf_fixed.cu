// FP32 + FP64-refinement RBF-FD kernels with compile-time system sizes: 2D
// m = 2 with n = 12 (K = 18) and 3D m = 2 with n = 20 (K = 30), all
// operators.  Their FP32 LU has every loop bound known at compile time
// (FixedLU), which removes most of the index arithmetic of the general one.
#include "rbf_kernels.cuh"

namespace hsm {

void* pick_fp32r_fixed(int dim, int nops, int K, int lanes) {
  if (dim == 2 && nops == 3 && K == 18) {
    switch (lanes) {
      case 4: return (void*)k_rbf_fp32r<2, 3, 4, 18>;
      case 8: return (void*)k_rbf_fp32r<2, 3, 8, 18>;
      case 16: return (void*)k_rbf_fp32r<2, 3, 16, 18>;
    }
  }
  if (dim == 3 && nops == 4 && K == 30) {
    switch (lanes) {
      case 8: return (void*)k_rbf_fp32r<3, 4, 8, 30>;
      case 16: return (void*)k_rbf_fp32r<3, 4, 16, 30>;
    }
  }
  return nullptr;
}
}  // namespace hsm
