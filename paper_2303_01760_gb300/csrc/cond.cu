// Per-stencil condition numbers kappa_2(M) = ||M|| ||M^-1|| of the weight
// systems (Section 2.1, "Computational stability"): the scaled MON matrix P^T
// of a regular node and the scaled augmented RBF-FD matrix [A P; P^T 0] of a
// scattered one, both in xi = (x - x_c) / s with s = max |x_i - x_c|.
//
// The RBF-FD matrix is symmetric, so kappa_2 is the ratio of the largest to
// the smallest eigenvalue magnitude; the MON matrix is not, so its singular
// values are the roots of the eigenvalues of P^T P.  Eigenvalues come from
// the cyclic Jacobi method (Rutishauser's rotation formulas), one thread per
// system, at most kJacobiSweeps sweeps.  A diagnostic, off the timed path.
#include <cfloat>

#include "common.cuh"

namespace hsm {
namespace {

constexpr int kJacobiSweeps = 40;

// Eigenvalues of the symmetric K x K matrix a (row stride ld, element stride
// es: a[i * ld * es + j * es]) by cyclic Jacobi; they are left on the diagonal.
__device__ void jacobi_eigen(double* a, int K, int ld, int es) {
  auto at = [&](int i, int j) -> double& { return a[((int64_t)i * ld + j) * es]; };
  for (int sweep = 0; sweep < kJacobiSweeps; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int i = 0; i < K; ++i) {
      diag += at(i, i) * at(i, i);
      for (int j = i + 1; j < K; ++j) off += at(i, j) * at(i, j);
    }
    if (off <= 1e-32 * diag || off == 0.0) break;
    for (int p = 0; p < K - 1; ++p)
      for (int q = p + 1; q < K; ++q) {
        const double apq = at(p, q);
        if (apq == 0.0) continue;
        const double app = at(p, p), aqq = at(q, q);
        const double theta = (aqq - app) / (2.0 * apq);
        const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < K; ++k) {
          const double akp = at(k, p), akq = at(k, q);
          at(k, p) = c * akp - s * akq;
          at(k, q) = s * akp + c * akq;
        }
        for (int k = 0; k < K; ++k) {
          const double apk = at(p, k), aqk = at(q, k);
          at(p, k) = c * apk - s * aqk;
          at(q, k) = s * apk + c * aqk;
        }
      }
  }
}

__device__ double spectrum_ratio(const double* a, int K, int ld, int es) {
  double lo = DBL_MAX, hi = 0.0;
  for (int i = 0; i < K; ++i) {
    const double v = fabs(a[((int64_t)i * ld + i) * es]);
    lo = fmin(lo, v);
    hi = fmax(hi, v);
  }
  return lo > 0.0 ? hi / lo : __longlong_as_double(0x7ff0000000000000ll);
}

// One thread per scattered node: the K x K matrix is kept in shared memory,
// element (i, j) of thread t at [(i K + j) * B + t] (B threads per block).
template <int DIM>
__global__ void k_cond_rbf(const double* __restrict__ coords, int64_t N, const int32_t* __restrict__ idx,
                           const int32_t* __restrict__ nodes, int64_t G, int n, int nm,
                           const int8_t* __restrict__ mono_exp, double* kappa) {
  extern __shared__ double smem[];
  const int B = blockDim.x, t = threadIdx.x;
  const int K = n + nm;
  double* a = smem + t;
  for (int64_t p = blockIdx.x * (int64_t)B + t; p < G; p += (int64_t)gridDim.x * B) {
    const int32_t c = nodes[p];
    double xc[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) xc[k] = coords[k * N + c];
    // the scale s = max |x_i - x_c|
    double s2 = 0.0;
    for (int j = 0; j < n; ++j) {
      const int32_t id = idx[(int64_t)j * G + p];
      double r2 = 0.0;
#pragma unroll
      for (int k = 0; k < DIM; ++k) {
        const double o = coords[k * N + id] - xc[k];
        r2 += o * o;
      }
      s2 = fmax(s2, r2);
    }
    const double s = s2 > 0.0 ? sqrt(s2) : 1.0;
    auto A = [&](int i, int j) -> double& { return a[((int64_t)i * K + j) * B]; };
    for (int i = 0; i < n; ++i) {
      const int32_t ii = idx[(int64_t)i * G + p];
      double xi[DIM];
#pragma unroll
      for (int k = 0; k < DIM; ++k) xi[k] = (coords[k * N + ii] - xc[k]) / s;
      A(i, i) = 0.0;
      for (int j = i + 1; j < n; ++j) {
        const int32_t jj = idx[(int64_t)j * G + p];
        double d2 = 0.0;
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
          const double d = xi[k] - (coords[k * N + jj] - xc[k]) / s;
          d2 += d * d;
        }
        const double r = sqrt(d2);
        A(i, j) = A(j, i) = r * r * r;
      }
      for (int q = 0; q < nm; ++q) {
        double v = 1.0;
#pragma unroll
        for (int k = 0; k < DIM; ++k)
          for (int e = 0; e < mono_exp[q * DIM + k]; ++e) v *= xi[k];
        A(i, n + q) = A(n + q, i) = v;
      }
    }
    for (int q = 0; q < nm; ++q)
      for (int r = 0; r < nm; ++r) A(n + q, n + r) = 0.0;
    jacobi_eigen(a, K, K, B);
    kappa[c] = spectrum_ratio(a, K, K, B);
  }
}

// One thread per regular node: the 2d+1 system P^T (rows = basis 1, xi_k,
// xi_k^2), kappa_2 = sqrt(lambda_max / lambda_min) of P^T P.
template <int DIM>
__global__ void k_cond_mon(const double* __restrict__ coords, int64_t N, const int32_t* __restrict__ idx,
                           const int32_t* __restrict__ nodes, int64_t G, double* kappa) {
  constexpr int K = 2 * DIM + 1;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < G; p += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = nodes[p];
    double xc[DIM], xi[K][DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) xc[k] = coords[k * N + c];
    double s2 = 0.0;
    for (int j = 0; j < K; ++j) {
      const int32_t id = idx[(int64_t)j * G + p];
      double r2 = 0.0;
#pragma unroll
      for (int k = 0; k < DIM; ++k) {
        xi[j][k] = coords[k * N + id] - xc[k];
        r2 += xi[j][k] * xi[j][k];
      }
      s2 = fmax(s2, r2);
    }
    const double s = s2 > 0.0 ? sqrt(s2) : 1.0;
    double P[K][K];  // P[node][basis]
    for (int j = 0; j < K; ++j) {
      P[j][0] = 1.0;
#pragma unroll
      for (int k = 0; k < DIM; ++k) {
        const double x = xi[j][k] / s;
        P[j][1 + 2 * k] = x;
        P[j][2 + 2 * k] = x * x;
      }
    }
    double g[K * K];  // (P^T)^T P^T = P P^T: same non-zero spectrum as P^T P
    for (int i = 0; i < K; ++i)
      for (int j = 0; j < K; ++j) {
        double v = 0.0;
        for (int b = 0; b < K; ++b) v += P[i][b] * P[j][b];
        g[i * K + j] = v;
      }
    jacobi_eigen(g, K, K, 1);
    kappa[c] = sqrt(spectrum_ratio(g, K, K, 1));
  }
}

}  // namespace

hsm_status launch_condition(hsm_plan p, double* kappa) {
  cudaStream_t s = p->stream;
  if (p->mon.count) {
    const int grid = (int)std::min<int64_t>(ceil_div(p->mon.count, 128), (int64_t)num_sms() * 8);
    if (p->dim == 2) k_cond_mon<2><<<grid, 128, 0, s>>>(p->coords, p->N, p->mon.idx, p->mon.nodes, p->mon.count, kappa);
    else k_cond_mon<3><<<grid, 128, 0, s>>>(p->coords, p->N, p->mon.idx, p->mon.nodes, p->mon.count, kappa);
    HSM_CUDA(p, cudaGetLastError());
    p->launches += 1;
  }
  if (p->rbf.count) {
    const int K = p->n + p->n_mono;
    const size_t per = (size_t)K * K * sizeof(double);
    const int threads = (int)std::max<size_t>(1, std::min<size_t>(64, (200 * 1024) / per));
    const size_t smem = per * threads;
    if (smem > 227 * 1024) return set_error(p, HSM_EINVAL, "RBF-FD system too large for the condition diagnostic");
    void* fn = p->dim == 2 ? (void*)k_cond_rbf<2> : (void*)k_cond_rbf<3>;
    HSM_CUDA(p, raise_smem_limit(fn, smem));
    const int grid = (int)std::min<int64_t>(ceil_div(p->rbf.count, threads), (int64_t)num_sms() * 4);
    const double* coords = p->coords;
    int64_t N = p->N, G = p->rbf.count;
    const int32_t* idx = p->rbf.idx;
    const int32_t* nodes = p->rbf.nodes;
    int n = p->n, nm = p->n_mono;
    const int8_t* ex = p->mono_exp;
    void* args[] = {(void*)&coords, (void*)&N, (void*)&idx, (void*)&nodes, (void*)&G, (void*)&n, (void*)&nm,
                    (void*)&ex, (void*)&kappa};
    HSM_CUDA(p, cudaLaunchKernel(fn, dim3(grid), dim3(threads), args, smem, s));
    p->launches += 1;
  }
  return HSM_OK;
}

}  // namespace hsm
