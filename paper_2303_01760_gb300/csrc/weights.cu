// Stencil weights of Eq. 1 (Section 2 and 2.1).
//
// MON (regular nodes): P^T w = L p over the 2d+1 monomials {1, x_k, x_k^2}
// (Section 2 footnote), one thread per node: the closed-form solution of the
// decoupled per-axis systems when the stencil is axis-aligned, otherwise the
// (2d+1) x (2d+1+ops) system by Gaussian elimination in a fixed order that
// needs no pivoting on lattice stencils.
//
// RBF-FD (scattered, boundary and demoted nodes): the augmented PHS system
//     [A P; P^T 0][w; lambda] = [L phi; L p],  phi(r) = r^3,
// with all monomials of degree <= m (Section 2, Section 4).  One group of
// LANES lanes solves one system held in shared memory: assembly, LU with
// partial pivoting applied to all right-hand sides at once, and back
// substitution.  Every elimination step spreads its (rows x columns) updates
// over the lanes as one flat index range, which keeps the FP64 pipe busy even
// when the active block is smaller than the lane count.  Both bases are solved
// in the scaled offset xi = (x - x_c)/s, s = max |x_i - x_c|; derivative
// weights are divided by s, Laplacian weights by s^2 afterwards.
//
// The FP32 variant factors the same system in FP32 and refines every
// right-hand side with residuals r = b - M x formed in FP64 against the FP64
// matrix, x += M32^-1 r, until the correction is below 3e-4 of |x| (the next
// iterate is then accurate to about 1e-7) or three corrections were taken;
// systems that do not converge are re-solved by the FP64 kernel.
#include <cfloat>

#include "common.cuh"

namespace hsm {
namespace {

struct OpsDesc {
  int kind[kMaxOps];  // 0,1,2 = d/dx_k ; 3 = Laplacian
};

__host__ OpsDesc make_ops(hsm_plan p, unsigned mask) {
  OpsDesc d{};
  int o = 0;
  for (int b = 0; b < 4; ++b)
    if (mask & (1u << b)) d.kind[o++] = b;
  return d;
}

// ---------------------------------------------------------------------------
// MON
// ---------------------------------------------------------------------------
// The system is ordered basis rows (1, xi_1, xi_1^2, xi_2, xi_2^2 [, xi_3,
// xi_3^2]) against node columns (c, c-e1, c+e1, c-e2, c+e2 [, c-e3, c+e3]).
// On (and within 1e-6 lattice units of) the lattice this order needs no
// pivoting: every pivot stays within rounding of 1, -1 or 2, so the
// elimination runs as straight-line code in registers.  A pivot below 1e-8
// (impossible for a lattice stencil) marks the node singular.
template <int DIM, int NOPS>
__global__ void __launch_bounds__(128) k_mon(const double* __restrict__ coords, int64_t N,
                                             const int32_t* __restrict__ idx, int64_t G, OpsDesc ops,
                                             double* __restrict__ w, uint8_t* __restrict__ status,
                                             const int32_t* __restrict__ nodes, unsigned* flags) {
  constexpr int K = 2 * DIM + 1;
  constexpr int C = K + NOPS;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < G; p += (int64_t)gridDim.x * blockDim.x) {
    double xi[K][DIM];
    const int32_t c = idx[p];
    double cx[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) cx[k] = coords[k * N + c];
    double s2 = 0.0;
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const int32_t id = idx[(int64_t)j * G + p];
      double r2 = 0.0;
#pragma unroll
      for (int k = 0; k < DIM; ++k) {
        const double o = coords[k * N + id] - cx[k];
        xi[j][k] = o;
        r2 += o * o;
      }
      s2 = fmax(s2, r2);
    }
    // Axis-aligned stencil (every neighbour offset is zero off its own axis,
    // as for nodes placed exactly on the lattice): the system decouples into
    // one 3-point Vandermonde system per axis, solved in closed form with
    // a = |x_c - x_{c-e}|, b = |x_{c+e} - x_c|, r = 1 / (a b (a + b)):
    //   d/dx_k : w(c-e) = -b^2 r, w(c+e) = a^2 r, w(c) = -(w(c-e) + w(c+e))
    //   lap    : w(c-e) = 2 b r,  w(c+e) = 2 a r, summed over the axes.
    bool aligned = true;
#pragma unroll
    for (int k = 0; k < DIM; ++k)
#pragma unroll
      for (int e = 0; e < DIM; ++e)
        if (e != k) aligned = aligned && xi[1 + 2 * k][e] == 0.0 && xi[2 + 2 * k][e] == 0.0;
    if (aligned) {
      double wm[DIM], wp[DIM], lm[DIM], lpl[DIM];
      bool okk = true;
#pragma unroll
      for (int k = 0; k < DIM; ++k) {
        const double a = -xi[1 + 2 * k][k], b = xi[2 + 2 * k][k];
        okk = okk && a > 0.0 && b > 0.0;
        const double r = 1.0 / (a * b * (a + b));
        wm[k] = -b * b * r;
        wp[k] = a * a * r;
        lm[k] = 2.0 * b * r;
        lpl[k] = 2.0 * a * r;
      }
#pragma unroll
      for (int o = 0; o < NOPS; ++o) {
        const int kd = ops.kind[o];
        double wc = 0.0;
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
          double m = 0.0, pl = 0.0;
          if (kd == 3) {
            m = lm[k];
            pl = lpl[k];
          } else if (kd == k) {
            m = wm[k];
            pl = wp[k];
          }
          wc -= m + pl;
          w[((int64_t)o * K + 1 + 2 * k) * G + p] = okk ? m : 0.0;
          w[((int64_t)o * K + 2 + 2 * k) * G + p] = okk ? pl : 0.0;
        }
        w[((int64_t)o * K) * G + p] = okk ? wc : 0.0;
      }
      if (!okk) atomicOr(flags, kDevSingular);
      if (status) status[nodes[p]] = okk ? HSM_NODE_OK : HSM_NODE_SINGULAR;
      continue;
    }
    const double s = sqrt(s2);
    const double inv_s = 1.0 / s;
    double a[K][C];
#pragma unroll
    for (int j = 0; j < K; ++j) {
      a[0][j] = 1.0;
#pragma unroll
      for (int k = 0; k < DIM; ++k) {
        const double x = xi[j][k] * inv_s;
        a[1 + 2 * k][j] = x;
        a[2 + 2 * k][j] = x * x;
      }
    }
#pragma unroll
    for (int b = 0; b < K; ++b)
#pragma unroll
      for (int o = 0; o < NOPS; ++o) {
        const int kd = ops.kind[o];
        // row b is 1 (b == 0), xi_k (b = 1 + 2k) or xi_k^2 (b = 2 + 2k)
        double v = 0.0;
        if (kd == 3) v = (b > 0 && (b % 2) == 0) ? 2.0 : 0.0;
        else v = (b == 1 + 2 * kd) ? 1.0 : 0.0;
        a[b][K + o] = v;
      }
    bool ok = s > 0.0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const double piv = a[k][k];
      ok = ok && fabs(piv) > 1e-8;
      const double inv = 1.0 / piv;
#pragma unroll
      for (int i = k + 1; i < K; ++i) {
        const double l = a[i][k] * inv;
#pragma unroll
        for (int j = k + 1; j < C; ++j) a[i][j] = fma(-l, a[k][j], a[i][j]);
      }
      a[k][k] = inv;
    }
#pragma unroll
    for (int k = K - 1; k >= 0; --k) {
#pragma unroll
      for (int o = 0; o < NOPS; ++o) {
        double x = a[k][K + o];
#pragma unroll
        for (int j = k + 1; j < K; ++j) x = fma(-a[k][j], a[j][K + o], x);
        a[k][K + o] = x * a[k][k];
      }
    }
#pragma unroll
    for (int o = 0; o < NOPS; ++o) {
      const double sc = ops.kind[o] == 3 ? inv_s * inv_s : inv_s;
#pragma unroll
      for (int j = 0; j < K; ++j) w[((int64_t)o * K + j) * G + p] = ok ? a[j][K + o] * sc : 0.0;
    }
    if (!ok) atomicOr(flags, kDevSingular);
    if (status) status[nodes[p]] = ok ? HSM_NODE_OK : HSM_NODE_SINGULAR;
  }
}

// ---------------------------------------------------------------------------
// RBF-FD: lane-group-per-system LU in shared memory
// ---------------------------------------------------------------------------
struct RbfArgs {
  const double* coords;
  int64_t N;
  const int32_t* list;     // positions to solve (nullptr = 0..count-1)
  int64_t count;
  const int32_t* idx;      // [n][G]
  int64_t G;
  const int32_t* nodes;    // [G] node ids of the group
  int n, n_mono, K, ld;
  const int8_t* mono_exp;  // [n_mono][dim]
  const uint16_t* pairs;   // [n(n-1)/2]
  OpsDesc ops;
  double* w;               // [nops][n][G]
  uint8_t* status;         // [N] or nullptr
  uint8_t status_demoted_mark;
  const uint8_t* is_regular;
  unsigned* flags;
  int32_t* fail_list;      // fp32r: positions that did not converge
  int* fail_count;
};

template <typename T>
struct AbsBits;
template <>
struct AbsBits<double> {
  static __device__ __forceinline__ unsigned long long get(double x) {
    return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
  }
};
template <>
struct AbsBits<float> {
  static __device__ __forceinline__ unsigned long long get(float x) {
    return (unsigned long long)(__float_as_uint(x) & 0x7fffffffu);
  }
};

template <typename T>
struct PivTol;
template <>
struct PivTol<double> {
  static constexpr double value = 1e-12;
};
template <>
struct PivTol<float> {
  static constexpr double value = 0.0;
};

__device__ __forceinline__ unsigned long long shfl_xor_u64(unsigned mask, unsigned long long v, int o, int w) {
  return (unsigned long long)__shfl_xor_sync(mask, (long long)v, o, w);
}

// Per-system shared memory layout (in doubles):
//   M      K x ld        (T = double) or K x K FP64 copy + K x ld T (fp32r)
//   xi     n x DIM
//   rc     n          |xi_j|, the scaled distance of node j from the centre
//   inv    K
//   b64    K x NOPS   (fp32r only)
//   x64    K x NOPS   (fp32r only)
template <int DIM, int NOPS, bool R32>
__host__ __device__ constexpr size_t sys_doubles(int K, int ld, int n) {
  return R32 ? ((size_t)K * K + ((size_t)K * ld + 1) / 2 + (size_t)n * (DIM + 1) + K + 2 * (size_t)K * NOPS +
                (K + 1) / 2)
             : ((size_t)K * ld + (size_t)n * (DIM + 1) + K);
}

// Assembles [A P | L phi; P^T 0 | L p] into Mt (row stride ld) for the scaled
// offsets xi.  Returns via *inv_s the inverse scale.
template <int DIM, int NOPS, int LANES, typename T>
__device__ __forceinline__ void assemble(const RbfArgs& a, int64_t pos, int lane, unsigned mask, double* xi,
                                         double* rc, T* Mt, int ldt, double* M64, double& inv_s_out, bool& ok) {
  const int n = a.n, K = a.K, nm = a.n_mono;
  const int32_t c = a.nodes[pos];
  unsigned long long b = 0ull;
  for (int j = lane; j < n; j += LANES) {
    const int32_t id = a.idx[(int64_t)j * a.G + pos];
    double r2 = 0.0;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      double o = a.coords[k * a.N + id] - a.coords[k * a.N + c];
      xi[j * DIM + k] = o;
      r2 += o * o;
    }
    const double r = sqrt(r2);
    rc[j] = r;
    // non-negative doubles order like their bit patterns
    const unsigned long long rb = (unsigned long long)__double_as_longlong(r);
    b = rb > b ? rb : b;
  }
#pragma unroll
  for (int o = LANES / 2; o > 0; o >>= 1) {
    unsigned long long t = shfl_xor_u64(mask, b, o, LANES);
    b = t > b ? t : b;
  }
  const double s = __longlong_as_double((long long)b);
  const double inv_s = 1.0 / s;
  inv_s_out = inv_s;
  ok = s > 0.0 && isfinite(s);
  __syncwarp(mask);
  for (int e = lane; e < n * DIM; e += LANES) xi[e] *= inv_s;
  for (int e = lane; e < n; e += LANES) rc[e] *= inv_s;
  __syncwarp(mask);
  // A block (zero diagonal, symmetric pairs)
  for (int e = lane; e < n; e += LANES) {
    Mt[e * ldt + e] = T(0);
    if (M64) M64[e * K + e] = 0.0;
  }
  const int npairs = n * (n - 1) / 2;
  for (int e = lane; e < npairs; e += LANES) {
    const uint16_t pr = a.pairs[e];
    const int i = pr >> 8, j = pr & 0xff;
    double d2 = 0.0;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      double d = xi[i * DIM + k] - xi[j * DIM + k];
      d2 += d * d;
    }
    const double v = d2 * sqrt(d2);
    Mt[i * ldt + j] = T(v);
    Mt[j * ldt + i] = T(v);
    if (M64) {
      M64[i * K + j] = v;
      M64[j * K + i] = v;
    }
  }
  // P and P^T blocks
  for (int e = lane; e < n * nm; e += LANES) {
    const int i = e / nm, q = e - (e / nm) * nm;
    double v = 1.0;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      const int ex = a.mono_exp[q * DIM + k];
      for (int t = 0; t < ex; ++t) v *= xi[i * DIM + k];
    }
    Mt[i * ldt + n + q] = T(v);
    Mt[(n + q) * ldt + i] = T(v);
    if (M64) {
      M64[i * K + n + q] = v;
      M64[(n + q) * K + i] = v;
    }
  }
  for (int e = lane; e < nm * nm; e += LANES) {
    const int i = e / nm, q = e - (e / nm) * nm;
    Mt[(n + i) * ldt + n + q] = T(0);
    if (M64) M64[(n + i) * K + n + q] = 0.0;
  }
  __syncwarp(mask);
}

// RHS value of operator o for stencil node e (PHS part); r = |xi_e|.
template <int DIM>
__device__ __forceinline__ double rhs_phi(const double* xi, const double* rc, int e, int kind) {
  const double r = rc[e];
  if (kind == 3) return 3.0 * (DIM + 1) * r;
  return -3.0 * r * xi[e * DIM + kind];
}
template <int DIM>
__device__ __forceinline__ double rhs_mono(const int8_t* ex, int q, int kind) {
  int deg = 0, mx = 0, which = -1;
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    int e = ex[q * DIM + k];
    deg += e;
    if (e > mx) {
      mx = e;
      which = k;
    }
  }
  if (kind == 3) return (deg == 2 && mx == 2) ? 2.0 : 0.0;
  return (deg == 1 && which == kind) ? 1.0 : 0.0;
}

// LU with partial pivoting of the K x (K+NOPS) matrix Mt (row stride ldt),
// in place, followed by back substitution; the solutions overwrite the
// right-hand-side columns.  inv[k] receives the inverse pivots.
template <int NOPS, int LANES, typename T>
__device__ __forceinline__ bool lu_solve(T* Mt, int ldt, int K, T* inv, int lane, unsigned mask, bool factor,
                                         int* perm = nullptr) {
  const int Ctot = K + NOPS;
  bool ok = true;
  if (factor) {
    for (int k = 0; k < K; ++k) {
      unsigned long long best = 0ull;
      int brow = K;
      for (int i = k + lane; i < K; i += LANES) {
        unsigned long long v = AbsBits<T>::get(Mt[i * ldt + k]);
        if (v > best || (v == best && i < brow)) {
          best = v;
          brow = i;
        }
      }
#pragma unroll
      for (int o = LANES / 2; o > 0; o >>= 1) {
        unsigned long long ob = shfl_xor_u64(mask, best, o, LANES);
        int orow = __shfl_xor_sync(mask, brow, o, LANES);
        if (ob > best || (ob == best && orow < brow)) {
          best = ob;
          brow = orow;
        }
      }
      if (brow != k && brow < K) {
        // whole rows, multipliers included, so the stored factor stays
        // consistent for later right-hand sides
        for (int j = (perm ? 0 : k) + lane; j < Ctot; j += LANES) {
          T t = Mt[k * ldt + j];
          Mt[k * ldt + j] = Mt[brow * ldt + j];
          Mt[brow * ldt + j] = t;
        }
        if (perm && lane == 0) {
          int t = perm[k];
          perm[k] = perm[brow];
          perm[brow] = t;
        }
      }
      __syncwarp(mask);
      const T piv = Mt[k * ldt + k];
      // the scaled system has entries of order one: a pivot below the
      // threshold means the system is singular to working precision
      if (!(fabs((double)piv) > PivTol<T>::value) || !isfinite((double)piv)) {
        ok = false;
        break;
      }
      const T ip = T(1) / piv;
      if (lane == 0) inv[k] = ip;
      for (int i = k + 1 + lane; i < K; i += LANES) Mt[i * ldt + k] *= ip;
      __syncwarp(mask);
      const int R = K - k - 1, C = Ctot - k - 1;
      const int total = R * C;
      if (total > 0) {
        int i = lane / C, j = lane - (lane / C) * C;
        const int dq = LANES / C, dr = LANES - (LANES / C) * C;
        const T* prow = Mt + k * ldt + k + 1;
        T* base = Mt + (k + 1) * ldt + k + 1;
        for (int e = lane; e < total; e += LANES) {
          T* row = base + i * ldt;
          row[j] = fma(-row[-1], prow[j], row[j]);
          j += dr;
          i += dq;
          if (j >= C) {
            j -= C;
            ++i;
          }
        }
      }
      __syncwarp(mask);
    }
  } else {
    // forward elimination of the right-hand sides only, with the stored
    // multipliers and the row order already applied to the factor
    for (int k = 0; k < K - 1; ++k) {
      for (int e = lane; e < (K - k - 1) * NOPS; e += LANES) {
        const int i = k + 1 + e / NOPS, o = e - (e / NOPS) * NOPS;
        Mt[i * ldt + K + o] = fma(-Mt[i * ldt + k], Mt[k * ldt + K + o], Mt[i * ldt + K + o]);
      }
      __syncwarp(mask);
    }
  }
  if (!ok) return false;
  for (int k = K - 1; k >= 0; --k) {
    for (int o = lane; o < NOPS; o += LANES) Mt[k * ldt + K + o] *= inv[k];
    __syncwarp(mask);
    for (int e = lane; e < k * NOPS; e += LANES) {
      const int i = e / NOPS, o = e - (e / NOPS) * NOPS;
      Mt[i * ldt + K + o] = fma(-Mt[i * ldt + k], Mt[k * ldt + K + o], Mt[i * ldt + K + o]);
    }
    __syncwarp(mask);
  }
  return true;
}

template <int DIM, int NOPS, int LANES>
__global__ void __launch_bounds__(128) k_rbf_fp64(RbfArgs a) {
  extern __shared__ double smem[];
  constexpr int SYS = 128 / LANES;
  const int sub = threadIdx.x / LANES, lane = threadIdx.x % LANES;
  const unsigned mask = LANES == 32 ? 0xffffffffu : (((1u << LANES) - 1u) << ((threadIdx.x & 31) / LANES * LANES));
  const int K = a.K, ld = a.ld, n = a.n;
  double* base = smem + (size_t)sub * sys_doubles<DIM, NOPS, false>(K, ld, n);
  double* M = base;
  double* xi = M + (size_t)K * ld;
  double* rc = xi + n * DIM;
  double* inv = rc + n;
  for (int64_t t = (int64_t)blockIdx.x * SYS + sub; t < a.count; t += (int64_t)gridDim.x * SYS) {
    const int64_t pos = a.list ? a.list[t] : t;
    double inv_s;
    bool ok;
    assemble<DIM, NOPS, LANES, double>(a, pos, lane, mask, xi, rc, M, ld, nullptr, inv_s, ok);
    for (int e = lane; e < n * NOPS; e += LANES) {
      const int i = e / NOPS, o = e - (e / NOPS) * NOPS;
      M[i * ld + K + o] = rhs_phi<DIM>(xi, rc, i, a.ops.kind[o]);
    }
    for (int e = lane; e < a.n_mono * NOPS; e += LANES) {
      const int q = e / NOPS, o = e - (e / NOPS) * NOPS;
      M[(n + q) * ld + K + o] = rhs_mono<DIM>(a.mono_exp, q, a.ops.kind[o]);
    }
    __syncwarp(mask);
    ok = lu_solve<NOPS, LANES, double>(M, ld, K, inv, lane, mask, true) && ok;
    for (int e = lane; e < n * NOPS; e += LANES) {
      const int j = e / NOPS, o = e - (e / NOPS) * NOPS;
      const double sc = a.ops.kind[o] == 3 ? inv_s * inv_s : inv_s;
      const double v = M[j * ld + K + o] * sc;
      a.w[((int64_t)o * n + j) * a.G + pos] = ok && isfinite(v) ? v : 0.0;
    }
    if (lane == 0) {
      const int32_t node = a.nodes[pos];
      if (!ok) atomicOr(a.flags, kDevSingular);
      if (a.status)
        a.status[node] = !ok ? HSM_NODE_SINGULAR
                             : (a.status_demoted_mark ? a.status_demoted_mark
                                                      : (a.is_regular[node] ? HSM_NODE_DEMOTED : HSM_NODE_OK));
    }
    __syncwarp(mask);
  }
}

template <int DIM, int NOPS, int LANES>
__global__ void __launch_bounds__(128) k_rbf_fp32r(RbfArgs a) {
  extern __shared__ double smem[];
  constexpr int SYS = 128 / LANES;
  constexpr int kMaxIt = 3;
  const int sub = threadIdx.x / LANES, lane = threadIdx.x % LANES;
  const unsigned mask = LANES == 32 ? 0xffffffffu : (((1u << LANES) - 1u) << ((threadIdx.x & 31) / LANES * LANES));
  const int K = a.K, n = a.n;
  const int ld32 = (K + NOPS) | 1;
  double* base = smem + (size_t)sub * sys_doubles<DIM, NOPS, true>(K, ld32, n);
  double* M64 = base;
  float* L32 = reinterpret_cast<float*>(M64 + (size_t)K * K);
  double* xi = M64 + (size_t)K * K + ((size_t)K * ld32 + 1) / 2;
  double* rc = xi + n * DIM;
  float* inv = reinterpret_cast<float*>(rc + n);
  double* b64 = rc + n + K;
  double* x64 = b64 + K * NOPS;
  int* perm = reinterpret_cast<int*>(x64 + K * NOPS);
  for (int64_t t = (int64_t)blockIdx.x * SYS + sub; t < a.count; t += (int64_t)gridDim.x * SYS) {
    const int64_t pos = a.list ? a.list[t] : t;
    double inv_s;
    bool ok;
    assemble<DIM, NOPS, LANES, float>(a, pos, lane, mask, xi, rc, L32, ld32, M64, inv_s, ok);
    for (int e = lane; e < K * NOPS; e += LANES) {
      const int i = e / NOPS, o = e - (e / NOPS) * NOPS;
      const double v = i < n ? rhs_phi<DIM>(xi, rc, i, a.ops.kind[o]) : rhs_mono<DIM>(a.mono_exp, i - n, a.ops.kind[o]);
      b64[i * NOPS + o] = v;
      L32[i * ld32 + K + o] = (float)v;
    }
    for (int i = lane; i < K; i += LANES) perm[i] = i;
    __syncwarp(mask);
    ok = lu_solve<NOPS, LANES, float>(L32, ld32, K, inv, lane, mask, true, perm) && ok;
    bool conv = false;
    if (ok) {
      for (int e = lane; e < K * NOPS; e += LANES) {
        const int i = e / NOPS, o = e - (e / NOPS) * NOPS;
        x64[i * NOPS + o] = (double)L32[i * ld32 + K + o];
      }
      __syncwarp(mask);
      for (int it = 0; it < kMaxIt && !conv; ++it) {
        // r = b - M x in FP64 (original equation order), rounded into the
        // FP32 right-hand-side columns in the factor's row order
        for (int e = lane; e < K * NOPS; e += LANES) {
          const int kf = e / NOPS, o = e - (e / NOPS) * NOPS;
          const int i = perm[kf];
          double r = b64[i * NOPS + o];
          const double* row = M64 + (size_t)i * K;
          for (int j = 0; j < K; ++j) r = fma(-row[j], x64[j * NOPS + o], r);
          L32[kf * ld32 + K + o] = (float)r;
        }
        __syncwarp(mask);
        lu_solve<NOPS, LANES, float>(L32, ld32, K, inv, lane, mask, false);
        // x += d ; converged when max|d| <= 3e-4 max|x| for every operator
        unsigned long long dmax[NOPS], xmax[NOPS];
#pragma unroll
        for (int o = 0; o < NOPS; ++o) dmax[o] = xmax[o] = 0ull;
        for (int e = lane; e < K * NOPS; e += LANES) {
          const int i = e / NOPS, o = e - (e / NOPS) * NOPS;
          const double d = (double)L32[i * ld32 + K + o];
          const double x = x64[i * NOPS + o] + d;
          x64[i * NOPS + o] = x;
#pragma unroll
          for (int q = 0; q < NOPS; ++q)
            if (q == o) {
              unsigned long long bd = AbsBits<double>::get(d), bx = AbsBits<double>::get(x);
              dmax[q] = bd > dmax[q] ? bd : dmax[q];
              xmax[q] = bx > xmax[q] ? bx : xmax[q];
            }
        }
        bool c = true;
#pragma unroll
        for (int o = 0; o < NOPS; ++o) {
#pragma unroll
          for (int s = LANES / 2; s > 0; s >>= 1) {
            unsigned long long t1 = shfl_xor_u64(mask, dmax[o], s, LANES);
            unsigned long long t2 = shfl_xor_u64(mask, xmax[o], s, LANES);
            dmax[o] = t1 > dmax[o] ? t1 : dmax[o];
            xmax[o] = t2 > xmax[o] ? t2 : xmax[o];
          }
          const double dm = __longlong_as_double((long long)dmax[o]);
          const double xm = __longlong_as_double((long long)xmax[o]);
          c = c && isfinite(xm) && dm <= 3e-4 * xm;
        }
        conv = c;
        __syncwarp(mask);
      }
    }
    const bool good = ok && conv;
    for (int e = lane; e < n * NOPS; e += LANES) {
      const int j = e / NOPS, o = e - (e / NOPS) * NOPS;
      const double sc = a.ops.kind[o] == 3 ? inv_s * inv_s : inv_s;
      a.w[((int64_t)o * n + j) * a.G + pos] = good ? x64[j * NOPS + o] * sc : 0.0;
    }
    if (lane == 0) {
      const int32_t node = a.nodes[pos];
      if (!good) {
        int slot = atomicAdd(a.fail_count, 1);
        a.fail_list[slot] = (int32_t)pos;
      } else if (a.status) {
        a.status[node] = a.is_regular[node] ? HSM_NODE_DEMOTED : HSM_NODE_OK;
      }
    }
    __syncwarp(mask);
  }
}

template <int DIM, int NOPS>
__global__ void k_to_f32(const double* __restrict__ w, float* __restrict__ w32, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    w32[i] = (float)w[i];
}

template <template <int, int, int> class KernelT>
struct Dispatch;

template <int DIM, int NOPS, int LANES>
struct Fp64Kernel {
  static void* ptr() { return (void*)k_rbf_fp64<DIM, NOPS, LANES>; }
};
template <int DIM, int NOPS, int LANES>
struct Fp32rKernel {
  static void* ptr() { return (void*)k_rbf_fp32r<DIM, NOPS, LANES>; }
};

template <template <int, int, int> class KT, int DIM, int NOPS>
void* pick_lanes(int lanes) {
  switch (lanes) {
    case 8: return KT<DIM, NOPS, 8>::ptr();
    case 16: return KT<DIM, NOPS, 16>::ptr();
    default: return KT<DIM, NOPS, 32>::ptr();
  }
}
template <template <int, int, int> class KT, int DIM>
void* pick_nops(int nops, int lanes) {
  switch (nops) {
    case 1: return pick_lanes<KT, DIM, 1>(lanes);
    case 2: return pick_lanes<KT, DIM, 2>(lanes);
    case 3: return pick_lanes<KT, DIM, 3>(lanes);
    default: return pick_lanes<KT, DIM, 4>(lanes);
  }
}
template <template <int, int, int> class KT>
void* pick(int dim, int nops, int lanes) {
  return dim == 2 ? pick_nops<KT, 2>(nops, lanes) : pick_nops<KT, 3>(nops, lanes);
}

size_t smem_bytes(int dim, int nops, bool r32, int K, int ld, int n) {
  size_t d = 0;
  const int ld32 = (K + nops) | 1;
  if (r32) d = (size_t)K * K + ((size_t)K * ld32 + 1) / 2 + (size_t)n * (dim + 1) + K + 2 * (size_t)K * nops +
               (K + 1) / 2;
  else d = (size_t)K * ld + (size_t)n * (dim + 1) + K;
  return d * sizeof(double);
}

hsm_status launch_rbf(hsm_plan p, bool r32, const int32_t* list, int64_t count, uint8_t* status,
                      int32_t* fail_list, int* fail_count, uint8_t mark) {
  if (count == 0) return HSM_OK;
  RbfArgs a;
  a.coords = p->coords;
  a.N = p->N;
  a.list = list;
  a.count = count;
  a.idx = p->rbf.idx;
  a.G = p->rbf.count;
  a.nodes = p->rbf.nodes;
  a.n = p->n;
  a.n_mono = p->n_mono;
  a.K = p->n + p->n_mono;
  a.ld = (a.K + p->nops) | 1;
  a.mono_exp = p->mono_exp;
  a.pairs = p->pairs;
  a.ops = make_ops(p, p->op_mask);
  a.w = p->rbf.w64;
  a.status = status;
  a.status_demoted_mark = mark;
  a.is_regular = p->is_regular;
  a.flags = p->dev_flags;
  a.fail_list = fail_list;
  a.fail_count = fail_count;
  int lanes = p->tune.rbf_lanes;
  const int sys_per_block = 128 / lanes;
  size_t per = smem_bytes(p->dim, p->nops, r32, a.K, a.ld, a.n);
  size_t smem = per * sys_per_block;
  while (smem > 200 * 1024 && lanes < 32) {
    lanes *= 2;
    smem = per * (128 / lanes);
  }
  if (smem > 220 * 1024) return set_error(p, HSM_EINVAL, "RBF-FD system too large for shared memory");
  void* fn = r32 ? pick<Fp32rKernel>(p->dim, p->nops, lanes) : pick<Fp64Kernel>(p->dim, p->nops, lanes);
  HSM_CUDA(p, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int blocks_per_sm = 0;
  HSM_CUDA(p, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, fn, 128, smem));
  if (blocks_per_sm < 1) blocks_per_sm = 1;
  const int spb = 128 / lanes;
  int64_t want = ceil_div(count, spb);
  int grid = (int)std::min<int64_t>(want, (int64_t)num_sms() * blocks_per_sm);
  void* args[] = {&a};
  HSM_CUDA(p, cudaLaunchKernel(fn, dim3(grid), dim3(128), args, smem, p->stream));
  p->launches += 1;
  return HSM_OK;
}

}  // namespace

size_t rbf_smem_per_system(int K, int ld, bool fp32) { return smem_bytes(3, 4, fp32, K, ld, kMaxStencil); }

cudaError_t launch_rbf_external(const RbfExternal& x, bool r32, const int32_t* list, int64_t count, uint8_t* status,
                                uint8_t mark, bool* too_big) {
  *too_big = false;
  if (count == 0) return cudaSuccess;
  RbfArgs a;
  a.coords = x.coords;
  a.N = x.N;
  a.list = list;
  a.count = count;
  a.idx = x.idx;
  a.G = x.G;
  a.nodes = x.idx;  // row 0 of the stencils holds the centres
  a.n = x.n;
  a.n_mono = x.n_mono;
  a.K = x.n + x.n_mono;
  a.ld = (a.K + x.nops) | 1;
  a.mono_exp = x.mono_exp;
  a.pairs = x.pairs;
  OpsDesc d{};
  int o = 0;
  for (int b = 0; b < 4; ++b)
    if (x.op_mask & (1u << b)) d.kind[o++] = b;
  a.ops = d;
  a.w = x.w;
  a.status = status;
  a.status_demoted_mark = mark;
  a.is_regular = nullptr;  // never read: status is either NULL or written with mark
  a.flags = x.flags;
  a.fail_list = x.fail_list;
  a.fail_count = x.fail_count;
  int lanes = 8;
  size_t per = smem_bytes(x.dim, x.nops, r32, a.K, a.ld, a.n);
  size_t smem = per * (128 / lanes);
  while (smem > 200 * 1024 && lanes < 32) {
    lanes *= 2;
    smem = per * (128 / lanes);
  }
  if (smem > 220 * 1024) {
    *too_big = true;
    return cudaSuccess;
  }
  void* fn = r32 ? pick<Fp32rKernel>(x.dim, x.nops, lanes) : pick<Fp64Kernel>(x.dim, x.nops, lanes);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int blocks_per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, fn, 128, smem);
  if (e != cudaSuccess) return e;
  if (blocks_per_sm < 1) blocks_per_sm = 1;
  const int64_t want = ceil_div(count, 128 / lanes);
  const int grid = (int)std::min<int64_t>(want, (int64_t)num_sms() * blocks_per_sm);
  void* args[] = {&a};
  return cudaLaunchKernel(fn, dim3(grid), dim3(128), args, smem, x.stream);
}

hsm_status compute_mon_weights(hsm_plan p, uint8_t* status) {
  const int64_t G = p->mon.count;
  if (G == 0) return HSM_OK;
  OpsDesc ops = make_ops(p, p->op_mask);
  const int T = 128;
  int grid = (int)std::min<int64_t>(ceil_div(G, T), (int64_t)num_sms() * 16);
#define HSM_MON(D, O)                                                                                      \
  k_mon<D, O><<<grid, T, 0, p->stream>>>(p->coords, p->N, p->mon.idx, G, ops, p->mon.w64, status, p->mon.nodes, \
                                         p->dev_flags)
  if (p->dim == 2) {
    switch (p->nops) {
      case 1: HSM_MON(2, 1); break;
      case 2: HSM_MON(2, 2); break;
      default: HSM_MON(2, 3); break;
    }
  } else {
    switch (p->nops) {
      case 1: HSM_MON(3, 1); break;
      case 2: HSM_MON(3, 2); break;
      case 3: HSM_MON(3, 3); break;
      default: HSM_MON(3, 4); break;
    }
  }
#undef HSM_MON
  HSM_CUDA(p, cudaGetLastError());
  p->launches += 1;
  return HSM_OK;
}

hsm_status compute_rbf_weights_fp64(hsm_plan p, const int32_t* list, int64_t count, uint8_t* status) {
  return launch_rbf(p, false, list, count, status, nullptr, nullptr, 0);
}

hsm_status compute_rbf_weights_fp64_marked(hsm_plan p, const int32_t* list, int64_t count, uint8_t* status,
                                           uint8_t mark) {
  return launch_rbf(p, false, list, count, status, nullptr, nullptr, mark);
}

hsm_status compute_rbf_weights_fp32r(hsm_plan p, const int32_t* list, int64_t count, uint8_t* status,
                                     int32_t* fail_list, int* fail_count) {
  return launch_rbf(p, true, list, count, status, fail_list, fail_count, 0);
}

hsm_status weights_to_f32(hsm_plan p) {
  const int T = 256;
  for (Group* g : {&p->mon, &p->rbf}) {
    const int64_t n = (int64_t)p->nops * g->width * g->count;
    if (!n) continue;
    int grid = (int)std::min<int64_t>(ceil_div(n, T), (int64_t)num_sms() * 8);
    k_to_f32<2, 1><<<grid, T, 0, p->stream>>>(g->w64, g->w32, n);
    p->launches += 1;
    HSM_CUDA(p, cudaGetLastError());
  }
  return HSM_OK;
}

}  // namespace hsm
