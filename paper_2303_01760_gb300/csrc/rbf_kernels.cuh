// RBF-FD weight kernels of Eq. 1 (Section 2, Section 4): argument block,
// shared-memory layouts, assembly, the lane-group LU factorizations and the
// FP64 and FP32 + FP64-refinement kernels.  Included by weights.cu (kernels
// for any system size) and rbf_fixed.cu (compile-time system sizes).
#pragma once
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

__device__ __forceinline__ unsigned long long shfl_xor_u64(unsigned mask, unsigned long long v, int o, int w) {
  return (unsigned long long)__shfl_xor_sync(mask, (long long)v, o, w);
}

// Per-system shared memory of the FP64 kernel (in doubles):
//   M      K x ld     matrix, LU factor and right-hand sides
//   xi     n x DIM    scaled offsets
//   rc     n          |xi_j|, the scaled distance of node j from the centre
//   inv    K          reciprocal pivots
template <int DIM, int NOPS, bool R32>
__host__ __device__ constexpr size_t sys_doubles(int K, int ld, int n) {
  return (size_t)K * ld + (size_t)n * (DIM + 1) + K;
}

// Per-system shared memory of the FP32 + FP64-refinement kernel: the FP64
// data first, then the FP32 factor (M = K - n monomials).
//   xi    n x DIM    scaled offsets                     (double)
//   rc    n          |xi_j|                             (double)
//   A64   n(n-1)/2   r^3 of every pair i < j, in pair-table order (double)
//   P64   n x M      monomials at xi                    (double)
//   x64   K x NOPS   current solution                   (double)
//   xf    n x DIM    xi rounded to FP32                 (float)
//   L32   K x ld32   FP32 matrix / LU factor, right-hand sides (float)
//   piv   K          reciprocal FP32 pivots             (float)
//   perm  K          equation order of the factor rows  (int)
//   iperm K          factor row of each equation        (int)
__host__ __device__ constexpr size_t r32_doubles(int dim, int nops, int K, int n) {
  return (size_t)n * dim + n + (size_t)n * (n - 1) / 2 + (size_t)n * (K - n) + (size_t)K * nops +
         ((size_t)n * dim + (size_t)K * ((K + nops) | 1) + 3 * (size_t)K + 1) / 2;
}

// Inverse scale 2^-t for the largest squared offset d2max in [2^e, 2^(e+1)):
// t = floor((e+1)/2) puts max |xi| in [2^-1/2, 2^1/2).  A power of two makes
// the scaling and unscaling exact; the weights do not depend on the scale.
__device__ __forceinline__ double pow2_inv_scale(unsigned long long d2bits) {
  const int e = (int)((d2bits >> 52) & 0x7ff) - 1023;
  const int t = (e + 1 + 2048) / 2 - 1024;
  return __longlong_as_double((long long)(1023 - t) << 52);
}

// Reciprocal by the Newton-Raphson iteration y <- y + y (1 - x y), started
// from the correctly rounded single-precision reciprocal: two steps take the
// seed's 2^-24 relative error below double rounding.  Arguments whose
// exponent lies outside single range take the division.
__device__ __forceinline__ double recip(double x) {
  const unsigned ex = (unsigned)((unsigned long long)__double_as_longlong(x) >> 52) & 0x7ffu;
  if (ex < 1023u - 120u || ex > 1023u + 120u) return 1.0 / x;
  double y = (double)__frcp_rn((float)x);
  double e = fma(-x, y, 1.0);
  y = fma(y, e, y);
  e = fma(-x, y, 1.0);
  return fma(y, e, y);
}
__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }

// |pivot| above the singularity threshold and finite, tested on the bits.
template <typename T>
__device__ __forceinline__ bool pivot_ok(T piv);
template <>
__device__ __forceinline__ bool pivot_ok<double>(double piv) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(piv) & 0x7fffffffffffffffull;
  return b > 0x3d719799812dea11ull /* 1e-12 */ && b < 0x7ff0000000000000ull;
}
template <>
__device__ __forceinline__ bool pivot_ok<float>(float piv) {
  const unsigned b = __float_as_uint(piv) & 0x7fffffffu;
  return b > 0u && b < 0x7f800000u;
}

// Assembles [A P | L phi; P^T 0 | L p] into Mt (row stride ld) for the scaled
// offsets xi = (x - x_c) * inv_s, inv_s a power of two (pow2_inv_scale).
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
      const double o = a.coords[k * a.N + id] - a.coords[k * a.N + c];
      xi[j * DIM + k] = o;
      r2 = fma(o, o, r2);
    }
    rc[j] = r2;
    // non-negative doubles order like their bit patterns
    const unsigned long long rb = (unsigned long long)__double_as_longlong(r2);
    b = rb > b ? rb : b;
  }
#pragma unroll
  for (int o = LANES / 2; o > 0; o >>= 1) {
    unsigned long long t = shfl_xor_u64(mask, b, o, LANES);
    b = t > b ? t : b;
  }
  const double inv_s = pow2_inv_scale(b);
  inv_s_out = inv_s;
  ok = b != 0ull && b < 0x7ff0000000000000ull;
  __syncwarp(mask);
  for (int e = lane; e < n * DIM; e += LANES) xi[e] *= inv_s;
  for (int e = lane; e < n; e += LANES) rc[e] = sqrt(rc[e] * (inv_s * inv_s));
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
      if (!pivot_ok<T>(piv)) {
        ok = false;
        break;
      }
      const T ip = recip(piv);
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

// LU with partial pivoting of a K x (K + NOPS) row-major system in shared
// memory (row stride LD), every loop bound known at compile time.  Step k
// deals the active columns k+1 .. C-1 to the lanes as k+1+lane+LANES*c, so a
// lane's share shrinks with the active block, the pivot-row values sit in
// registers for the whole step and every address is an immediate offset from
// a per-lane base.  Whole rows are swapped so the stored multipliers stay with
// their equation; perm records the equation order of the factor rows.
template <int K, int NOPS, int LANES, typename T>
struct FixedLU {
  static constexpr int C = K + NOPS;
  static constexpr int LD = C | 1;

  __device__ static bool factor(T* M, T* inv, int* perm, int lane, unsigned mask) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      unsigned long long best = 0ull;
      int brow = K;
#pragma unroll
      for (int c = 0; c < (K - k + LANES - 1) / LANES; ++c) {
        const int i = k + lane + LANES * c;
        if (c < (K - k) / LANES || i < K) {
          const unsigned long long v = AbsBits<T>::get(M[i * LD + k]);
          if (v > best) {
            best = v;
            brow = i;
          }
        }
      }
#pragma unroll
      for (int o = LANES / 2; o > 0; o >>= 1) {
        const unsigned long long ob = shfl_xor_u64(mask, best, o, LANES);
        const int orow = __shfl_xor_sync(mask, brow, o, LANES);
        if (ob > best || (ob == best && orow < brow)) {
          best = ob;
          brow = orow;
        }
      }
      if (brow != k && brow < K) {
#pragma unroll
        for (int c = 0; c < (C + LANES - 1) / LANES; ++c) {
          const int j = lane + LANES * c;
          if (c < C / LANES || j < C) {
            const T t = M[k * LD + j];
            M[k * LD + j] = M[brow * LD + j];
            M[brow * LD + j] = t;
          }
        }
        if (perm && lane == 0) {
          const int t = perm[k];
          perm[k] = perm[brow];
          perm[brow] = t;
        }
      }
      __syncwarp(mask);
      const T piv = M[k * LD + k];
      if (!pivot_ok<T>(piv)) return false;
      const T ip = recip(piv);
      if (lane == 0) inv[k] = ip;
#pragma unroll
      for (int c = 0; c < (K - 1 - k + LANES - 1) / LANES; ++c) {
        const int i = k + 1 + lane + LANES * c;
        if (c < (K - 1 - k) / LANES || i < K) M[i * LD + k] *= ip;
      }
      // active columns NA and chunks NC: constants once the k loop is unrolled
      const int NA = C - 1 - k;
      const int NC = (NA + LANES - 1) / LANES;
      constexpr int NCMAX = (C - 1 + LANES - 1) / LANES;
      T pr[NCMAX];
#pragma unroll
      for (int c = 0; c < NCMAX; ++c) {
        const int j = k + 1 + lane + LANES * c;
        if (c < NC) pr[c] = (c < NA / LANES || j < C) ? M[k * LD + j] : T(0);
      }
      __syncwarp(mask);
#pragma unroll
      for (int i = k + 1; i < K; ++i) {
        const T l = M[i * LD + k];
#pragma unroll
        for (int c = 0; c < NCMAX; ++c) {
          const int j = k + 1 + lane + LANES * c;
          if (c < NC && (c < NA / LANES || j < C)) M[i * LD + j] = fma(-l, pr[c], M[i * LD + j]);
        }
      }
      __syncwarp(mask);
    }
    return true;
  }

  // Forward elimination of the right-hand-side columns with the stored
  // multipliers (rows already in the factor's order).
  __device__ static void forward(T* M, int lane, unsigned mask) {
#pragma unroll
    for (int k = 0; k < K - 1; ++k) {
      T rk[NOPS];
#pragma unroll
      for (int o = 0; o < NOPS; ++o) rk[o] = M[k * LD + K + o];
#pragma unroll
      for (int c = 0; c < (K - 1 - k + LANES - 1) / LANES; ++c) {
        const int i = k + 1 + lane + LANES * c;
        if (c < (K - 1 - k) / LANES || i < K) {
          const T l = M[i * LD + k];
#pragma unroll
          for (int o = 0; o < NOPS; ++o) M[i * LD + K + o] = fma(-l, rk[o], M[i * LD + K + o]);
        }
      }
      __syncwarp(mask);
    }
  }

  // Back substitution; the solution overwrites the right-hand-side columns.
  __device__ static void backward(T* M, const T* inv, int lane, unsigned mask) {
#pragma unroll
    for (int k = K - 1; k >= 0; --k) {
      const T ik = inv[k];
      T xk[NOPS];
#pragma unroll
      for (int o = 0; o < NOPS; ++o) xk[o] = M[k * LD + K + o] * ik;
#pragma unroll
      for (int c = 0; c < (k + LANES - 1) / LANES; ++c) {
        const int i = lane + LANES * c;
        if (c < k / LANES || i < k) {
          const T u = M[i * LD + k];
#pragma unroll
          for (int o = 0; o < NOPS; ++o) M[i * LD + K + o] = fma(-u, xk[o], M[i * LD + K + o]);
        }
      }
      if (lane < NOPS) {
#pragma unroll
        for (int o = 0; o < NOPS; ++o)
          if (o == lane) M[k * LD + K + o] = xk[o];
      }
      __syncwarp(mask);
    }
  }
};

template <int DIM, int NOPS, int LANES>
__global__ void __launch_bounds__(256) k_rbf_fp64(RbfArgs a) {
  extern __shared__ double smem[];
  const int SYS = blockDim.x / LANES;
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
    // the flat (row, column) update of lu_solve fills every lane of each FP64
    // instruction, which matters more here than its index arithmetic
    ok = lu_solve<NOPS, LANES, double>(M, ld, K, inv, lane, mask, true) && ok;
    for (int e = lane; e < n * NOPS; e += LANES) {
      const int j = e / NOPS, o = e - (e / NOPS) * NOPS;
      const double sc = a.ops.kind[o] == 3 ? inv_s * inv_s : inv_s;
      const double v = M[j * ld + K + o] * sc;
      const bool fin = ((unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull) < 0x7ff0000000000000ull;
      a.w[((int64_t)o * n + j) * a.G + pos] = ok && fin ? v : 0.0;
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

// FP32 factorization with FP64 iterative refinement.  The FP32 matrix is
// assembled in FP32 from the rounded offsets; FP64 holds only what the
// residual r = b - M x needs (offsets, |xi|, the pair values r^3, the
// monomials and the solution).  The residual skips the zero block and reads
// the symmetric A block from its upper triangle.
template <int DIM, int NOPS, int LANES, int KF>
__global__ void __launch_bounds__(256) k_rbf_fp32r(RbfArgs a) {
  extern __shared__ double smem[];
  const int SYS = blockDim.x / LANES;
  constexpr int kMaxIt = 3;
  const int sub = threadIdx.x / LANES, lane = threadIdx.x % LANES;
  const unsigned mask = LANES == 32 ? 0xffffffffu : (((1u << LANES) - 1u) << ((threadIdx.x & 31) / LANES * LANES));
  const int K = a.K, n = a.n, M = a.n_mono;
  const int ld32 = (K + NOPS) | 1;
  const int npairs = n * (n - 1) / 2;
  double* xi = smem + (size_t)sub * r32_doubles(DIM, NOPS, K, n);
  double* rc = xi + n * DIM;
  double* A64 = rc + n;
  double* P64 = A64 + npairs;
  double* x64 = P64 + n * M;
  float* xf = reinterpret_cast<float*>(x64 + K * NOPS);
  float* L32 = xf + n * DIM;
  float* piv = L32 + K * ld32;
  int* perm = reinterpret_cast<int*>(piv + K);
  int* iperm = perm + K;
  for (int64_t t = (int64_t)blockIdx.x * SYS + sub; t < a.count; t += (int64_t)gridDim.x * SYS) {
    const int64_t pos = a.list ? a.list[t] : t;
    const int32_t c = a.nodes[pos];
    // ---- offsets and the scale
    unsigned long long bmax = 0ull;
    for (int j = lane; j < n; j += LANES) {
      const int32_t id = a.idx[(int64_t)j * a.G + pos];
      double r2 = 0.0;
#pragma unroll
      for (int k = 0; k < DIM; ++k) {
        const double o = a.coords[k * a.N + id] - a.coords[k * a.N + c];
        xi[j * DIM + k] = o;
        r2 = fma(o, o, r2);
      }
      rc[j] = r2;
      const unsigned long long rb = (unsigned long long)__double_as_longlong(r2);
      bmax = rb > bmax ? rb : bmax;
    }
#pragma unroll
    for (int o = LANES / 2; o > 0; o >>= 1) {
      const unsigned long long u = shfl_xor_u64(mask, bmax, o, LANES);
      bmax = u > bmax ? u : bmax;
    }
    bool ok = bmax != 0ull && bmax < 0x7ff0000000000000ull;
    const double inv_s = pow2_inv_scale(bmax);
    __syncwarp(mask);
    for (int e = lane; e < n * DIM; e += LANES) {
      const double v = xi[e] * inv_s;
      xi[e] = v;
      xf[e] = (float)v;
    }
    for (int j = lane; j < n; j += LANES) rc[j] = sqrt(rc[j] * (inv_s * inv_s));
    __syncwarp(mask);
    // ---- pair values: r^3 in FP64 (kept) and in FP32 (into the matrix)
    for (int e = lane; e < npairs; e += LANES) {
      const uint16_t pr = a.pairs[e];
      const int i = pr >> 8, j = pr & 0xff;
      double d2 = 0.0;
      float f2 = 0.f;
#pragma unroll
      for (int k = 0; k < DIM; ++k) {
        const double d = xi[i * DIM + k] - xi[j * DIM + k];
        d2 = fma(d, d, d2);
        const float df = xf[i * DIM + k] - xf[j * DIM + k];
        f2 = fmaf(df, df, f2);
      }
      // r = sqrt(d2) by one step of the coupled (Goldschmidt) Newton-Raphson
      // iteration g <- g + h (d2 - g^2), h ~ 1/(2g), from the single-precision
      // root of the FP32 distance: relative error ~1e-12, which moves the
      // refinement's fixed point by about cond * 1e-12
      const float gf = sqrtf(f2);
      double g = (double)gf;
      g = fma((double)(0.5f / gf), fma(-g, g, d2), g);
      A64[e] = d2 * g;
      const float vf = f2 * gf;
      L32[i * ld32 + j] = vf;
      L32[j * ld32 + i] = vf;
    }
    for (int i = lane; i < n; i += LANES) L32[i * ld32 + i] = 0.f;
    // ---- monomial block (FP64 kept, FP32 into the matrix) and its zero block
    for (int e = lane; e < n * M; e += LANES) {
      const int i = e / M, q = e - (e / M) * M;
      double v = 1.0;
      float vf = 1.f;
#pragma unroll
      for (int k = 0; k < DIM; ++k) {
        const int ex = a.mono_exp[q * DIM + k];
        for (int u = 0; u < ex; ++u) {
          v *= xi[i * DIM + k];
          vf *= xf[i * DIM + k];
        }
      }
      P64[e] = v;
      L32[i * ld32 + n + q] = vf;
      L32[(n + q) * ld32 + i] = vf;
    }
    for (int e = lane; e < M * M; e += LANES) {
      const int i = e / M, q = e - (e / M) * M;
      L32[(n + i) * ld32 + n + q] = 0.f;
    }
    // ---- FP32 right-hand sides
    for (int e = lane; e < K * NOPS; e += LANES) {
      const int i = e / NOPS, o = e - (e / NOPS) * NOPS;
      const int kind = a.ops.kind[o];
      float v;
      if (i < n) {
        float r2 = 0.f;
#pragma unroll
        for (int k = 0; k < DIM; ++k) r2 = fmaf(xf[i * DIM + k], xf[i * DIM + k], r2);
        const float r = sqrtf(r2);
        v = kind == 3 ? 3.f * (DIM + 1) * r : -3.f * r * xf[i * DIM + kind];
      } else {
        v = (float)rhs_mono<DIM>(a.mono_exp, i - n, kind);
      }
      L32[i * ld32 + K + o] = v;
    }
    for (int i = lane; i < K; i += LANES) perm[i] = i;
    __syncwarp(mask);
    if constexpr (KF > 0) {
      ok = ok && FixedLU<KF, NOPS, LANES, float>::factor(L32, piv, perm, lane, mask);
      if (ok) FixedLU<KF, NOPS, LANES, float>::backward(L32, piv, lane, mask);
    } else {
      ok = lu_solve<NOPS, LANES, float>(L32, ld32, K, piv, lane, mask, true, perm) && ok;
    }
    bool conv = false;
    if (ok) {
      for (int e = lane; e < K * NOPS; e += LANES) {
        const int i = e / NOPS, o = e - (e / NOPS) * NOPS;
        x64[e] = (double)L32[i * ld32 + K + o];
      }
      for (int kf = lane; kf < K; kf += LANES) iperm[perm[kf]] = kf;
      __syncwarp(mask);
      for (int it = 0; it < kMaxIt && !conv; ++it) {
        // residual of the PHS rows, then of the monomial rows, written into
        // the FP32 right-hand-side columns in the factor's row order
        for (int e = lane; e < n * NOPS; e += LANES) {
          const int i = e / NOPS, o = e - (e / NOPS) * NOPS;
          double r = rhs_phi<DIM>(xi, rc, i, a.ops.kind[o]);
          // pairs (j, i), j < i: index of (j, i) in the pair table
          int pj = i - 1;
          for (int j = 0; j < i; ++j) {
            r = fma(-A64[pj], x64[j * NOPS + o], r);
            pj += n - j - 2;
          }
          // pairs (i, j), j > i: contiguous from (i, i+1)
          const double* Ai = A64 + (i * (2 * n - i - 1)) / 2 - (i + 1);
          for (int j = i + 1; j < n; ++j) r = fma(-Ai[j], x64[j * NOPS + o], r);
          const double* Pi = P64 + i * M;
          for (int q = 0; q < M; ++q) r = fma(-Pi[q], x64[(n + q) * NOPS + o], r);
          L32[iperm[i] * ld32 + K + o] = (float)r;
        }
        for (int e = lane; e < M * NOPS; e += LANES) {
          const int q = e / NOPS, o = e - (e / NOPS) * NOPS;
          double r = rhs_mono<DIM>(a.mono_exp, q, a.ops.kind[o]);
          for (int j = 0; j < n; ++j) r = fma(-P64[j * M + q], x64[j * NOPS + o], r);
          L32[iperm[n + q] * ld32 + K + o] = (float)r;
        }
        __syncwarp(mask);
        if constexpr (KF > 0) {
          FixedLU<KF, NOPS, LANES, float>::forward(L32, lane, mask);
          FixedLU<KF, NOPS, LANES, float>::backward(L32, piv, lane, mask);
        } else {
          lu_solve<NOPS, LANES, float>(L32, ld32, K, piv, lane, mask, false);
        }
        // x += d ; converged when max|d| <= 3e-4 max|x| for every operator
        unsigned long long dmax[NOPS], xmax[NOPS];
#pragma unroll
        for (int o = 0; o < NOPS; ++o) dmax[o] = xmax[o] = 0ull;
        for (int e = lane; e < K * NOPS; e += LANES) {
          const int i = e / NOPS, o = e - (e / NOPS) * NOPS;
          const float d = L32[i * ld32 + K + o];
          const double x = x64[e] + (double)d;
          x64[e] = x;
          const unsigned long long bd = AbsBits<float>::get(d), bx = AbsBits<double>::get(x);
#pragma unroll
          for (int q = 0; q < NOPS; ++q)
            if (q == o) {
              dmax[q] = bd > dmax[q] ? bd : dmax[q];
              xmax[q] = bx > xmax[q] ? bx : xmax[q];
            }
        }
        bool cv = true;
#pragma unroll
        for (int o = 0; o < NOPS; ++o) {
#pragma unroll
          for (int sh = LANES / 2; sh > 0; sh >>= 1) {
            const unsigned long long t1 = shfl_xor_u64(mask, dmax[o], sh, LANES);
            const unsigned long long t2 = shfl_xor_u64(mask, xmax[o], sh, LANES);
            dmax[o] = t1 > dmax[o] ? t1 : dmax[o];
            xmax[o] = t2 > xmax[o] ? t2 : xmax[o];
          }
          const double dm = (double)__uint_as_float((unsigned)dmax[o]);
          const double xm = __longlong_as_double((long long)xmax[o]);
          cv = cv && xmax[o] < 0x7ff0000000000000ull && dm <= 3e-4 * xm;
        }
        conv = cv;
        __syncwarp(mask);
      }
    }
    const bool good = ok && conv;
    for (int e = lane; e < n * NOPS; e += LANES) {
      const int j = e / NOPS, o = e - (e / NOPS) * NOPS;
      const double sc = a.ops.kind[o] == 3 ? inv_s * inv_s : inv_s;
      a.w[((int64_t)o * n + j) * a.G + pos] = good ? x64[e] * sc : 0.0;
    }
    if (lane == 0) {
      const int32_t node = a.nodes[pos];
      if (!good) {
        int slot = atomicAdd(a.fail_count, 1);
        a.fail_list[slot] = (int32_t)pos;
      } else if (a.status) {
        a.status[node] = a.status_demoted_mark
                             ? a.status_demoted_mark
                             : (a.is_regular[node] ? HSM_NODE_DEMOTED : HSM_NODE_OK);
      }
    }
    __syncwarp(mask);
  }
}

}  // namespace
}  // namespace hsm
