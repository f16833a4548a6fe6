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
  int32_t* sing_list;      // fp64: positions whose system was singular (nullptr: not recorded)
  int* sing_count;
  int64_t sing_cap;        // entries sing_list holds; later ones are counted, not stored
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

// Per-system shared memory of the FP64 kernel (in doubles), m monomials,
// r = n - m, ldB = (r + NOPS) | 1:
//   xi    n x DIM          scaled offsets
//   rc    n                |xi_j|
//   Ap    max(n(n-1)/2 + 1, r ldB) A in pivot order, strict upper triangle
//                          packed by rows, then one zero for the diagonal (A
//                          is symmetric with a zero diagonal); later
//                          [S | Z^T b], then y
//   Pw    (n + NOPS) x m   LU of P; rows m..n-1 become X, rows n.. the
//                          monomial right-hand sides, then w_t
//   Bm    n x ldB          [A Z | f - A w_t]
//   inv   n                reciprocal pivots of P (m), then of S (r)
//   perm  n ints           stencil position of each pivot-order row
__host__ __device__ constexpr size_t ns_apsize(int nops, int n, int m) {
  return (size_t)n * (n - 1) / 2 + 1 > (size_t)(n - m) * ((n - m + nops) | 1)
             ? (size_t)n * (n - 1) / 2 + 1
             : (size_t)(n - m) * ((n - m + nops) | 1);
}
__host__ __device__ constexpr size_t sys_doubles(int dim, int nops, int n, int m) {
  return (size_t)n * (dim + 1) + ns_apsize(nops, n, m) + (size_t)(n + nops) * m + (size_t)n * ((n - m + nops) | 1) +
         n + (n + 1) / 2;
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

// Seeds for the FP64 iterations below are formed in single precision; the
// conversions between the formats are done on the integer pipes, which keeps
// them off the FP64 pipe, the bound of the weight kernels.
// f32_trunc: x truncated to single precision (relative error < 2^-23), for x
// whose binary exponent lies in single precision's normal range.
__device__ __forceinline__ float f32_trunc(double x) {
  const unsigned hi = (unsigned)__double2hiint(x);
  const unsigned lo = (unsigned)__double2loint(x);
  const unsigned mag = (((hi & 0x7fffffffu) - (896u << 20)) << 3) | (lo >> 29);
  return __uint_as_float(mag | (hi & 0x80000000u));
}
// f64_of: exact widening of a normal single-precision value.
__device__ __forceinline__ double f64_of(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned hi = (((b & 0x7fffffffu) >> 3) + (896u << 20)) | (b & 0x80000000u);
  return __hiloint2double((int)hi, (int)(b << 29));
}
// Biased binary exponent of x.
__device__ __forceinline__ unsigned f64_exp(double x) { return ((unsigned)__double2hiint(x) >> 20) & 0x7ffu; }
// x > 0 with its binary exponent within 120 of zero (the sign bit makes the
// shifted high word exceed the range), tested on the bits.
__device__ __forceinline__ bool f64_pos_in_f32(double x) {
  return ((unsigned)__double2hiint(x) >> 20) - (1023u - 120u) <= 240u;
}

// Reciprocal by the Newton-Raphson iteration y <- y + y (1 - x y), started
// from the single-precision reciprocal of x truncated to single precision:
// two steps take the seed's 2^-22 relative error below double rounding.
__device__ __forceinline__ double recip_core(double x) {
  double y = f64_of(__frcp_rn(f32_trunc(x)));
  double e = fma(-x, y, 1.0);
  y = fma(y, e, y);
  e = fma(-x, y, 1.0);
  return fma(y, e, y);
}
// 2^k for -1022 <= k <= 1023, from the bits.
__device__ __forceinline__ double pow2i(int k) { return __longlong_as_double((long long)(1023 + k) << 52); }
// Arguments outside single range are scaled by powers of two into it and
// back (exact); zeros, infinities and NaNs are answered from the bits.  No
// library division, whose out-of-line slow path would cost the kernels
// their registers.
__device__ __forceinline__ double recip(double x) {
  const unsigned ex = f64_exp(x);
  if (ex >= 1023u - 120u && ex <= 1023u + 120u) return recip_core(x);
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned long long sign = b & 0x8000000000000000ull;
  if (ex == 0x7ffu) return (b & 0x000fffffffffffffull) ? x : __longlong_as_double((long long)sign);
  if ((b << 1) == 0ull) return __longlong_as_double((long long)(sign | 0x7ff0000000000000ull));
  const double pre = ex == 0u ? 0x1p+64 : 1.0;  // subnormal: 1/x = 2^64 / (2^64 x)
  const double xs = x * pre;
  const int t = (int)f64_exp(xs) - 1023, t1 = t / 2, t2 = t - t1;
  return recip_core(xs * pow2i(-t1) * pow2i(-t2)) * pow2i(-t1) * pow2i(-t2) * pre;
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

// Square-root arguments outside single range: x = x1 4^k with x1 in range,
// sqrt x = 2^k sqrt x1 (exact scalings); zero, infinity and NaN return
// themselves, negative arguments NaN.
template <typename F>
__device__ __forceinline__ double sqrt_wide(double x, F&& core) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned ex = f64_exp(x);
  if ((b << 1) == 0ull || (ex == 0x7ffu && !(b >> 63))) return x;
  if (b >> 63) return __longlong_as_double(0x7ff8000000000000ll);
  const bool sub = ex == 0u;
  const double xs = sub ? x * 0x1p+64 : x;
  const int t = ((int)f64_exp(xs) - 1023) & ~1, t1 = t / 2, t2 = t - t1;
  const double r = core(xs * pow2i(-t1) * pow2i(-t2));
  return r * pow2i(t / 2) * (sub ? 0x1p-32 : 1.0);
}

// sqrt(x) for x > 0 by two steps of Goldschmidt's coupled iteration
//   r = 1/2 - g h,  g <- g + g r  (-> sqrt x),  h <- h + h r  (-> 1/(2 sqrt x)),
// started from the single-precision reciprocal square root (g = x y, h = y/2).
// Each step squares the relative error: ~2^-22 -> ~2^-43 -> below double
// rounding.  Arguments outside single precision's normal range go through
// sqrt_wide.
__device__ __forceinline__ double sqrt_gs_core(double x) {
  const double y = f64_of(rsqrtf(f32_trunc(x)));
  double g = x * y, h = 0.5 * y;
  double r = fma(-g, h, 0.5);
  g = fma(g, r, g);
  h = fma(h, r, h);
  r = fma(-g, h, 0.5);
  return fma(g, r, g);
}
__device__ __forceinline__ double sqrt_gs(double x) {
  if (!f64_pos_in_f32(x)) return sqrt_wide(x, [](double v) { return sqrt_gs_core(v); });
  return sqrt_gs_core(x);
}

// sqrt(x) by one Newton-Raphson step g + (x - g^2) / (2g) from the
// single-precision root g of x truncated to single precision.  The relative
// error is the seed's (below 2^-23) squared over two plus the seed's times
// that of the single-precision 1/(2g) (2^-24): below 1.5e-14.  Arguments
// outside single precision's normal range go through sqrt_wide.
__device__ __forceinline__ double sqrt_nr1_core(double x) {
  const float gf = sqrtf(f32_trunc(x));
  const double g = f64_of(gf);
  return fma(f64_of(0.5f * __frcp_rn(gf)), fma(-g, g, x), g);
}
__device__ __forceinline__ double sqrt_nr1(double x) {
  if (!f64_pos_in_f32(x)) return sqrt_wide(x, [](double v) { return sqrt_nr1_core(v); });
  return sqrt_nr1_core(x);
}

// Monomial q of the basis is monomial par[q] times coordinate cor[q] (the
// exponent vector minus one unit in its first non-zero coordinate), so each
// monomial costs one product.  par[q] = -1 for the constant and -2 where the
// basis lacks that lower monomial (such entries take the exponent loop).
// Filled by the block's first n_mono threads; the caller synchronises.
__device__ __forceinline__ void mono_parents(const int8_t* ex, int nm, int dim, int8_t* par, int8_t* cor) {
  const int q = threadIdx.x;
  if (q >= nm) return;
  int k0 = -1;
  for (int k = 0; k < dim; ++k)
    if (k0 < 0 && ex[q * dim + k] > 0) k0 = k;
  int pq = -1;
  if (k0 >= 0) {
    pq = -2;
    for (int p = 0; p < nm && pq == -2; ++p) {
      bool eq = true;
      for (int k = 0; k < dim; ++k) eq = eq && ex[p * dim + k] == ex[q * dim + k] - (k == k0 ? 1 : 0);
      if (eq) pq = p;
    }
  }
  par[q] = (int8_t)pq;
  cor[q] = (int8_t)(k0 < 0 ? 0 : k0);
}

// Monomials of node j into row[0..nm) (row[q] = p_q(xi_j)), by the parent
// table: linear terms are copies, every higher one is one multiplication.
template <int DIM, typename T>
__device__ __forceinline__ T mono_value(const T* row, const T* x, int q, const int8_t* par, const int8_t* cor,
                                        const int8_t* ex) {
  const int pq = par[q];
  if (pq == -1) return T(1);
  if (pq == 0) return x[cor[q]];
  if (pq > 0) return row[pq] * x[cor[q]];
  T v = T(1);
#pragma unroll
  for (int k = 0; k < DIM; ++k)
    for (int t = 0; t < ex[q * DIM + k]; ++t) v *= x[k];
  return v;
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

// Position of A[i][j], i < j, in the strict upper triangle of an n x n
// matrix packed by rows (the pair table's order).
__device__ __forceinline__ int tri_index(int n, int i, int j) { return ((i * (2 * n - i - 1)) >> 1) + (j - i - 1); }

// Calls f(i, j) for every (i, j) of [0, R) x [0, C), dealt to the lanes in
// row-major order so that every lane of each instruction has work.
template <int LANES, typename F>
__device__ __forceinline__ void flat2(int R, int C, int lane, F&& f) {
  const int total = R * C;
  if (total <= 0) return;
  int i = lane / C, j = lane - (lane / C) * C;
  const int dq = LANES / C, dr = LANES - (LANES / C) * C;
  for (int e = lane; e < total; e += LANES) {
    f(i, j);
    j += dr;
    i += dq;
    if (j >= C) {
      j -= C;
      ++i;
    }
  }
}

// FP64 RBF-FD weights of Eq. 1 by the null-space method for the saddle-point
// system [A P; P^T 0] [w; lambda] = [f; g] (Section 2.1).  Only w is needed:
//   1. P = Pi^T [L1; L2] U by Gaussian elimination with row pivoting (Pi the
//      row order, L1 unit lower m x m, L2 r x m, U upper);
//   2. every w with P^T w = g is w = Pi^T ([w_t; 0] + Z y), where
//      Z = [-X; I], X = L1^-T L2^T spans the null space of P^T and
//      w_t = L1^-T U^-T g;
//   3. (Z^T A Z) y = Z^T (f - A w_t): an r x r system, r = n - m.  r^3 is
//      conditionally positive definite of order 2 and the monomials include
//      all linear ones, so Z^T A Z is positive definite.
// In exact arithmetic this is the solution of the augmented system; it takes
// about half the FP64 operations of an LU of the (n + m) x (n + m) matrix.
// FP64 RBF-FD systems at positions t0, t0 + stride, ... < t_end of the
// launch's list, solved by the lane group whose system memory starts at xi
// (sys_doubles doubles); par and cor are the monomial parent tables of the
// block.  The group size (the stride of idx and w) is a.G, or G_arg when
// DEV_G (a size read on the device).
template <int DIM, int NOPS, int LANES, bool DEV_G = false>
__device__ __forceinline__ void rbf64_systems(const RbfArgs& a, int64_t t0, int64_t t_end, int64_t stride, int lane,
                                              unsigned mask, double* xi, const int8_t* par, const int8_t* cor,
                                              int64_t G_arg = 0) {
  const int n = a.n, m = a.n_mono, r = n - m, rc_ = r + NOPS;
  const int ldB = rc_ | 1;
  double* rc = xi + n * DIM;
  double* Ap = rc + n;
  double* Sm = Ap;  // Ap is dead once Bm is formed
  double* Pw = Ap + ns_apsize(NOPS, n, m);
  double* Bm = Pw + (n + NOPS) * m;
  double* inv = Bm + n * ldB;
  int* perm = reinterpret_cast<int*>(inv + n);
  for (int64_t t = t0; t < t_end; t += stride) {
    const int64_t pos = a.list ? a.list[t] : t;
    const int32_t c = a.nodes[pos];
    // ---- offsets, the power-of-two scale, |xi| and the monomial rows of P
    unsigned long long bmax = 0ull;
    for (int j = lane; j < n; j += LANES) {
      const int32_t id = a.idx[(int64_t)j * (DEV_G ? G_arg : a.G) + pos];
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
      bmax = rb > bmax ? rb : bmax;
    }
  #pragma unroll
    for (int o = LANES / 2; o > 0; o >>= 1) {
      const unsigned long long u = shfl_xor_u64(mask, bmax, o, LANES);
      bmax = u > bmax ? u : bmax;
    }
    const double inv_s = pow2_inv_scale(bmax);
    bool ok = bmax != 0ull && bmax < 0x7ff0000000000000ull;
    __syncwarp(mask);
    for (int j = lane; j < n; j += LANES) {
      double* x = xi + j * DIM;
  #pragma unroll
      for (int k = 0; k < DIM; ++k) x[k] *= inv_s;
      double* row = Pw + j * m;
      for (int q = 0; q < m; ++q) row[q] = mono_value<DIM, double>(row, x, q, par, cor, a.mono_exp);
      perm[j] = j;
    }
    // |xi_j| comes with the pair values (the centre, node 0, sits at xi = 0)
    if (lane == 0) rc[0] = 0.0;
    __syncwarp(mask);
    // ---- 1. P = Pi^T [L1; L2] U, whole rows swapped, multipliers in place
    for (int k = 0; k < m && ok; ++k) {
      unsigned long long best = 0ull;
      int brow = n;
      for (int i = k + lane; i < n; i += LANES) {
        const unsigned long long v = AbsBits<double>::get(Pw[i * m + k]);
        if (v > best || (v == best && i < brow)) {
          best = v;
          brow = i;
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
      if (brow != k && brow < n) {
        for (int j = lane; j < m; j += LANES) {
          const double tmp = Pw[k * m + j];
          Pw[k * m + j] = Pw[brow * m + j];
          Pw[brow * m + j] = tmp;
        }
        if (lane == 0) {
          const int tp = perm[k];
          perm[k] = perm[brow];
          perm[brow] = tp;
        }
      }
      __syncwarp(mask);
      const double piv = Pw[k * m + k];
      // a pivot below the threshold: the stencil is not unisolvent for the
      // monomials to working precision
      if (!pivot_ok<double>(piv)) {
        ok = false;
        break;
      }
      const double ip = recip(piv);
      if (lane == 0) inv[k] = ip;
      for (int i = k + 1 + lane; i < n; i += LANES) Pw[i * m + k] *= ip;
      __syncwarp(mask);
      const double* urow = Pw + k * m + k + 1;
      double* base = Pw + (k + 1) * m + k + 1;
      flat2<LANES>(n - k - 1, m - k - 1, lane, [&](int i, int j) {
        double* row = base + i * m;
        row[j] = fma(-row[-1], urow[j], row[j]);
      });
      __syncwarp(mask);
    }
    if (ok) {
      // ---- 2a. U^T z = g, column by column; z_i is finished (scaled by
      // 1/u_ii) by the step that removes its last term
      flat2<LANES>(NOPS, m, lane, [&](int o, int q) {
        const double g = rhs_mono<DIM>(a.mono_exp, q, a.ops.kind[o]);
        Pw[(n + o) * m + q] = q == 0 ? g * inv[0] : g;
      });
      __syncwarp(mask);
      for (int i = 0; i + 1 < m; ++i) {
        flat2<LANES>(NOPS, m - i - 1, lane, [&](int o, int tt) {
          const int q = i + 1 + tt;
          double* z = Pw + (n + o) * m;
          const double v = fma(-Pw[i * m + q], z[i], z[q]);
          z[q] = tt == 0 ? v * inv[q] : v;
        });
        __syncwarp(mask);
      }
      // ---- 2b. L1^T [X | w_t] = [L2^T | z]: rows m .. n + NOPS - 1 of Pw
      for (int i = m - 1; i > 0; --i) {
        flat2<LANES>(rc_, i, lane, [&](int cc, int q) {
          double* col = Pw + (m + cc) * m;
          col[q] = fma(-Pw[i * m + q], col[i], col[q]);
        });
        __syncwarp(mask);
      }
      // ---- A and f in pivot order
      const int npairs = n * (n - 1) / 2;
      for (int e = lane; e < npairs; e += LANES) {
        const uint16_t pr = a.pairs[e];
        const int i = pr >> 8, j = pr & 0xff;
        const int ni = perm[i], nj = perm[j];
        const double* xa = xi + ni * DIM;
        const double* xb = xi + nj * DIM;
        double d2 = 0.0;
  #pragma unroll
        for (int k = 0; k < DIM; ++k) {
          const double d = xa[k] - xb[k];
          d2 = fma(d, d, d2);
        }
        // one Newton step: the pair values' relative error (< 1e-14) moves
        // the weights by about 1e-12 on the worst-conditioned test sets
        const double g = sqrt_nr1(d2);
        Ap[e] = d2 * g;
        if (ni == 0) rc[nj] = g;
        if (nj == 0) rc[ni] = g;
      }
      if (lane == 0) Ap[npairs] = 0.0;
      __syncwarp(mask);
      flat2<LANES>(n, NOPS, lane, [&](int i, int o) { Bm[i * ldB + r + o] = rhs_phi<DIM>(xi, rc, perm[i], a.ops.kind[o]); });
      __syncwarp(mask);
      // ---- [A Z | f - A w_t]: column cc < r is A_{:,m+cc} - A_{:,0..m} X_{:,cc}
      {
        // (the flat loop written out: as a lambda it was not inlined)
        const int C = rc_;
        int i = lane / C, cc = lane - (lane / C) * C;
        const int dq = LANES / C, dr = LANES - (LANES / C) * C;
        for (int e = lane; e < n * C; e += LANES) {
          const double* xc = Pw + (m + cc) * m;
          double v;
          if (cc < r) {
            const int jc = m + cc;
            v = Ap[jc == i ? npairs : tri_index(n, min(i, jc), max(i, jc))];
          } else {
            v = Bm[i * ldB + cc];
          }
          // every lane runs the same m products; the diagonal A[i][i] = 0
          // is read from the zero kept after the triangle
          for (int q = 0; q < m; ++q) v = fma(-Ap[q == i ? npairs : tri_index(n, min(i, q), max(i, q))], xc[q], v);
          Bm[i * ldB + cc] = v;
          cc += dr;
          i += dq;
          if (cc >= C) {
            cc -= C;
            ++i;
          }
        }
      }
      __syncwarp(mask);
      // ---- [Z^T A Z | Z^T b] over Ap's storage
      flat2<LANES>(r, rc_, lane, [&](int j, int cc) {
        const double* xj = Pw + (m + j) * m;
        double v = Bm[(m + j) * ldB + cc];
        for (int q = 0; q < m; ++q) v = fma(-xj[q], Bm[q * ldB + cc], v);
        Sm[j * ldB + cc] = v;
      });
      __syncwarp(mask);
      // ---- 3. the r x r positive definite system: y in columns r ..
      ok = lu_solve<NOPS, LANES, double>(Sm, ldB, r, inv + m, lane, mask, true);
    }
    // ---- w = Pi^T ([w_t - X y; y]), unscaled, in stencil order
    if (ok) {
      const double inv_s2 = inv_s * inv_s;
      auto put = [&](int i, int o, double v) {
        v *= a.ops.kind[o] == 3 ? inv_s2 : inv_s;
        const bool fin = ((unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull) < 0x7ff0000000000000ull;
        a.w[((int64_t)o * n + perm[i]) * (DEV_G ? G_arg : a.G) + pos] = fin ? v : 0.0;
      };
      flat2<LANES>(m, NOPS, lane, [&](int i, int o) {
        double v = Pw[(n + o) * m + i];
        for (int j = 0; j < r; ++j) v = fma(-Pw[(m + j) * m + i], Sm[j * ldB + r + o], v);
        put(i, o, v);
      });
      flat2<LANES>(r, NOPS, lane, [&](int j, int o) { put(m + j, o, Sm[j * ldB + r + o]); });
    } else {
      flat2<LANES>(n, NOPS, lane,
                   [&](int i, int o) { a.w[((int64_t)o * n + i) * (DEV_G ? G_arg : a.G) + pos] = 0.0; });
    }
    if (lane == 0) {
      const int32_t node = a.nodes[pos];
      if (!ok) atomicOr(a.flags, kDevSingular);
      if (!ok && a.sing_list) {
        const int slot = atomicAdd(a.sing_count, 1);
        if (slot < a.sing_cap) a.sing_list[slot] = (int32_t)pos;
      }
      if (a.status)
        a.status[node] = !ok ? HSM_NODE_SINGULAR
                             : (a.status_demoted_mark ? a.status_demoted_mark
                                                      : (a.is_regular[node] ? HSM_NODE_DEMOTED : HSM_NODE_OK));
    }
    __syncwarp(mask);
  }
}

template <int DIM, int NOPS, int LANES>
__global__ void __launch_bounds__(256) k_rbf_fp64(RbfArgs a) {
  extern __shared__ double smem[];
  const int SYS = blockDim.x / LANES;
  const int sub = threadIdx.x / LANES, lane = threadIdx.x % LANES;
  const unsigned mask = LANES == 32 ? 0xffffffffu : (((1u << LANES) - 1u) << ((threadIdx.x & 31) / LANES * LANES));
  double* xi = smem + (size_t)sub * sys_doubles(DIM, NOPS, a.n, a.n_mono);
  __shared__ int8_t par[kMaxMonomials], cor[kMaxMonomials];
  mono_parents(a.mono_exp, a.n_mono, DIM, par, cor);
  __syncthreads();
  rbf64_systems<DIM, NOPS, LANES>(a, (int64_t)blockIdx.x * SYS + sub, a.count, (int64_t)gridDim.x * SYS, lane, mask,
                                  xi, par, cor);
}

// The same solve for chunk `chunk` of `nchunks` equal chunks of the whole
// group, whose size G is read on the device (the stencil build enqueues it
// before the group sizes reach the host): positions [chunk C, chunk C + C)
// clipped to G, C = ceil(G / nchunks).  Blocks past the chunk return at once.
template <int DIM, int NOPS, int LANES>
__global__ void __launch_bounds__(256) k_rbf_fp64_chunk(RbfArgs a, const int* __restrict__ G_dev, int chunk,
                                                         int nchunks) {
  extern __shared__ double smem[];
  const int64_t G = *G_dev;
  const int64_t C = (G + nchunks - 1) / nchunks;
  const int64_t lo = min(G, (int64_t)chunk * C), hi = min(G, lo + C);
  const int SYS = blockDim.x / LANES;
  if ((int64_t)blockIdx.x * SYS >= hi - lo) return;
  const int sub = threadIdx.x / LANES, lane = threadIdx.x % LANES;
  const unsigned mask = LANES == 32 ? 0xffffffffu : (((1u << LANES) - 1u) << ((threadIdx.x & 31) / LANES * LANES));
  double* xi = smem + (size_t)sub * sys_doubles(DIM, NOPS, a.n, a.n_mono);
  __shared__ int8_t par[kMaxMonomials], cor[kMaxMonomials];
  mono_parents(a.mono_exp, a.n_mono, DIM, par, cor);
  __syncthreads();
  rbf64_systems<DIM, NOPS, LANES, true>(a, lo + (int64_t)blockIdx.x * SYS + sub, hi, (int64_t)gridDim.x * SYS, lane,
                                        mask, xi, par, cor, G);
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
  __shared__ int8_t par[kMaxMonomials], cor[kMaxMonomials];
  mono_parents(a.mono_exp, a.n_mono, DIM, par, cor);
  __syncthreads();
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
    for (int j = lane; j < n; j += LANES) rc[j] = sqrt_gs(rc[j] * (inv_s * inv_s));
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
    for (int i = lane; i < n; i += LANES) {
      double* prow = P64 + i * M;
      float* frow = L32 + i * ld32 + n;
      for (int q = 0; q < M; ++q) {
        prow[q] = mono_value<DIM, double>(prow, xi + i * DIM, q, par, cor, a.mono_exp);
        const float vf = mono_value<DIM, float>(frow, xf + i * DIM, q, par, cor, a.mono_exp);
        frow[q] = vf;
        L32[(n + q) * ld32 + i] = vf;
      }
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
