// Aggregation multigrid for the pressure operator of the Boussinesq step
// (Section 3: the Poisson problem of Chorin's projection), the right
// preconditioner of its BiCGSTAB solve.
//
// Aggregates are geometric: level l+1 groups the rows of level l whose nodes
// fall into one cell of edge 2^(l+1) h.  Cell indices of every level are the
// finest cell indices shifted right by l, so the cells nest exactly, and each
// aggregate is numbered by the rank of its lowest node id, which makes the
// hierarchy independent of thread timing.  Prolongation is piecewise
// constant; the coarse operators are the Galerkin products A_c = P^T A P,
// assembled one coarse row per thread from its member rows in ascending
// order.  Coarsening stops at kMgCoarsest rows, whose bordered system
// [A_c 1; 1^T 0] (the Neumann operator's constant null space, as in the fine
// bordered system) is inverted densely once.
//
// The cycle is V(2,2) with damped Jacobi (omega = 2/3); the coarse correction
// is scaled by alpha, the over-correction plain aggregation needs (1.8 in 2D,
// 1.5 in 3D, set on the seeded node sets).  Everything is FP64: rounding of an
// FP32 cycle makes the preconditioner slightly nonlinear, and BiCGSTAB then
// needed 1.6x the iterations.
#include <algorithm>
#include <vector>

#include "amg.cuh"

namespace hsm {
namespace {

constexpr unsigned long long kEmptyKey = ~0ull;
constexpr int kMaxProbe = 256;

// Grid-stride over the rows of a level: blocks [0, bm) take group 0, the rest group 1.
__device__ __forceinline__ void mg_rows(const MgLevel& L, int& g, int64_t& p, int64_t& stride) {
  if ((int)blockIdx.x < L.bm) {
    g = 0;
    p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    stride = (int64_t)L.bm * blockDim.x;
  } else {
    g = 1;
    p = (blockIdx.x - L.bm) * (int64_t)blockDim.x + threadIdx.x;
    stride = (int64_t)(gridDim.x - L.bm) * blockDim.x;
  }
}
__device__ __forceinline__ int64_t mg_row_id(const MgLevel& L, int g, int64_t p) {
  return L.nodes[g] ? (int64_t)L.nodes[g][p] : p;
}
__device__ __forceinline__ void mg_locate(const MgLevel& L, int64_t r, int& g, int64_t& p) {
  if (L.kind) {
    g = L.kind[r];
    p = L.pos[r];
  } else {
    g = 0;
    p = r;
  }
}
// sum over the W entries e of an ELL row ([W][G] column-major, position p) of
// val[e] * t(idx[e]), accumulated with FMAs in the order e = 0, 1, ...
// (Loading the entries eight at a time before the FMAs made the cycle slower:
// the padding of short rows cost loads and FP64 work, and the compiler
// already overlaps the loads of this loop.)
template <class TF>
__device__ __forceinline__ double ell_dot(const int32_t* __restrict__ idx, const double* __restrict__ val,
                                          int64_t G, int64_t p, int W, TF term) {
  double s = 0.0;
  for (int e = 0; e < W; ++e) s = fma(val[(int64_t)e * G + p], term(idx[(int64_t)e * G + p]), s);
  return s;
}

__device__ __forceinline__ double row_dot(const MgLevel& L, int g, int64_t p, const double* __restrict__ x) {
  return ell_dot(L.idx[g], L.val[g], L.count[g], p, L.width[g], [&](int32_t j) { return x[j]; });
}

// ---- cycle -------------------------------------------------------------------
// x = w f + w (f - A w f), w = omega D^-1: two Jacobi sweeps from zero.
__global__ void __launch_bounds__(kMgThreads) k_mg_pre(MgLevel L, const double* __restrict__ f, const double* done) {
  if (done && *done != 0.0) return;
  int g;
  int64_t p, stride;
  mg_rows(L, g, p, stride);
  const int W = L.width[g];
  const int64_t G = L.count[g];
  for (; p < G; p += stride) {
    const int64_t i = mg_row_id(L, g, p);
    const double acc = ell_dot(L.idx[g], L.val[g], G, p, W, [&](int32_t j) { return L.odinv[j] * f[j]; });
    const double fi = f[i], di = L.odinv[i];
    L.x[i] = di * fi + di * (fi - acc);
  }
}

// fc[I] = sum over the rows r of aggregate I of (f - A x)_r (fixed order).
// Up to kBatch rows are fetched level by level (row ids, their place in the
// matrix, then their stencils) so their dependent loads overlap.
__global__ void __launch_bounds__(kMgThreads) k_mg_restrict(MgLevel L, const double* __restrict__ f,
                                                            double* __restrict__ fc, int64_t nc, const double* done) {
  constexpr int kBatch = 8;
  if (done && *done != 0.0) return;
  for (int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; I < nc; I += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    const int32_t m1 = L.mstart[I + 1];
    for (int32_t m0 = L.mstart[I]; m0 < m1; m0 += kBatch) {
      int32_t r[kBatch], g[kBatch];
      int64_t pp[kBatch];
#pragma unroll
      for (int k = 0; k < kBatch; ++k) r[k] = m0 + k < m1 ? L.mlist[m0 + k] : -1;
#pragma unroll
      for (int k = 0; k < kBatch; ++k)
        if (r[k] >= 0) mg_locate(L, r[k], g[k], pp[k]);
#pragma unroll
      for (int k = 0; k < kBatch; ++k)
        if (r[k] >= 0) s += f[r[k]] - row_dot(L, g[k], pp[k], L.x);
    }
    fc[I] = s;
  }
}

// y = x' + w (f - A x'), x' = x + alpha P xc (prolongation on the fly).
__global__ void __launch_bounds__(kMgThreads) k_mg_post1(MgLevel L, const double* __restrict__ f,
                                                         const double* __restrict__ xc, double alpha,
                                                         const double* done) {
  if (done && *done != 0.0) return;
  int g;
  int64_t p, stride;
  mg_rows(L, g, p, stride);
  const int W = L.width[g];
  const int64_t G = L.count[g];
  for (; p < G; p += stride) {
    const int64_t i = mg_row_id(L, g, p);
    const double acc =
        ell_dot(L.idx[g], L.val[g], G, p, W, [&](int32_t j) { return fma(alpha, xc[L.agg[j]], L.x[j]); });
    const double xi = fma(alpha, xc[L.agg[i]], L.x[i]);
    L.y[i] = fma(L.odinv[i], f[i] - acc, xi);
  }
}

// out = y + w (f - A y); on level 0 the border entry passes through.
__global__ void __launch_bounds__(kMgThreads) k_mg_post2(MgLevel L, const double* __restrict__ f,
                                                         double* __restrict__ out, int border,
                                                         const double* done) {
  if (done && *done != 0.0) return;
  int g;
  int64_t p, stride;
  mg_rows(L, g, p, stride);
  for (; p < L.count[g]; p += stride) {
    const int64_t i = mg_row_id(L, g, p);
    out[i] = fma(L.odinv[i], f[i] - row_dot(L, g, p, L.y), L.y[i]);
  }
  if (border && blockIdx.x == 0 && threadIdx.x == 0) out[L.n] = f[L.n];
}

// x = Binv f, one warp per row; border >= 0 copies f[border] to x[border].
__global__ void __launch_bounds__(kMgThreads) k_mg_coarse(const double* __restrict__ binv, int m,
                                                          const double* __restrict__ f, double* __restrict__ x,
                                                          int64_t border, const double* done) {
  if (done && *done != 0.0) return;
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t r = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); r < m; r += warps) {
    double s = 0.0;
    for (int c = lane; c < m; c += 32) s = fma(binv[r * m + c], f[c], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) x[r] = s;
  }
  if (border >= 0 && blockIdx.x == 0 && threadIdx.x == 0) x[border] = f[border];
}

// ---- V(1,1): one sweep each way ------------------------------------------------
// Pre-smoothing from zero is x = w f, with no gather; the down phase stores
// it and restricts the residual: fc[I] = sum over the rows r of I of
// (f - A w f)_r (fixed order).
__global__ void __launch_bounds__(kMgThreads) k_mg_restrict1(MgLevel L, const double* __restrict__ f,
                                                             double* __restrict__ fc, int64_t nc,
                                                             const double* done) {
  if (done && *done != 0.0) return;
  for (int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; I < nc; I += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    const int32_t m1 = L.mstart[I + 1];
    for (int32_t m0 = L.mstart[I]; m0 < m1; ++m0) {
      const int32_t r = L.mlist[m0];
      int g;
      int64_t p;
      mg_locate(L, r, g, p);
      const double fr = f[r];
      L.x[r] = L.odinv[r] * fr;
      s += fr - ell_dot(L.idx[g], L.val[g], L.count[g], p, L.width[g],
                        [&](int32_t j) { return L.odinv[j] * f[j]; });
    }
    fc[I] = s;
  }
}

// The one post-smoothing sweep: out = x' + w (f - A x'), x' = x + alpha P xc
// (k_mg_post1's formula), written to out; on level 0 the border entry passes.
__global__ void __launch_bounds__(kMgThreads) k_mg_post1o(MgLevel L, const double* __restrict__ f,
                                                          const double* __restrict__ xc, double alpha,
                                                          double* __restrict__ out, int border, const double* done) {
  if (done && *done != 0.0) return;
  int g;
  int64_t p, stride;
  mg_rows(L, g, p, stride);
  const int W = L.width[g];
  const int64_t G = L.count[g];
  for (; p < G; p += stride) {
    const int64_t i = mg_row_id(L, g, p);
    const double acc =
        ell_dot(L.idx[g], L.val[g], G, p, W, [&](int32_t j) { return fma(alpha, xc[L.agg[j]], L.x[j]); });
    const double xi = fma(alpha, xc[L.agg[i]], L.x[i]);
    out[i] = fma(L.odinv[i], f[i] - acc, xi);
  }
  if (border && blockIdx.x == 0 && threadIdx.x == 0) out[L.n] = f[L.n];
}

// ---- fused forms: two phases of a level in one kernel -------------------------
// On the small levels a kernel is one chain of dependent L2 loads and costs a
// launch; the fused forms recompute the first phase's values at a row's
// stencil neighbours instead of waiting for another kernel (the matrix rows
// are read twice, the launches halve).  Same formulas, same term order.
__device__ __forceinline__ double pre_x(const MgLevel& L, const double* __restrict__ f, int64_t j) {
  int g;
  int64_t p;
  mg_locate(L, j, g, p);
  const double acc =
      ell_dot(L.idx[g], L.val[g], L.count[g], p, L.width[g], [&](int32_t k) { return L.odinv[k] * f[k]; });
  const double fj = f[j], dj = L.odinv[j];
  return dj * fj + dj * (fj - acc);
}

// k_mg_pre + k_mg_restrict: x of the aggregate's rows (stored for the way
// up) and fc[I] = sum over the rows r of I of (f - A x)_r.
__global__ void __launch_bounds__(kMgThreads) k_mg_down(MgLevel L, const double* __restrict__ f,
                                                        double* __restrict__ fc, int64_t nc, const double* done) {
  if (done && *done != 0.0) return;
  for (int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; I < nc; I += (int64_t)gridDim.x * blockDim.x) {
    double sum = 0.0;
    const int32_t m1 = L.mstart[I + 1];
    for (int32_t m0 = L.mstart[I]; m0 < m1; ++m0) {
      const int32_t r = L.mlist[m0];
      int g;
      int64_t p;
      mg_locate(L, r, g, p);
      const int W = L.width[g];
      const int64_t G = L.count[g];
      double acc = 0.0;
      bool own = false;
      for (int e = 0; e < W; ++e) {
        const int32_t j = L.idx[g][(int64_t)e * G + p];
        const double xj = pre_x(L, f, j);
        if (j == r) {  // the row's own entry (always present on level 0)
          L.x[r] = xj;
          own = true;
        }
        acc = fma(L.val[g][(int64_t)e * G + p], xj, acc);
      }
      if (!own) L.x[r] = pre_x(L, f, r);
      sum += f[r] - acc;
    }
    fc[I] = sum;
  }
}

__device__ __forceinline__ double post1_y(const MgLevel& L, const double* __restrict__ f,
                                          const double* __restrict__ xc, double alpha, int64_t j) {
  int g;
  int64_t p;
  mg_locate(L, j, g, p);
  const double acc = ell_dot(L.idx[g], L.val[g], L.count[g], p, L.width[g],
                             [&](int32_t k) { return fma(alpha, xc[L.agg[k]], L.x[k]); });
  const double xj = fma(alpha, xc[L.agg[j]], L.x[j]);
  return fma(L.odinv[j], f[j] - acc, xj);
}

// k_mg_post1 + k_mg_post2: out = y + w (f - A y), y = x' + w (f - A x'),
// x' = x + alpha P xc, y recomputed at every stencil neighbour.  out must not
// alias L.x (level >= 1 writes L.y); on level 0 the border entry passes.
__global__ void __launch_bounds__(kMgThreads) k_mg_up(MgLevel L, const double* __restrict__ f,
                                                      const double* __restrict__ xc, double alpha,
                                                      double* __restrict__ out, int border, const double* done) {
  if (done && *done != 0.0) return;
  int g;
  int64_t p, stride;
  mg_rows(L, g, p, stride);
  const int W = L.width[g];
  const int64_t G = L.count[g];
  for (; p < G; p += stride) {
    const int64_t i = mg_row_id(L, g, p);
    double acc = 0.0, yi = 0.0;
    bool own = false;
    for (int e = 0; e < W; ++e) {
      const int32_t j = L.idx[g][(int64_t)e * G + p];
      const double yj = post1_y(L, f, xc, alpha, j);
      if (j == i) {
        yi = yj;
        own = true;
      }
      acc = fma(L.val[g][(int64_t)e * G + p], yj, acc);
    }
    if (!own) yi = post1_y(L, f, xc, alpha, i);
    out[i] = fma(L.odinv[i], f[i] - acc, yi);
  }
  if (border && blockIdx.x == 0 && threadIdx.x == 0) out[L.n] = f[L.n];
}

// ---- the coarse levels in one thread-block cluster -------------------------
// Levels lt..L-1 of a cycle (their smoothing, restriction, the dense coarsest
// solve and the way back up) run in one launch of one cluster of CTAs, the
// phases separated by the cluster's hardware barrier instead of kernel
// boundaries: on these levels every phase is a chain of a few dependent L2
// loads over a few thousand rows, so a launch per phase costs more than its
// work.  Vectors written inside the kernel (x, y, f of the levels) are read
// through L2 (ld.global.cg): the barrier orders the writes of one CTA before
// the reads of another at cluster scope, and no stale L1 line of another SM
// can be hit.  Level descriptors are read from device memory.
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cluster_size() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ double row_dot_cg(const MgLevel& L, int64_t p, const double* x) {
  return ell_dot(L.idx[0], L.val[0], L.count[0], p, L.width[0], [&](int32_t j) { return __ldcg(x + j); });
}

__global__ void __launch_bounds__(1024, 1) k_mg_tail(const MgLevel* __restrict__ lev, int lt, int L,
                                                    const double* __restrict__ binv, int m, double alpha,
                                                    const double* done) {
  if (done && *done != 0.0) return;  // the same value for every thread of the cluster
  const int64_t t0 = (int64_t)cluster_rank() * blockDim.x + threadIdx.x;
  const int64_t T = (int64_t)cluster_size() * blockDim.x;
  for (int l = lt; l + 1 < L; ++l) {
    const MgLevel F = lev[l];
    // x = w f + w (f - A w f)
    for (int64_t i = t0; i < F.n; i += T) {
      const double acc = ell_dot(F.idx[0], F.val[0], F.count[0], i, F.width[0],
                                 [&](int32_t j) { return F.odinv[j] * __ldcg(F.f + j); });
      const double fi = __ldcg(F.f + i), di = F.odinv[i];
      __stcg(F.x + i, di * fi + di * (fi - acc));
    }
    cluster_sync_all();
    // fc[I] = sum over the rows of aggregate I of (f - A x)
    const int64_t nc = lev[l + 1].n;
    double* fc = lev[l + 1].f;
    for (int64_t I = t0; I < nc; I += T) {
      double sum = 0.0;
      const int32_t m1 = F.mstart[I + 1];
      for (int32_t k = F.mstart[I]; k < m1; ++k) {
        const int32_t r = F.mlist[k];
        sum += __ldcg(F.f + r) - row_dot_cg(F, r, F.x);
      }
      __stcg(fc + I, sum);
    }
    cluster_sync_all();
  }
  // coarsest level: x = Binv f, one warp per row
  {
    const MgLevel C = lev[L - 1];
    const int lane = threadIdx.x & 31;
    const int64_t w0 = t0 >> 5, nw = T >> 5;
    for (int64_t r = w0; r < m; r += nw) {
      double acc = 0.0;
      for (int c = lane; c < m; c += 32) acc = fma(binv[r * m + c], __ldcg(C.f + c), acc);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) __stcg(C.x + r, acc);
    }
  }
  cluster_sync_all();
  for (int l = L - 2; l >= lt; --l) {
    const MgLevel F = lev[l];
    const double* xc = lev[l + 1].x;
    // y = x' + w (f - A x'), x' = x + alpha P xc
    for (int64_t i = t0; i < F.n; i += T) {
      const double acc = ell_dot(F.idx[0], F.val[0], F.count[0], i, F.width[0], [&](int32_t j) {
        return fma(alpha, __ldcg(xc + F.agg[j]), __ldcg(F.x + j));
      });
      const double xi = fma(alpha, __ldcg(xc + F.agg[i]), __ldcg(F.x + i));
      __stcg(F.y + i, fma(F.odinv[i], __ldcg(F.f + i) - acc, xi));
    }
    cluster_sync_all();
    // x = y + w (f - A y)
    for (int64_t i = t0; i < F.n; i += T)
      __stcg(F.x + i, fma(F.odinv[i], __ldcg(F.f + i) - row_dot_cg(F, i, F.y), __ldcg(F.y + i)));
    cluster_sync_all();
  }
}

// ---- the whole cycle in one cooperative kernel -------------------------------
// Every phase of the V-cycle -- pre-smoothing and restriction of each level
// on the way down, the dense coarsest solve, the two post-smoothing sweeps of
// each level on the way up -- runs in one launch whose blocks are all
// resident at once (cooperative launch), separated by a grid-wide barrier
// instead of a kernel boundary.  Each phase computes what the per-level
// kernel of the same name computes, row by row and in the same term order.
// Vectors written inside the kernel are read and written through L2
// (ld/st.global.cg), so no stale L1 line of another SM is read after a
// barrier; the cycle's input and the matrices go through L1.
//
// The barrier: each block's thread 0 reads the generation, publishes the
// block's writes (they are ordered before it by __syncthreads, and the
// device-scope fence is cumulative) and arrives on the counter; the last
// arrival resets the counter and advances the generation, the others wait
// for the generation to move.  The wait is bounded: after kMgBarrierSpins
// polls it sets the timeout flag and goes on, so the kernel always ends (its
// results are then void and the caller reports HSM_ETIMEOUT).
constexpr long kMgBarrierSpins = 1L << 20;

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void grid_barrier(unsigned* bar) {
  __syncthreads();
  // once a barrier has timed out the cycle is void: the later ones do not wait
  if (threadIdx.x == 0 && ld_acquire_u32(bar + 2) == 0u) {
    const unsigned gen = ld_acquire_u32(bar + 1);
    __threadfence();
    if (atomicAdd(bar, 1u) == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long spins = 0;
      while (ld_acquire_u32(bar + 1) == gen) {
        if (++spins > kMgBarrierSpins || ld_acquire_u32(bar + 2) != 0u) {
          atomicOr(bar + 2, 1u);
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
  }
  __syncthreads();
}

struct CycleArgs {
  const MgLevel* lev;  // device copy of the levels
  int L;
  const double* binv;
  int m;
  double alpha;
  const double* in;
  double* out;
  const double* done;
  unsigned* bar;
};

// a vector of the cycle: the input through L1, the kernel's own through L2
__device__ __forceinline__ double vld(const double* p, bool own) { return own ? __ldcg(p) : *p; }

__device__ __forceinline__ double row_dot_own(const MgLevel& L, int g, int64_t p, const double* x) {
  return ell_dot(L.idx[g], L.val[g], L.count[g], p, L.width[g], [&](int32_t j) { return __ldcg(x + j); });
}

// rows of a level, both groups as one range
__device__ __forceinline__ void cyc_row(const MgLevel& F, int64_t q, int& g, int64_t& p, int64_t& i) {
  g = q < F.count[0] ? 0 : 1;
  p = g ? q - F.count[0] : q;
  i = F.nodes[g] ? (int64_t)F.nodes[g][p] : p;
}

// k_mg_pre
__device__ void cyc_pre(const MgLevel& F, const double* f, bool own, int64_t t0, int64_t T) {
  const int64_t R = F.count[0] + F.count[1];
  for (int64_t q = t0; q < R; q += T) {
    int g;
    int64_t p, i;
    cyc_row(F, q, g, p, i);
    const double acc = ell_dot(F.idx[g], F.val[g], F.count[g], p, F.width[g],
                               [&](int32_t j) { return F.odinv[j] * vld(f + j, own); });
    const double fi = vld(f + i, own), di = F.odinv[i];
    __stcg(F.x + i, di * fi + di * (fi - acc));
  }
}

// k_mg_restrict
__device__ void cyc_restrict(const MgLevel& F, const double* f, bool own, double* fc, int64_t nc, int64_t t0,
                             int64_t T) {
  constexpr int kBatch = 8;
  for (int64_t I = t0; I < nc; I += T) {
    double s = 0.0;
    const int32_t m1 = F.mstart[I + 1];
    for (int32_t m0 = F.mstart[I]; m0 < m1; m0 += kBatch) {
      int32_t r[kBatch], g[kBatch];
      int64_t pp[kBatch];
#pragma unroll
      for (int k = 0; k < kBatch; ++k) r[k] = m0 + k < m1 ? F.mlist[m0 + k] : -1;
#pragma unroll
      for (int k = 0; k < kBatch; ++k)
        if (r[k] >= 0) mg_locate(F, r[k], g[k], pp[k]);
#pragma unroll
      for (int k = 0; k < kBatch; ++k)
        if (r[k] >= 0) s += vld(f + r[k], own) - row_dot_own(F, g[k], pp[k], F.x);
    }
    __stcg(fc + I, s);
  }
}

// k_mg_coarse (one warp per row)
__device__ void cyc_coarse(const MgLevel& C, const double* binv, int m, int64_t t0, int64_t T) {
  const int lane = threadIdx.x & 31;
  for (int64_t r = t0 >> 5; r < m; r += T >> 5) {
    double s = 0.0;
    for (int c = lane; c < m; c += 32) s = fma(binv[r * m + c], __ldcg(C.f + c), s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) __stcg(C.x + r, s);
  }
}

// k_mg_post1
__device__ void cyc_post1(const MgLevel& F, const double* f, bool own, const double* xc, double alpha, int64_t t0,
                          int64_t T) {
  const int64_t R = F.count[0] + F.count[1];
  for (int64_t q = t0; q < R; q += T) {
    int g;
    int64_t p, i;
    cyc_row(F, q, g, p, i);
    const double acc = ell_dot(F.idx[g], F.val[g], F.count[g], p, F.width[g], [&](int32_t j) {
      return fma(alpha, __ldcg(xc + F.agg[j]), __ldcg(F.x + j));
    });
    const double xi = fma(alpha, __ldcg(xc + F.agg[i]), __ldcg(F.x + i));
    __stcg(F.y + i, fma(F.odinv[i], vld(f + i, own) - acc, xi));
  }
}

// k_mg_post2
__device__ void cyc_post2(const MgLevel& F, const double* f, bool own, double* out, int64_t t0, int64_t T) {
  const int64_t R = F.count[0] + F.count[1];
  for (int64_t q = t0; q < R; q += T) {
    int g;
    int64_t p, i;
    cyc_row(F, q, g, p, i);
    __stcg(out + i, fma(F.odinv[i], vld(f + i, own) - row_dot_own(F, g, p, F.y), __ldcg(F.y + i)));
  }
}

__global__ void __launch_bounds__(kMgCycleThreads) k_mg_cycle(CycleArgs a) {
  if (a.done && *a.done != 0.0) return;  // the same value for every block
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t T = (int64_t)gridDim.x * blockDim.x;
  const int L = a.L;
  for (int l = 0; l + 1 < L; ++l) {
    const MgLevel& F = a.lev[l];
    const double* f = l == 0 ? a.in : F.f;
    cyc_pre(F, f, l > 0, t0, T);
    grid_barrier(a.bar);
    cyc_restrict(F, f, l > 0, a.lev[l + 1].f, a.lev[l + 1].n, t0, T);
    grid_barrier(a.bar);
  }
  cyc_coarse(a.lev[L - 1], a.binv, a.m, t0, T);
  grid_barrier(a.bar);
  for (int l = L - 2; l >= 0; --l) {
    const MgLevel& F = a.lev[l];
    const double* f = l == 0 ? a.in : F.f;
    cyc_post1(F, f, l > 0, a.lev[l + 1].x, a.alpha, t0, T);
    grid_barrier(a.bar);
    cyc_post2(F, f, l > 0, l == 0 ? a.out : F.x, t0, T);
    if (l > 0) grid_barrier(a.bar);
  }
  // the border entry of the bordered system passes through
  if (t0 == 0) a.out[a.lev[0].n] = a.in[a.lev[0].n];
}

// ---- set-up ------------------------------------------------------------------
__global__ void k_mg_odinv0(MgLevel L, double omega) {
  int g;
  int64_t p, stride;
  mg_rows(L, g, p, stride);
  for (; p < L.count[g]; p += stride) {
    const double d = L.val[g][p];  // the centre is the first stencil entry
    L.odinv[mg_row_id(L, g, p)] = (d != 0.0 && isfinite(d)) ? omega / d : 0.0;
  }
}

__device__ __forceinline__ unsigned long long ordered_bits(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}

__global__ void k_mg_min_coords(const double* __restrict__ coords, int64_t N, int dim, unsigned long long* lo) {
  unsigned long long m[3] = {~0ull, ~0ull, ~0ull};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    for (int k = 0; k < dim; ++k) m[k] = min(m[k], ordered_bits(coords[k * N + i]));
  for (int k = 0; k < dim; ++k) {
    unsigned long long v = m[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = min(v, (unsigned long long)__shfl_xor_sync(0xffffffffu, (long long)v, o));
    if ((threadIdx.x & 31) == 0) atomicMin(&lo[k], v);
  }
}

__global__ void k_mg_cells(const double* __restrict__ coords, int64_t N, int dim, double lo0, double lo1, double lo2,
                           double inv_c, int32_t* cell) {
  const double lo[3] = {lo0, lo1, lo2};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    for (int k = 0; k < dim; ++k) cell[k * N + i] = (int32_t)floor((coords[k * N + i] - lo[k]) * inv_c);
}

__device__ __forceinline__ unsigned long long cell_key(const int32_t* cell, int64_t N, int dim, int64_t i, int l) {
  unsigned long long key = 0ull;
  for (int k = 0; k < dim; ++k) key = (key << 21) | (unsigned long long)((cell[k * N + i] >> l) & 0x1fffff);
  return key;
}
__device__ __forceinline__ unsigned long long mix(unsigned long long k) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  return k;
}

// Inserts every node's level-l cell; the slot keeps the lowest node id.
__global__ void k_mg_insert(const int32_t* __restrict__ cell, int64_t N, int dim, int l, unsigned long long* keys,
                            int32_t* owner, int32_t* slot, unsigned long long mask, unsigned* overflow) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long key = cell_key(cell, N, dim, i, l);
    unsigned long long h = mix(key) & mask;
    int probe = 0;
    for (; probe < kMaxProbe; ++probe) {
      const unsigned long long prev = atomicCAS(&keys[h], kEmptyKey, key);
      if (prev == kEmptyKey || prev == key) break;
      h = (h + 1) & mask;
    }
    if (probe == kMaxProbe) {
      atomicOr(overflow, 1u);
      slot[i] = -1;
      continue;
    }
    atomicMin(&owner[h], (int32_t)i);
    slot[i] = (int32_t)h;
  }
}

__global__ void k_mg_leader(const int32_t* __restrict__ slot, const int32_t* __restrict__ owner, int64_t N,
                            uint8_t* lead) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    lead[i] = (slot[i] >= 0 && owner[slot[i]] == (int32_t)i) ? 1 : 0;
}

// cid[i] = coarse index of node i's cell; agg of the finer level's rows.
__global__ void k_mg_cid(const int32_t* __restrict__ slot, const int32_t* __restrict__ owner,
                         const int32_t* __restrict__ rank, const int32_t* __restrict__ cid_prev, int64_t N,
                         int32_t* cid, int32_t* agg) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = rank[owner[slot[i]]];
    cid[i] = c;
    // every node of a finer row lies in the same coarse cell: equal writes
    agg[cid_prev ? cid_prev[i] : i] = c;
  }
}

__global__ void k_mg_count(const int32_t* __restrict__ agg, int64_t n, int32_t* cnt) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&cnt[agg[r]], 1);
}
__global__ void k_mg_fill(const int32_t* __restrict__ agg, int64_t n, const int32_t* __restrict__ start,
                          int32_t* cursor, int32_t* list) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    const int32_t I = agg[r];
    list[start[I] + atomicAdd(&cursor[I], 1)] = (int32_t)r;
  }
}
// members of each aggregate in ascending order (fixed summation order)
__global__ void k_mg_sort(const int32_t* __restrict__ start, int64_t nc, int32_t* list) {
  for (int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; I < nc; I += (int64_t)gridDim.x * blockDim.x) {
    const int32_t a = start[I], b = start[I + 1];
    for (int32_t k = a + 1; k < b; ++k) {
      const int32_t v = list[k];
      int32_t j = k - 1;
      while (j >= a && list[j] > v) {
        list[j + 1] = list[j];
        --j;
      }
      list[j + 1] = v;
    }
  }
}

// Galerkin coarse row I = sum of its member rows with columns mapped by agg.
// Pass 1 counts distinct columns (max into *maxw); pass 2 writes the ELL row
// sorted by column, padded with (I, 0), and omega / diagonal.
template <bool FILL>
__global__ void k_mg_assemble(MgLevel L, int64_t nc, int Wc, int32_t* cidx, double* cval, double* codinv,
                              double omega, int* maxw, unsigned* overflow) {
  for (int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; I < nc; I += (int64_t)gridDim.x * blockDim.x) {
    int32_t cols[kMgMaxRow];
    double vals[kMgMaxRow];
    int cnt = 0;
    bool over = false;
    for (int32_t m = L.mstart[I]; m < L.mstart[I + 1]; ++m) {
      int g;
      int64_t p;
      mg_locate(L, L.mlist[m], g, p);
      const int W = L.width[g];
      const int64_t G = L.count[g];
      for (int e = 0; e < W; ++e) {
        const int32_t J = L.agg[L.idx[g][(int64_t)e * G + p]];
        const double a = L.val[g][(int64_t)e * G + p];
        int k = 0;
        while (k < cnt && cols[k] != J) ++k;
        if (k < cnt) {
          vals[k] += a;
        } else if (cnt < kMgMaxRow) {
          cols[cnt] = J;
          vals[cnt] = a;
          ++cnt;
        } else {
          over = true;
        }
      }
    }
    if (over) atomicOr(overflow, 2u);
    if (!FILL) {
      atomicMax(maxw, cnt);
      continue;
    }
    for (int k = 1; k < cnt; ++k) {
      const int32_t c = cols[k];
      const double v = vals[k];
      int j = k - 1;
      while (j >= 0 && cols[j] > c) {
        cols[j + 1] = cols[j];
        vals[j + 1] = vals[j];
        --j;
      }
      cols[j + 1] = c;
      vals[j + 1] = v;
    }
    double diag = 0.0;
    for (int k = 0; k < Wc; ++k) {
      const bool have = k < cnt;
      cidx[(int64_t)k * nc + I] = have ? cols[k] : (int32_t)I;
      cval[(int64_t)k * nc + I] = have ? vals[k] : 0.0;
      if (have && cols[k] == (int32_t)I) diag = vals[k];
    }
    codinv[I] = (diag != 0.0 && isfinite(diag)) ? omega / diag : 0.0;
  }
}

// Dense bordered matrix [A 1; 1^T 0] of the coarsest level, row-major (m+1)^2.
__global__ void k_mg_dense(MgLevel L, int m, double* B) {
  const int n1 = m + 1;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m; r += (int64_t)gridDim.x * blockDim.x) {
    int g;
    int64_t p;
    mg_locate(L, r, g, p);
    const int W = L.width[g];
    const int64_t G = L.count[g];
    for (int e = 0; e < W; ++e) B[r * n1 + L.idx[g][(int64_t)e * G + p]] += L.val[g][(int64_t)e * G + p];
    B[r * n1 + m] = 1.0;
    B[(int64_t)m * n1 + r] = 1.0;
  }
}

// Gauss-Jordan inversion with partial pivoting of the n1 x n1 matrix B into
// the right half of the n1 x 2n1 workspace M, one block; writes the leading
// m x m block of the inverse to binv.  *singular is set when a pivot vanishes.
__global__ void __launch_bounds__(1024) k_mg_invert(const double* B, int n1, double* M, double* binv,
                                                    unsigned* singular) {
  __shared__ double sv[1024];
  __shared__ int si[1024];
  __shared__ double fac[1024];
  const int t = threadIdx.x, T = blockDim.x, w = 2 * n1;
  for (int64_t e = t; e < (int64_t)n1 * w; e += T) {
    const int r = (int)(e / w), c = (int)(e % w);
    M[e] = c < n1 ? B[(int64_t)r * n1 + c] : (c - n1 == r ? 1.0 : 0.0);
  }
  __syncthreads();
  for (int k = 0; k < n1; ++k) {
    double best = -1.0;
    int brow = k;
    for (int r = k + t; r < n1; r += T) {
      const double v = fabs(M[(int64_t)r * w + k]);
      if (v > best) {
        best = v;
        brow = r;
      }
    }
    sv[t] = best;
    si[t] = brow;
    __syncthreads();
    for (int s = T / 2; s > 0; s >>= 1) {
      if (t < s && (sv[t + s] > sv[t] || (sv[t + s] == sv[t] && si[t + s] < si[t]))) {
        sv[t] = sv[t + s];
        si[t] = si[t + s];
      }
      __syncthreads();
    }
    const int pr = si[0];
    const double pv = sv[0];
    __syncthreads();
    if (!(pv > 0.0) || !isfinite(pv)) {
      if (t == 0) *singular = 1u;
      return;
    }
    if (pr != k)
      for (int c = t; c < w; c += T) {
        const double a = M[(int64_t)k * w + c];
        M[(int64_t)k * w + c] = M[(int64_t)pr * w + c];
        M[(int64_t)pr * w + c] = a;
      }
    __syncthreads();
    const double ip = 1.0 / M[(int64_t)k * w + k];
    __syncthreads();
    for (int c = t; c < w; c += T) M[(int64_t)k * w + c] *= ip;
    for (int r = t; r < n1; r += T) fac[r] = r == k ? 0.0 : M[(int64_t)r * w + k];
    __syncthreads();
    for (int64_t e = t; e < (int64_t)n1 * w; e += T) {
      const int r = (int)(e / w), c = (int)(e % w);
      if (r != k) M[e] = fma(-fac[r], M[(int64_t)k * w + c], M[e]);
    }
    __syncthreads();
  }
  const int m = n1 - 1;
  for (int64_t e = t; e < (int64_t)m * m; e += T) {
    const int r = (int)(e / m), c = (int)(e % m);
    binv[e] = M[(int64_t)r * w + n1 + c];
  }
}

int grid_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, kMgThreads), (int64_t)num_sms() * 8)); }

}  // namespace

hsm_status amg_setup(hsm_plan pl, const double* wp_mon, const double* wp_rbf, double alpha, Amg* amg) {
  cudaStream_t s = pl->stream;
  const int64_t N = pl->N;
  const int dim = pl->dim;
  amg->alpha = alpha;
  const double omega = amg->omega;
  MgLevel& L0 = amg->lev[0];
  L0.n = N;
  L0.nodes[0] = pl->mon.nodes;
  L0.nodes[1] = pl->rbf.nodes;
  L0.idx[0] = pl->mon.idx;
  L0.idx[1] = pl->rbf.idx;
  L0.val[0] = wp_mon;
  L0.val[1] = wp_rbf;
  L0.count[0] = pl->mon.count;
  L0.count[1] = pl->rbf.count;
  L0.width[0] = pl->mon.width;
  L0.width[1] = pl->rbf.width;
  L0.bm = pl->mon.count ? grid_for(pl->mon.count) : 0;
  L0.blocks = L0.bm + (pl->rbf.count ? grid_for(pl->rbf.count) : 0);
  L0.kind = pl->kind;
  L0.pos = pl->pos;
  HSM_CUDA(pl, dev_alloc(&L0.odinv, N, s));
  HSM_CUDA(pl, dev_alloc(&L0.x, N, s));
  HSM_CUDA(pl, dev_alloc(&L0.y, N, s));
  k_mg_odinv0<<<L0.blocks, kMgThreads, 0, s>>>(L0, omega);
  pl->launches += 1;

  // finest cells: edge 2h from the lower corner of the node set
  unsigned long long* lo_d = nullptr;
  HSM_CUDA(pl, dev_alloc(&lo_d, 3, s));
  HSM_CUDA(pl, cudaMemsetAsync(lo_d, 0xff, 3 * sizeof(unsigned long long), s));
  k_mg_min_coords<<<grid_for(N), kMgThreads, 0, s>>>(pl->coords, N, dim, lo_d);
  unsigned long long lo_h[3] = {0, 0, 0};
  HSM_CUDA(pl, cudaMemcpyAsync(lo_h, lo_d, sizeof(lo_h), cudaMemcpyDeviceToHost, s));
  HSM_CUDA(pl, cudaStreamSynchronize(s));
  double lo[3] = {0.0, 0.0, 0.0};
  for (int k = 0; k < dim; ++k) {
    unsigned long long b = lo_h[k];
    b = (b & 0x8000000000000000ull) ? (b & 0x7fffffffffffffffull) : ~b;
    memcpy(&lo[k], &b, sizeof(double));
  }
  unsigned long long cap = 1;
  while (cap < 2ull * (unsigned long long)N) cap <<= 1;
  int32_t *cell = nullptr, *owner = nullptr, *slot = nullptr, *rank = nullptr, *list = nullptr, *cid = nullptr,
          *cid_prev = nullptr, *cnt = nullptr, *scan_ws = nullptr;
  unsigned long long* keys = nullptr;
  uint8_t* lead = nullptr;
  unsigned* flags = nullptr;
  int* maxw = nullptr;
  auto release = [&]() {
    for (void** ptr : {(void**)&cell, (void**)&owner, (void**)&slot, (void**)&rank, (void**)&list, (void**)&cid,
                       (void**)&cid_prev, (void**)&cnt, (void**)&scan_ws, (void**)&keys, (void**)&lead,
                       (void**)&flags, (void**)&maxw, (void**)&lo_d})
      dev_free(ptr, s);
  };
  cudaError_t ce = cudaSuccess;
  for (auto e : {dev_alloc(&cell, (size_t)dim * N, s), dev_alloc(&owner, cap, s), dev_alloc(&slot, N, s),
                 dev_alloc(&rank, N, s), dev_alloc(&list, N, s), dev_alloc(&cid, N, s), dev_alloc(&cid_prev, N, s),
                 dev_alloc(&cnt, N + 1, s), dev_alloc(&scan_ws, scan_scratch(N + 1), s), dev_alloc(&keys, cap, s),
                 dev_alloc(&lead, N, s), dev_alloc(&flags, 2, s), dev_alloc(&maxw, 1, s)})
    if (e != cudaSuccess) ce = e;
  if (ce != cudaSuccess) {
    release();
    return cuda_fail(pl, ce, "multigrid set-up allocation");
  }
  k_mg_cells<<<grid_for(N), kMgThreads, 0, s>>>(pl->coords, N, dim, lo[0], lo[1], lo[2], 0.5 / pl->h, cell);
  HSM_CUDA(pl, cudaMemsetAsync(flags, 0, 2 * sizeof(unsigned), s));
  int l = 0;
  bool first = true;
  for (; l + 1 < kMgMaxLevels && amg->lev[l].n > kMgCoarsest; ++l) {
    MgLevel& F = amg->lev[l];
    // aggregates: the level-(l+1) cells of the nodes, numbered by lowest node id
    HSM_CUDA(pl, cudaMemsetAsync(keys, 0xff, cap * sizeof(unsigned long long), s));
    HSM_CUDA(pl, cudaMemsetAsync(owner, 0x7f, cap * sizeof(int32_t), s));
    k_mg_insert<<<grid_for(N), kMgThreads, 0, s>>>(cell, N, dim, l, keys, owner, slot, cap - 1, flags);
    k_mg_leader<<<grid_for(N), kMgThreads, 0, s>>>(slot, owner, N, lead);
    HSM_CUDA(pl, select_indices(lead, 1, N, list, rank, cnt, s, scan_ws));
    int nc_h = 0;
    unsigned fl = 0;
    HSM_CUDA(pl, cudaMemcpyAsync(&nc_h, cnt, sizeof(int), cudaMemcpyDeviceToHost, s));
    HSM_CUDA(pl, cudaMemcpyAsync(&fl, flags, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    HSM_CUDA(pl, cudaStreamSynchronize(s));
    if (fl) {
      release();
      return set_error(pl, HSM_ECUDA, "multigrid aggregation hash overflowed");
    }
    if (nc_h >= F.n || nc_h < 1) break;  // no coarsening: this level is the coarsest
    const int64_t nc = nc_h;
    HSM_CUDA(pl, dev_alloc(&F.agg, F.n, s));
    k_mg_cid<<<grid_for(N), kMgThreads, 0, s>>>(slot, owner, rank, first ? nullptr : cid_prev, N, cid, F.agg);
    first = false;
    std::swap(cid, cid_prev);
    // rows of each aggregate, ascending
    HSM_CUDA(pl, dev_alloc(&F.mstart, nc + 1, s));
    HSM_CUDA(pl, dev_alloc(&F.mlist, F.n, s));
    HSM_CUDA(pl, cudaMemsetAsync(cnt, 0, (nc + 1) * sizeof(int32_t), s));
    k_mg_count<<<grid_for(F.n), kMgThreads, 0, s>>>(F.agg, F.n, cnt);
    HSM_CUDA(pl, exclusive_scan_i32(cnt, F.mstart, nc, s, scan_ws));
    HSM_CUDA(pl, cudaMemsetAsync(cnt, 0, (nc + 1) * sizeof(int32_t), s));
    k_mg_fill<<<grid_for(F.n), kMgThreads, 0, s>>>(F.agg, F.n, F.mstart, cnt, F.mlist);
    k_mg_sort<<<grid_for(nc), kMgThreads, 0, s>>>(F.mstart, nc, F.mlist);
    F.cblocks = grid_for(nc);
    // Galerkin coarse operator
    HSM_CUDA(pl, cudaMemsetAsync(maxw, 0, sizeof(int), s));
    k_mg_assemble<false><<<grid_for(nc), kMgThreads, 0, s>>>(F, nc, 0, nullptr, nullptr, nullptr, omega, maxw, flags);
    int wc = 0;
    HSM_CUDA(pl, cudaMemcpyAsync(&wc, maxw, sizeof(int), cudaMemcpyDeviceToHost, s));
    HSM_CUDA(pl, cudaMemcpyAsync(&fl, flags, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    HSM_CUDA(pl, cudaStreamSynchronize(s));
    if (fl) {
      release();
      return set_error(pl, HSM_ECUDA, "a coarse multigrid row has more than 64 columns");
    }
    MgLevel& C = amg->lev[l + 1];
    C.n = nc;
    C.count[0] = nc;
    C.width[0] = std::max(wc, 1);
    C.bm = C.blocks = grid_for(nc);
    HSM_CUDA(pl, dev_alloc(&C.own_idx, (size_t)C.width[0] * nc, s));
    HSM_CUDA(pl, dev_alloc(&C.own_val, (size_t)C.width[0] * nc, s));
    HSM_CUDA(pl, dev_alloc(&C.odinv, nc, s));
    HSM_CUDA(pl, dev_alloc(&C.f, nc, s));
    HSM_CUDA(pl, dev_alloc(&C.x, nc, s));
    HSM_CUDA(pl, dev_alloc(&C.y, nc, s));
    C.idx[0] = C.own_idx;
    C.val[0] = C.own_val;
    k_mg_assemble<true><<<grid_for(nc), kMgThreads, 0, s>>>(F, nc, C.width[0], C.own_idx, C.own_val, C.odinv, omega,
                                                            maxw, flags);
    pl->launches += 8;
  }
  amg->L = l + 1;
  // coarsest level: dense inverse of its bordered system
  const MgLevel& Cs = amg->lev[l];
  if (Cs.n + 1 > 1024) {  // the dense inversion runs in one block of 1024 threads
    release();
    return set_error(pl, HSM_EINVAL, "multigrid coarsening stalled above 1023 rows");
  }
  const int m = (int)Cs.n, n1 = m + 1;
  amg->m = m;
  double *B = nullptr, *M = nullptr;
  HSM_CUDA(pl, dev_alloc(&B, (size_t)n1 * n1, s));
  HSM_CUDA(pl, dev_alloc(&M, (size_t)n1 * 2 * n1, s));
  HSM_CUDA(pl, dev_alloc(&amg->binv, (size_t)m * m, s));
  HSM_CUDA(pl, cudaMemsetAsync(B, 0, (size_t)n1 * n1 * sizeof(double), s));
  HSM_CUDA(pl, cudaMemsetAsync(flags, 0, 2 * sizeof(unsigned), s));
  k_mg_dense<<<grid_for(m), kMgThreads, 0, s>>>(Cs, m, B);
  k_mg_invert<<<1, 1024, 0, s>>>(B, n1, M, amg->binv, flags);
  pl->launches += 2;
  unsigned sing = 0;
  HSM_CUDA(pl, cudaMemcpyAsync(&sing, flags, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  HSM_CUDA(pl, cudaStreamSynchronize(s));
  dev_free(&B, s);
  dev_free(&M, s);
  release();
  if (sing) return set_error(pl, HSM_ESINGULAR, "the coarsest multigrid system is singular");
  return HSM_OK;
}

static cudaError_t launch_tail(const Amg& A, int lt, const double* done, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)A.tail_ctas;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)A.tail_ctas);
  cfg.blockDim = dim3(1024);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_mg_tail, (const MgLevel*)A.dlev, lt, A.L, (const double*)A.binv, A.m, A.alpha,
                            done);
}

// One V-cycle: levels below lt (all, when lt = 0) with their own kernels --
// the fused down/up forms from level lf on -- and levels lt..L-1 in the
// cluster tail.
static cudaError_t vcycle_lt(const Amg& A, int lt, int lf, const double* in, double* out, const double* done,
                             cudaStream_t s) {
  const int cg = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div((int64_t)A.m, kMgThreads / 32), 1024));
  if (A.L == 1) {
    k_mg_coarse<<<cg, kMgThreads, 0, s>>>(A.binv, A.m, in, out, A.lev[0].n, done);
    return cudaGetLastError();
  }
  if (A.nu == 1) {
    // V(1,1): two kernels per level
    const double* f = in;
    for (int l = 0; l + 1 < A.L; ++l) {
      const MgLevel& F = A.lev[l];
      k_mg_restrict1<<<F.cblocks, kMgThreads, 0, s>>>(F, f, A.lev[l + 1].f, A.lev[l + 1].n, done);
      f = A.lev[l + 1].f;
    }
    const MgLevel& Cs = A.lev[A.L - 1];
    k_mg_coarse<<<cg, kMgThreads, 0, s>>>(A.binv, A.m, Cs.f, Cs.x, -1, done);
    const double* xc = Cs.x;
    for (int l = A.L - 2; l >= 0; --l) {
      const MgLevel& F = A.lev[l];
      double* res = l == 0 ? out : F.y;
      k_mg_post1o<<<F.blocks, kMgThreads, 0, s>>>(F, l == 0 ? in : F.f, xc, A.alpha, res, l == 0 ? 1 : 0, done);
      xc = res;
    }
    return cudaGetLastError();
  }
  const int stop = lt > 0 ? lt : A.L - 1;  // first level not handled by per-level kernels
  const double* f = in;
  for (int l = 0; l < stop; ++l) {
    const MgLevel& F = A.lev[l];
    if (l >= lf) {
      k_mg_down<<<F.cblocks, kMgThreads, 0, s>>>(F, f, A.lev[l + 1].f, A.lev[l + 1].n, done);
    } else {
      k_mg_pre<<<F.blocks, kMgThreads, 0, s>>>(F, f, done);
      k_mg_restrict<<<F.cblocks, kMgThreads, 0, s>>>(F, f, A.lev[l + 1].f, A.lev[l + 1].n, done);
    }
    f = A.lev[l + 1].f;
  }
  if (lt > 0) {
    cudaError_t e = launch_tail(A, lt, done, s);
    if (e != cudaSuccess) return e;
  } else {
    const MgLevel& Cs = A.lev[A.L - 1];
    k_mg_coarse<<<cg, kMgThreads, 0, s>>>(A.binv, A.m, Cs.f, Cs.x, -1, done);
  }
  // the corrected iterate of level stop: x of the coarsest level or the tail's
  const double* xc = A.lev[stop].x;
  for (int l = stop - 1; l >= 0; --l) {
    const MgLevel& F = A.lev[l];
    const double* fl = l == 0 ? in : F.f;
    if (l >= lf) {
      double* res = l == 0 ? out : F.y;  // the fused form reads F.x throughout
      k_mg_up<<<F.blocks, kMgThreads, 0, s>>>(F, fl, xc, A.alpha, res, l == 0 ? 1 : 0, done);
      xc = res;
    } else {
      k_mg_post1<<<F.blocks, kMgThreads, 0, s>>>(F, fl, xc, A.alpha, done);
      double* res = l == 0 ? out : F.x;
      k_mg_post2<<<F.blocks, kMgThreads, 0, s>>>(F, fl, res, l == 0 ? 1 : 0, done);
      xc = res;
    }
  }
  return cudaGetLastError();
}

static cudaError_t launch_cycle(const Amg& A, const double* in, double* out, const double* done, cudaStream_t s) {
  CycleArgs a{A.dlev, A.L, A.binv, A.m, A.alpha, in, out, done, A.gbar};
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.gridDim = dim3((unsigned)A.pblocks);
  cfg.blockDim = dim3(kMgCycleThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_mg_cycle, a);
}

cudaError_t amg_vcycle(const Amg& A, const double* in, double* out, const double* done, cudaStream_t s) {
  if (A.persist) return launch_cycle(A, in, out, done, s);
  return vcycle_lt(A, A.lt, A.lf, in, out, done, s);
}

cudaError_t amg_reset_barrier(const Amg& A, cudaStream_t s) {
  if (!A.gbar) return cudaSuccess;
  return cudaMemsetAsync(A.gbar, 0, 4 * sizeof(unsigned), s);
}

const unsigned* amg_timeout_flag(const Amg& A) { return A.persist && A.gbar ? A.gbar + 2 : nullptr; }

int amg_kernels_per_cycle(const Amg& A) {
  if (A.L == 1) return 1;
  if (A.persist) return 1;
  if (A.nu == 1) return 2 * (A.L - 1) + 1;
  const int stop = A.lt > 0 ? A.lt : A.L - 1;
  int k = 1;
  for (int l = 0; l < stop; ++l) k += l >= A.lf ? 2 : 4;
  return k;
}

hsm_status amg_tune_tail(hsm_plan pl, Amg* A, int tail_from, int fused_from, int persistent) {
  cudaStream_t s = pl->stream;
  A->lt = 0;
  A->lf = A->L;
  A->persist = 0;
  A->persist_ms = -1.f;
  for (int l = 0; l < kMgMaxLevels; ++l) A->tail_ms[l] = A->fuse_ms[l] = -1.f;
  if (A->L < 2) return HSM_OK;
  if (A->nu == 1) {
    // V(1,1) has one shape (two kernels per level)
    if (tail_from > 0 || fused_from > 0 || persistent > 0)
      return set_error(pl, HSM_EINVAL, "the cycle shapes apply to V(2,2) only (mg_sweeps = 2)");
    return HSM_OK;
  }
  // the largest cluster the device schedules with 1024-thread CTAs
  int ctas = 0;
  for (int cl : {16, 8}) {
    if (cl > 8 && cudaFuncSetAttribute(k_mg_tail, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)cl;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)cl);
    cfg.blockDim = dim3(1024);
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, k_mg_tail, &cfg) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (nclusters >= 1) {
      ctas = cl;
      break;
    }
  }
  A->tail_ctas = ctas;
  // every block of the cooperative cycle resident at once
  int dev = 0, coop = 0, per_sm = 0;
  HSM_CUDA(pl, cudaGetDevice(&dev));
  HSM_CUDA(pl, cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (coop && persistent >= 0 &&
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mg_cycle, kMgCycleThreads, 0) == cudaSuccess &&
      per_sm >= 1)
    A->pblocks = num_sms() * std::min(per_sm, 2);
  else
    A->pblocks = 0;
  cudaGetLastError();
  if (persistent > 0 && A->pblocks == 0)
    return set_error(pl, HSM_EINVAL, "the cooperative multigrid cycle cannot be launched on this device");
  if (ctas || A->pblocks) {
    HSM_CUDA(pl, dev_alloc(&A->dlev, A->L, s));
    HSM_CUDA(pl, cudaMemcpyAsync(A->dlev, A->lev, A->L * sizeof(MgLevel), cudaMemcpyHostToDevice, s));
  }
  if (A->pblocks) HSM_CUDA(pl, dev_alloc(&A->gbar, 4, s));
  // time each choice of the first tail level on zero vectors
  const int64_t N1 = A->lev[0].n + 1;
  double *in = nullptr, *out = nullptr, *done = nullptr;
  HSM_CUDA(pl, dev_alloc(&in, N1, s));
  HSM_CUDA(pl, dev_alloc(&out, N1, s));
  HSM_CUDA(pl, dev_alloc(&done, 1, s));
  HSM_CUDA(pl, cudaMemsetAsync(in, 0, N1 * sizeof(double), s));
  HSM_CUDA(pl, cudaMemsetAsync(done, 0, sizeof(double), s));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  HSM_CUDA(pl, cudaEventCreate(&e0));
  HSM_CUDA(pl, cudaEventCreate(&e1));
  float best = 1e30f;
  int best_lt = 0, best_lf = A->L;
  cudaError_t ce = cudaSuccess;
  for (int lt = 0; lt < A->L && ce == cudaSuccess; ++lt) {
    if (lt > 0 && (!ctas || A->lev[lt].n > kMgTailMaxRows)) continue;
    if (tail_from != 0 && lt != (tail_from > 0 ? tail_from : 0)) continue;  // fixed by the caller
    // lf: first level of the fused down/up kernels (L: none)
    for (int lf = A->L; lf >= 0 && ce == cudaSuccess; --lf) {
      if (lt > 0 && lf > lt && lf != A->L) continue;  // past the tail: same cycle as lf = L
      if (fused_from != 0 && lf != (fused_from > 0 ? std::min(fused_from - 1, A->L) : A->L)) continue;
      float ms = 0.f;
      for (int rep = 0; rep < 2 && ce == cudaSuccess; ++rep) {  // the first pass warms up
        ce = cudaEventRecord(e0, s);
        for (int k = 0; k < 10 && ce == cudaSuccess; ++k) ce = vcycle_lt(*A, lt, lf, in, out, done, s);
        if (ce == cudaSuccess) ce = cudaEventRecord(e1, s);
        if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
        if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
      }
      if (ce != cudaSuccess) break;
      if (lf == A->L) A->tail_ms[lt] = ms;
      if (lt == 0 && lf < kMgMaxLevels) A->fuse_ms[lf] = ms;
      if (ms < best) {
        best = ms;
        best_lt = lt;
        best_lf = lf;
      }
    }
  }
  // the cooperative cycle, against the best of the shapes above
  bool use_persist = false;
  if (ce == cudaSuccess && A->pblocks) {
    Amg P = *A;
    P.persist = 1;
    float ms = 0.f;
    unsigned flag = 0;
    ce = amg_reset_barrier(P, s);
    for (int rep = 0; rep < 2 && ce == cudaSuccess; ++rep) {
      ce = cudaEventRecord(e0, s);
      for (int k = 0; k < 10 && ce == cudaSuccess; ++k) ce = launch_cycle(P, in, out, done, s);
      if (ce == cudaSuccess) ce = cudaEventRecord(e1, s);
      if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
      if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (ce == cudaSuccess) ce = cudaMemcpy(&flag, A->gbar + 2, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (ce == cudaSuccess) ce = amg_reset_barrier(P, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce == cudaSuccess && flag == 0) {
      A->persist_ms = ms;
      use_persist = persistent > 0 || (persistent == 0 && tail_from == 0 && fused_from == 0 && ms < best);
    }
    if (ce == cudaSuccess && flag != 0 && persistent > 0) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      dev_free(&in, s);
      dev_free(&out, s);
      dev_free(&done, s);
      return set_error(pl, HSM_ETIMEOUT, "a grid barrier of the cooperative multigrid cycle timed out");
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  dev_free(&in, s);
  dev_free(&out, s);
  dev_free(&done, s);
  if (ce != cudaSuccess) return cuda_fail(pl, ce, "multigrid cycle timing");
  if (best >= 1e30f && !use_persist)
    return set_error(pl, HSM_EINVAL, "the requested multigrid cycle shape is not available");
  A->lt = best_lt;
  A->lf = best_lf;
  A->persist = use_persist ? 1 : 0;
  return HSM_OK;
}

void amg_free(Amg* A, cudaStream_t s) {
  for (int l = 0; l < kMgMaxLevels; ++l) {
    MgLevel& L = A->lev[l];
    dev_free(&L.odinv, s);
    dev_free(&L.agg, s);
    dev_free(&L.mstart, s);
    dev_free(&L.mlist, s);
    dev_free(&L.f, s);
    dev_free(&L.x, s);
    dev_free(&L.y, s);
    dev_free(&L.own_idx, s);
    dev_free(&L.own_val, s);
  }
  dev_free(&A->binv, s);
  dev_free(&A->dlev, s);
  dev_free(&A->gbar, s);
  A->L = 0;
  A->lt = 0;
  A->lf = kMgMaxLevels;
}

}  // namespace hsm
