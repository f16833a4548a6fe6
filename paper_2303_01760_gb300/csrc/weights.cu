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
#include <vector>

#include <map>
#include <mutex>

#include "common.cuh"
#include "rbf_kernels.cuh"

namespace hsm {

// The maximum dynamic shared memory of a kernel is one attribute per
// function, while shapes are cached per system size: the attribute is only
// ever raised, so a cached shape of a larger system stays launchable after a
// smaller one was computed.
cudaError_t raise_smem_limit(void* fn, size_t smem) {
  static std::mutex mu;
  static std::map<std::pair<int, void*>, size_t> limit;  // per device and kernel
  int dev = 0;
  cudaError_t de = cudaGetDevice(&dev);
  if (de != cudaSuccess) return de;
  std::lock_guard<std::mutex> g(mu);
  size_t& cur = limit[{dev, fn}];
  if (smem <= cur) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) cur = smem;
  return e;
}

// Kernels with compile-time system sizes (rbf_fixed.cu); nullptr when the
// size or lane count has none.
void* pick_fp32r_fixed(int dim, int nops, int K, int lanes);

namespace {

// ---------------------------------------------------------------------------
// MON
// ---------------------------------------------------------------------------
// The system is ordered basis rows (1, xi_1, xi_1^2, xi_2, xi_2^2 [, xi_3,
// xi_3^2]) against node columns (c, c-e1, c+e1, c-e2, c+e2 [, c-e3, c+e3]).
// On (and within 1e-6 lattice units of) the lattice this order needs no
// pivoting: every pivot stays within rounding of 1, -1 or 2, so the
// elimination runs as straight-line code in registers.  A pivot below 1e-8
// (impossible for a lattice stencil) marks the node singular.
// MON weights of the nodes at positions p0, p0 + stride, ... < G of the group.
template <int DIM, int NOPS>
__device__ __forceinline__ void mon_nodes(const double* __restrict__ coords, int64_t N,
                                          const int32_t* __restrict__ idx, int64_t G, const OpsDesc& ops,
                                          double* __restrict__ w, uint8_t* __restrict__ status,
                                          const int32_t* __restrict__ nodes, unsigned* flags, int64_t p0,
                                          int64_t stride) {
  constexpr int K = 2 * DIM + 1;
  constexpr int C = K + NOPS;
  for (int64_t p = p0; p < G; p += stride) {
    int32_t id[K];
#pragma unroll
    for (int j = 0; j < K; ++j) id[j] = idx[(int64_t)j * G + p];
    const int32_t c = id[0];
    double cx[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) cx[k] = coords[k * N + c];
    // Axis-aligned stencil (each neighbour c -+ e_k shares every other
    // coordinate with c, as for nodes placed exactly on the lattice), tested
    // on the coordinates' bits: the system decouples into one 3-point
    // Vandermonde system per axis, solved in closed form with
    // a = x_c - x_{c-e}, b = x_{c+e} - x_c, r = 1 / (a b (a + b)):
    //   d/dx_k : w(c-e) = -b^2 r, w(c+e) = a^2 r, w(c) = -(w(c-e) + w(c+e))
    //   lap    : w(c-e) = 2 b r,  w(c+e) = 2 a r, summed over the axes.
    bool aligned = true;
#pragma unroll
    for (int k = 0; k < DIM; ++k)
#pragma unroll
      for (int e = 0; e < DIM; ++e)
        if (e != k) {
          const long long ce = __double_as_longlong(cx[e]);
          aligned = aligned && __double_as_longlong(coords[e * N + id[1 + 2 * k]]) == ce &&
                    __double_as_longlong(coords[e * N + id[2 + 2 * k]]) == ce;
        }
    if (aligned) {
      double wm[DIM], wp[DIM], lm[DIM], lpl[DIM];
      bool okk = true;
#pragma unroll
      for (int k = 0; k < DIM; ++k) {
        const double a = cx[k] - coords[k * N + id[1 + 2 * k]], b = coords[k * N + id[2 + 2 * k]] - cx[k];
        // a, b > 0 and finite, on the bits
        const unsigned long long ab = (unsigned long long)__double_as_longlong(a),
                                 bb = (unsigned long long)__double_as_longlong(b);
        okk = okk && ab - 1ull < 0x7fefffffffffffffull && bb - 1ull < 0x7fefffffffffffffull;
        const double r = recip(a * b * (a + b));
        const double br = b * r, ar = a * r;
        wm[k] = -b * br;
        wp[k] = a * ar;
        lm[k] = br + br;
        lpl[k] = ar + ar;
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
          if (kd == 3 || kd == k) wc -= m + pl;
          w[((int64_t)o * K + 1 + 2 * k) * G + p] = okk ? m : 0.0;
          w[((int64_t)o * K + 2 + 2 * k) * G + p] = okk ? pl : 0.0;
        }
        w[((int64_t)o * K) * G + p] = okk ? wc : 0.0;
      }
      if (!okk) atomicOr(flags, kDevSingular);
      if (status) status[nodes[p]] = okk ? HSM_NODE_OK : HSM_NODE_SINGULAR;
      continue;
    }
    double xi[K][DIM];
    double s2 = 0.0;
#pragma unroll
    for (int j = 0; j < K; ++j) {
      double r2 = 0.0;
#pragma unroll
      for (int k = 0; k < DIM; ++k) {
        const double o = coords[k * N + id[j]] - cx[k];
        xi[j][k] = o;
        r2 += o * o;
      }
      s2 = fmax(s2, r2);
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

template <int DIM, int NOPS>
__global__ void __launch_bounds__(128) k_mon(const double* __restrict__ coords, int64_t N,
                                             const int32_t* __restrict__ idx, int64_t G, OpsDesc ops,
                                             double* __restrict__ w, uint8_t* __restrict__ status,
                                             const int32_t* __restrict__ nodes, unsigned* flags,
                                             const int* __restrict__ G_dev) {
  // the group size is read on the device when the launch is part of the
  // stencil build (it is known on the host only after the build)
  if (G_dev) G = *G_dev;
  mon_nodes<DIM, NOPS>(coords, N, idx, G, ops, w, status, nodes, flags, blockIdx.x * (int64_t)blockDim.x + threadIdx.x,
                       (int64_t)gridDim.x * blockDim.x);
}

// MON group of a grouped launch.
struct MonArgs {
  const double* coords;
  int64_t N;
  const int32_t* idx;
  int64_t G;
  OpsDesc ops;
  double* w;
  uint8_t* status;
  const int32_t* nodes;
  unsigned* flags;
};

// Weights of both stencil groups, systems of uneven size, in one persistent
// launch: every block takes work items from one queue (an atomic counter)
// until it is empty.  An item is a batch of SYS = blockDim / LANES RBF-FD
// systems (one per lane group, FP64 null-space solve: the FP64 pipe bounds
// the launch) or a chunk of blockDim MON nodes (one per thread: a few loads
// and stores, memory-bound).  The M MON chunks are spread evenly over the
// T items (item i is the MON chunk f(i) when f(i+1) > f(i), f(i) =
// floor(i M / T), else the RBF-FD batch i - f(i)), so memory-bound and
// FP64-bound blocks share the SMs.  No block waits on another.
template <int DIM, int NOPS, int LANES>
__global__ void __launch_bounds__(256) k_weights_grouped(RbfArgs a, MonArgs mo, int64_t mon_items, int64_t items,
                                                         int* queue) {
  extern __shared__ double smem[];
  const int SYS = blockDim.x / LANES;
  const int sub = threadIdx.x / LANES, lane = threadIdx.x % LANES;
  const unsigned mask = LANES == 32 ? 0xffffffffu : (((1u << LANES) - 1u) << ((threadIdx.x & 31) / LANES * LANES));
  double* xi = smem + (size_t)sub * sys_doubles(DIM, NOPS, a.n, a.n_mono);
  __shared__ int8_t par[kMaxMonomials], cor[kMaxMonomials];
  __shared__ int item_s;
  mono_parents(a.mono_exp, a.n_mono, DIM, par, cor);
  __syncthreads();
  for (;;) {
    if (threadIdx.x == 0) item_s = atomicAdd(queue, 1);
    __syncthreads();
    const int64_t item = item_s;
    __syncthreads();
    if (item >= items) break;
    const int64_t f0 = item * mon_items / items, f1 = (item + 1) * mon_items / items;
    if (f1 == f0) {
      const int64_t t = (item - f0) * SYS + sub;
      rbf64_systems<DIM, NOPS, LANES>(a, t, t + 1 < a.count ? t + 1 : a.count, 1, lane, mask, xi, par, cor);
    } else {
      const int64_t p = f0 * blockDim.x + threadIdx.x;
      mon_nodes<DIM, NOPS>(mo.coords, mo.N, mo.idx, mo.G, mo.ops, mo.w, mo.status, mo.nodes, mo.flags, p, mo.G);
    }
  }
}

template <int DIM, int NOPS, int LANES>
struct GroupedKernel {
  static void* ptr() { return (void*)k_weights_grouped<DIM, NOPS, LANES>; }
};

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
struct Fp64ChunkKernel {
  static void* ptr() { return (void*)k_rbf_fp64_chunk<DIM, NOPS, LANES>; }
};
template <int DIM, int NOPS, int LANES>
struct Fp32rKernel {
  static void* ptr() { return (void*)k_rbf_fp32r<DIM, NOPS, LANES, 0>; }
};

template <template <int, int, int> class KT, int DIM, int NOPS>
void* pick_lanes(int lanes) {
  switch (lanes) {
    case 4: return KT<DIM, NOPS, 4>::ptr();
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
  const size_t d = r32 ? r32_doubles(dim, nops, K, n) : sys_doubles(dim, nops, n, K - n);
  return d * sizeof(double);
}

// Launch shape of an RBF-FD kernel: the lane count (the requested one,
// doubled while a system does not fit) and the block size that keeps the most
// systems resident per SM.  Shapes are cached per kernel and system size.
struct RbfShape {
  void* fn = nullptr;
  int lanes = 0, threads = 0, blocks_per_sm = 0;
  size_t smem = 0;
};

// kind (FP64): 0 k_rbf_fp64, 1 k_weights_grouped, 2 k_rbf_fp64_chunk
cudaError_t rbf_shape(bool r32, int dim, int nops, int K, int ld, int n, int lanes, RbfShape* out, int kind = 0) {
  struct Entry {
    void* fn;
    size_t per;
    RbfShape shape;
  };
  thread_local std::vector<Entry> cache;
  const size_t per = smem_bytes(dim, nops, r32, K, ld, n);
  for (; lanes <= 32; lanes *= 2) {
    void* fn = r32 ? pick_fp32r_fixed(dim, nops, K, lanes) : nullptr;
    if (!fn)
      fn = r32 ? pick<Fp32rKernel>(dim, nops, lanes)
               : kind == 1 ? pick<GroupedKernel>(dim, nops, lanes)
                           : (kind == 2 ? pick<Fp64ChunkKernel>(dim, nops, lanes) : pick<Fp64Kernel>(dim, nops, lanes));
    for (const Entry& e : cache)
      if (e.fn == fn && e.per == per) {
        *out = e.shape;
        return cudaSuccess;
      }
    RbfShape best;
    int best_sys = 0;
    for (int threads : {64, 96, 128, 160, 192, 256}) {
      if (threads < lanes) continue;
      const size_t smem = per * (size_t)(threads / lanes);
      if (smem > 220 * 1024) continue;
      cudaError_t e = raise_smem_limit(fn, smem);
      if (e != cudaSuccess) return e;
      int bps = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, threads, smem);
      if (e != cudaSuccess) return e;
      const int sys = bps * (threads / lanes);
      if (sys > best_sys) {
        best_sys = sys;
        best.fn = fn;
        best.lanes = lanes;
        best.threads = threads;
        best.blocks_per_sm = bps;
        best.smem = smem;
      }
    }
    if (best_sys > 0) {
      cache.push_back({fn, per, best});
      *out = best;
      return cudaSuccess;
    }
  }
  *out = RbfShape{};
  return cudaSuccess;
}

hsm_status launch_rbf(hsm_plan p, bool r32, const int32_t* list, int64_t count, uint8_t* status,
                      int32_t* fail_list, int* fail_count, uint8_t mark, int degree = 0,
                      int32_t* sing_out = nullptr) {
  if (count == 0) return HSM_OK;
  // degree > 0: the monomials of total degree <= degree only (the first
  // C(degree + d, d) of the graded table)
  int n_mono = p->n_mono;
  if (degree > 0) {
    n_mono = 1;
    for (int i = 1; i <= p->dim; ++i) n_mono = n_mono * (degree + i) / i;
  }
  RbfArgs a{};
  a.coords = p->coords;
  a.N = p->N;
  a.list = list;
  a.count = count;
  a.idx = p->rbf.idx;
  a.G = p->rbf.count;
  a.nodes = p->rbf.nodes;
  a.n = p->n;
  a.n_mono = n_mono;
  a.K = p->n + n_mono;
  a.ld = (a.K + p->nops) | 1;
  a.mono_exp = p->mono_exp;
  a.pairs = p->pairs;
  a.ops = make_ops(p, p->op_mask);
  a.w = p->rbf.w64;
  // the FP64 solve records its singular systems (for the lower-degree retry)
  // once the plan holds a list for every system of the group
  const bool rec = !r32 && p->sing_list && p->sing_cap >= p->rbf.count;
  a.sing_list = rec ? (sing_out ? sing_out : p->sing_list) : nullptr;
  a.sing_count = rec ? p->dev_count + 1 : nullptr;
  a.sing_cap = rec ? p->rbf.count : 0;
  a.status = status;
  a.status_demoted_mark = mark;
  a.is_regular = p->is_regular;
  a.flags = p->dev_flags;
  a.fail_list = fail_list;
  a.fail_count = fail_count;
  RbfShape sh;
  HSM_CUDA(p, rbf_shape(r32, p->dim, p->nops, a.K, a.ld, a.n, r32 ? p->tune.rbf_lanes32 : p->tune.rbf_lanes, &sh));
  if (!sh.fn) return set_error(p, HSM_EINVAL, "RBF-FD system too large for shared memory");
  const int spb = sh.threads / sh.lanes;
  const int grid = (int)std::min<int64_t>(ceil_div(count, spb), (int64_t)num_sms() * sh.blocks_per_sm);
  void* args[] = {&a};
  HSM_CUDA(p, cudaLaunchKernel(sh.fn, dim3(grid), dim3(sh.threads), args, sh.smem, p->stream));
  p->launches += 1;
  return HSM_OK;
}

// Both groups' FP64 weights in one k_weights_grouped launch.
hsm_status launch_grouped_fp64(hsm_plan p, uint8_t* status) {
  RbfArgs a{};
  a.coords = p->coords;
  a.N = p->N;
  a.list = nullptr;
  a.count = p->rbf.count;
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
  a.status_demoted_mark = 0;
  a.is_regular = p->is_regular;
  a.flags = p->dev_flags;
  const bool rec = p->sing_list && p->sing_cap >= p->rbf.count;
  a.sing_list = rec ? p->sing_list : nullptr;
  a.sing_count = rec ? p->dev_count + 1 : nullptr;
  a.sing_cap = rec ? p->rbf.count : 0;
  MonArgs mo{p->coords, p->N, p->mon.idx, p->mon.count, make_ops(p, p->op_mask), p->mon.w64, status,
             p->mon.nodes, p->dev_flags};
  RbfShape sh;
  HSM_CUDA(p, rbf_shape(false, p->dim, p->nops, a.K, a.ld, a.n, p->tune.rbf_lanes, &sh, 1));
  if (!sh.fn) return set_error(p, HSM_EINVAL, "RBF-FD system too large for shared memory");
  const int spb = sh.threads / sh.lanes;
  const int64_t mon_items = ceil_div(p->mon.count, sh.threads);
  const int64_t items = ceil_div(p->rbf.count, spb) + mon_items;
  if (items == 0) return HSM_OK;
  if (items >= ((int64_t)1 << 31) - (int64_t)num_sms() * sh.blocks_per_sm)
    return set_error(p, HSM_EINVAL, "too many weight systems for one grouped launch");
  const int grid = (int)std::min<int64_t>(items, (int64_t)num_sms() * sh.blocks_per_sm);
  int* queue = p->dev_count + 2;
  HSM_CUDA(p, cudaMemsetAsync(queue, 0, sizeof(int), p->stream));
  void* args[] = {&a, &mo, (void*)&mon_items, (void*)&items, &queue};
  HSM_CUDA(p, cudaLaunchKernel(sh.fn, dim3(grid), dim3(sh.threads), args, sh.smem, p->stream));
  p->launches += 1;
  return HSM_OK;
}

}  // namespace

hsm_status compute_weights_grouped_fp64(hsm_plan p, uint8_t* status) { return launch_grouped_fp64(p, status); }

// Arguments of the FP64 solve of the whole RBF-FD group into w, the group
// size left to the device (chunk launches of the stencil build).
static RbfArgs chunk_args(hsm_plan p, double* w) {
  RbfArgs a{};
  a.coords = p->coords;
  a.N = p->N;
  a.list = nullptr;
  a.idx = p->rbf.idx;
  a.nodes = p->rbf.nodes;
  a.n = p->n;
  a.n_mono = p->n_mono;
  a.K = p->n + p->n_mono;
  a.ld = (a.K + p->nops) | 1;
  a.mono_exp = p->mono_exp;
  a.pairs = p->pairs;
  a.ops = make_ops(p, p->op_mask);
  a.w = w;
  a.status = nullptr;
  a.is_regular = p->is_regular;
  // its own status word (the second of the plan's four): the build reads the
  // first back as its own status, and the weights call reads this one
  a.flags = p->dev_flags + 1;
  // singular systems are recorded for the lower-degree retry of the weights
  // call; the list has room for every node
  const bool rec = p->sing_list && p->sing_cap >= p->N;
  a.sing_list = rec ? p->sing_list : nullptr;
  a.sing_count = rec ? p->dev_count + 1 : nullptr;
  a.sing_cap = rec ? p->sing_cap : 0;
  return a;
}

static cudaError_t rbf_chunk_shape(hsm_plan p, RbfShape* sh) {
  const int K = p->n + p->n_mono;
  return rbf_shape(false, p->dim, p->nops, K, (K + p->nops) | 1, p->n, p->tune.rbf_lanes, sh, 2);
}

cudaError_t rbf_chunk_ready(hsm_plan p) {
  RbfShape sh;
  cudaError_t e = rbf_chunk_shape(p, &sh);
  if (e != cudaSuccess) return e;
  return sh.fn ? cudaSuccess : cudaErrorInvalidConfiguration;
}

cudaError_t enqueue_rbf_chunk(hsm_plan p, const int* G_dev, double* w, int chunk, int nchunks, cudaStream_t s) {
  RbfShape sh;
  cudaError_t e = rbf_chunk_shape(p, &sh);
  if (e != cudaSuccess) return e;
  if (!sh.fn) return cudaErrorInvalidConfiguration;
  RbfArgs a = chunk_args(p, w);
  const int spb = sh.threads / sh.lanes;
  // sized for the largest possible chunk; blocks past the real one return
  const int grid = (int)std::min<int64_t>(ceil_div(ceil_div(p->N, nchunks), spb), (int64_t)num_sms() * sh.blocks_per_sm);
  void* args[] = {&a, (void*)&G_dev, &chunk, &nchunks};
  return cudaLaunchKernel(sh.fn, dim3(grid), dim3(sh.threads), args, sh.smem, s);
}

cudaError_t launch_rbf_external(const RbfExternal& x, bool r32, const int32_t* list, int64_t count, uint8_t* status,
                                uint8_t mark, bool* too_big) {
  *too_big = false;
  if (count == 0) return cudaSuccess;
  RbfArgs a{};
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
  RbfShape sh;
  cudaError_t e = rbf_shape(r32, x.dim, x.nops, a.K, a.ld, a.n, 8, &sh);
  if (e != cudaSuccess) return e;
  if (!sh.fn) {
    *too_big = true;
    return cudaSuccess;
  }
  const int spb = sh.threads / sh.lanes;
  const int grid = (int)std::min<int64_t>(ceil_div(count, spb), (int64_t)num_sms() * sh.blocks_per_sm);
  void* args[] = {&a};
  return cudaLaunchKernel(sh.fn, dim3(grid), dim3(sh.threads), args, sh.smem, x.stream);
}

cudaError_t rbf_external_fits(const RbfExternal& x, bool r32, bool* fits) {
  *fits = false;
  const int K = x.n + x.n_mono;
  RbfShape sh;
  cudaError_t e = rbf_shape(r32, x.dim, x.nops, K, (K + x.nops) | 1, x.n, 8, &sh);
  if (e != cudaSuccess) return e;
  *fits = sh.fn != nullptr;
  return cudaSuccess;
}

// MON weights of the G (or *G_dev) nodes of the MON group into w, on stream s.
static cudaError_t launch_mon(hsm_plan p, int64_t G, const int* G_dev, double* w, uint8_t* status,
                              cudaStream_t s) {
  OpsDesc ops = make_ops(p, p->op_mask);
  const int T = 128;
  int grid = (int)std::min<int64_t>(ceil_div(G, T), (int64_t)num_sms() * 16);
#define HSM_MON(D, O)                                                                                         \
  k_mon<D, O><<<grid, T, 0, s>>>(p->coords, p->N, p->mon.idx, G, ops, w, status, p->mon.nodes, p->dev_flags, \
                                 G_dev)
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
  return cudaGetLastError();
}

cudaError_t enqueue_mon_weights(hsm_plan p, const int* count_dev, double* w, cudaStream_t s) {
  return launch_mon(p, p->N, count_dev, w, nullptr, s);
}

hsm_status compute_mon_weights(hsm_plan p, uint8_t* status) {
  if (p->mon.count == 0) return HSM_OK;
  HSM_CUDA(p, launch_mon(p, p->mon.count, nullptr, p->mon.w64, status, p->stream));
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

hsm_status compute_rbf_weights_fp64_degree(hsm_plan p, const int32_t* list, int64_t count, uint8_t* status,
                                           int degree, int32_t* sing_out) {
  return launch_rbf(p, false, list, count, status, nullptr, nullptr, HSM_NODE_REDUCED_DEGREE, degree, sing_out);
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
