// Operator application, Eq. 1: (L u)(x_c) = sum_i w_i u(x_i).
//
// One launch covers both stencil groups: the first blocks walk the MON group
// (width 2d+1), the rest the RBF-FD group (width n), so regular and scattered
// stencils of uneven size share one grid.  One thread owns one stencil and
// all requested operators: the index stream is read once, every weight stream
// once, and the field gathered once per stencil entry.  Index and weight arrays are index-major ([j][node] and
// [op][j][node]), so consecutive threads read consecutive addresses (fully
// coalesced 128-byte lines); the gathered field values come from L1/L2 because
// nodes are spatially sorted.
#include "common.cuh"

namespace hsm {
namespace {

struct ApplyGroup {
  const int32_t* nodes;
  const int32_t* idx;
  const void* w;   // double* or float* [nops_plan][width][count]
  int64_t count;
  int width;
};

template <int NOPS>
struct Slots {
  int s[NOPS];
};

template <typename T>
__device__ __forceinline__ T ldg_stream(const T* p) {
  return __ldcs(p);
}

// The stencil sum runs in the storage type (FP64 for f64 fields; FP32 for
// f32 fields, whose n-term sums stay within (n+2) 2^-24 of the exact sum
// relative to sum |w u|, and whose FP32 pipe is 64x wider than the FP64 one
// on this part); every output is stored in FP64.
template <int W, int NOPS, typename TU, typename TW>
__device__ __forceinline__ void apply_one(const ApplyGroup& g, int width, int64_t p, Slots<NOPS> sl,
                                          const TU* __restrict__ u, double* __restrict__ out, int64_t N) {
  typedef TW Acc;
  const int Wd = W > 0 ? W : width;
  const TW* __restrict__ w = reinterpret_cast<const TW*>(g.w);
  const int64_t G = g.count;
  Acc acc[NOPS];
#pragma unroll
  for (int o = 0; o < NOPS; ++o) acc[o] = Acc(0);
  if (W > 0) {
    int32_t id[W > 0 ? W : 1];
#pragma unroll
    for (int j = 0; j < (W > 0 ? W : 1); ++j) id[j] = ldg_stream(g.idx + (int64_t)j * G + p);
    Acc uv[W > 0 ? W : 1];
#pragma unroll
    for (int j = 0; j < (W > 0 ? W : 1); ++j) uv[j] = (Acc)__ldg(u + id[j]);
#pragma unroll
    for (int o = 0; o < NOPS; ++o) {
      const TW* wo = w + (int64_t)sl.s[o] * Wd * G + p;
#pragma unroll
      for (int j = 0; j < (W > 0 ? W : 1); ++j) acc[o] = fma((Acc)ldg_stream(wo + (int64_t)j * G), uv[j], acc[o]);
    }
  } else {
    for (int j = 0; j < Wd; ++j) {
      const int32_t id = ldg_stream(g.idx + (int64_t)j * G + p);
      const Acc uv = (Acc)__ldg(u + id);
#pragma unroll
      for (int o = 0; o < NOPS; ++o)
        acc[o] = fma((Acc)ldg_stream(w + ((int64_t)sl.s[o] * Wd + j) * G + p), uv, acc[o]);
    }
  }
  const int32_t node = g.nodes[p];
#pragma unroll
  for (int o = 0; o < NOPS; ++o) __stcs(out + (int64_t)o * N + node, (double)acc[o]);
}

template <int WM, int WR, int NOPS, typename TU, typename TW>
__global__ void __launch_bounds__(256) k_apply(ApplyGroup gm, ApplyGroup gr, int64_t blocks_mon, Slots<NOPS> sl,
                                               const TU* __restrict__ u, double* __restrict__ out, int64_t N) {
  if (blockIdx.x < blocks_mon) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < gm.count; p += blocks_mon * blockDim.x)
      apply_one<WM, NOPS, TU, TW>(gm, gm.width, p, sl, u, out, N);
  } else {
    const int64_t b = blockIdx.x - blocks_mon, nb = gridDim.x - blocks_mon;
    for (int64_t p = b * blockDim.x + threadIdx.x; p < gr.count; p += nb * blockDim.x)
      apply_one<WR, NOPS, TU, TW>(gr, gr.width, p, sl, u, out, N);
  }
}

template <int WM, int NOPS, typename TU, typename TW>
void* pick_wr(int wr) {
  switch (wr) {
    case 12: return (void*)k_apply<WM, 12, NOPS, TU, TW>;
    case 20: return (void*)k_apply<WM, 20, NOPS, TU, TW>;
    case 30: return (void*)k_apply<WM, 30, NOPS, TU, TW>;
    case 40: return (void*)k_apply<WM, 40, NOPS, TU, TW>;
    default: return (void*)k_apply<WM, 0, NOPS, TU, TW>;
  }
}
template <int NOPS, typename TU, typename TW>
void* pick_wm(int wm, int wr) {
  return wm == 5 ? pick_wr<5, NOPS, TU, TW>(wr) : pick_wr<7, NOPS, TU, TW>(wr);
}
template <typename TU, typename TW>
void* pick_nops(int nops, int wm, int wr) {
  switch (nops) {
    case 1: return pick_wm<1, TU, TW>(wm, wr);
    case 2: return pick_wm<2, TU, TW>(wm, wr);
    case 3: return pick_wm<3, TU, TW>(wm, wr);
    default: return pick_wm<4, TU, TW>(wm, wr);
  }
}

// Average Nusselt number of Section 4.1: scale * mean_i |n_i . grad T(x_i)|
// over the listed nodes, one block; each thread sums its nodes in order and
// the block adds the partial sums in a fixed tree, so the result does not
// depend on timing.  The node ids come from the caller: an id outside [0, N)
// is not followed, and the result is then a quiet NaN.
constexpr int kFluxThreads = 256;

template <int DIM>
__global__ void __launch_bounds__(kFluxThreads) k_wall_flux(
    const double* __restrict__ T, const int32_t* __restrict__ nodes, int64_t count,
    const double* __restrict__ normals, int64_t N, const uint8_t* __restrict__ kind, const int32_t* __restrict__ pos,
    const int32_t* __restrict__ idx_m, const double* __restrict__ w_m, int64_t cnt_m, int width_m,
    const int32_t* __restrict__ idx_r, const double* __restrict__ w_r, int64_t cnt_r, int width_r, Slots<3> slot,
    double scale, double* out) {
  __shared__ double part[kFluxThreads];
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < count; i += kFluxThreads) {
    const int32_t c = nodes[i];
    if (c < 0 || (int64_t)c >= N) {
      bad = 1;
      continue;
    }
    const bool mon = kind[c] == 0;
    const int32_t* idx = mon ? idx_m : idx_r;
    const double* w = mon ? w_m : w_r;
    const int64_t G = mon ? cnt_m : cnt_r;
    const int W = mon ? width_m : width_r;
    const int64_t p = pos[c];
    double flux = 0.0;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      double g = 0.0;
      for (int j = 0; j < W; ++j) g = fma(w[((int64_t)slot.s[k] * W + j) * G + p], T[idx[(int64_t)j * G + p]], g);
      flux = fma(normals[k * N + c], g, flux);
    }
    acc += fabs(flux);
  }
  part[threadIdx.x] = acc;
  __syncthreads();
  for (int h = kFluxThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) part[threadIdx.x] += part[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = bad ? __longlong_as_double(0x7ff8000000000000ll) : scale * part[0] / (double)count;
}

}  // namespace

hsm_status launch_apply(hsm_plan p, unsigned op_mask, hsm_dtype dt, const void* u, double* out, cudaStream_t s) {
  int slots[kMaxOps];
  int nops = 0, slot = 0;
  for (int b = 0; b < 4; ++b) {
    if (p->op_mask & (1u << b)) {
      if (op_mask & (1u << b)) slots[nops++] = slot;
      ++slot;
    }
  }
  const bool f32 = dt == HSM_F32;
  ApplyGroup gm{p->mon.nodes, p->mon.idx, f32 ? (const void*)p->mon.w32 : (const void*)p->mon.w64, p->mon.count,
                p->mon.width};
  ApplyGroup gr{p->rbf.nodes, p->rbf.idx, f32 ? (const void*)p->rbf.w32 : (const void*)p->rbf.w64, p->rbf.count,
                p->rbf.width};
  const int T = p->tune.apply_threads;
  // grid: enough resident blocks to fill every SM, split in proportion to the
  // bytes each group streams
  const int64_t bytes_m = gm.count * (int64_t)gm.width * (4 + nops * (f32 ? 4 : 8));
  const int64_t bytes_r = gr.count * (int64_t)gr.width * (4 + nops * (f32 ? 4 : 8));
  const int64_t full = (int64_t)num_sms() * (2048 / T) * 4;
  int64_t bm = gm.count ? std::max<int64_t>(1, std::min<int64_t>(ceil_div(gm.count, T),
                                                                 full * bytes_m / std::max<int64_t>(1, bytes_m + bytes_r) + 1))
                        : 0;
  int64_t br = gr.count ? std::max<int64_t>(1, std::min<int64_t>(ceil_div(gr.count, T),
                                                                 full * bytes_r / std::max<int64_t>(1, bytes_m + bytes_r) + 1))
                        : 0;
  if (bm + br == 0) return HSM_OK;
  void* fn = nullptr;
  const int wm = p->mon.width;
  const int wr = p->rbf.width;
  switch (nops) {
    default: break;
  }
  Slots<4> sl4{};
  for (int o = 0; o < nops; ++o) sl4.s[o] = slots[o];
  if (f32) fn = pick_nops<float, float>(nops, wm, wr);
  else fn = pick_nops<double, double>(nops, wm, wr);
  int64_t N = p->N;
  // Slots<NOPS> is a prefix of Slots<4>; the kernel reads only its first NOPS ints
  void* args[] = {&gm, &gr, &bm, &sl4, &u, &out, &N};
  HSM_CUDA(p, cudaLaunchKernel(fn, dim3((unsigned)(bm + br)), dim3(T), args, 0, s));
  p->launches += 1;
  return HSM_OK;
}

hsm_status launch_wall_flux(hsm_plan p, const double* T, const int32_t* nodes, int64_t count, const double* normals,
                            double scale, double* out) {
  Slots<3> sl{};
  for (int k = 0; k < p->dim; ++k) {
    sl.s[k] = -1;
    for (int o = 0; o < p->nops; ++o)
      if (p->ops[o] == (1 << k)) sl.s[k] = o;
    if (sl.s[k] < 0) return set_error(p, HSM_EINVAL, "the plan's op mask lacks a first derivative");
  }
  if (p->dim == 2)
    k_wall_flux<2><<<1, kFluxThreads, 0, p->stream>>>(T, nodes, count, normals, p->N, p->kind, p->pos, p->mon.idx,
                                                      p->mon.w64, p->mon.count, p->mon.width, p->rbf.idx, p->rbf.w64,
                                                      p->rbf.count, p->rbf.width, sl, scale, out);
  else
    k_wall_flux<3><<<1, kFluxThreads, 0, p->stream>>>(T, nodes, count, normals, p->N, p->kind, p->pos, p->mon.idx,
                                                      p->mon.w64, p->mon.count, p->mon.width, p->rbf.idx, p->rbf.w64,
                                                      p->rbf.count, p->rbf.width, sl, scale, out);
  HSM_CUDA(p, cudaGetLastError());
  p->launches += 1;
  return HSM_OK;
}

}  // namespace hsm
