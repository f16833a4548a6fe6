// Device-wide exclusive scan and stream compaction: block sums, then a
// block-local scan plus the block's offset (the offsets come from a scan of
// the block sums in one block, or, for at most 1,024 blocks, from each block
// summing its predecessors' sums itself).
#include "common.cuh"

namespace hsm {
namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int warp_incl_scan(int v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Exclusive scan of one value per thread over the block; returns the block total.
__device__ __forceinline__ int block_excl_scan(int v, int* total) {
  __shared__ int warp_sums[kScanThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int incl = warp_incl_scan(v);
  if (lane == 31) warp_sums[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int ws = (lane < kScanThreads / 32) ? warp_sums[lane] : 0;
    int wi = warp_incl_scan(ws);
    if (lane < kScanThreads / 32) warp_sums[lane] = wi - ws;
    if (lane == kScanThreads / 32 - 1) *total = wi;
  }
  __syncthreads();
  int r = incl - v + warp_sums[wid];
  __syncthreads();
  return r;
}

struct CountsIn {
  const int32_t* in;
  __device__ int operator()(int64_t i) const { return in[i]; }
};
struct KeyEq {
  const uint8_t* key;
  uint8_t want;
  __device__ int operator()(int64_t i) const { return key[i] == want ? 1 : 0; }
};

template <typename F>
__global__ void k_block_sums(F f, int64_t n, int32_t* sums) {
  __shared__ int total;
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int v = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k)
    if (base + k < n) v += f(base + k);
  block_excl_scan(v, &total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void k_scan_sums(int32_t* sums, int nb, int32_t* grand, int64_t n, int32_t* rest) {
  __shared__ int total;
  int carry = 0;
  for (int s = 0; s < nb; s += kScanThreads) {
    int i = s + threadIdx.x;
    int v = i < nb ? sums[i] : 0;
    int e = block_excl_scan(v, &total);
    if (i < nb) sums[i] = carry + e;
    carry += total;
    __syncthreads();
  }
  if (threadIdx.x == 0 && grand) *grand = carry;
  if (threadIdx.x == 0 && rest) *rest = (int32_t)(n - carry);
}

template <typename F, typename W>
__global__ void k_block_write(F f, int64_t n, const int32_t* sums, W w) {
  __shared__ int total;
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int vals[kScanItems];
  int v = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    vals[k] = (base + k < n) ? f(base + k) : 0;
    v += vals[k];
  }
  int e = block_excl_scan(v, &total) + sums[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < n) w(base + k, e, vals[k]);
    e += vals[k];
  }
}

// Second pass with the offsets of the earlier blocks summed in the block
// itself (no separate scan of the block sums): nb reads per block, so it is
// used when there are at most kFoldBlocks blocks.  The last block writes the
// totals.
constexpr int kFoldBlocks = 1024;
template <typename F, typename W>
__global__ void k_block_write_fold(F f, int64_t n, const int32_t* sums, W w, int32_t* grand, int32_t* rest) {
  __shared__ int before, total;
  int part = 0;
  for (int i = threadIdx.x; i < (int)blockIdx.x; i += blockDim.x) part += sums[i];
  block_excl_scan(part, &before);
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int vals[kScanItems];
  int v = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    vals[k] = (base + k < n) ? f(base + k) : 0;
    v += vals[k];
  }
  int e = block_excl_scan(v, &total) + before;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < n) w(base + k, e, vals[k]);
    e += vals[k];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
    if (grand) *grand = before + total;
    if (rest) *rest = (int32_t)(n - (before + total));
  }
}

struct WriteExcl {
  int32_t* out;
  __device__ void operator()(int64_t i, int e, int) const { out[i] = e; }
};
// Stable partition by a 0/1 key: e counts the selected items before i, so an
// unselected item goes to place i - e of the second list.
struct WritePartition {
  int32_t* first;
  int32_t* second;
  int32_t* pos;
  __device__ void operator()(int64_t i, int e, int v) const {
    const int32_t q = v ? e : (int32_t)(i - e);
    (v ? first : second)[q] = (int32_t)i;
    pos[i] = q;
  }
};
struct WriteSelect {
  int32_t* list;
  int32_t* pos;
  __device__ void operator()(int64_t i, int e, int v) const {
    if (v) {
      list[e] = (int32_t)i;
      if (pos) pos[i] = e;
    }
  }
};

template <typename F, typename W>
cudaError_t run_scan(F f, W w, int64_t n, int32_t* grand, cudaStream_t s, int32_t* ws, int32_t* rest = nullptr) {
  int nb = (int)ceil_div(n > 0 ? n : 1, kScanTile);
  int32_t* sums = ws;
  cudaError_t e = cudaSuccess;
  if (!sums) {
    e = dev_alloc(&sums, nb, s);
    if (e != cudaSuccess) return e;
  }
  k_block_sums<<<nb, kScanThreads, 0, s>>>(f, n, sums);
  if (nb <= kFoldBlocks) {
    k_block_write_fold<<<nb, kScanThreads, 0, s>>>(f, n, sums, w, grand, rest);
  } else {
    k_scan_sums<<<1, kScanThreads, 0, s>>>(sums, nb, grand, n, rest);
    k_block_write<<<nb, kScanThreads, 0, s>>>(f, n, sums, w);
  }
  e = cudaGetLastError();
  if (!ws) dev_free(&sums, s);
  return e;
}

}  // namespace

cudaError_t exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, cudaStream_t s, int32_t* ws) {
  return run_scan(CountsIn{in}, WriteExcl{out}, n, out + n, s, ws);
}

int scan_kernels(int64_t n) { return ceil_div(n > 0 ? n : 1, kScanTile) <= kFoldBlocks ? 2 : 3; }

cudaError_t select_indices(const uint8_t* key, uint8_t want, int64_t n, int32_t* out_list,
                           int32_t* out_pos, int* count_dev, cudaStream_t s, int32_t* ws) {
  return run_scan(KeyEq{key, want}, WriteSelect{out_list, out_pos}, n, count_dev, s, ws);
}

cudaError_t partition_indices(const uint8_t* key, uint8_t want, int64_t n, int32_t* first, int32_t* second,
                              int32_t* pos, int* count_first, int* count_second, cudaStream_t s, int32_t* ws) {
  return run_scan(KeyEq{key, want}, WritePartition{first, second, pos}, n, count_first, s, ws, count_second);
}

int64_t scan_scratch(int64_t n) { return ceil_div(n > 0 ? n : 1, kScanTile); }

}  // namespace hsm
