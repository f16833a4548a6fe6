// Stencil selection (Section 2: "a set of n neighbouring nodes").
//
// Regular nodes keep the symmetric 2d+1 lattice stencil, found through a
// lattice map (integer coordinates round(x/h) -> lowest node id): a dense
// array over the lattice's extents when it has at most 4N + 1024 points, an
// open-addressing hash otherwise.
// All other nodes take the n nodes of smallest (d2, id), where
// d2 = ((dx*dx) + (dy*dy)) + (dz*dz) is evaluated in FP64 with explicit
// round-to-nearest intrinsics (never contracted to FMA), so the selection is
// bit-identical to any other evaluation of the same expression.  Boundary
// nodes search among interior nodes only (plus themselves).  The search uses
// a uniform cell grid (cell edge = lattice spacing), one thread per query,
// visiting square (cube) shells of cells until no unvisited cell can hold a
// closer node.  Boundary nodes keep themselves first and search the n-1
// interior nodes nearest to x_c - h n_c, so their one-sided stencils reach
// several node layers.
#include <cfloat>
#include <cmath>

#include "common.cuh"

namespace hsm {
namespace {

constexpr double kLatticeTol = 1e-6;

__device__ __forceinline__ unsigned long long ordered_bits(double x) {
  unsigned long long b = (unsigned long long)__double_as_longlong(x);
  return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double from_ordered(unsigned long long b) {
  b = (b & 0x8000000000000000ull) ? (b & 0x7fffffffffffffffull) : ~b;
  return __longlong_as_double((long long)b);
}
__host__ __device__ inline double host_from_ordered(unsigned long long b) {
  b = (b & 0x8000000000000000ull) ? (b & 0x7fffffffffffffffull) : ~b;
  double d;
  memcpy(&d, &b, sizeof(d));
  return d;
}

// Lattice map: open-addressing hash table from packed lattice coordinates
// (21 bits per axis) to the lowest node id on that lattice point; capacity a
// power of two >= 2N, linear probing, every probe loop bounded by the
// capacity.
struct LatticeHash {
  unsigned long long* keys;  // ~0ull = empty slot
  int32_t* vals;             // kEmpty = no node
  unsigned long long mask;
  int dim;
  template <int DIM>
  __device__ __forceinline__ unsigned long long key(const int* q) const {
    unsigned long long k = 0;
#pragma unroll
    for (int a = DIM - 1; a >= 0; --a) k = (k << 21) | (unsigned long long)(q[a] + (1 << 20));
    return k;
  }
  static __device__ __forceinline__ unsigned long long hash(unsigned long long x) {
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdull;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ull;
    return x ^ (x >> 33);
  }
  template <int DIM>
  __device__ __forceinline__ void insert(const int* q, int32_t id) const {
    const unsigned long long k = key<DIM>(q);
    unsigned long long h = hash(k) & mask;
    for (unsigned long long probe = 0; probe <= mask; ++probe) {
      const unsigned long long prev = atomicCAS(&keys[h], ~0ull, k);
      if (prev == ~0ull || prev == k) {
        atomicMin(&vals[h], id);
        return;
      }
      h = (h + 1) & mask;
    }
  }
  // owner of lattice point q, or kEmpty
  template <int DIM>
  __device__ __forceinline__ int32_t find(const int* q) const {
#pragma unroll
    for (int a = 0; a < DIM; ++a)
      if (q[a] <= -(1 << 20) || q[a] >= (1 << 20)) return kEmpty;
    const unsigned long long k = key<DIM>(q);
    unsigned long long h = hash(k) & mask;
    for (unsigned long long probe = 0; probe <= mask; ++probe) {
      const unsigned long long cur = keys[h];
      if (cur == k) return vals[h];
      if (cur == ~0ull) return kEmpty;
      h = (h + 1) & mask;
    }
    return kEmpty;
  }
};

// Extents of the dense lattice map, written on the device once the lattice
// extents are known.
struct LatticeDense {
  int lo[kMaxDim];
  int ext[kMaxDim];
  long long size;  // product of the extents
  int dense;       // 1: the dense array holds the map; 0: the hash does
};

// The lattice map used by the kernels: the dense array when the lattice is
// compact, the hash otherwise.  load() reads the device-side extents; the
// choice is the same for every thread of a launch.
struct LatticeMap {
  LatticeHash hash;
  int32_t* dmap;  // [size] owner ids, kEmpty = no node
  const LatticeDense* desc;
  int lo[kMaxDim], ext[kMaxDim];
  int dense;
  __device__ __forceinline__ void load() {
    const LatticeDense d = *desc;
    dense = d.dense;
#pragma unroll
    for (int k = 0; k < kMaxDim; ++k) {
      lo[k] = d.lo[k];
      ext[k] = d.ext[k];
    }
  }
  template <int DIM>
  __device__ __forceinline__ long long slot(const int* q) const {
    long long l = 0;
#pragma unroll
    for (int k = DIM - 1; k >= 0; --k) {
      const int t = q[k] - lo[k];
      if (t < 0 || t >= ext[k]) return -1;
      l = l * ext[k] + t;
    }
    return l;
  }
  template <int DIM>
  __device__ __forceinline__ int32_t find(const int* q) const {
    if (!dense) return hash.find<DIM>(q);
    const long long l = slot<DIM>(q);
    return l < 0 ? kEmpty : dmap[l];
  }
  template <int DIM>
  __device__ __forceinline__ void insert(const int* q, int32_t id) const {
    if (!dense) {
      hash.insert<DIM>(q, id);
      return;
    }
    const long long l = slot<DIM>(q);
    if (l >= 0) atomicMin(&dmap[l], id);
  }
};

struct CellGrid;
struct LatticeDense;
// Cell grid of the bounding box, and the dense lattice map's extents (defined
// below); run by the last block of k_bounds once every block's minima and
// maxima are in.
__device__ void grid_setup(const unsigned long long* bbox, int dim, double h, int64_t N, CellGrid* out);
__device__ void lattice_setup(const int* lat_lo, const int* lat_hi, int dim, long long dense_cap, LatticeDense* desc);

// Adding 1.5 * 2^52 to a double of magnitude below 2^51 rounds it to an
// integer: the sum lies in [2^52, 2^53), where one unit in the last place is
// 1, and the integer is the sum's bit pattern minus that of 1.5 * 2^52.
constexpr double kRoundMagic = 6755399441055744.0;
constexpr long long kRoundMagicBits = 0x4338000000000000ll;
constexpr long long kLatticeRangeI = 1ll << 20;  // |lattice coordinate| < 2^20 (21-bit key fields)
constexpr int kBoundsThreads = 256;
constexpr int kBoundsItems = 2;  // nodes per thread per pass, their loads issued together

// Block-wide extrema of each thread's running ones; valid in thread 0.
__device__ __forceinline__ void block_extrema(unsigned long long* bmin, unsigned long long* bmax, int* lmin, int* lmax, int dim) {
  __shared__ unsigned long long sb[2][kMaxDim][kBoundsThreads / 32];
  __shared__ int sl[2][kMaxDim][kBoundsThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kMaxDim; ++k) {
    if (k >= dim) break;
    for (int o = 16; o > 0; o >>= 1) {
      unsigned long long a = __shfl_xor_sync(0xffffffffu, bmin[k], o);
      unsigned long long b = __shfl_xor_sync(0xffffffffu, bmax[k], o);
      int c = __shfl_xor_sync(0xffffffffu, lmin[k], o);
      int d = __shfl_xor_sync(0xffffffffu, lmax[k], o);
      bmin[k] = a < bmin[k] ? a : bmin[k];
      bmax[k] = b > bmax[k] ? b : bmax[k];
      lmin[k] = min(lmin[k], c);
      lmax[k] = max(lmax[k], d);
    }
    if (lane == 0) {
      sb[0][k][wid] = bmin[k];
      sb[1][k][wid] = bmax[k];
      sl[0][k][wid] = lmin[k];
      sl[1][k][wid] = lmax[k];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < kMaxDim; ++k)
      for (int w = 1; w < kBoundsThreads / 32 && k < dim; ++w) {
        bmin[k] = sb[0][k][w] < bmin[k] ? sb[0][k][w] : bmin[k];
        bmax[k] = sb[1][k][w] > bmax[k] ? sb[1][k][w] : bmax[k];
        lmin[k] = min(lmin[k], sl[0][k][w]);
        lmax[k] = max(lmax[k], sl[1][k][w]);
      }
  }
}

// Bounding box (ordered-bit keys), each node's nearest lattice point and
// whether it lies on it, and the lattice extents.  Each block writes its own
// slot of extrema partials (bpart, lpart: [gridDim.x][2 kMaxDim], interleaved
// [min_k, max_k]); the last block to arrive reduces them into bbox and
// lat[0, 2 kMaxDim) (lattice extents; an empty lattice keeps 0x7f7f7f7f /
// 0x80808080), sets up the cell grid and the lattice map, and zeroes the
// build's counters for the kernels after it: the status flags, the weights
// call's counts, lat[2 kMaxDim, +4) (demoted, n_mon, n_rbf, flags copy) and
// the arrival count lat[2 kMaxDim + 4], which starts at zero on allocation.
__global__ void __launch_bounds__(kBoundsThreads) k_bounds(const double* __restrict__ coords, int64_t N, int dim,
                                                           double inv_h, unsigned long long* bpart, int* lpart,
                                                           int32_t* ijk, uint8_t* on_lat, unsigned long long* bbox,
                                                           int* lat, unsigned* flags, int* counts, double h,
                                                           long long dense_cap, CellGrid* cg_out,
                                                           LatticeDense* ld_out) {
  unsigned long long bmin[kMaxDim], bmax[kMaxDim];
  int lmin[kMaxDim], lmax[kMaxDim];
#pragma unroll
  for (int k = 0; k < kMaxDim; ++k) {
    bmin[k] = ~0ull;
    bmax[k] = 0ull;
    lmin[k] = 0x7fffffff;
    lmax[k] = -0x7fffffff;
  }
  const int64_t stride = (int64_t)gridDim.x * blockDim.x * kBoundsItems;
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x * kBoundsItems + threadIdx.x; i0 < N; i0 += stride) {
    double x[kBoundsItems][kMaxDim];
#pragma unroll
    for (int u = 0; u < kBoundsItems; ++u) {
      const int64_t i = i0 + (int64_t)u * blockDim.x;
#pragma unroll
      for (int k = 0; k < kMaxDim; ++k) x[u][k] = (i < N && k < dim) ? coords[k * N + i] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kBoundsItems; ++u) {
      const int64_t i = i0 + (int64_t)u * blockDim.x;
      if (i >= N) break;
      bool on = true;
      int q[kMaxDim];
#pragma unroll
      for (int k = 0; k < kMaxDim; ++k) {
        if (k >= dim) break;
        const double xk = x[u][k];
        const unsigned long long ob = ordered_bits(xk);
        bmin[k] = ob < bmin[k] ? ob : bmin[k];
        bmax[k] = ob > bmax[k] ? ob : bmax[k];
        // nearest lattice coordinate r of x / h (the product rounded once,
        // with the magic constant); NaN, infinities and |x / h| >= 2^20 give
        // a sum outside (magic - 2^20, magic + 2^20)
        const double s = __fma_rn(xk, inv_h, kRoundMagic);
        const long long r = (long long)__double_as_longlong(s) - kRoundMagicBits;
        const double d = __fma_rn(xk, inv_h, -__dsub_rn(s, kRoundMagic));  // x / h - r
        if (!(r > -kLatticeRangeI && r < kLatticeRangeI && fabs(d) <= kLatticeTol)) on = false;
        q[k] = on ? (int)r : 0;
      }
      on_lat[i] = on ? 1 : 0;
#pragma unroll
      for (int k = 0; k < kMaxDim; ++k) {
        if (k >= dim) break;
        ijk[k * N + i] = q[k];
        if (on) {
          lmin[k] = min(lmin[k], q[k]);
          lmax[k] = max(lmax[k], q[k]);
        }
      }
    }
  }
  block_extrema(bmin, bmax, lmin, lmax, dim);
  __shared__ bool last;
  if (threadIdx.x == 0) {
    unsigned long long* bp = bpart + (size_t)blockIdx.x * 2 * kMaxDim;
    int* lp = lpart + (size_t)blockIdx.x * 2 * kMaxDim;
#pragma unroll
    for (int k = 0; k < kMaxDim; ++k) {
      if (k >= dim) break;
      bp[2 * k] = bmin[k];
      bp[2 * k + 1] = bmax[k];
      lp[2 * k] = lmin[k];
      lp[2 * k + 1] = lmax[k];
    }
    __threadfence();
    unsigned* arrivals = reinterpret_cast<unsigned*>(lat + 2 * kMaxDim + 4);
    last = atomicAdd(arrivals, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  // the last block: every other block's partials are visible
  __threadfence();
#pragma unroll
  for (int k = 0; k < kMaxDim; ++k) {
    bmin[k] = ~0ull;
    bmax[k] = 0ull;
    lmin[k] = 0x7fffffff;
    lmax[k] = -0x7fffffff;
  }
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
    const unsigned long long* bp = bpart + (size_t)b * 2 * kMaxDim;
    const int* lp = lpart + (size_t)b * 2 * kMaxDim;
#pragma unroll
    for (int k = 0; k < kMaxDim; ++k) {
      if (k >= dim) break;
      const unsigned long long a = __ldcg(bp + 2 * k), c = __ldcg(bp + 2 * k + 1);
      bmin[k] = a < bmin[k] ? a : bmin[k];
      bmax[k] = c > bmax[k] ? c : bmax[k];
      lmin[k] = min(lmin[k], __ldcg(lp + 2 * k));
      lmax[k] = max(lmax[k], __ldcg(lp + 2 * k + 1));
    }
  }
  block_extrema(bmin, bmax, lmin, lmax, dim);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < kMaxDim; ++k) {
      const bool any = k < dim && lmin[k] <= lmax[k];
      bbox[2 * k] = k < dim ? bmin[k] : ~0ull;
      bbox[2 * k + 1] = k < dim ? bmax[k] : 0ull;
      lat[k] = any ? lmin[k] : 0x7f7f7f7f;
      lat[kMaxDim + k] = any ? lmax[k] : (int)0x80808080u;
    }
    grid_setup(bbox, dim, h, N, cg_out);
    lattice_setup(lat, lat + kMaxDim, dim, dense_cap, ld_out);
    for (int t = 0; t < 4; ++t) {
      flags[t] = 0u;
      counts[t] = 0;
      lat[2 * kMaxDim + t] = 0;
    }
    lat[2 * kMaxDim + 4] = 0;  // arrivals, for the next launch
  }
}


// Dense map extents from the lattice extents; the dense array is used when
// the lattice has at most dense_cap points.
__device__ void lattice_setup(const int* lat_lo, const int* lat_hi, int dim, long long dense_cap, LatticeDense* desc) {
  LatticeDense d;
  long long size = 1;
  bool fits = true;
  for (int k = 0; k < kMaxDim; ++k) {
    const int lo = k < dim ? __ldcg(lat_lo + k) : 0, hi = k < dim ? __ldcg(lat_hi + k) : 0;
    d.lo[k] = lo;
    const long long e = k < dim ? (long long)hi - lo + 1 : 1;
    d.ext[k] = e > 0 && e < (1ll << 30) ? (int)e : 0;
    if (e <= 0) size = 0;  // no node on the lattice
    if (e >= (1ll << 30)) fits = false;
    if (fits && size > 0) {
      size *= e;
      if (size > dense_cap) fits = false;
    }
  }
  d.size = fits ? size : 0;
  d.dense = fits ? 1 : 0;
  *desc = d;
}

// Empties the map in use: the dense array's first size entries, or the hash.
__global__ void k_lattice_clear(LatticeMap g, unsigned long long hcap) {
  g.load();
  const long long n = g.dense ? g.desc->size : (long long)hcap;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    if (g.dense) {
      g.dmap[i] = kEmpty;
    } else {
      g.hash.keys[i] = ~0ull;
      g.hash.vals[i] = kEmpty;
    }
  }
}

// Lattice point of every on-lattice node into the map (owner = lowest id).
template <int DIM>
__global__ void k_lattice_insert(const int32_t* __restrict__ ijk, const uint8_t* __restrict__ on_lat, int64_t N,
                                 LatticeMap g) {
  g.load();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    if (!on_lat[i]) continue;
    int q[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) q[k] = ijk[k * N + i];
    g.insert<DIM>(q, (int32_t)i);
  }
}

// kind = 0 (MON) when the node is regular, interior, owns its lattice point and
// has all 2d lattice neighbours; 1 (RBF-FD) otherwise.
template <int DIM>
__device__ __forceinline__ void classify_node(const int32_t* __restrict__ ijk, const uint8_t* __restrict__ on_lat,
                                              const uint8_t* __restrict__ is_regular,
                                              const uint8_t* __restrict__ is_boundary, int64_t N,
                                              const LatticeMap& g, int64_t i, uint8_t* kind, int* n_demoted) {
  bool reg = is_regular[i] != 0;
  bool mon = reg && on_lat[i] && !(is_boundary && is_boundary[i]);
  if (mon) {
    int q[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) q[k] = ijk[k * N + i];
    // every lookup is made (no short circuit), so their loads are in flight together
    bool all = g.find<DIM>(q) == (int32_t)i;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
#pragma unroll
      for (int s = -1; s <= 1; s += 2) {
        q[k] += s;
        all = all & (g.find<DIM>(q) != kEmpty);
        q[k] -= s;
      }
    }
    mon = all;
  }
  kind[i] = mon ? 0 : 1;
  if (reg && !mon) atomicAdd(n_demoted, 1);
}

// MON stencils; the group size is read on the device.
template <int DIM>
__global__ void k_mon_stencil(const int32_t* __restrict__ ijk, const int32_t* __restrict__ mon_nodes,
                              const int* __restrict__ count_dev, int64_t N, LatticeMap g, int32_t* idx) {
  g.load();
  const int64_t count = *count_dev;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < count;
       p += (int64_t)gridDim.x * blockDim.x) {
    int32_t c = mon_nodes[p];
    int q[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) q[k] = ijk[k * N + c];
    idx[p] = c;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
#pragma unroll
      for (int s = -1; s <= 1; s += 2) {
        q[k] += s;
        idx[(int64_t)(1 + 2 * k + (s + 1) / 2) * count + p] = g.find<DIM>(q);
        q[k] -= s;
      }
    }
  }
}

// ---- uniform cell grid ----------------------------------------------------
struct CellGrid {
  double lo[kMaxDim];
  double inv_cell;
  double cell;
  int g[kMaxDim];
  int dim;
  // floor((x - lo) / cell) clamped to the grid: the conversion rounds down
  // and saturates, the clamp is integer arithmetic (a NaN lands in cell 0)
  __device__ __forceinline__ int cell_of(double x, int k) const {
    const int c = __double2int_rd(__dmul_rn(__dsub_rn(x, lo[k]), inv_cell));
    return min(max(c, 0), g[k] - 1);
  }
};

// Cell grid of the bounding box: cell edge h, enlarged by 1.5x until the
// grid has at most 4N + 1024 cells (the scan buffers are sized for that).
__device__ void grid_setup(const unsigned long long* bbox, int dim, double h, int64_t N, CellGrid* out) {
  CellGrid cg;
  cg.dim = dim;
  double lo[kMaxDim], hi[kMaxDim];
  for (int k = 0; k < kMaxDim; ++k) {
    lo[k] = k < dim ? from_ordered(__ldcg(bbox + 2 * k)) : 0.0;
    hi[k] = k < dim ? from_ordered(__ldcg(bbox + 2 * k + 1)) : 0.0;
    cg.lo[k] = lo[k];
  }
  double cell = h;
  for (int tries = 0; tries < 64; ++tries) {
    int64_t ncell = 1;
    for (int k = 0; k < kMaxDim; ++k) {
      cg.g[k] = k < dim ? (int)fmin(floor((hi[k] - lo[k]) / cell) + 1.0, 1e9) : 1;
      ncell *= cg.g[k];
    }
    if (ncell <= 4 * N + 1024) break;
    cell *= 1.5;
  }
  cg.cell = cell;
  cg.inv_cell = 1.0 / cell;
  *out = cg;
}

// One pass over the nodes: the MON / RBF-FD classification (the lattice map
// is complete) and each node's cell with the per-cell counts (the cell grid
// is set up by k_bounds).
template <int DIM>
__global__ void k_classify_count(const int32_t* __restrict__ ijk, const uint8_t* __restrict__ on_lat,
                                 const uint8_t* __restrict__ is_regular, const uint8_t* __restrict__ is_boundary,
                                 int64_t N, LatticeMap g, uint8_t* kind, int* n_demoted,
                                 const double* __restrict__ coords, const CellGrid* __restrict__ cgp,
                                 int32_t* cell_of, int32_t* counts) {
  g.load();
  const CellGrid cg = *cgp;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    classify_node<DIM>(ijk, on_lat, is_regular, is_boundary, N, g, i, kind, n_demoted);
    int64_t l = 0;
#pragma unroll
    for (int k = DIM - 1; k >= 0; --k) l = l * cg.g[k] + cg.cell_of(coords[k * N + i], k);
    cell_of[i] = (int32_t)l;
    atomicAdd(&counts[l], 1);
  }
}

// The build's status words beside its counters for the one read-back: st[3]
// the status bits, st[5] the in-build solve's singular-system count, st[6]
// its status bits (st[0..2]: demoted, n_mon, n_rbf; st[4]: k_bounds' arrivals).
constexpr int kReadbackWords = 7;
__global__ void k_build_status(const unsigned* __restrict__ flags, const int* __restrict__ counts, int* st) {
  st[3] = (int)flags[0];
  st[5] = counts[1];
  st[6] = (int)flags[1];
}

__global__ void k_cell_scatter(const double* __restrict__ coords, const uint8_t* __restrict__ is_boundary,
                               int64_t N, int dim, const int32_t* __restrict__ cell_of,
                               const int32_t* __restrict__ start, int32_t* cursor, int32_t* sorted_id,
                               double* sorted_xyz, uint8_t* sorted_bnd) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t l = cell_of[i];
    // the cursors are the cell counts, counted down to zero: the next build's
    // counting starts from zero without a memset
    int32_t s = start[l] + atomicSub(&cursor[l], 1) - 1;
    sorted_id[s] = (int32_t)i;
    for (int k = 0; k < dim; ++k) sorted_xyz[(int64_t)s * kMaxDim + k] = coords[k * N + i];
    sorted_bnd[s] = is_boundary ? is_boundary[i] : 0;
  }
}

// (d2, id) lexicographic key comparison (integer compare of the d2 bits;
// d2 is non-negative and finite).
__device__ __forceinline__ bool key_less(double d2a, int32_t ia, double d2b, int32_t ib) {
  const unsigned long long a = (unsigned long long)__double_as_longlong(d2a);
  const unsigned long long b = (unsigned long long)__double_as_longlong(d2b);
  return a < b || (a == b && ia < ib);
}

template <int DIM>
__device__ __forceinline__ double sq_dist(const double* a, const double* b) {
  double d = __dsub_rn(a[0], b[0]);
  double s = __dmul_rn(d, d);
#pragma unroll
  for (int k = 1; k < DIM; ++k) {
    double e = __dsub_rn(a[k], b[k]);
    s = __dadd_rn(s, __dmul_rn(e, e));
  }
  return s;
}

// QT threads per query (a "quad" of consecutive lanes).  Every thread keeps
// its own sorted top-n list of (d2, id) keys in shared memory ([n][blockDim]
// structure of arrays, bank-conflict free) and prunes candidates against its
// own n-th key and the quad's merged n-th key of the previous pass.
//
// The first pass scans the whole window of rings 0..R0 around the search
// point's cell; each later pass scans one more ring.  After every pass the
// quad leader merges the QT lists to find the quad's n-th key, and the search
// stops once that distance is below the distance from the search point to the
// scanned region's edge; at the end the leader merges the lists into the
// stencil.  The result does not depend on R0: any region that passes the
// stopping test holds the n smallest keys.  R0 only decides how much one pass
// scans.  It is set per query from the local spacing hs (the plan's spacing
// array, else h): R0 = floor(rfac * hs / cell) + 1, clamped to [1, RMAX], with
// rfac * hs an estimate of the n-th neighbour distance (from n and the
// dimension, set by the caller; a boundary node's search point lies h inside
// the wall, where about half the disc or ball is outside the domain, so it
// takes 2^(1/DIM) more).  The distance to the window's edge lies in
// [R0, R0 + 1/2) cells, so the window holds the n-th neighbour with R0 cells
// to spare in the common case.
//
// Scanning rings one by one, with a dependent chain of loads per cell (the
// cell's range, then its nodes), left each query's thread waiting on memory
// for about fifty cells in a row.  A row of the window, and the top and bottom
// rows of a ring, are runs of cells that are consecutive in the cell order,
// so their nodes are one contiguous range of the sorted arrays: one pair of
// range loads per row, the next row's pair loaded while the current row is
// scanned (window pass), and the node loads of a range issued BATCH at a
// time before any of them is used.  The rows of a pass are dealt round-robin
// to the quad's threads, and so are the single side cells of a ring.
template <int DIM, int QT>
__global__ void __launch_bounds__(32 * QT, 1) k_knn(const double* __restrict__ coords, int64_t N,
                                             const uint8_t* __restrict__ is_boundary,
                                             const double* __restrict__ normals, double h,
                                             const double* __restrict__ spacing,
                                             const int32_t* __restrict__ queries, const int* __restrict__ nq_dev,
                                             int n_full, double rfac, const CellGrid* __restrict__ cgp,
                                             const int32_t* __restrict__ start, const int32_t* __restrict__ sorted_id,
                                             const double* __restrict__ sorted_xyz,
                                             const uint8_t* __restrict__ sorted_bnd, int32_t* __restrict__ out_idx,
                                             unsigned* flags, int chunk, int nchunks) {
  constexpr int RMAX = DIM == 2 ? 6 : 4;
  // node loads in flight per thread: 8 when a query has several threads (a
  // 2D window row of ~7 nodes in one round trip), 4 with one thread per query
  // (fewer registers, more resident queries for large query counts)
  constexpr int BATCH = QT == 1 ? 4 : 8;
  extern __shared__ unsigned char smem_raw[];
  const int B = blockDim.x;
  const int64_t nq = *nq_dev;  // the stride of out_idx
  // this launch's queries: chunk `chunk` of `nchunks` equal chunks
  const int64_t qc = (nq + nchunks - 1) / nchunks;
  const int64_t q_lo = min(nq, (int64_t)chunk * qc), q_hi = min(nq, q_lo + qc);
  const CellGrid cg = *cgp;
  double* kd = reinterpret_cast<double*>(smem_raw);
  int32_t* ki = reinterpret_cast<int32_t*>(kd + (size_t)n_full * B);
  const int t = threadIdx.x, sub = t % QT, lead = t - sub;
  const int lane = t & 31;
  const unsigned qmask = ((1u << QT) - 1u) << (lane - sub);
  const int64_t qpb = B / QT;
  for (int64_t qi = q_lo + blockIdx.x * qpb + t / QT; qi < q_hi; qi += (int64_t)gridDim.x * qpb) {
    const int32_t c = queries[qi];
    const bool bnd_center = is_boundary && is_boundary[c];
    // boundary nodes: search the n-1 interior nodes nearest to x_c - h n_c
    const int n = bnd_center ? n_full - 1 : n_full;
    double q[DIM];
    int cq[DIM];
    // one local spacing inside: h(x_c) of a refined node set, else h
    const double hs = spacing ? spacing[c] : h;
    const double hc = bnd_center ? hs : h;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      q[k] = coords[k * N + c];
      if (bnd_center && normals) q[k] = __dsub_rn(q[k], __dmul_rn(hc, normals[k * N + c]));
      cq[k] = cg.cell_of(q[k], k);
    }
    const double rf = bnd_center ? rfac * (DIM == 2 ? 1.4142135623730951 : 1.2599210498948732) : rfac;
    const int r0 = (int)fmin(fmax(floor(rf * hs * cg.inv_cell) + 1.0, 1.0), (double)RMAX);
    int cnt = 0;
    double qd = DBL_MAX;  // quad's n-th key after the last pass (pruning bound)
    int32_t qid = 0x7fffffff;
    // nodes [s0, s1) of the sorted arrays, loads issued BATCH at a time
    auto scan = [&](int32_t s0, int32_t s1) {
      for (int32_t s = s0; s < s1; s += BATCH) {
        int32_t id[BATCH];
        bool use[BATCH];
        double x[BATCH][DIM];
#pragma unroll
        for (int u = 0; u < BATCH; ++u) {
          const int32_t su = min(s + u, s1 - 1);
          id[u] = sorted_id[su];
          use[u] = s + u < s1 && !(bnd_center && sorted_bnd[su]);
#pragma unroll
          for (int k = 0; k < DIM; ++k) x[u][k] = sorted_xyz[(int64_t)su * kMaxDim + k];
        }
#pragma unroll
        for (int u = 0; u < BATCH; ++u) {
          if (!use[u]) continue;
          const double d2 = sq_dist<DIM>(x[u], q);
          if (!key_less(d2, id[u], qd, qid)) continue;
          if (cnt == n && !key_less(d2, id[u], kd[(n - 1) * B + t], ki[(n - 1) * B + t])) continue;
          int j = (cnt < n) ? cnt++ : n - 1;
          while (j > 0 && key_less(d2, id[u], kd[(j - 1) * B + t], ki[(j - 1) * B + t])) {
            kd[j * B + t] = kd[(j - 1) * B + t];
            ki[j * B + t] = ki[(j - 1) * B + t];
            --j;
          }
          kd[j * B + t] = d2;
          ki[j * B + t] = id[u];
        }
      }
    };
    for (int r = r0;; ++r) {
      int lo[DIM], hi[DIM];
      bool any_inside = false;
#pragma unroll
      for (int k = 0; k < DIM; ++k) {
        lo[k] = cq[k] - r;
        hi[k] = cq[k] + r;
        if (lo[k] >= 0 || hi[k] < cg.g[k]) any_inside = true;
      }
      if (r > r0 && !any_inside) break;
      const bool window = r == r0;
      int turn = 0;  // row / side-cell counter; this thread takes turn % QT == sub
      const int xa = max(lo[0], 0), xb = min(hi[0], cg.g[0] - 1);
      const int zlo = DIM == 3 ? max(lo[DIM - 1], 0) : 0, zhi = DIM == 3 ? min(hi[DIM - 1], cg.g[DIM - 1] - 1) : 0;
      if (window) {
        // every row of the window is one node range; this thread's rows (i =
        // sub, sub + QT, ...) with the next row's range loaded while the
        // current one is scanned
        const int ylo = max(lo[1], 0), yhi = min(hi[1], cg.g[1] - 1);
        // (y, z) of this thread's next row, advanced QT rows at a time
        int y = ylo + sub, z = zlo;
        auto advance = [&](int& yy, int& zz) {
          yy += QT;
#pragma unroll 1
          while (yy > yhi) {
            yy -= yhi - ylo + 1;
            ++zz;
          }
        };
#pragma unroll 1
        while (y > yhi && z <= zhi) {
          y -= yhi - ylo + 1;
          ++z;
        }
        int32_t a0 = 0, a1 = 0;
        if (z <= zhi) {
          const int64_t rb = ((int64_t)z * cg.g[1] + y) * cg.g[0];
          a0 = start[rb + xa];
          a1 = start[rb + xb + 1];
        }
        while (z <= zhi) {
          const int32_t s0 = a0, s1 = a1;
          advance(y, z);
          if (z <= zhi) {
            const int64_t rb = ((int64_t)z * cg.g[1] + y) * cg.g[0];
            a0 = start[rb + xa];
            a1 = start[rb + xb + 1];
          }
          scan(s0, s1);
        }
      }
      for (int z = zlo; z <= zhi && !window; ++z) {
        const bool zedge = DIM == 3 && (z == lo[DIM - 1] || z == hi[DIM - 1]);
        for (int y = max(lo[1], 0); y <= min(hi[1], cg.g[1] - 1); ++y) {
          const int64_t row = ((int64_t)z * cg.g[1] + y) * cg.g[0];
          if (window || zedge || y == lo[1] || y == hi[1]) {
            if ((turn++ % QT) != sub) continue;
            scan(start[row + xa], start[row + xb + 1]);
          } else {
#pragma unroll
            for (int e = 0; e < 2; ++e) {
              const int x = e ? hi[0] : lo[0];
              if (x < 0 || x >= cg.g[0]) continue;
              if ((turn++ % QT) != sub) continue;
              scan(start[row + x], start[row + x + 1]);
            }
          }
        }
      }
      // quad's n-th key: the leader merges the QT sorted lists
      __syncwarp(qmask);
      double nd = DBL_MAX;
      int32_t nid = 0x7fffffff;
      int total = 0;
      // list lengths of the quad (every thread shares its cnt)
      int lens[QT];
#pragma unroll
      for (int u = 0; u < QT; ++u) lens[u] = __shfl_sync(qmask, cnt, (lane - sub) + u);
#pragma unroll
      for (int u = 0; u < QT; ++u) total += lens[u];
      if (sub == 0 && total >= n) {
        int pos[QT];
#pragma unroll
        for (int u = 0; u < QT; ++u) pos[u] = 0;
        for (int k = 0; k < n; ++k) {
          int best = -1;
          double bd = DBL_MAX;
          int32_t bi = 0x7fffffff;
#pragma unroll
          for (int u = 0; u < QT; ++u) {
            if (pos[u] < lens[u]) {
              const double dd = kd[pos[u] * B + lead + u];
              const int32_t ii = ki[pos[u] * B + lead + u];
              if (best < 0 || key_less(dd, ii, bd, bi)) {
                best = u;
                bd = dd;
                bi = ii;
              }
            }
          }
          ++pos[best];
          nd = bd;
          nid = bi;
        }
      }
      nd = __shfl_sync(qmask, nd, lane - sub);
      nid = __shfl_sync(qmask, nid, lane - sub);
      if (total >= n) {
        qd = nd;
        qid = nid;
        double bound = DBL_MAX;
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
          if (lo[k] > 0) bound = fmin(bound, q[k] - (cg.lo[k] + lo[k] * cg.cell));
          if (hi[k] < cg.g[k] - 1) bound = fmin(bound, (cg.lo[k] + (hi[k] + 1) * cg.cell) - q[k]);
        }
        if (bound == DBL_MAX) break;
        bound *= (1.0 - 1e-9);
        if (bound > 0.0 && nd < bound * bound) break;
      }
    }
    // final merge of the quad's lists by the leader
    __syncwarp(qmask);
    int lens[QT];
#pragma unroll
    for (int u = 0; u < QT; ++u) lens[u] = __shfl_sync(qmask, cnt, (lane - sub) + u);
    if (sub == 0) {
      int pos[QT];
#pragma unroll
      for (int u = 0; u < QT; ++u) pos[u] = 0;
      const int off = bnd_center ? 1 : 0;
      if (bnd_center) out_idx[qi] = c;
      int got = 0;
      for (int k = 0; k < n; ++k) {
        int best = -1;
        double bd = DBL_MAX;
        int32_t bi = 0x7fffffff;
#pragma unroll
        for (int u = 0; u < QT; ++u) {
          if (pos[u] < lens[u]) {
            const double dd = kd[pos[u] * B + lead + u];
            const int32_t ii = ki[pos[u] * B + lead + u];
            if (best < 0 || key_less(dd, ii, bd, bi)) {
              best = u;
              bd = dd;
              bi = ii;
            }
          }
        }
        int32_t v = c;
        if (best >= 0) {
          ++pos[best];
          v = bi;
          ++got;
        }
        out_idx[(int64_t)(k + off) * nq + qi] = v;
      }
      if (got < n) atomicOr(flags, kDevKnnShort);
    }
    __syncwarp(qmask);
  }
}

}  // namespace

// The workspace of the build depends only on N, dim and n, so it is
// allocated once per plan; the group node lists and index arrays are sized for
// the largest possible group.
hsm_status alloc_build_ws(hsm_plan p) {
  BuildWs& w = p->ws;
  if (w.ready) return HSM_OK;
  cudaStream_t s = p->stream;
  const int64_t N = p->N;
  const int64_t ncell_max = 4 * N + 1024;
  unsigned long long cap = 1;
  while (cap < 2ull * (unsigned long long)N) cap <<= 1;
  w.hcap = cap;
  CellGrid* cg = nullptr;
  HSM_CUDA(p, dev_alloc(&w.bbox, 2 * kMaxDim, s));
  HSM_CUDA(p, dev_alloc(&w.lat, 2 * kMaxDim + kReadbackWords, s));
  HSM_CUDA(p, cudaMemsetAsync(w.lat, 0, (2 * kMaxDim + kReadbackWords) * sizeof(int), s));  // k_bounds' arrival count
  const int64_t bgrid = (int64_t)num_sms() * 8;  // k_bounds' largest grid
  HSM_CUDA(p, dev_alloc(&w.bpart, bgrid * 2 * kMaxDim, s));
  HSM_CUDA(p, dev_alloc(&w.lpart, bgrid * 2 * kMaxDim, s));
  HSM_CUDA(p, dev_alloc(&w.ijk, (size_t)p->dim * N, s));
  HSM_CUDA(p, dev_alloc(&w.on_lat, N, s));
  HSM_CUDA(p, dev_alloc(&w.hkeys, cap, s));
  HSM_CUDA(p, dev_alloc(&w.hvals, cap, s));
  HSM_CUDA(p, dev_alloc(&w.dmap, 4 * N + 1024, s));
  // empty lattice map (kEmpty is the byte 0x7f repeated; empty hash keys are all ones)
  HSM_CUDA(p, cudaMemsetAsync(w.dmap, 0x7f, (size_t)(4 * N + 1024) * sizeof(int32_t), s));
  HSM_CUDA(p, cudaMemsetAsync(w.hkeys, 0xff, (size_t)cap * sizeof(unsigned long long), s));
  HSM_CUDA(p, cudaMemsetAsync(w.hvals, 0x7f, (size_t)cap * sizeof(int32_t), s));
  {
    LatticeDense* ld = nullptr;
    HSM_CUDA(p, dev_alloc(&ld, 1, s));
    w.ldesc = ld;
  }
  HSM_CUDA(p, dev_alloc(&cg, 1, s));
  w.cgd = cg;
  HSM_CUDA(p, dev_alloc(&w.cell_of, N, s));
  HSM_CUDA(p, dev_alloc(&w.cstart, ncell_max + 1, s));
  HSM_CUDA(p, dev_alloc(&w.ccount, ncell_max, s));
  HSM_CUDA(p, cudaMemsetAsync(w.ccount, 0, ncell_max * sizeof(int32_t), s));  // then every scatter leaves zeros
  HSM_CUDA(p, dev_alloc(&w.sorted_id, N, s));
  HSM_CUDA(p, dev_alloc(&w.sorted_xyz, (size_t)N * kMaxDim, s));
  HSM_CUDA(p, dev_alloc(&w.mon_w64, (size_t)p->nops * (2 * p->dim + 1) * N, s));
  HSM_CUDA(p, dev_alloc(&w.sorted_bnd, N, s));
  HSM_CUDA(p, dev_alloc(&w.scan_ws, scan_scratch(ncell_max), s));
  HSM_CUDA(p, dev_alloc(&w.scan_ws2, scan_scratch(N), s));
  HSM_CUDA(p, dev_alloc(&p->kind, N, s));
  HSM_CUDA(p, dev_alloc(&p->pos, N, s));
  HSM_CUDA(p, dev_alloc(&p->dev_flags, 4, s));
  HSM_CUDA(p, dev_alloc(&p->dev_count, 4, s));
  p->mon.width = 2 * p->dim + 1;
  p->rbf.width = p->n;
  HSM_CUDA(p, dev_alloc(&p->mon.nodes, N, s));
  HSM_CUDA(p, dev_alloc(&p->rbf.nodes, N, s));
  HSM_CUDA(p, dev_alloc(&p->mon.idx, (size_t)p->mon.width * N, s));
  HSM_CUDA(p, dev_alloc(&p->rbf.idx, (size_t)p->rbf.width * N, s));
  HSM_CUDA(p, cudaMallocHost((void**)&w.readback, kReadbackWords * sizeof(int)));
  HSM_CUDA(p, cudaStreamCreateWithFlags(&w.cap, cudaStreamNonBlocking));
  HSM_CUDA(p, cudaStreamCreateWithFlags(&w.side, cudaStreamNonBlocking));
  HSM_CUDA(p, cudaStreamCreateWithFlags(&w.side2, cudaStreamNonBlocking));
  HSM_CUDA(p, cudaStreamCreateWithFlags(&w.side3, cudaStreamNonBlocking));
  for (cudaEvent_t* e : {&w.ev_fork, &w.ev_join, &w.ev_fork2, &w.ev_join2, &w.ev_join3})
    HSM_CUDA(p, cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  for (cudaEvent_t& e : w.ev_chunk) HSM_CUDA(p, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  w.ready = true;
  return HSM_OK;
}

void free_build_ws(hsm_plan p) {
  BuildWs& w = p->ws;
  cudaStream_t s = p->stream;
  if (w.graph) cudaGraphExecDestroy(w.graph);
  w.graph = nullptr;
  for (void** ptr : {(void**)&w.bbox, (void**)&w.lat, (void**)&w.ijk, (void**)&w.on_lat, (void**)&w.hkeys,
                     (void**)&w.hvals, (void**)&w.dmap, (void**)&w.ldesc, (void**)&w.cgd, (void**)&w.cell_of, (void**)&w.cstart, (void**)&w.ccount,
                     (void**)&w.sorted_id, (void**)&w.sorted_xyz, (void**)&w.mon_w64, (void**)&w.sorted_bnd, (void**)&w.scan_ws,
                     (void**)&w.scan_ws2, (void**)&w.bpart, (void**)&w.lpart})
    dev_free(ptr, s);
  if (w.readback) cudaFreeHost(w.readback);
  w.readback = nullptr;
  if (w.cap) cudaStreamDestroy(w.cap);
  if (w.side) cudaStreamDestroy(w.side);
  if (w.side2) cudaStreamDestroy(w.side2);
  if (w.side3) cudaStreamDestroy(w.side3);
  for (cudaEvent_t& e : w.ev_chunk) {
    if (e) cudaEventDestroy(e);
    e = nullptr;
  }
  for (cudaEvent_t* e : {&w.ev_fork, &w.ev_join, &w.ev_fork2, &w.ev_join2, &w.ev_join3}) {
    if (*e) cudaEventDestroy(*e);
    *e = nullptr;
  }
  w.cap = w.side = w.side2 = w.side3 = nullptr;
  w.ready = false;
}

namespace {

#define HSM_TRY(x)                       \
  do {                                   \
    cudaError_t e_ = (x);                \
    if (e_ != cudaSuccess) return e_;    \
  } while (0)

// Enqueues the whole build on stream s without reading anything back: the
// lattice map is a hash table sized from N, the cell grid is derived from the
// bounding box on the device, group sizes stay in device memory and the
// kernels that need them read them there.  The last node copies the group
// sizes, the demotion count and the status bits to pinned host memory.
// Returns the number of kernels enqueued in *nk.
cudaError_t enqueue_build(hsm_plan p, cudaStream_t s, int qt, int* nk) {
  BuildWs& w = p->ws;
  const int64_t N = p->N;
  const int dim = p->dim;
  const int T = 256;
  const int grid = (int)std::min<int64_t>(ceil_div(N, T), (int64_t)num_sms() * 8);
  int k = 0;

  // ---- bounds and lattice coordinates
  // [0,6): lattice extents, [6]: demoted, [7]: n_mon, [8]: n_rbf, [9]: flags, [10]: k_bounds' arrivals
  int* lat = w.lat;
  // k_bounds also zeroes the status flags and counters for the kernels after it
  const int bgrid = (int)std::min<int64_t>(ceil_div(N, kBoundsThreads * kBoundsItems), (int64_t)num_sms() * 8);
  k_bounds<<<bgrid, kBoundsThreads, 0, s>>>(p->coords, N, dim, 1.0 / p->h, w.bpart, w.lpart, w.ijk, w.on_lat,
                                            w.bbox, lat, p->dev_flags, p->dev_count, p->h,
                                            (long long)(4 * N + 1024), static_cast<CellGrid*>(w.cgd),
                                            static_cast<LatticeDense*>(w.ldesc));
  ++k;
  HSM_TRY(cudaGetLastError());
  // lattice map: dense over the lattice's extents when they hold at most
  // 4N + 1024 points, else the hash
  LatticeMap lh;
  lh.hash.dim = dim;
  lh.hash.mask = w.hcap - 1;
  lh.hash.keys = w.hkeys;
  lh.hash.vals = w.hvals;
  lh.dmap = w.dmap;
  lh.desc = static_cast<const LatticeDense*>(w.ldesc);
  // the cell counts start at zero: zeroed at allocation, and every scatter
  // counts its cursors back down to zero
  const int64_t ncell_max = 4 * N + 1024;
  // the map starts empty: cleared once at allocation and by every build
  // after its last reader (the MON stencils, on the side branch)
  if (dim == 2) k_lattice_insert<2><<<grid, T, 0, s>>>(w.ijk, w.on_lat, N, lh);
  else k_lattice_insert<3><<<grid, T, 0, s>>>(w.ijk, w.on_lat, N, lh);
  ++k;
  HSM_TRY(cudaGetLastError());

  // ---- classification
  int* d_demoted = lat + 2 * kMaxDim;
  int* counts = lat + 2 * kMaxDim + 1;
  CellGrid* cgd = static_cast<CellGrid*>(w.cgd);  // set up by k_bounds
  if (dim == 2)
    k_classify_count<2><<<grid, T, 0, s>>>(w.ijk, w.on_lat, p->is_regular, p->is_boundary, N, lh, p->kind, d_demoted,
                                           p->coords, cgd, w.cell_of, w.ccount);
  else
    k_classify_count<3><<<grid, T, 0, s>>>(w.ijk, w.on_lat, p->is_regular, p->is_boundary, N, lh, p->kind, d_demoted,
                                           p->coords, cgd, w.cell_of, w.ccount);
  ++k;
  HSM_TRY(cudaGetLastError());

  // ---- cell scan and scatter on a branch of their own, beside the group
  // partition (each scan with its own block sums); the kNN search joins both
  HSM_TRY(cudaEventRecord(w.ev_fork2, s));
  HSM_TRY(cudaStreamWaitEvent(w.side2, w.ev_fork2, 0));
  HSM_TRY(exclusive_scan_i32(w.ccount, w.cstart, ncell_max, w.side2, w.scan_ws));
  k += scan_kernels(ncell_max);
  k_cell_scatter<<<grid, T, 0, w.side2>>>(p->coords, p->is_boundary, N, dim, w.cell_of, w.cstart, w.ccount,
                                          w.sorted_id, w.sorted_xyz, w.sorted_bnd);
  ++k;
  HSM_TRY(cudaGetLastError());
  HSM_TRY(cudaEventRecord(w.ev_join2, w.side2));

  // ---- group lists (ascending node ids) and positions
  HSM_TRY(partition_indices(p->kind, 0, N, p->mon.nodes, p->rbf.nodes, p->pos, counts, counts + 1, s, w.scan_ws2));
  k += scan_kernels(N);
  // MON stencils on a side branch of the graph, joined before the read-back
  HSM_TRY(cudaEventRecord(w.ev_fork, s));
  HSM_TRY(cudaStreamWaitEvent(w.side, w.ev_fork, 0));
  if (dim == 2) k_mon_stencil<2><<<grid, T, 0, w.side>>>(w.ijk, p->mon.nodes, counts, N, lh, p->mon.idx);
  else k_mon_stencil<3><<<grid, T, 0, w.side>>>(w.ijk, p->mon.nodes, counts, N, lh, p->mon.idx);
  // the map's last reader: empty it for the next build, off the critical path
  k_lattice_clear<<<grid, T, 0, w.side>>>(lh, w.hcap);
  k += 2;
  HSM_TRY(cudaGetLastError());
  // MON weights on the same branch (unless the plan solves both groups in the
  // grouped weights launch): they need only the MON stencils and run beside
  // the kNN search, which leaves most of each SM idle
  if (p->tune.arrange != 1) {
    HSM_TRY(enqueue_mon_weights(p, counts, w.mon_w64, w.side));
    ++k;
  }
  HSM_TRY(cudaEventRecord(w.ev_join, w.side));

  // ---- kNN for the RBF-FD group, once the cells are sorted
  HSM_TRY(cudaStreamWaitEvent(s, w.ev_join2, 0));
  {
    // qt threads per query (1, 2 or 4), blocks of 32 * qt; with the weights
    // in the build, the queries in nch chunks, the RBF-FD weights of chunk c
    // solved on a branch of their own while the search runs on chunk c + 1
    const int nch = p->tune.arrange == 2 ? p->tune.chunks : 1;
    const int KT = 32 * qt;
    size_t smem = (size_t)p->n * KT * (sizeof(double) + sizeof(int32_t));
    int gk = (int)std::min<int64_t>(ceil_div(ceil_div(N, nch), 32), (int64_t)num_sms() * 16);
    void* fn = nullptr;
    if (dim == 2) fn = qt == 4 ? (void*)k_knn<2, 4> : (qt == 2 ? (void*)k_knn<2, 2> : (void*)k_knn<2, 1>);
    else fn = qt == 4 ? (void*)k_knn<3, 4> : (qt == 2 ? (void*)k_knn<3, 2> : (void*)k_knn<3, 1>);
    const double* coords = p->coords;
    const uint8_t* isb = p->is_boundary;
    const double* nrm = p->normals;
    double hh = p->h;
    const double* spc = p->spacing;
    const int32_t* qlist = p->rbf.nodes;
    const int* nqd = counts + 1;
    int nf = p->n;
    int32_t* outp = p->rbf.idx;
    unsigned* fl = p->dev_flags;
    int64_t NN = N;
    int32_t* cs = w.cstart;
    int32_t* sid = w.sorted_id;
    double* sxyz = w.sorted_xyz;
    uint8_t* sb = w.sorted_bnd;
    // first-window radius factor: the radius of the disc (ball) that holds n
    // nodes at density 1, widened by 1.1 for the lower density of a scattered
    // set than of the lattice
    const double omega = dim == 2 ? M_PI : 4.0 * M_PI / 3.0;
    double rfac = 1.1 * std::pow((double)p->n / omega, 1.0 / dim);
    int c = 0, nc = nch;
    void* args[] = {(void*)&coords, (void*)&NN, (void*)&isb, (void*)&nrm, (void*)&hh, (void*)&spc, (void*)&qlist,
                    (void*)&nqd, (void*)&nf, (void*)&rfac, (void*)&cgd, (void*)&cs, (void*)&sid, (void*)&sxyz,
                    (void*)&sb, (void*)&outp, (void*)&fl, (void*)&c, (void*)&nc};
    for (c = 0; c < nch; ++c) {
      HSM_TRY(cudaLaunchKernel(fn, dim3(gk), dim3(KT), args, smem, s));
      ++k;
      if (p->tune.arrange != 2) continue;
      HSM_TRY(cudaEventRecord(w.ev_chunk[c], s));
      HSM_TRY(cudaStreamWaitEvent(w.side3, w.ev_chunk[c], 0));
      if (c == 0 && p->timing)
        HSM_TRY(cudaEventRecordWithFlags(p->ev[2 * HSM_PHASE_RBF], w.side3, cudaEventRecordExternal));
      HSM_TRY(enqueue_rbf_chunk(p, nqd, p->rbf.w64, c, nch, w.side3));
      ++k;
    }
    if (p->tune.arrange == 2) {
      if (p->timing)
        HSM_TRY(cudaEventRecordWithFlags(p->ev[2 * HSM_PHASE_RBF + 1], w.side3, cudaEventRecordExternal));
      HSM_TRY(cudaEventRecord(w.ev_join3, w.side3));
      HSM_TRY(cudaStreamWaitEvent(s, w.ev_join3, 0));
    }
  }
  // ---- status words next to the counters, then the one read-back
  HSM_TRY(cudaStreamWaitEvent(s, w.ev_join, 0));
  k_build_status<<<1, 1, 0, s>>>(p->dev_flags, p->dev_count, lat + 2 * kMaxDim);
  ++k;
  HSM_TRY(cudaGetLastError());
  HSM_TRY(cudaMemcpyAsync(w.readback, lat + 2 * kMaxDim, kReadbackWords * sizeof(int), cudaMemcpyDeviceToHost, s));
  *nk = k;
  return cudaSuccess;
}

#undef HSM_TRY

}  // namespace

// The build is captured once per plan (and kNN variant) as a CUDA graph on a
// private stream and replayed on the plan's stream: one graph launch and one
// synchronisation per build instead of some fifty API calls.
hsm_status build_stencils(hsm_plan p) {
  hsm_status st = alloc_build_ws(p);
  if (st != HSM_OK) return st;
  BuildWs& w = p->ws;
  cudaStream_t s = p->stream;
  const int qt = p->tune.knn_qt == 4 ? 4 : (p->tune.knn_qt == 2 ? 2 : 1);
  const bool in_build = p->tune.arrange == 2;
  if (in_build) {
    // the in-build solve writes the plan's RBF-FD weight array and singular
    // list, sized here for a group of every node (the graph keeps the pointers)
    const int64_t need = (int64_t)p->nops * p->n * p->N;
    if (!p->rbf.w64 || p->rbf.w64_cap < need) {
      dev_free(&p->rbf.w64, s);
      p->rbf.w64_cap = 0;
      HSM_CUDA(p, dev_alloc(&p->rbf.w64, (size_t)need, s));
      p->rbf.w64_cap = need;
    }
    if (p->m >= 2 && p->sing_cap < p->N) {
      dev_free(&p->sing_list, s);
      p->sing_cap = 0;
      HSM_CUDA(p, dev_alloc(&p->sing_list, 2 * (size_t)p->N, s));
      p->sing_cap = p->N;
    }
    if (rbf_chunk_ready(p) != cudaSuccess)
      return set_error(p, HSM_EINVAL, "RBF-FD system too large for the in-build weights arrangement");
    if (p->timing && !p->ev[2 * HSM_PHASE_RBF]) {
      HSM_CUDA(p, cudaEventCreate(&p->ev[2 * HSM_PHASE_RBF]));
      HSM_CUDA(p, cudaEventCreate(&p->ev[2 * HSM_PHASE_RBF + 1]));
    }
  }
  const bool timing = in_build && p->timing;
  if (!w.graph || w.graph_qt != qt || w.graph_spacing != p->spacing || w.graph_arrange != p->tune.arrange ||
      w.graph_chunks != p->tune.chunks || w.graph_timing != timing ||
      (in_build && (w.graph_w64 != p->rbf.w64 || w.graph_sing != p->sing_list))) {
    if (w.graph) cudaGraphExecDestroy(w.graph);
    w.graph = nullptr;
    // kernel attributes are set outside the capture
    const size_t smem = (size_t)p->n * 32 * qt * (sizeof(double) + sizeof(int32_t));
    void* fn = nullptr;
    if (p->dim == 2) fn = qt == 4 ? (void*)k_knn<2, 4> : (qt == 2 ? (void*)k_knn<2, 2> : (void*)k_knn<2, 1>);
    else fn = qt == 4 ? (void*)k_knn<3, 4> : (qt == 2 ? (void*)k_knn<3, 2> : (void*)k_knn<3, 1>);
    if (smem > 48 * 1024) HSM_CUDA(p, raise_smem_limit(fn, smem));
    // the workspace allocations must be complete before the captured work runs
    HSM_CUDA(p, cudaStreamSynchronize(s));
    HSM_CUDA(p, cudaStreamBeginCapture(w.cap, cudaStreamCaptureModeThreadLocal));
    int nk = 0;
    cudaError_t e = enqueue_build(p, w.cap, qt, &nk);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(w.cap, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&w.graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      w.graph = nullptr;
      HSM_CUDA(p, e);
    }
    w.graph_qt = qt;
    w.graph_spacing = p->spacing;
    w.graph_arrange = p->tune.arrange;
    w.graph_chunks = p->tune.chunks;
    w.graph_timing = timing;
    w.graph_w64 = p->rbf.w64;
    w.graph_sing = p->sing_list;
    w.graph_kernels = nk;
  }
  HSM_CUDA(p, cudaGraphLaunch(w.graph, s));
  p->launches += w.graph_kernels;
  p->counters_fresh = true;  // k_bounds cleared the weights call's status words
  p->rbf_from_build = in_build;
  if (timing) p->ev_used[HSM_PHASE_RBF] = true;
  HSM_CUDA(p, cudaStreamSynchronize(s));
  const int* rb = w.readback;
  p->n_demoted = rb[0];
  p->mon.count = rb[1];
  p->rbf.count = rb[2];
  p->build_flags = (unsigned)rb[3];
  p->build_sing = rb[5];
  p->build_solve_flags = (unsigned)rb[6];
  p->mon.w64 = w.mon_w64;
  if ((unsigned)rb[3] & kDevKnnShort)
    return set_error(p, HSM_EINVAL, "not enough candidate nodes for an RBF-FD stencil");
  p->stencils_built = true;
  return HSM_OK;
}

}  // namespace hsm
