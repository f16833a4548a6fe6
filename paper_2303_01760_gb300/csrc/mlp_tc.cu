// Fused forward pass of the learned-weight MLP on the 5th-generation tensor
// cores.  One CTA per SM walks its 128-row tiles two at a time (two slots,
// each with its own activation buffer and tensor-memory accumulator), and a
// tile goes through every layer without leaving the SM:
//
//   * warp 0 streams each tile's padded bf16 inputs into its slot's
//     activation buffer and the weight matrices (64-column K slices, two
//     stages) into shared memory with TMA (cp.async.bulk.tensor, 128-byte
//     swizzle);
//   * warp 1 owns two 128 x 256 FP32 accumulators in tensor memory (512
//     columns) and issues tcgen05.mma (M = 128, N = layer width, K = 16 per
//     instruction) with both operands K-major in shared memory, alternating
//     the slots layer by layer and committing to mbarriers;
//   * warps 4..19 drain an accumulator with tcgen05.ld (each warp its lane
//     quarter, a quarter of the columns), add the bias, apply GELU and write
//     the bf16 activations straight back into the slot's buffer in the
//     swizzled K-major layout the next layer's MMA reads; the last layer adds
//     its bias and writes FP32 outputs to global memory.
//
// While the epilogue drains one slot the tensor cores run the other slot's
// layer.  Only the inputs and outputs touch HBM.  Every wait on an mbarrier
// is bounded: on expiry the kernel records an error flag, every role leaves
// its loop and the tensor memory is released.
#include <cuda.h>

#include "gelu.cuh"
#include "mlp.cuh"

namespace hsm {
namespace {

constexpr int kThreads = 640;
constexpr int kTileRows = 128;
constexpr int kEpiWarps = 16;  // warps 4..19: four per TMEM lane quarter
constexpr int kStages = 2;
constexpr int kSlots = 2;
constexpr int kMaxLayers = 4;
constexpr int kActBytes = 4 * 16384;     // 128 rows x 256 bf16, four 64-column K slices; inputs land in slice 0
constexpr int kWStageBytes = 256 * 128;  // up to 256 rows x 64 bf16
constexpr int kBiasBytes = kMaxLayers * 256 * 4;
constexpr int kSmemBytes = kSlots * kActBytes + kStages * kWStageBytes + kBiasBytes + 256 + 1024;
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kMaxSpins = 1u << 20;

struct TcArgs {
  int nl;
  int din[kMaxLayers], dout[kMaxLayers];
  const float* bias[kMaxLayers];
  int64_t rows;
  float* Y;
  int ldy, ncols;
  unsigned* err;
  int hold_loads;  // test hook: the producer issues nothing, so the consumers' bounded waits expire
};

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(b)) : "memory");
}
// Waits for the phase of parity `par` to complete; false after kMaxSpins
// polls or once another role has given up.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t par, volatile int* abort_flag, unsigned* err) {
  const uint32_t a = saddr(b);
  for (uint32_t it = 0; it < kMaxSpins; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(a), "r"(par)
        : "memory");
    if (ok) return true;
    if (*abort_flag) return false;
  }
  *abort_flag = 1;
  atomicOr(err, 1u);
  return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          saddr(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(saddr(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major tile with 128-byte rows and
// the 128-byte swizzle: 8-row groups 1024 bytes apart (stride byte offset),
// descriptor version 1, swizzle mode 2.  The leading byte offset is not used
// by swizzled K-major layouts.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// Instruction descriptor of kind::f16: FP32 accumulator, bf16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__device__ __forceinline__ uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void umma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(
          d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
               : "memory");
}

// 32 consecutive FP32 columns of this thread's accumulator row.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__global__ void __launch_bounds__(kThreads, 1)
    k_mlp_tc(TcArgs a, const __grid_constant__ CUtensorMap tx, const __grid_constant__ CUtensorMap tw0,
             const __grid_constant__ CUtensorMap tw1, const __grid_constant__ CUtensorMap tw2,
             const __grid_constant__ CUtensorMap tw3) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t* act = base;                      // [slot][4 slices][128 rows][128 B]
  uint8_t* wb = act + kSlots * kActBytes;   // [stage][<=256 rows][128 B]
  float* sbias = reinterpret_cast<float*>(wb + kStages * kWStageBytes);  // [layer][256]
  uint64_t* bars = reinterpret_cast<uint64_t*>(sbias + kMaxLayers * 256);
  uint64_t* wfull = bars;                   // [stage]
  uint64_t* wempty = wfull + kStages;       // [stage]
  uint64_t* xfull = wempty + kStages;       // [slot] inputs landed
  uint64_t* actfree = xfull + kSlots;       // [slot] last layer's MMAs done: buffer free for new inputs
  uint64_t* accfull = actfree + kSlots;     // [slot] a layer's MMAs done
  uint64_t* accempty = accfull + kSlots;    // [slot] a layer's epilogue done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accempty + kSlots);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&wfull[s], 1);
      mbar_init(&wempty[s], 1);
    }
    for (int s = 0; s < kSlots; ++s) {
      mbar_init(&xfull[s], 1);
      mbar_init(&actfree[s], 1);
      mbar_init(&accfull[s], 1);
      mbar_init(&accempty[s], kEpiWarps);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int i = threadIdx.x; i < kMaxLayers * 256; i += blockDim.x) {
    const int l = i >> 8, c = i & 255;
    sbias[i] = (l < a.nl && c < a.dout[l]) ? a.bias[l][c] : 0.f;
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int64_t ntiles = (a.rows + kTileRows - 1) / kTileRows;
  const int64_t mine = ntiles > blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;  // tiles of this CTA
  const int64_t npairs = (mine + 1) / 2;
  const CUtensorMap* tw[kMaxLayers] = {&tw0, &tw1, &tw2, &tw3};
  // tile of slot s in pair p, or -1
  auto tile_of = [&](int64_t p, int s) -> int64_t {
    const int64_t j = 2 * p + s;
    return j < mine ? blockIdx.x + j * (int64_t)gridDim.x : -1;
  };

  if (warp == 0 && lane == 0 && !a.hold_loads) {
    // ---- producer: each slot's inputs, then the weight slices in MMA order
    uint32_t seq = 0, nx[kSlots] = {0, 0};
    bool ok = true;
    for (int64_t p = 0; p < npairs && ok; ++p) {
      for (int s = 0; s < kSlots && ok; ++s) {
        const int64_t tile = tile_of(p, s);
        if (tile < 0) continue;
        ok = mbar_wait(&actfree[s], (nx[s] & 1) ^ 1, abort_flag, a.err);
        if (!ok) break;
        ++nx[s];
        mbar_expect_tx(&xfull[s], 16384u);
        tma_load_2d(act + s * kActBytes, &tx, 0, (int)(tile * kTileRows), &xfull[s]);
      }
      for (int l = 0; l < a.nl && ok; ++l)
        for (int s = 0; s < kSlots && ok; ++s) {
          if (tile_of(p, s) < 0) continue;
          for (int c = 0; c < a.din[l] / 64 && ok; ++c, ++seq) {
            const uint32_t st = seq % kStages, u = seq / kStages;
            ok = mbar_wait(&wempty[st], (u & 1) ^ 1, abort_flag, a.err);
            if (!ok) break;
            mbar_expect_tx(&wfull[st], (uint32_t)a.dout[l] * 128u);
            tma_load_2d(wb + st * kWStageBytes, tw[l], c * 64, 0, &wfull[st]);
          }
        }
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer: layer by layer, alternating the slots
    uint32_t seq = 0, nx[kSlots] = {0, 0}, njob[kSlots] = {0, 0};
    bool ok = true;
    for (int64_t p = 0; p < npairs && ok; ++p)
      for (int l = 0; l < a.nl && ok; ++l)
        for (int s = 0; s < kSlots && ok; ++s) {
          if (tile_of(p, s) < 0) continue;
          ok = mbar_wait(&accempty[s], (njob[s] & 1) ^ 1, abort_flag, a.err);
          ++njob[s];
          if (ok && l == 0) {
            ok = mbar_wait(&xfull[s], nx[s] & 1, abort_flag, a.err);
            ++nx[s];
          }
          if (!ok) break;
          tc_fence_after();
          const uint32_t idesc = idesc_bf16(kTileRows, a.dout[l]);
          const uint32_t d = tmem + (uint32_t)(s * 256);
          for (int c = 0; c < a.din[l] / 64; ++c, ++seq) {
            const uint32_t st = seq % kStages, u = seq / kStages;
            ok = mbar_wait(&wfull[st], u & 1, abort_flag, a.err);
            if (!ok) break;
            tc_fence_after();
            const uint64_t ad = sw128_desc(saddr(act + s * kActBytes + c * 16384));
            const uint64_t bd = sw128_desc(saddr(wb + st * kWStageBytes));
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)  // K = 16 per MMA: 32 bytes along the swizzled row
              umma(d, ad + 2 * kk, bd + 2 * kk, idesc, (c | kk) != 0 ? 1u : 0u);
            umma_commit(&wempty[st]);
          }
          if (!ok) break;
          umma_commit(&accfull[s]);
          if (l == a.nl - 1) umma_commit(&actfree[s]);
        }
  } else if (warp >= 4) {
    // ---- epilogue: TMEM -> bias (+ GELU) -> the slot's activations or global outputs
    const int q = warp & 3, part = (warp - 4) >> 2;  // lane quarter, column quarter
    const int r = 32 * q + lane;
    uint32_t njob[kSlots] = {0, 0};
    bool ok = true;
    for (int64_t p = 0; p < npairs && ok; ++p)
      for (int l = 0; l < a.nl && ok; ++l)
        for (int s = 0; s < kSlots && ok; ++s) {
          const int64_t tile = tile_of(p, s);
          if (tile < 0) continue;
          ok = mbar_wait(&accfull[s], njob[s] & 1, abort_flag, a.err);
          ++njob[s];
          ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld needs the whole warp
          if (!ok) break;
          tc_fence_after();
          const uint32_t trow = tmem + (uint32_t)(s * 256) + ((uint32_t)(32 * q) << 16);
          uint8_t* sact = act + s * kActBytes;
          const int N = a.dout[l], c0 = part * (N / 4);
          const float* bias = sbias + l * 256;
          const bool last = l == a.nl - 1;
          for (int cc = c0; cc < c0 + N / 4; cc += 32) {
            float v[32];
            tmem_ld32(trow + (uint32_t)cc, v);
            if (!last) {
#pragma unroll
              for (int j = 0; j < 32; j += 8) {
                uint32_t pk[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                  const float g0 = gelu(v[j + 2 * t] + bias[cc + j + 2 * t]);
                  const float g1 = gelu(v[j + 2 * t + 1] + bias[cc + j + 2 * t + 1]);
                  const __nv_bfloat162 h2 = __floats2bfloat162_rn(g0, g1);
                  pk[t] = *reinterpret_cast<const uint32_t*>(&h2);
                }
                const int k = cc + j;  // the next layer's K index
                const uint32_t dst =
                    saddr(sact + (k >> 6) * 16384 + r * 128 + ((((k & 63) >> 3) ^ (r & 7)) << 4));
                asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(dst), "r"(pk[0]), "r"(pk[1]),
                             "r"(pk[2]), "r"(pk[3])
                             : "memory");
              }
            } else {
              const int64_t row = tile * kTileRows + r;
              if (row < a.rows) {
                float* y = a.Y + row * (int64_t)a.ldy;
#pragma unroll
                for (int j = 0; j < 32; ++j)
                  if (cc + j < a.ncols) y[cc + j] = v[j] + bias[cc + j];
              }
            }
          }
          tc_fence_before();
          // the activations written here are read next by the tensor cores (async proxy)
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          __syncwarp();
          if (lane == 0) mbar_arrive(&accempty[s]);
        }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// 2D bf16 row-major [outer][inner] tensor, boxes of [box_outer][64] with the
// 128-byte swizzle (64 bf16 = one 128-byte row).
bool make_map(CUtensorMap* m, const void* ptr, uint64_t inner, uint64_t outer, uint32_t box_outer) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {inner, outer};
  const cuuint64_t strides[1] = {inner * 2};
  const cuuint32_t box[2] = {64, box_outer};
  const cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 2D bf16 row-major tensor [outer][inner] with row stride ld elements, boxes
// of [box_outer][64] with the 128-byte swizzle.
bool make_map_ld(CUtensorMap* m, const void* ptr, uint64_t inner, uint64_t outer, uint64_t ld, uint32_t box_outer) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {inner, outer};
  const cuuint64_t strides[1] = {ld * 2};
  const cuuint32_t box[2] = {64, box_outer};
  const cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// ---- training GEMMs ------------------------------------------------------------
// C[M x N] = A[M x K] B[N x K]^T with A and B bf16 K-major in global memory
// (row-major [M][K] and [N][K]), FP32 accumulation in tensor memory.  One
// 128 x BN output tile per CTA (BN = 64 or 128):
//
//   * warp 0 streams 64-column K slices of A and B into a four-stage ring with
//     TMA (128-byte swizzle);
//   * warp 1 allocates BN tensor-memory columns and issues tcgen05.mma
//     (M = 128, N = BN, K = 16 per instruction), committing each stage back
//     to the producer and, after the last slice, to the epilogue;
//   * warps 4..7 drain the accumulator with tcgen05.ld (warp 4 + q reads lane
//     quarter q: rows 32q .. 32q + 31) and apply the layer's epilogue.
//
// Every mbarrier wait is bounded.  On expiry the error flag is set and every
// role leaves its loop; the producer then waits (bounded) for the copies it
// issued, the MMA issuer for its issued MMAs, and only then is the tensor
// memory released.
constexpr int kGThreads = 256;
constexpr int kGStages = 4;
constexpr int kGStageBytes = 128 * 128;  // 128 rows x 64 bf16
constexpr int kGSmemBytes = 2 * kGStages * kGStageBytes + 256 + 1024;

struct GemmTcArgs {
  int M, N, K, BN, epi;
  const float* bias;   // [N] (MLP_EPI_BIAS_GELU, MLP_EPI_BIAS)
  const float* Zin;    // [M][N] pre-activations (MLP_EPI_DGELU)
  float* Cf;           // [M][N] FP32 output (MLP_EPI_BIAS, MLP_EPI_F32)
  float* Zout;         // [M][N] pre-activations (MLP_EPI_BIAS_GELU)
  __nv_bfloat16* Ch;   // [M][N] bf16 output (MLP_EPI_BIAS_GELU, MLP_EPI_DGELU)
  __nv_bfloat16* Cht;  // [N][ldt] its transpose, or nullptr
  int64_t ldt;
  unsigned* err;
};

// d GELU / dz = Phi(z) + z phi(z), with the erf of gelu()
__device__ __forceinline__ float gelu_grad(float z) {
  const float e = erf_as(fabsf(z) * 0.70710678118654752f);
  const float Phi = 0.5f * (1.0f + (z < 0.0f ? -e : e));
  return fmaf(z * 0.39894228040143268f, __expf(-0.5f * z * z), Phi);
}

// a bounded wait that ignores the abort flag (draining after an abort)
__device__ __forceinline__ void mbar_drain(uint64_t* b, uint32_t par) {
  const uint32_t a = saddr(b);
  for (uint32_t it = 0; it < kMaxSpins; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(a), "r"(par)
        : "memory");
    if (ok) return;
  }
}

__global__ void __launch_bounds__(kGThreads, 1)
    k_gemm_tc(GemmTcArgs a, const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t* sa = base;                          // [stage][128 rows][128 B]
  uint8_t* sb = sa + kGStages * kGStageBytes;  // [stage][BN rows][128 B]
  uint64_t* full = reinterpret_cast<uint64_t*>(sb + kGStages * kGStageBytes);
  uint64_t* empty = full + kGStages;
  uint64_t* accfull = empty + kGStages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accfull + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  int* issued = const_cast<int*>(abort_flag) + 1;    // K slices the producer issued
  int* consumed = issued + 1;                        // K slices the MMA issuer consumed
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * 128, n0 = blockIdx.x * a.BN;
  const int KT = a.K / 64;
  if (threadIdx.x == 0) {
    for (int st = 0; st < kGStages; ++st) {
      mbar_init(&full[st], 1);
      mbar_init(&empty[st], 1);
    }
    mbar_init(accfull, 1);
    *abort_flag = 0;
    *issued = 0;
    *consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(tmem_slot)),
                 "r"((uint32_t)a.BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  bool mma_done = false;
  if (warp == 0 && lane == 0) {
    // ---- producer
    int c = 0;
    for (; c < KT; ++c) {
      const int st = c % kGStages;
      const uint32_t u = (uint32_t)(c / kGStages);
      if (!mbar_wait(&empty[st], (u & 1) ^ 1, abort_flag, a.err)) break;
      mbar_expect_tx(&full[st], (uint32_t)(128 + a.BN) * 128u);
      tma_load_2d(sa + st * kGStageBytes, &ta, c * 64, m0, &full[st]);
      tma_load_2d(sb + st * kGStageBytes, &tb, c * 64, n0, &full[st]);
    }
    *issued = c;
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer
    const uint32_t idesc = idesc_bf16(128, a.BN);
    int c = 0;
    for (; c < KT; ++c) {
      const int st = c % kGStages;
      const uint32_t u = (uint32_t)(c / kGStages);
      if (!mbar_wait(&full[st], u & 1, abort_flag, a.err)) break;
      tc_fence_after();
      const uint64_t ad = sw128_desc(saddr(sa + st * kGStageBytes));
      const uint64_t bd = sw128_desc(saddr(sb + st * kGStageBytes));
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) umma(tmem, ad + 2 * kk, bd + 2 * kk, idesc, (c | kk) != 0 ? 1u : 0u);
      umma_commit(&empty[st]);
    }
    *consumed = c;
    // the accumulator is complete (or, after an abort, every issued MMA has
    // finished) when this commit arrives
    umma_commit(accfull);
    mma_done = c == KT;
  } else if (warp >= 4) {
    // ---- epilogue
    const int q = warp & 3;
    const int64_t row = m0 + 32 * q + lane;
    bool ok = mbar_wait(accfull, 0, abort_flag, a.err);
    ok = __all_sync(0xffffffffu, ok) && !*abort_flag;
    if (ok) {
      tc_fence_after();
      const uint32_t trow = tmem + ((uint32_t)(32 * q) << 16);
      for (int cc = 0; cc < a.BN; cc += 32) {
        float v[32];
        tmem_ld32(trow + (uint32_t)cc, v);
        const int n = n0 + cc;
        const int64_t o = row * a.N + n;
        if (a.epi == MLP_EPI_BIAS_GELU) {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const float z = v[j] + a.bias[n + j];
            a.Zout[o + j] = z;
            v[j] = gelu(z);
          }
        } else if (a.epi == MLP_EPI_BIAS) {
#pragma unroll
          for (int j = 0; j < 32; ++j) a.Cf[o + j] = v[j] + a.bias[n + j];
          continue;
        } else if (a.epi == MLP_EPI_DGELU) {
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] *= gelu_grad(a.Zin[o + j]);
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j) a.Cf[o + j] = v[j];
          continue;
        }
        // bf16 outputs: the row, and its transpose (consecutive rows of a warp
        // are consecutive entries of a transposed row)
#pragma unroll
        for (int j = 0; j < 32; j += 8) {
          uint4 pk;
          uint32_t* w = reinterpret_cast<uint32_t*>(&pk);
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[j + 2 * t], v[j + 2 * t + 1]);
            w[t] = *reinterpret_cast<const uint32_t*>(&h2);
          }
          *reinterpret_cast<uint4*>(a.Ch + o + j) = pk;
        }
        if (a.Cht)
#pragma unroll
          for (int j = 0; j < 32; ++j) a.Cht[(int64_t)(n + j) * a.ldt + row] = __float2bfloat16(v[j]);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  // after an abort: the copies issued and not consumed, and the issued MMAs,
  // finish before the shared and tensor memory are given up
  if (warp == 0 && lane == 0) {
    for (int c = *consumed; c < *issued; ++c) mbar_drain(&full[c % kGStages], (uint32_t)(c / kGStages) & 1);
  }
  if (warp == 1 && lane == 0 && !mma_done) mbar_drain(accfull, 0);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)a.BN) : "memory");
  }
}

}  // namespace

hsm_status mlp_gemm_tc(Mlp& m, const MlpGemm& g) {
  if (g.M % 128 || g.K % 64 || g.N % 64 || g.M <= 0 || g.N <= 0 || g.K <= 0) return HSM_EINVAL;
  cudaStream_t s = m.stream;
  if (!m.tc_err) {
    if (dev_alloc(&m.tc_err, 1, s) != cudaSuccess) return HSM_ENOMEM;
    if (cudaMemsetAsync(m.tc_err, 0, sizeof(unsigned), s) != cudaSuccess) return HSM_ECUDA;
  }
  GemmTcArgs a{};
  a.M = g.M;
  a.N = g.N;
  a.K = g.K;
  a.BN = g.N % 128 == 0 ? 128 : 64;
  a.epi = g.epi;
  a.bias = g.bias;
  a.Zin = g.Zin;
  a.Cf = g.Cf;
  a.Zout = g.Zout;
  a.Ch = g.Ch;
  a.Cht = g.Cht;
  a.ldt = g.ldt;
  a.err = m.tc_err;
  CUtensorMap ta, tb;
  memset(&ta, 0, sizeof(ta));
  memset(&tb, 0, sizeof(tb));
  if (!make_map_ld(&ta, g.A, (uint64_t)g.K, (uint64_t)g.M, (uint64_t)g.lda, 128) ||
      !make_map_ld(&tb, g.B, (uint64_t)g.K, (uint64_t)g.N, (uint64_t)g.ldb, (uint32_t)a.BN))
    return HSM_ECUDA;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kGSmemBytes) != cudaSuccess)
      return HSM_ECUDA;
    attr = true;
  }
  k_gemm_tc<<<dim3((unsigned)(g.N / a.BN), (unsigned)(g.M / 128)), kGThreads, kGSmemBytes, s>>>(a, ta, tb);
  return cudaGetLastError() == cudaSuccess ? HSM_OK : HSM_ECUDA;
}

bool mlp_forward_tc_supported(const Mlp& m) {
  if (m.nl < 2 || m.nl > kMaxLayers || m.din[0] != 64) return false;
  for (int l = 0; l < m.nl; ++l) {
    if (m.din[l] % 64 || m.din[l] > 256) return false;
    if (m.dout[l] != 128 && m.dout[l] != 256) return false;
    if (l + 1 < m.nl && m.din[l + 1] != m.dout[l]) return false;
  }
  return encode_fn() != nullptr;
}

hsm_status mlp_forward_tc(Mlp& m, const __nv_bfloat16* X, int64_t rows, float* Y, int ldy) {
  if (rows <= 0) return HSM_OK;
  cudaStream_t s = m.stream;
  if (!m.tc_err) {
    if (dev_alloc(&m.tc_err, 1, s) != cudaSuccess) return HSM_ENOMEM;
    if (cudaMemsetAsync(m.tc_err, 0, sizeof(unsigned), s) != cudaSuccess) return HSM_ECUDA;
  }
  TcArgs a{};
  a.nl = m.nl;
  CUtensorMap maps[1 + kMaxLayers];
  memset(maps, 0, sizeof(maps));
  const int64_t rows_pad = (rows + kTileRows - 1) / kTileRows * kTileRows;
  if (!make_map(&maps[0], X, 64, (uint64_t)rows_pad, kTileRows)) return HSM_ECUDA;
  for (int l = 0; l < m.nl; ++l) {
    a.din[l] = m.din[l];
    a.dout[l] = m.dout[l];
    a.bias[l] = m.master + m.b_off[l];
    if (!make_map(&maps[1 + l], m.wbf + m.wbf_off[l], (uint64_t)m.din[l], (uint64_t)m.dout[l], (uint32_t)m.dout[l]))
      return HSM_ECUDA;
  }
  for (int l = m.nl; l < kMaxLayers; ++l) maps[1 + l] = maps[1];
  a.rows = rows;
  a.Y = Y;
  a.ldy = ldy;
  a.ncols = m.n_out;
  a.err = m.tc_err;
  a.hold_loads = m.fault_hold_loads;
  m.fault_hold_loads = 0;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(k_mlp_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes) != cudaSuccess)
      return HSM_ECUDA;
    attr = true;
  }
  const int64_t ntiles = rows_pad / kTileRows;
  const int grid = (int)std::min<int64_t>(ntiles, (int64_t)num_sms());
  k_mlp_tc<<<grid, kThreads, kSmemBytes, s>>>(a, maps[0], maps[1], maps[2], maps[3], maps[4]);
  return cudaGetLastError() == cudaSuccess ? HSM_OK : HSM_ECUDA;
}

}  // namespace hsm
