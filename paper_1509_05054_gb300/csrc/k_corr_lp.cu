// Reduced-precision correlations on tcgen05 tensor cores: alpha0 = D^T y for a
// tile of 128 signals with BF16 operands (kind::f16) or E4M3 operands with
// per-signal and per-atom scales (kind::f8f6f4), FP32 accumulation in TMEM.
// This is the mixed-precision form of Algorithm 1 step 1; the OMP loop that
// consumes alpha0 stays FP32.
//
// Operands are converted once into padded row-major buffers (row = one signal
// or one atom, rows padded to a multiple of 128 bytes with zeros), so one TMA
// box of 128 bytes x rows covers K in 128-byte swizzle chunks.  Per CTA: TMA
// the A tile (128 signals), then per block of 256 atoms TMA the B block, issue
// 4 MMAs per 128-byte chunk (K = 16 BF16 or 32 E4M3 per MMA), commit, and drain
// TMEM with tcgen05.ld; E4M3 results are multiplied by the two inverse scales.
// Every mbarrier wait is bounded (ERR_TIMEOUT on expiry).
#include "dl_internal.cuh"
#include "tc_ptx.cuh"

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cudaTypedefs.h>
#include <stdint.h>

namespace dlk {
namespace {

using namespace tc;

constexpr int LP_THREADS = 128;
constexpr int TILE_M = 128;
constexpr int BLOCK_N = 256;
constexpr int CHUNK_BYTES = 128;

template <int KIND>
struct LpTraits;
template <>
struct LpTraits<LP_BF16> {
  static constexpr int esize = 2;
  // kind::f16: D F32, A/B BF16, K-major, N = 256, M = 128
  static constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) |
                                    ((uint32_t)(BLOCK_N >> 3) << 17) | ((uint32_t)(TILE_M >> 4) << 24);
};
template <>
struct LpTraits<LP_E4M3> {
  static constexpr int esize = 1;
  // kind::f8f6f4: D F32, A/B E4M3 (format 0), K-major, N = 256, M = 128
  static constexpr uint32_t idesc = (1u << 4) | (0u << 7) | (0u << 10) |
                                    ((uint32_t)(BLOCK_N >> 3) << 17) | ((uint32_t)(TILE_M >> 4) << 24);
};

constexpr size_t kAChunk = (size_t)TILE_M * CHUNK_BYTES;   // 16 KB
constexpr size_t kBChunk = (size_t)BLOCK_N * CHUNK_BYTES;  // 32 KB

template <int KIND>
__global__ void __launch_bounds__(LP_THREADS, 1)
    corr_lp_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   int64_t rows_a, int n, int kb, const float* __restrict__ row_scale,
                   const float* __restrict__ col_scale, float* __restrict__ C, int64_t ldc,
                   int* __restrict__ err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* As = base;
  uint8_t* Bs = base + kb * kAChunk;
  uint64_t* bars = (uint64_t*)(Bs + kb * kBChunk);
  uint32_t* tmem_slot = (uint32_t*)(bars + 4);
  __shared__ int s_fail;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i0 = (int64_t)blockIdx.x * TILE_M;
  const int nblocks = (n + BLOCK_N - 1) / BLOCK_N;
  const uint32_t ncols = nblocks <= 1 ? 256u : 512u;

  if (threadIdx.x == 0) {
    s_fail = 0;
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    mbar_init(&bars[2], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  constexpr int EPC = CHUNK_BYTES / LpTraits<KIND>::esize;  // elements per chunk

  if (threadIdx.x == 0) {
    mbar_expect_tx(&bars[0], (uint32_t)(kb * kAChunk));
    for (int q = 0; q < kb; ++q) tma_load_2d(As + q * kAChunk, &tmA, &bars[0], q * EPC, (int)i0);
    bool ok = mbar_wait(&bars[0], 0);
    for (int nb = 0; nb < nblocks && ok; ++nb) {
      mbar_expect_tx(&bars[1], (uint32_t)(kb * kBChunk));
      for (int q = 0; q < kb; ++q)
        tma_load_2d(Bs + q * kBChunk, &tmB, &bars[1], q * EPC, nb * BLOCK_N);
      ok = mbar_wait(&bars[1], (uint32_t)(nb & 1));
      if (!ok) break;
      tc_fence_after();
      const uint32_t dcol = tmem + (uint32_t)(nb * BLOCK_N);
      uint32_t accum = 0;
      for (int q = 0; q < kb; ++q) {
        const uint64_t ad = sw128_desc(As + q * kAChunk);
        const uint64_t bd = sw128_desc(Bs + q * kBChunk);
#pragma unroll
        for (int k = 0; k < 4; ++k) {  // 32 bytes of K per MMA
          if constexpr (KIND == LP_BF16)
            mma_f16(dcol, ad + (uint64_t)(2 * k), bd + (uint64_t)(2 * k), LpTraits<KIND>::idesc, accum);
          else
            mma_f8f6f4(dcol, ad + (uint64_t)(2 * k), bd + (uint64_t)(2 * k), LpTraits<KIND>::idesc, accum);
          accum = 1;
        }
      }
      mma_commit(&bars[2]);
      ok = mbar_wait(&bars[2], (uint32_t)(nb & 1));
    }
    if (!ok) s_fail = 1;
  }
  __syncthreads();
  tc_fence_after();
  if (!s_fail) {
    const int64_t row = i0 + warp * 32 + lane;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    const float rs = (KIND == LP_E4M3 && row < rows_a) ? row_scale[row] : 1.f;
    for (int c0 = 0; c0 < n; c0 += 16) {
      uint32_t r[16];
      tmem_ld16(tmem + lane_base + (uint32_t)c0, r);
      if (row < rows_a) {
        float v[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          v[q] = __uint_as_float(r[q]);
          if (KIND == LP_E4M3) v[q] *= rs * __ldg(col_scale + c0 + q);
        }
        float4* dst = (float4*)(C + row * ldc + c0);
#pragma unroll
        for (int q = 0; q < 4; ++q) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
      }
    }
  } else if (threadIdx.x == 0) {
    atomicOr(err, ERR_TIMEOUT);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols)
                 : "memory");
}

// rows x p FP32 -> rows x ld BF16 (zero padded).
__global__ void to_bf16_kernel(const float* __restrict__ src, int64_t rows, int p, int ld,
                               __nv_bfloat16* __restrict__ dst) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * ld) return;
  const int64_t r = e / ld;
  const int c = (int)(e - r * ld);
  dst[e] = __float2bfloat16_rn(c < p ? src[r * p + c] : 0.f);
}

// rows x p FP32 -> rows x ld E4M3 (zero padded), one warp per row: the row is
// scaled so that its largest magnitude maps to 448 (the E4M3 maximum);
// inv_scale[r] = max|row| / 448 undoes it.
__global__ void to_e4m3_kernel(const float* __restrict__ src, int64_t rows, int p, int ld,
                               uint8_t* __restrict__ dst, float* __restrict__ inv_scale) {
  const int lane = threadIdx.x & 31;
  const int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= rows) return;
  float mx = 0.f;
  for (int c = lane; c < p; c += 32) mx = fmaxf(mx, fabsf(src[r * p + c]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  const float scale = mx > 0.f ? 448.f / mx : 1.f;
  for (int c = lane; c < ld; c += 32) {
    const float v = c < p ? src[r * p + c] * scale : 0.f;
    dst[r * ld + c] = (uint8_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
  }
  if (lane == 0) inv_scale[r] = mx > 0.f ? mx / 448.f : 1.f;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

bool make_map_lp(CUtensorMap* map, const void* ptr, int64_t rows, int ld, int esize, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * esize};
  cuuint32_t box[2] = {(cuuint32_t)(CHUNK_BYTES / esize), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  const CUtensorMapDataType dt =
      esize == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8;
  return fn(map, dt, 2, (void*)ptr, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}


// ---- BF16 correlations, persistent and pipelined --------------------------------
// The same warp-specialised structure as the split-TF32 kernel (k_corr_tc.cu),
// with FP32 signals converted to BF16 on chip instead of split:
//   * warp 4, one thread: TMA of this CTA's 128-atom BF16 block of D once (it
//     stays resident), then of the FP32 signal tiles into a two-slot ring;
//   * warps 6-11: convert each arrived FP32 tile to a BF16 tile (128-byte
//     swizzled rows, the MMA operand layout) in the same slot;
//   * warp 5, one thread: tcgen05.mma kind::f16 (M=128, N=128, K=16) into one of
//     four 128-column TMEM accumulators;
//   * warps 0-3 and 12-15: drain an accumulator (tcgen05.ld; two warps per TMEM
//     lane quadrant, 64 columns each) through swizzled staging into TMA stores
//     of FP32 alpha0.
// Y is read once, in FP32, by this kernel: no separate conversion pass.  Every
// mbarrier wait is bounded; on timeout the kernel flags ERR_TIMEOUT, frees its
// TMEM and returns.
constexpr int BW_THREADS = 512;
constexpr int BW_CONV = 192;               // warps 6-11
constexpr int BW_EPI = 8;                  // epilogue warps 0-3 and 12-15
constexpr int BW_M = 128;                  // signals per tile (MMA M)
constexpr int BW_N = 128;                  // atoms per block (MMA N)
constexpr int BW_RING = 4;                 // TMEM accumulators
constexpr int BW_BOX = 32;                 // TMA store box: 32 rows x 32 floats
constexpr int BW_STAGES = 2;               // store boxes in flight per epilogue warp
// kind::f16: D F32, A/B BF16, K-major, N = 128, M = 128
constexpr uint32_t kBwIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BW_N >> 3) << 17) |
                              ((uint32_t)(BW_M >> 4) << 24);
struct BwSmem {  // byte offsets from the 1024-aligned base
  static constexpr size_t chunk = (size_t)128 * 128;  // 128 rows x 128 bytes
  static constexpr size_t b = 0;                      // BF16 block of D (1 chunk)
  static constexpr size_t a0 = chunk;                 // slot s: FP32 tile (2 chunks), BF16 tile
  static constexpr size_t a_slot = 3 * chunk;
  static constexpr size_t stage = a0 + 2 * a_slot;    // 8 warps x BW_STAGES boxes
  static constexpr size_t box = (size_t)BW_BOX * BW_BOX * 4;
  static constexpr size_t bars = stage + BW_EPI * BW_STAGES * box;
  static constexpr size_t total = bars + 15 * 8 + 16;
  static constexpr size_t dyn = total + 1024;
};
static_assert(BwSmem::dyn <= 232448, "shared memory budget");
constexpr int W_BFULL = 0, W_AFULL = 1, W_AFREE = 3, W_ACONV = 5, W_TFULL = 7, W_TEMPTY = 11;
constexpr int kBwBars = 15;

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *(const uint32_t*)&v;
}

template <bool OUTB>
__global__ void __launch_bounds__(BW_THREADS, 1)
    corr_bf16_ws_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                        const __grid_constant__ CUtensorMap tmC, int64_t rows, int64_t tiles, int n,
                        int kbf, int nq, int* __restrict__ err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(base + BwSmem::bars);
  uint32_t* tmem_slot = (uint32_t*)(bars + kBwBars);
  volatile int* fail = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int blk_n = blockIdx.x % nq;
  const int64_t gi = blockIdx.x / nq, groups = gridDim.x / nq;
  const int nitems = gi < tiles ? (int)((tiles - 1 - gi) / groups + 1) : 0;

  if (threadIdx.x == 0) {
    *fail = 0;
    mbar_init(&bars[W_BFULL], 1);
    for (int q = 0; q < 2; ++q) {
      mbar_init(&bars[W_AFULL + q], 1);
      mbar_init(&bars[W_AFREE + q], 1);
      mbar_init(&bars[W_ACONV + q], BW_CONV);
    }
    for (int q = 0; q < BW_RING; ++q) {
      mbar_init(&bars[W_TFULL + q], 1);
      mbar_init(&bars[W_TEMPTY + q], BW_EPI);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(BW_RING * BW_N)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  auto fslot = [&](int sl) { return base + BwSmem::a0 + sl * BwSmem::a_slot; };  // FP32 tile
  auto hslot = [&](int sl) { return fslot(sl) + 2 * BwSmem::chunk; };            // BF16 tile

  if (warp == 4) {
    // ---------------- TMA issuer: the B block once, then the FP32 signal tiles ----------------
    if (lane == 0 && nitems > 0) {
      mbar_expect_tx(&bars[W_BFULL], (uint32_t)BwSmem::chunk);
      tma_load_2d(base + BwSmem::b, &tmB, &bars[W_BFULL], 0, blk_n * BW_N);
      for (int v = 0; v < nitems && !*fail; ++v) {
        const int sl = v & 1;
        // the slot is free once the MMAs of the tile two back have completed
        if (v >= 2 && !mbar_wait(&bars[W_AFREE + sl], (uint32_t)((v / 2 - 1) & 1))) {
          *fail = 1;
          break;
        }
        const int64_t t = gi + (int64_t)v * groups;
        mbar_expect_tx(&bars[W_AFULL + sl], (uint32_t)(kbf * BwSmem::chunk));
        for (int q = 0; q < kbf; ++q)
          tma_load_2d(fslot(sl) + q * BwSmem::chunk, &tmA, &bars[W_AFULL + sl], q * 32,
                      (int)(t * BW_M));
      }
    }
  } else if (warp == 5) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      bool ok = nitems == 0 || mbar_wait(&bars[W_BFULL], 0);
      const uint64_t bd = sw128_desc(base + BwSmem::b);
      for (int v = 0; v < nitems && ok && !*fail; ++v) {
        const int sl = v & 1, blk = v & (BW_RING - 1);
        ok = mbar_wait(&bars[W_ACONV + sl], (uint32_t)((v / 2) & 1));
        ok = ok && (v < BW_RING ||
                    mbar_wait(&bars[W_TEMPTY + blk], (uint32_t)(((v / BW_RING) - 1) & 1)));
        if (!ok) break;
        tc_fence_after();
        const uint64_t ad = sw128_desc(hslot(sl));
        const uint32_t dcol = tmem + (uint32_t)(blk * BW_N);
#pragma unroll
        for (int k = 0; k < 4; ++k)  // 16 BF16 = 32 bytes of K per MMA
          mma_f16(dcol, ad + (uint64_t)(2 * k), bd + (uint64_t)(2 * k), kBwIdesc, k > 0 ? 1u : 0u);
        mma_commit(&bars[W_AFREE + sl]);
        mma_commit(&bars[W_TFULL + blk]);
      }
      if (!ok) *fail = 1;
    }
  } else if (warp >= 6 && warp < 12) {
    // ---------------- converters: FP32 tile -> BF16 tile (swizzled rows) ----------------
    const int pt = threadIdx.x - 192;
    for (int v = 0; v < nitems; ++v) {
      if (*fail) break;
      const int sl = v & 1;
      if (!mbar_wait(&bars[W_AFULL + sl], (uint32_t)((v / 2) & 1))) {
        *fail = 1;
        break;
      }
      const uint8_t* F = fslot(sl);
      uint8_t* H = hslot(sl);
      // unit e: row r, 16-byte output unit u (BF16 columns 8u .. 8u + 7), read from
      // FP32 chunk u / 4, input units 2 (u mod 4) and + 1; 128-byte swizzle on both
      for (int e = pt; e < BW_M * 8; e += BW_CONV) {
        const int r = e >> 3, u = e & 7, c = u >> 2, u0 = 2 * (u & 3), sw = r & 7;
        uint4 o = make_uint4(0u, 0u, 0u, 0u);
        if (c < kbf) {  // columns past the loaded chunks are zero
          const uint8_t* frow = F + c * BwSmem::chunk + r * 128;
          const float4 x0 = *(const float4*)(frow + ((u0 ^ sw) << 4));
          const float4 x1 = *(const float4*)(frow + (((u0 + 1) ^ sw) << 4));
          o = make_uint4(pack_bf16x2(x0.x, x0.y), pack_bf16x2(x0.z, x0.w),
                         pack_bf16x2(x1.x, x1.y), pack_bf16x2(x1.z, x1.w));
        }
        *(uint4*)(H + r * 128 + ((u ^ sw) << 4)) = o;
      }
      fence_async_smem();
      mbar_arrive(&bars[W_ACONV + sl]);
    }
  } else {
    // ---------------- epilogue warps: TMEM lanes 32 (warp mod 4) .. + 31, the
    // accumulator's left (warps 0-3) or right (warps 12-15) 64 columns ----------------
    const int ew = warp < 4 ? warp : warp - 8;  // 0..7
    const int quad = warp & 3, half = warp >= 12 ? 1 : 0;
    float* stg0 = (float*)(base + BwSmem::stage + (size_t)(BW_STAGES * ew) * BwSmem::box);
    const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
    int sb = 0;
    for (int v = 0; v < nitems; ++v) {
      if (__shfl_sync(0xffffffffu, *fail, 0)) continue;
      const int64_t t = gi + (int64_t)v * groups;
      const int blk = v & (BW_RING - 1);
      const bool ok = __all_sync(0xffffffffu,
                                 mbar_wait(&bars[W_TFULL + blk], (uint32_t)((v / BW_RING) & 1)));
      if (!ok) {
        if (lane == 0) *fail = 1;
        continue;
      }
      tc_fence_after();
      const int64_t row0 = t * BW_M + quad * 32;
      if (OUTB && row0 < rows) {
        // BF16 alpha0: this warp's 64 columns as one 32-row x 128-byte box
        const int col0 = blk_n * BW_N + 64 * half;
        if (col0 < n) {
          uint32_t r0[32], r1[32];
          tmem_ld32(tmem + lane_base + (uint32_t)(blk * BW_N + 64 * half), r0);
          tmem_ld32(tmem + lane_base + (uint32_t)(blk * BW_N + 64 * half + 32), r1);
          float* stg = stg0 + sb * (BW_BOX * BW_BOX);
          if (lane == 0) bulk_wait_read<BW_STAGES - 1>();
          __syncwarp();
          uint8_t* rowp = (uint8_t*)stg + lane * 128;
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const uint32_t* rr = c < 4 ? r0 : r1;
            const int b = 8 * (c & 3);
            *(uint4*)(rowp + ((c ^ (lane & 7)) << 4)) = make_uint4(
                pack_bf16x2(__uint_as_float(rr[b]), __uint_as_float(rr[b + 1])),
                pack_bf16x2(__uint_as_float(rr[b + 2]), __uint_as_float(rr[b + 3])),
                pack_bf16x2(__uint_as_float(rr[b + 4]), __uint_as_float(rr[b + 5])),
                pack_bf16x2(__uint_as_float(rr[b + 6]), __uint_as_float(rr[b + 7])));
          }
          fence_async_smem();
          __syncwarp();
          if (lane == 0) {
            tma_store_2d(&tmC, stg, col0, (int)row0);
            bulk_commit();
          }
          sb = (sb + 1) % BW_STAGES;
        }
      } else if (row0 < rows) {
        for (int j = 2 * half; j < 2 * half + 2; ++j) {
          const int col0 = blk_n * BW_N + j * BW_BOX;
          if (col0 >= n) break;
          uint32_t r[32];
          tmem_ld32(tmem + lane_base + (uint32_t)(blk * BW_N + j * BW_BOX), r);
          float* stg = stg0 + sb * (BW_BOX * BW_BOX);
          if (lane == 0) bulk_wait_read<BW_STAGES - 1>();  // this staging box is free again
          __syncwarp();
          uint8_t* rowp = (uint8_t*)stg + lane * 128;
#pragma unroll
          for (int c = 0; c < 8; ++c)
            *(uint4*)(rowp + ((c ^ (lane & 7)) << 4)) =
                make_uint4(r[4 * c], r[4 * c + 1], r[4 * c + 2], r[4 * c + 3]);
          fence_async_smem();
          __syncwarp();
          if (lane == 0) {
            tma_store_2d(&tmC, stg, col0, (int)row0);
            bulk_commit();
          }
          sb = (sb + 1) % BW_STAGES;
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bars[W_TEMPTY + blk]);
    }
    if (lane == 0) bulk_wait<0>();
    __syncwarp();
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(BW_RING * BW_N)
                 : "memory");
  if (threadIdx.x == 0 && *fail) atomicOr(err, ERR_TIMEOUT);
}

// rows x p row-major FP32 matrix, box = 32 floats x box_rows, 128-byte swizzle.
bool make_map_f32(CUtensorMap* map, const float* ptr, int64_t rows, int p, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)p, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)p * 4};
  cuuint32_t box[2] = {32u, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)ptr, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// rows x n row-major output with leading dimension ldc (elements): FP32 with 32 x 32
// store boxes, or BF16 with 64-column x 32-row boxes (128-byte rows either way).
bool make_map_out(CUtensorMap* map, void* ptr, bool bf16, int64_t rows, int n, int64_t ldc) {
  auto fn = encode_fn();
  if (!fn) return false;
  const int es = bf16 ? 2 : 4;
  cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ldc * es};
  cuuint32_t box[2] = {(cuuint32_t)(128 / es), (cuuint32_t)BW_BOX};
  cuuint32_t estr[2] = {1, 1};
  return fn(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
            (void*)ptr, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

int lp_row_elems(int kind, int p) {
  const int epc = CHUNK_BYTES / (kind == LP_BF16 ? 2 : 1);
  return (p + epc - 1) / epc * epc;
}

bool corr_lp_supported(int kind, int p, int n, int64_t ldc) {
  const int kb = lp_row_elems(kind, p) * (kind == LP_BF16 ? 2 : 1) / CHUNK_BYTES;
  return (kind == LP_BF16 || kind == LP_E4M3) && p >= 1 && kb <= 2 && n >= 1 && n <= 512 &&
         (ldc % 4) == 0 && ldc >= (int64_t)(n + 15) / 16 * 16 && encode_fn() != nullptr;
}

cudaError_t to_lowp(int kind, const float* src, int64_t rows, int p, void* dst, float* inv_scale,
                    cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  const int ld = lp_row_elems(kind, p);
  if (kind == LP_BF16) {
    const int64_t tot = rows * ld;
    to_bf16_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(src, rows, p, ld,
                                                                 (__nv_bfloat16*)dst);
  } else {
    to_e4m3_kernel<<<(unsigned)((rows + 7) / 8), 256, 0, st>>>(src, rows, p, ld, (uint8_t*)dst,
                                                               inv_scale);
  }
  return cudaGetLastError();
}

bool corr_bf16_ws_supported(const float* Y, int p, int n, int64_t ldc) {
  return p >= 1 && p <= 64 && (p % 4) == 0 && ((uintptr_t)Y % 16) == 0 && n >= 1 && n <= 1024 &&
         (ldc % 4) == 0 && ldc >= (int64_t)(n + 15) / 16 * 16 && encode_fn() != nullptr;
}

cudaError_t corr_bf16_ws(const float* Y, int64_t rows, const void* Dbf, int n, int p, void* C,
                         bool out_bf16, int64_t ldc, int* err, cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  if (((uintptr_t)C % 16) != 0 || (ldc % 8) != 0) return cudaErrorInvalidValue;
  const int ld = lp_row_elems(LP_BF16, p);
  CUtensorMap ma, mb, mc;
  if (!make_map_f32(&ma, Y, rows, p, BW_M) || !make_map_lp(&mb, Dbf, n, ld, 2, BW_N) ||
      !make_map_out(&mc, C, out_bf16, rows, n, ldc))
    return cudaErrorInvalidValue;
  auto kern = out_bf16 ? corr_bf16_ws_kernel<true> : corr_bf16_ws_kernel<false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)BwSmem::dyn);
  if (e != cudaSuccess) return e;
  const int64_t tiles = (rows + BW_M - 1) / BW_M;
  const int nq = (n + BW_N - 1) / BW_N;
  int64_t groups = num_sms() / nq;
  if (groups < 1) groups = 1;
  if (groups > tiles) groups = tiles;
  const int kbf = (p + 31) / 32;
  kern<<<(unsigned)(groups * nq), BW_THREADS, BwSmem::dyn, st>>>(ma, mb, mc, rows, tiles, n, kbf,
                                                                   nq, err);
  return cudaGetLastError();
}

cudaError_t corr_lp(int kind, const void* A, int64_t rows_a, const float* a_inv_scale,
                    const void* B, const float* b_inv_scale, int n, int p, float* C, int64_t ldc,
                    int* err, cudaStream_t st) {
  if (rows_a <= 0) return cudaSuccess;
  const int esize = kind == LP_BF16 ? 2 : 1;
  const int ld = lp_row_elems(kind, p);
  const int kb = ld * esize / CHUNK_BYTES;
  CUtensorMap ma, mb;
  if (!make_map_lp(&ma, A, rows_a, ld, esize, TILE_M) || !make_map_lp(&mb, B, n, ld, esize, BLOCK_N))
    return cudaErrorInvalidValue;
  size_t smem = 1024 + kb * (kAChunk + kBChunk) + 64;
  // one CTA per SM when it holds all 512 TMEM columns
  if (n > BLOCK_N && smem < 120 * 1024) smem = 120 * 1024;
  const unsigned grid = (unsigned)((rows_a + TILE_M - 1) / TILE_M);
  cudaError_t e;
  if (kind == LP_BF16) {
    e = cudaFuncSetAttribute(corr_lp_kernel<LP_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    corr_lp_kernel<LP_BF16><<<grid, LP_THREADS, smem, st>>>(ma, mb, rows_a, n, kb, a_inv_scale,
                                                            b_inv_scale, C, ldc, err);
  } else {
    e = cudaFuncSetAttribute(corr_lp_kernel<LP_E4M3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    corr_lp_kernel<LP_E4M3><<<grid, LP_THREADS, smem, st>>>(ma, mb, rows_a, n, kb, a_inv_scale,
                                                            b_inv_scale, C, ldc, err);
  }
  return cudaGetLastError();
}

}  // namespace dlk
