// FP32-accurate correlations on the 5th-generation tensor cores (tcgen05):
//   C[i][j] = sum_r A[i][r] * B[j][r]
// with A the signals Y (alpha0 = D^T y for every signal, Algorithm 1 step 1)
// or the atoms D (the Gram matrix G = D^T D of Batch-OMP), and B the atoms D.
// One launch can compute two such products with the same B (the correlations
// of all signals and the Gram matrix of a DL iteration).
//
// Split-TF32 ("3xTF32") arithmetic: every operand is split into a TF32 head
// and a TF32 tail, a = a_hi + a_lo with a_hi = rna_tf32(a), a_lo = a - a_hi;
// C = A_hi B_hi + A_hi B_lo + A_lo B_hi accumulated in FP32 in tensor memory.
// The dropped A_lo B_lo term and the TF32 rounding of the tails leave a
// relative error near 2^-21 per product, i.e. FP32 accuracy.
//
// Work split: the columns of C are cut into blocks of 128 atoms; CTA c owns
// block c % nq (nq = ceil(n/128)) and keeps that block's pre-split B (head and
// tail, 64 KB at p <= 64) resident in shared memory for its whole life; the
// CTAs owning a block share out the 128-row tiles of A (both products' tiles
// in one list).  Warp roles, 384 threads, each waiting only on mbarriers:
//   * warp 4, one thread: TMA of the B block once, then of the A tiles into a
//     two-slot ring (SWIZZLE_128B), each as soon as its slot is free;
//   * warps 6-11: split each arrived tile in place into A_hi / A_lo;
//   * warp 5, one thread: per split tile, 3 x (K/8) tcgen05.mma kind::tf32
//     (M=128, N=128, K=8) into one of four 128-column TMEM accumulators;
//   * warps 0-3 (epilogue): drain an accumulator with tcgen05.ld (warp w owns
//     TMEM lanes 32w..32w+31 = rows), stage 32x32 boxes in 128-byte-swizzled
//     shared memory and write them with TMA stores (two boxes in flight per
//     warp), then hand the accumulator back.
// A tiles stream in while the previous tile multiplies and older tiles drain,
// and B is read from L2 once per CTA.  Every wait on an mbarrier is bounded
// (2 s of %globaltimer); on timeout the kernel flags ERR_TIMEOUT, skips the
// remaining work, frees its TMEM and returns.
#include "dl_internal.cuh"
#include "tc_ptx.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>
#include <stdint.h>

namespace dlk {
namespace {

constexpr int WS_THREADS = 384;
constexpr int SPLIT_THREADS = WS_THREADS - 192;  // warps 6..
constexpr int TILE_M = 128;
constexpr int BLOCK_N = 128;  // atoms per column block (MMA N)
constexpr int KCHUNK = 32;    // floats per 128-byte swizzle row
constexpr int TMEM_RING = 4;
constexpr int BOX = 32;       // TMA store box: 32 rows x 32 floats
using namespace tc;
// Instruction descriptor: kind::tf32, A/B TF32 K-major, D FP32, M = 128, N = 128.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BLOCK_N >> 3) << 17) |
                            ((uint32_t)(TILE_M >> 4) << 24);

struct WsSmem {  // byte offsets from the 1024-aligned base
  static constexpr size_t chunk = (size_t)TILE_M * KCHUNK * 4;  // 16 KB (= BLOCK_N * KCHUNK * 4)
  static constexpr size_t b_hi = 0;                  // 2 chunks (K <= 64), then 2 tail chunks
  static constexpr size_t b_lo = 2 * chunk;
  static constexpr size_t a0 = 4 * chunk;            // slot s: 2 head chunks, then 2 tail chunks
  static constexpr size_t a_slot = 4 * chunk;
  static constexpr size_t stage = a0 + 2 * a_slot;   // 4 warps x 2 boxes
  static constexpr size_t box = (size_t)BOX * BOX * 4;
  static constexpr size_t bars = stage + 8 * box;
  static constexpr size_t total = bars + 15 * 8 + 16;
  static constexpr size_t dyn = total + 1024;
};
static_assert(WsSmem::dyn <= 232448, "shared memory budget");

// barrier indices
constexpr int B_BFULL = 0, B_AFULL = 1, B_AFREE = 3, B_ASPLIT = 5, B_TFULL = 7, B_TEMPTY = 11;
constexpr int kBars = 15;

// tiles0 tiles of product 0 (A0 -> C0, rows0 rows), then those of product 1.
__global__ void __launch_bounds__(WS_THREADS, 1)
    corr_tf32x3_kernel(const __grid_constant__ CUtensorMap tmA0, const __grid_constant__ CUtensorMap tmA1,
                       const __grid_constant__ CUtensorMap tmBhi, const __grid_constant__ CUtensorMap tmBlo,
                       const __grid_constant__ CUtensorMap tmC0, const __grid_constant__ CUtensorMap tmC1,
                       int64_t rows0, int64_t rows1, int64_t tiles0, int64_t tiles, int n, int kb,
                       int nq, int* __restrict__ err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(base + WsSmem::bars);
  uint32_t* tmem_slot = (uint32_t*)(bars + kBars);
  volatile int* fail = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int blk_n = blockIdx.x % nq;              // this CTA's column block
  const int64_t gi = blockIdx.x / nq, groups = gridDim.x / nq;
  const int nitems = gi < tiles ? (int)((tiles - 1 - gi) / groups + 1) : 0;

  if (threadIdx.x == 0) {
    *fail = 0;
    mbar_init(&bars[B_BFULL], 1);
    for (int q = 0; q < 2; ++q) {
      mbar_init(&bars[B_AFULL + q], 1);
      mbar_init(&bars[B_AFREE + q], 1);
      mbar_init(&bars[B_ASPLIT + q], SPLIT_THREADS);
    }
    for (int q = 0; q < TMEM_RING; ++q) {
      mbar_init(&bars[B_TFULL + q], 1);
      mbar_init(&bars[B_TEMPTY + q], 4);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TMEM_RING * BLOCK_N)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  auto aslot = [&](int sl) { return (float*)(base + WsSmem::a0 + sl * WsSmem::a_slot); };
  if (warp == 4) {
    // ---------------- TMA issuer: the B block once, then the A tiles ----------------
    if (lane == 0 && nitems > 0) {
      mbar_expect_tx(&bars[B_BFULL], (uint32_t)(2 * kb * WsSmem::chunk));
      for (int q = 0; q < kb; ++q) {
        tma_load_2d(base + WsSmem::b_hi + q * WsSmem::chunk, &tmBhi, &bars[B_BFULL], q * KCHUNK,
                    blk_n * BLOCK_N);
        tma_load_2d(base + WsSmem::b_lo + q * WsSmem::chunk, &tmBlo, &bars[B_BFULL], q * KCHUNK,
                    blk_n * BLOCK_N);
      }
      for (int v = 0; v < nitems && !*fail; ++v) {
        const int sl = v & 1;
        // the slot is free once the MMAs of the tile two back have completed
        if (v >= 2 && !mbar_wait(&bars[B_AFREE + sl], (uint32_t)((v / 2 - 1) & 1))) {
          *fail = 1;
          break;
        }
        const int64_t T = gi + (int64_t)v * groups;
        const bool second = T >= tiles0;
        const int64_t t = second ? T - tiles0 : T;
        float* dst = aslot(sl);
        mbar_expect_tx(&bars[B_AFULL + sl], (uint32_t)(kb * WsSmem::chunk));
        for (int q = 0; q < kb; ++q)
          tma_load_2d(dst + q * TILE_M * KCHUNK, second ? &tmA1 : &tmA0, &bars[B_AFULL + sl],
                      q * KCHUNK, (int)(t * TILE_M));
      }
    }
  } else if (warp == 5) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      bool ok = nitems == 0 || mbar_wait(&bars[B_BFULL], 0);
      for (int v = 0; v < nitems && ok && !*fail; ++v) {
        const int sl = v & 1, blk = v & (TMEM_RING - 1);
        ok = mbar_wait(&bars[B_ASPLIT + sl], (uint32_t)((v / 2) & 1));
        ok = ok && (v < TMEM_RING ||
                    mbar_wait(&bars[B_TEMPTY + blk], (uint32_t)(((v / TMEM_RING) - 1) & 1)));
        if (!ok) break;
        tc_fence_after();
        const float* Ahi = aslot(sl);
        const float* Alo = Ahi + 2 * TILE_M * KCHUNK;
        const uint32_t dcol = tmem + (uint32_t)(blk * BLOCK_N);
        uint32_t accum = 0;
        // small terms first: A_hi B_lo, A_lo B_hi, then A_hi B_hi
        for (int pass = 0; pass < 3; ++pass) {
          const float* Ap = pass == 1 ? Alo : Ahi;
          const uint8_t* Bp = base + (pass == 0 ? WsSmem::b_lo : WsSmem::b_hi);
          for (int q = 0; q < kb; ++q) {
            const uint64_t ad = sw128_desc(Ap + q * TILE_M * KCHUNK);
            const uint64_t bd = sw128_desc(Bp + q * WsSmem::chunk);
#pragma unroll
            for (int k = 0; k < KCHUNK / 8; ++k) {
              // advance 8 TF32 = 32 bytes along K inside the swizzle row
              mma_tf32(dcol, ad + (uint64_t)(2 * k), bd + (uint64_t)(2 * k), kIdesc, accum);
              accum = 1;
            }
          }
        }
        mma_commit(&bars[B_AFREE + sl]);
        mma_commit(&bars[B_TFULL + blk]);
      }
      if (!ok) *fail = 1;
    }
  } else if (warp >= 6) {
    // ---------------- splitters: A tile -> A_hi / A_lo in place ----------------
    const int pt = threadIdx.x - 192;
    for (int v = 0; v < nitems; ++v) {
      if (*fail) break;
      const int sl = v & 1;
      if (!mbar_wait(&bars[B_AFULL + sl], (uint32_t)((v / 2) & 1))) {
        *fail = 1;
        break;
      }
      float* Ahi = aslot(sl);
      float* Alo = Ahi + 2 * TILE_M * KCHUNK;
      const int total = kb * TILE_M * KCHUNK;
      for (int e = pt * 4; e < total; e += SPLIT_THREADS * 4) {
        float4 x = *(float4*)(Ahi + e);
        float4 h = make_float4(tf32_rna(x.x), tf32_rna(x.y), tf32_rna(x.z), tf32_rna(x.w));
        *(float4*)(Ahi + e) = h;
        *(float4*)(Alo + e) = make_float4(x.x - h.x, x.y - h.y, x.z - h.z, x.w - h.w);
      }
      fence_async_smem();
      mbar_arrive(&bars[B_ASPLIT + sl]);
    }
  } else {
    // ---------------- epilogue warps ----------------
    float* stg0 = (float*)(base + WsSmem::stage + (size_t)(2 * warp) * WsSmem::box);
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    int sb = 0;
    for (int v = 0; v < nitems; ++v) {
      if (__shfl_sync(0xffffffffu, *fail, 0)) continue;
      const int64_t T = gi + (int64_t)v * groups;
      const bool second = T >= tiles0;
      const int64_t t = second ? T - tiles0 : T;
      const int64_t rows = second ? rows1 : rows0;
      const CUtensorMap* tmC = second ? &tmC1 : &tmC0;
      const int blk = v & (TMEM_RING - 1);
      const bool ok = __all_sync(0xffffffffu,
                                 mbar_wait(&bars[B_TFULL + blk], (uint32_t)((v / TMEM_RING) & 1)));
      if (!ok) {
        if (lane == 0) *fail = 1;
        continue;
      }
      tc_fence_after();
      const int64_t row0 = t * TILE_M + warp * 32;
      if (row0 < rows) {
        for (int j = 0; j < BLOCK_N / BOX; ++j) {
          const int col0 = blk_n * BLOCK_N + j * BOX;
          if (col0 >= n) break;
          uint32_t r[32];
          tmem_ld32(tmem + lane_base + (uint32_t)(blk * BLOCK_N + j * BOX), r);
          float* stg = stg0 + sb * (BOX * BOX);
          if (lane == 0) bulk_wait_read<1>();
          __syncwarp();
          // 128-byte swizzle: 16-byte chunk c of row `lane` sits at chunk c ^ (lane & 7)
          uint8_t* rowp = (uint8_t*)stg + lane * 128;
#pragma unroll
          for (int c = 0; c < 8; ++c)
            *(uint4*)(rowp + ((c ^ (lane & 7)) << 4)) =
                make_uint4(r[4 * c], r[4 * c + 1], r[4 * c + 2], r[4 * c + 3]);
          fence_async_smem();
          __syncwarp();
          if (lane == 0) {
            tma_store_2d(tmC, stg, col0, (int)row0);
            bulk_commit();
          }
          sb ^= 1;
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bars[B_TEMPTY + blk]);
    }
    if (lane == 0) bulk_wait<0>();
    __syncwarp();
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_RING * BLOCK_N)
                 : "memory");
  if (threadIdx.x == 0 && *fail) atomicOr(err, ERR_TIMEOUT);
}

// Split B into TF32 head and tail (row-major, same layout as B).
__global__ void split_kernel(const float* __restrict__ B, int64_t count, float* __restrict__ hi,
                             float* __restrict__ lo) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= count) return;
  const float v = B[e];
  const float h = tf32_rna(v);
  hi[e] = h;
  lo[e] = v - h;
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

// rows x p row-major FP32 matrix, box = 32 floats (K) x box_rows, 128-byte swizzle.
bool make_map(CUtensorMap* map, const float* ptr, int64_t rows, int p, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)p, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)p * 4};
  cuuint32_t box[2] = {(cuuint32_t)KCHUNK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)ptr, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// rows x n row-major FP32 output with leading dimension ldc; 32 x 32 store boxes.
bool make_map_out(CUtensorMap* map, float* ptr, int64_t rows, int n, int64_t ldc) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ldc * 4};
  cuuint32_t box[2] = {(cuuint32_t)BOX, (cuuint32_t)BOX};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)ptr, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace

bool corr_tc_supported(const float* A, int p, int n, int64_t ldc) {
  return p >= 1 && p <= 64 && (p % 4) == 0 && n >= 1 && n <= 1024 && (ldc % 4) == 0 &&
         ldc >= (int64_t)(n + 15) / 16 * 16 && ((uintptr_t)A % 16) == 0 && encode_fn() != nullptr;
}


cudaError_t split_tf32(const float* B, int64_t count, float* hi, float* lo, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  split_kernel<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(B, count, hi, lo);
  return cudaGetLastError();
}

cudaError_t corr_tf32x3_pair(const float* A0, int64_t rows0, float* C0, int64_t ldc0,
                             const float* A1, int64_t rows1, float* C1, int64_t ldc1,
                             const float* Bhi, const float* Blo, int n, int p, int* err,
                             cudaStream_t st) {
  if (!A1) rows1 = 0;
  if (rows0 <= 0 && rows1 <= 0) return cudaSuccess;
  if (rows0 <= 0) return corr_tf32x3_pair(A1, rows1, C1, ldc1, nullptr, 0, nullptr, 0, Bhi, Blo, n,
                                          p, err, st);
  if (((uintptr_t)C0 % 16) != 0 || (rows1 > 0 && ((uintptr_t)C1 % 16) != 0))
    return cudaErrorInvalidValue;
  CUtensorMap ma0, ma1, mbh, mbl, mc0, mc1;
  if (!make_map(&ma0, A0, rows0, p, TILE_M) || !make_map(&mbh, Bhi, n, p, BLOCK_N) ||
      !make_map(&mbl, Blo, n, p, BLOCK_N) || !make_map_out(&mc0, C0, rows0, n, ldc0))
    return cudaErrorInvalidValue;
  if (rows1 > 0) {
    if (!make_map(&ma1, A1, rows1, p, TILE_M) || !make_map_out(&mc1, C1, rows1, n, ldc1))
      return cudaErrorInvalidValue;
  } else {
    ma1 = ma0;
    mc1 = mc0;
  }
  const int kb = (p + KCHUNK - 1) / KCHUNK;
  cudaError_t e = cudaFuncSetAttribute(corr_tf32x3_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)WsSmem::dyn);
  if (e != cudaSuccess) return e;
  const int64_t tiles0 = (rows0 + TILE_M - 1) / TILE_M;
  const int64_t tiles = tiles0 + (rows1 + TILE_M - 1) / TILE_M;
  const int nq = (n + BLOCK_N - 1) / BLOCK_N;
  int64_t groups = num_sms() / nq;
  if (groups < 1) groups = 1;
  if (groups > tiles) groups = tiles;
  corr_tf32x3_kernel<<<(unsigned)(groups * nq), WS_THREADS, WsSmem::dyn, st>>>(
      ma0, ma1, mbh, mbl, mc0, mc1, rows0, rows1, tiles0, tiles, n, kb, nq, err);
  return cudaGetLastError();
}

cudaError_t corr_tf32x3(const float* A, int64_t rows_a, const float* Bhi, const float* Blo, int n,
                        int p, float* C, int64_t ldc, int* err, cudaStream_t st) {
  return corr_tf32x3_pair(A, rows_a, C, ldc, nullptr, 0, nullptr, 0, Bhi, Blo, n, p, err, st);
}

}  // namespace dlk
