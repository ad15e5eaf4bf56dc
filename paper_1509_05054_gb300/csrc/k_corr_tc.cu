// FP32-accurate correlations on the 5th-generation tensor cores (tcgen05):
//   C[i][j] = sum_r A[i][r] * B[j][r]
// with A the signals Y (alpha0 = D^T y for every signal, Algorithm 1 step 1)
// or the atoms D (the Gram matrix G = D^T D of Batch-OMP), and B the atoms D.
//
// Split-TF32 ("3xTF32") arithmetic: every operand is split into a TF32 head
// and a TF32 tail, a = a_hi + a_lo with a_hi = rna_tf32(a), a_lo = a - a_hi;
// C = A_hi B_hi + A_hi B_lo + A_lo B_hi accumulated in FP32 in tensor memory.
// The dropped A_lo B_lo term and the TF32 rounding of the tails leave a
// relative error near 2^-21 per product, i.e. FP32 accuracy.
//
// The output is a grid of units (128-row tile t, 128-column block nb); the
// units are dealt to a persistent grid (one CTA per SM) in contiguous ranges,
// so a CTA walks its tiles block by block.  Warp roles, 256 threads:
//   * warps 4-7 (producer group): on a tile change, TMA the A tile (128 rows x
//     64 K, SWIZZLE_128B) and split it in place into A_hi / A_lo; thread 128
//     keeps a two-slot ring of pre-split B blocks (TMA, one unit ahead) and
//     issues 3 x (K/8) tcgen05.mma kind::tf32 (M=128, N=128, K=8) per unit
//     into one of four 128-column TMEM accumulators;
//   * warps 0-3 (epilogue): drain an accumulator with tcgen05.ld (warp w owns
//     TMEM lanes 32w..32w+31 = rows), stage 32x32 boxes in 128-byte-swizzled
//     shared memory and write them with TMA stores (two boxes in flight per
//     warp), then hand the accumulator back.
// So the stores of one unit overlap the loads and MMAs of the next ones and
// every global write is a full line.  Every wait on an mbarrier is bounded
// (2 s of %globaltimer); on timeout the kernel flags ERR_TIMEOUT, skips the
// remaining work, frees its TMEM and returns.
#include "dl_internal.cuh"
#include "tc_ptx.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>
#include <stdint.h>

namespace dlk {
namespace {

constexpr int WS_THREADS = 256;
constexpr int TILE_M = 128;
constexpr int UNIT_N = 128;  // columns per unit (MMA N)
constexpr int KCHUNK = 32;   // floats per 128-byte swizzle row
constexpr int TMEM_RING = 4;
constexpr int BOX = 32;      // TMA store box: 32 rows x 32 floats
using namespace tc;
// Instruction descriptor: kind::tf32, A/B TF32 K-major, D FP32, M = 128, N = 128.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(UNIT_N >> 3) << 17) |
                            ((uint32_t)(TILE_M >> 4) << 24);

struct WsSmem {  // byte offsets from the 1024-aligned base
  static constexpr size_t chunk_a = (size_t)TILE_M * KCHUNK * 4;  // 16 KB
  static constexpr size_t chunk_b = (size_t)UNIT_N * KCHUNK * 4;  // 16 KB
  static constexpr size_t a_hi = 0;
  static constexpr size_t a_lo = 2 * chunk_a;
  static constexpr size_t b0 = 4 * chunk_a;          // slot s: hi chunks, then lo chunks
  static constexpr size_t b_slot = 4 * chunk_b;
  static constexpr size_t stage = b0 + 2 * b_slot;   // 4 warps x 2 boxes
  static constexpr size_t box = (size_t)BOX * BOX * 4;
  static constexpr size_t bars = stage + 8 * box;
  static constexpr size_t total = bars + 14 * 8 + 16;
  static constexpr size_t dyn = total + 1024;
};
static_assert(WsSmem::dyn <= 232448, "shared memory budget");

// barrier indices
constexpr int B_AFULL = 0, B_AFREE = 1, B_BFULL = 2, B_BFREE = 4, B_TFULL = 6, B_TEMPTY = 10;

__device__ __forceinline__ void group_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

__global__ void __launch_bounds__(WS_THREADS, 1)
    corr_tf32x3_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmBhi,
                       const __grid_constant__ CUtensorMap tmBlo, const __grid_constant__ CUtensorMap tmC,
                       int64_t rows_a, int n, int kb, int64_t units, int* __restrict__ err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(base + WsSmem::bars);
  uint32_t* tmem_slot = (uint32_t*)(bars + 14);
  volatile int* fail = (volatile int*)(tmem_slot + 1);
  float* Ahi = (float*)(base + WsSmem::a_hi);
  float* Alo = (float*)(base + WsSmem::a_lo);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int NB = (n + UNIT_N - 1) / UNIT_N;
  const int64_t ubeg = units * blockIdx.x / gridDim.x;
  const int nv = (int)(units * (blockIdx.x + 1) / gridDim.x - ubeg);

  if (threadIdx.x == 0) {
    *fail = 0;
    mbar_init(&bars[B_AFULL], 1);
    mbar_init(&bars[B_AFREE], 1);
    for (int q = 0; q < 2; ++q) {
      mbar_init(&bars[B_BFULL + q], 1);
      mbar_init(&bars[B_BFREE + q], 1);
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
                 "r"(TMEM_RING * UNIT_N)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp >= 4) {
    // ---------------- producer group ----------------
    const int pt = threadIdx.x - 128;
    const bool leader = pt == 0;
    auto bslot = [&](int slot) { return base + WsSmem::b0 + slot * WsSmem::b_slot; };
    auto load_b = [&](int v) {
      const int slot = v & 1, nb = (int)((ubeg + v) % NB);
      uint8_t* bs = bslot(slot);
      mbar_expect_tx(&bars[B_BFULL + slot], (uint32_t)(2 * kb * WsSmem::chunk_b));
      for (int q = 0; q < kb; ++q) {
        tma_load_2d(bs + q * WsSmem::chunk_b, &tmBhi, &bars[B_BFULL + slot], q * KCHUNK, nb * UNIT_N);
        tma_load_2d(bs + (2 + q) * WsSmem::chunk_b, &tmBlo, &bars[B_BFULL + slot], q * KCHUNK,
                    nb * UNIT_N);
      }
    };
    if (leader && nv > 0) load_b(0);
    int64_t tcur = -1;
    int ka = 0;
    // No early exit: every thread of the group runs the same iterations and
    // reaches every group_sync(); after a failure the work is skipped.
    for (int v = 0; v < nv; ++v) {
      const int64_t u = ubeg + v, t = u / NB;
      if (t != tcur) {
        if (leader && !*fail) {
          if (ka == 0 || mbar_wait(&bars[B_AFREE], (uint32_t)((ka - 1) & 1))) {
            mbar_expect_tx(&bars[B_AFULL], (uint32_t)(kb * WsSmem::chunk_a));
            for (int q = 0; q < kb; ++q)
              tma_load_2d(Ahi + q * TILE_M * KCHUNK, &tmA, &bars[B_AFULL], q * KCHUNK,
                          (int)(t * TILE_M));
          } else {
            *fail = 1;
          }
        }
        if (!*fail && !mbar_wait(&bars[B_AFULL], (uint32_t)(ka & 1))) *fail = 1;
        if (!*fail) {
          const int total = kb * TILE_M * KCHUNK;
          for (int e = pt * 4; e < total; e += 128 * 4) {
            float4 x = *(float4*)(Ahi + e);
            float4 h = make_float4(tf32_rna(x.x), tf32_rna(x.y), tf32_rna(x.z), tf32_rna(x.w));
            *(float4*)(Ahi + e) = h;
            *(float4*)(Alo + e) = make_float4(x.x - h.x, x.y - h.y, x.z - h.z, x.w - h.w);
          }
          fence_async_smem();
        }
        group_sync();
        ++ka;
        tcur = t;
      }
      if (leader && !*fail) {
        const int blk = v & (TMEM_RING - 1), slot = v & 1;
        bool ok = v < TMEM_RING ||
                  mbar_wait(&bars[B_TEMPTY + blk], (uint32_t)(((v / TMEM_RING) - 1) & 1));
        ok = ok && mbar_wait(&bars[B_BFULL + slot], (uint32_t)((v >> 1) & 1));
        if (ok) {
          tc_fence_after();
          const uint32_t dcol = tmem + (uint32_t)(blk * UNIT_N);
          const uint8_t* bs = bslot(slot);
          uint32_t accum = 0;
          // small terms first: A_hi B_lo, A_lo B_hi, then A_hi B_hi
          for (int pass = 0; pass < 3; ++pass) {
            const float* Ap = pass == 1 ? Alo : Ahi;
            const uint8_t* Bp = pass == 0 ? bs + 2 * WsSmem::chunk_b : bs;
            for (int q = 0; q < kb; ++q) {
              const uint64_t ad = sw128_desc(Ap + q * TILE_M * KCHUNK);
              const uint64_t bd = sw128_desc(Bp + q * WsSmem::chunk_b);
#pragma unroll
              for (int k = 0; k < KCHUNK / 8; ++k) {
                // advance 8 TF32 = 32 bytes along K inside the swizzle row
                mma_tf32(dcol, ad + (uint64_t)(2 * k), bd + (uint64_t)(2 * k), kIdesc, accum);
                accum = 1;
              }
            }
          }
          mma_commit(&bars[B_BFREE + slot]);
          mma_commit(&bars[B_TFULL + blk]);
          if (v + 1 == nv || (u + 1) / NB != t) mma_commit(&bars[B_AFREE]);
          if (v + 1 < nv) {
            ok = v < 1 || mbar_wait(&bars[B_BFREE + ((v + 1) & 1)], (uint32_t)(((v - 1) >> 1) & 1));
            if (ok) load_b(v + 1);
          }
        }
        if (!ok) *fail = 1;
      }
    }
  } else {
    // ---------------- epilogue warps ----------------
    float* stg0 = (float*)(base + WsSmem::stage + (size_t)(2 * warp) * WsSmem::box);
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    int sb = 0;
    for (int v = 0; v < nv; ++v) {
      if (__shfl_sync(0xffffffffu, *fail, 0)) continue;
      const int64_t u = ubeg + v, t = u / NB;
      const int nb = (int)(u % NB), blk = v & (TMEM_RING - 1);
      const bool ok = __all_sync(0xffffffffu,
                                 mbar_wait(&bars[B_TFULL + blk], (uint32_t)((v / TMEM_RING) & 1)));
      if (!ok) {
        if (lane == 0) *fail = 1;
        continue;
      }
      tc_fence_after();
      const int64_t row0 = t * TILE_M + warp * 32;
      if (row0 < rows_a) {
        for (int j = 0; j < UNIT_N / BOX; ++j) {
          const int col0 = nb * UNIT_N + j * BOX;
          if (col0 >= n) break;
          uint32_t r[32];
          tmem_ld32(tmem + lane_base + (uint32_t)(blk * UNIT_N + j * BOX), r);
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
            tma_store_2d(&tmC, stg, col0, (int)row0);
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
                 "r"(TMEM_RING * UNIT_N)
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

cudaError_t corr_tf32x3(const float* A, int64_t rows_a, const float* Bhi, const float* Blo, int n,
                        int p, float* C, int64_t ldc, int* err, cudaStream_t st) {
  if (rows_a <= 0) return cudaSuccess;
  if (((uintptr_t)C % 16) != 0) return cudaErrorInvalidValue;
  CUtensorMap ma, mbh, mbl, mc;
  if (!make_map(&ma, A, rows_a, p, TILE_M) || !make_map(&mbh, Bhi, n, p, UNIT_N) ||
      !make_map(&mbl, Blo, n, p, UNIT_N) || !make_map_out(&mc, C, rows_a, n, ldc))
    return cudaErrorInvalidValue;
  const int kb = (p + KCHUNK - 1) / KCHUNK;
  cudaError_t e = cudaFuncSetAttribute(corr_tf32x3_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)WsSmem::dyn);
  if (e != cudaSuccess) return e;
  const int64_t tiles = (rows_a + TILE_M - 1) / TILE_M;
  const int64_t units = tiles * ((n + UNIT_N - 1) / UNIT_N);
  const unsigned grid = (unsigned)(units < num_sms() ? units : num_sms());
  corr_tf32x3_kernel<<<grid, WS_THREADS, WsSmem::dyn, st>>>(ma, mbh, mbl, mc, rows_a, n, kb, units,
                                                            err);
  return cudaGetLastError();
}

}  // namespace dlk
