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
// One CTA computes a 128-row tile of C for all columns (n <= 512):
//   * TMA loads the A tile (128 rows x 64 K, SWIZZLE_128B) into shared memory;
//     the CTA's threads split it in place into A_hi / A_lo;
//   * per block of 256 columns, TMA loads B_hi and B_lo (pre-split on the
//     device), one thread issues 3 x (K/8) tcgen05.mma kind::tf32
//     (M=128, N=256, K=8) into a 256-column TMEM accumulator;
//   * the four warps read the accumulator back with tcgen05.ld (warp w owns
//     TMEM lanes 32w..32w+31 = rows) and store rows of C with 16-byte stores.
// Every wait on an mbarrier is bounded (2 s of %globaltimer); on timeout the
// kernel flags ERR_TIMEOUT, frees its TMEM and returns.
#include "dl_internal.cuh"
#include "tc_ptx.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>
#include <stdint.h>

namespace dlk {
namespace {

constexpr int TC_THREADS = 128;
constexpr int TILE_M = 128;
constexpr int BLOCK_N = 256;
constexpr int KCHUNK = 32;  // floats per 128-byte swizzle row
using namespace tc;
// Instruction descriptor: kind::tf32, A/B TF32 K-major, D FP32, M = 128, N = 256.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BLOCK_N >> 3) << 17) |
                            ((uint32_t)(TILE_M >> 4) << 24);

struct TcSmem {
  // byte offsets from the 1024-aligned base
  static constexpr size_t a_chunk = (size_t)TILE_M * KCHUNK * 4;   // 16 KB
  static constexpr size_t b_chunk = (size_t)BLOCK_N * KCHUNK * 4;  // 32 KB
  static size_t bytes(int kb) { return 1024 + kb * (2 * a_chunk + 2 * b_chunk) + 64; }
};

__global__ void __launch_bounds__(TC_THREADS, 1)
    corr_tf32x3_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmBhi,
                       const __grid_constant__ CUtensorMap tmBlo, int64_t rows_a, int n, int kb,
                       float* __restrict__ C, int64_t ldc, int* __restrict__ err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  float* Ahi = (float*)base;
  float* Alo = (float*)(base + kb * TcSmem::a_chunk);
  float* Bhi = (float*)(base + 2 * kb * TcSmem::a_chunk);
  float* Blo = (float*)(base + 2 * kb * TcSmem::a_chunk + kb * TcSmem::b_chunk);
  uint64_t* bars = (uint64_t*)(base + 2 * kb * (TcSmem::a_chunk + TcSmem::b_chunk));
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

  // ---- A tile: TMA, then split into head / tail in place
  if (threadIdx.x == 0) {
    mbar_expect_tx(&bars[0], (uint32_t)(kb * TcSmem::a_chunk));
    for (int q = 0; q < kb; ++q)
      tma_load_2d(Ahi + q * TILE_M * KCHUNK, &tmA, &bars[0], q * KCHUNK, (int)i0);
  }
  if (!mbar_wait(&bars[0], 0)) s_fail = 1;
  __syncthreads();
  if (!s_fail) {
    const int total = kb * TILE_M * KCHUNK;
    for (int e = threadIdx.x * 4; e < total; e += TC_THREADS * 4) {
      float4 v = *(float4*)(Ahi + e);
      float4 h = make_float4(tf32_rna(v.x), tf32_rna(v.y), tf32_rna(v.z), tf32_rna(v.w));
      *(float4*)(Ahi + e) = h;
      *(float4*)(Alo + e) = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
    }
    fence_async_smem();
  }
  __syncthreads();

  // ---- per 256-column block: TMA the pre-split B, issue the MMAs
  for (int nb = 0; nb < nblocks && !s_fail; ++nb) {
    if (threadIdx.x == 0) {
      mbar_expect_tx(&bars[1], (uint32_t)(2 * kb * TcSmem::b_chunk));
      for (int q = 0; q < kb; ++q) {
        tma_load_2d(Bhi + q * BLOCK_N * KCHUNK, &tmBhi, &bars[1], q * KCHUNK, nb * BLOCK_N);
        tma_load_2d(Blo + q * BLOCK_N * KCHUNK, &tmBlo, &bars[1], q * KCHUNK, nb * BLOCK_N);
      }
      bool ok = mbar_wait(&bars[1], (uint32_t)(nb & 1));
      if (ok) {
        tc_fence_after();
        const uint32_t dcol = tmem + (uint32_t)(nb * BLOCK_N);
        uint32_t accum = 0;
        // small terms first: A_hi B_lo, A_lo B_hi, then A_hi B_hi
        for (int pass = 0; pass < 3; ++pass) {
          const float* Ap = pass == 1 ? Alo : Ahi;
          const float* Bp = pass == 0 ? Blo : Bhi;
          for (int q = 0; q < kb; ++q) {
            const uint64_t ad = sw128_desc(Ap + q * TILE_M * KCHUNK);
            const uint64_t bd = sw128_desc(Bp + q * BLOCK_N * KCHUNK);
#pragma unroll
            for (int k = 0; k < KCHUNK / 8; ++k) {
              // advance 8 TF32 = 32 bytes along K inside the swizzle row
              mma_tf32(dcol, ad + (uint64_t)(2 * k), bd + (uint64_t)(2 * k), kIdesc, accum);
              accum = 1;
            }
          }
        }
        mma_commit(&bars[2]);
        ok = mbar_wait(&bars[2], (uint32_t)(nb & 1));
      }
      if (!ok) s_fail = 1;
    }
    __syncthreads();
  }

  // ---- epilogue: TMEM -> registers -> C rows
  tc_fence_after();
  if (!s_fail) {
    const int64_t row = i0 + warp * 32 + lane;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    for (int c0 = 0; c0 < n; c0 += 16) {
      uint32_t r[16];
      tmem_ld16(tmem + lane_base + (uint32_t)c0, r);
      if (row < rows_a) {
        float4* dst = (float4*)(C + row * ldc + c0);
#pragma unroll
        for (int q = 0; q < 4; ++q)
          dst[q] = make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                               __uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]));
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

}  // namespace

bool corr_tc_supported(const float* A, int p, int n, int64_t ldc) {
  return p >= 1 && p <= 64 && (p % 4) == 0 && n >= 1 && n <= 512 && (ldc % 4) == 0 &&
         ldc >= (int64_t)(n + 15) / 16 * 16 && ((uintptr_t)A % 16) == 0 && encode_fn() != nullptr;
}

size_t corr_tc_smem(int p) { return TcSmem::bytes((p + KCHUNK - 1) / KCHUNK); }

cudaError_t split_tf32(const float* B, int64_t count, float* hi, float* lo, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  split_kernel<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(B, count, hi, lo);
  return cudaGetLastError();
}

cudaError_t corr_tf32x3(const float* A, int64_t rows_a, const float* Bhi, const float* Blo, int n,
                        int p, float* C, int64_t ldc, int* err, cudaStream_t st) {
  if (rows_a <= 0) return cudaSuccess;
  CUtensorMap ma, mbh, mbl;
  if (!make_map(&ma, A, rows_a, p, TILE_M) || !make_map(&mbh, Bhi, n, p, BLOCK_N) ||
      !make_map(&mbl, Blo, n, p, BLOCK_N))
    return cudaErrorInvalidValue;
  const int kb = (p + KCHUNK - 1) / KCHUNK;
  const size_t smem = corr_tc_smem(p);
  cudaError_t e = cudaFuncSetAttribute(corr_tf32x3_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)((rows_a + TILE_M - 1) / TILE_M);
  corr_tf32x3_kernel<<<grid, TC_THREADS, smem, st>>>(ma, mbh, mbl, rows_a, n, kb, C, ldc, err);
  return cudaGetLastError();
}

}  // namespace dlk
