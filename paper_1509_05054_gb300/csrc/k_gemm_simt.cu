// FP32 CUDA-core GEMM C = A B^T with both operands K-major (rows of length p).
// Used for the Gram matrix G = D^T D (Batch-OMP, [RZE08] as cited in Section 4)
// and, as the FP32 reference path, for the correlations D^T Y (Algorithm 1 step 1).
#include "dl_internal.cuh"

namespace dlk {
namespace {

constexpr int TM = 128, TN = 128, TK = 32, NTHR = 256;

__global__ void __launch_bounds__(NTHR) gemm_nt_kernel(const float* __restrict__ A, int64_t rows_a,
                                                       const float* __restrict__ B, int rows_b, int p,
                                                       float* __restrict__ C, int64_t ldc) {
  __shared__ float As[TK][TM + 1];
  __shared__ float Bs[TK][TN + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t i0 = (int64_t)blockIdx.x * TM;
  const int j0 = blockIdx.y * TN;
  float acc[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;

  for (int k0 = 0; k0 < p; k0 += TK) {
    for (int e = tid; e < TM * TK; e += NTHR) {
      const int r = e / TK, c = e % TK;
      const int64_t gi = i0 + r;
      As[c][r] = (gi < rows_a && k0 + c < p) ? A[gi * p + k0 + c] : 0.f;
      const int gj = j0 + r;
      Bs[c][r] = (gj < rows_b && k0 + c < p) ? B[(int64_t)gj * p + k0 + c] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < TK; ++kk) {
      float a[8], b[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        a[q] = As[kk][ty + 16 * q];
        b[q] = Bs[kk][tx + 16 * q];
      }
#pragma unroll
      for (int x = 0; x < 8; ++x)
#pragma unroll
        for (int y = 0; y < 8; ++y) acc[x][y] = fmaf(a[x], b[y], acc[x][y]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int x = 0; x < 8; ++x) {
    const int64_t gi = i0 + ty + 16 * x;
    if (gi >= rows_a) continue;
#pragma unroll
    for (int y = 0; y < 8; ++y) {
      const int gj = j0 + tx + 16 * y;
      if (gj < rows_b) C[gi * ldc + gj] = acc[x][y];
    }
  }
}

}  // namespace

cudaError_t gemm_nt_simt(const float* A, int64_t rows_a, const float* B, int rows_b, int p, float* C,
                         int64_t ldc, cudaStream_t st) {
  if (rows_a <= 0 || rows_b <= 0) return cudaSuccess;
  dim3 grid((unsigned)((rows_a + TM - 1) / TM), (unsigned)((rows_b + TN - 1) / TN));
  gemm_nt_kernel<<<grid, NTHR, 0, st>>>(A, rows_a, B, rows_b, p, C, ldc);
  return cudaGetLastError();
}

}  // namespace dlk
