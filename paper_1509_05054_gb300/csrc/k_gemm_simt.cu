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

// ---- Gram matrix G = D D^T (n x n, row-major; D n x p row-major) ----------------
// The Gram matrix of Batch-OMP and of the residual-form OMP's Cholesky rows, as
// one short launch: a CTA per 32 x 32 block of the upper triangle (136 CTAs at
// n = 512, one SM each), 256 threads of 2 x 2 entries, the two 32-atom row
// blocks in shared memory (odd pitch: no bank conflicts), FP32 sums in row
// order; each block is written with its mirror, so G is exactly symmetric.
namespace dlk {
namespace {

constexpr int GT = 32, GK = 64;

__global__ void __launch_bounds__(256) gram_kernel(const float* __restrict__ D, int n, int p,
                                                   float* __restrict__ G, int tiles) {
  __shared__ float Dj[GT][GK + 1];
  __shared__ float Dk[GT][GK + 1];
  // block b -> (jt, kt) with jt <= kt, row by row of the upper triangle
  int b = blockIdx.x, jt = 0;
  while (b >= tiles - jt) {
    b -= tiles - jt;
    ++jt;
  }
  const int kt = jt + b;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
  for (int k0 = 0; k0 < p; k0 += GK) {
    __syncthreads();
    for (int e = tid; e < GT * GK; e += 256) {
      const int r = e / GK, c = e % GK;
      const int j = jt * GT + r, k = kt * GT + r;
      Dj[r][c] = (j < n && k0 + c < p) ? __ldg(D + (size_t)j * p + k0 + c) : 0.f;
      Dk[r][c] = (k < n && k0 + c < p) ? __ldg(D + (size_t)k * p + k0 + c) : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int c = 0; c < GK; ++c) {
      const float a0 = Dj[2 * ty][c], a1 = Dj[2 * ty + 1][c];
      const float b0 = Dk[2 * tx][c], b1 = Dk[2 * tx + 1][c];
      acc[0][0] = fmaf(a0, b0, acc[0][0]);
      acc[0][1] = fmaf(a0, b1, acc[0][1]);
      acc[1][0] = fmaf(a1, b0, acc[1][0]);
      acc[1][1] = fmaf(a1, b1, acc[1][1]);
    }
  }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int j = jt * GT + 2 * ty + a, k = kt * GT + 2 * tx + c;
      if (j < n && k < n) {
        G[(size_t)j * n + k] = acc[a][c];
        G[(size_t)k * n + j] = acc[a][c];
      }
    }
}

}  // namespace

cudaError_t gram_simt(const float* D, int n, int p, float* G, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int tiles = (n + GT - 1) / GT;
  gram_kernel<<<tiles * (tiles + 1) / 2, 256, 0, st>>>(D, n, p, G, tiles);
  return cudaGetLastError();
}

}  // namespace dlk
