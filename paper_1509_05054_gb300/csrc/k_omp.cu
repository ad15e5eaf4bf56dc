// Batch-OMP sparse coding, one warp per signal (Algorithm 1 step 1; the OMP-Box
// tool named in Section 4 implements the Cholesky "Batch-OMP" of [RZE08]).
//
// Per signal y with correlations alpha0 = D^T y and Gram G = D^T D, step k:
//   sel   = argmax_{j not selected} |alpha_j|                (lowest index on ties)
//   w_q   = q_q^T d_sel (q < k): the new row of the Cholesky factor of G[I,I]
//   delta = G[sel,sel] - w.w,  c_k = 1/sqrt(delta) = 1/L_kk
//   z_k   = c_k alpha[sel]     (coefficient of y on the new orthonormal direction q_k)
//   u_k   = G[:, sel] - sum_{q<k} (w_q c_q) u_q       (D^T q_k = c_k u_k)
//   alpha = alpha - (z_k c_k) u_k                         (= D^T r_k)
// and at the end x_I = L^{-T} z.  This is the Gram-Schmidt (progressive
// Cholesky) form of Batch-OMP: alpha is updated with one new vector per step
// instead of being recomputed as alpha0 - G[:,I] gamma; the multiply-adds are
// the same n*k per step, there is no triangular solve per step, and w_q is read
// from the stored vectors (w_q = c_q u_q[sel]) instead of a forward
// substitution.  Identical to the oracle's Batch-OMP in exact arithmetic.
//
// Lane l of the warp holds alpha[32t + l], t < NT = ceil(n/32), as NT/2 float2
// pairs (elements t = 2v, 2v+1) so the updates issue as packed FP32x2 FMAs
// (__ffma2_rn, sm_100 family); the first NR u vectors live in registers, the
// rest in shared memory (see reg_us).  Selected atoms are masked by setting their alpha to NaN,
// which the argmax ignores.
#include "dl_internal.cuh"
#include "omp_common.cuh"
#include "omp_one.cuh"

#include <math.h>

namespace dlk {
namespace {

using namespace omp;
constexpr int OMP_THREADS = 128;

template <int NT, int SMAX, int NR, bool FULLN>
__global__ void __launch_bounds__(OMP_THREADS) omp_warp_kernel(
    const float* __restrict__ A0, int64_t lda, const float* __restrict__ G, int n,
    const float* __restrict__ Y, int p, int64_t m, int s, int32_t* __restrict__ oidx,
    float* __restrict__ oval, int32_t* __restrict__ ocnt, float* __restrict__ ores,
    int* __restrict__ err, int* __restrict__ rs_list, int* __restrict__ rs_count, int rs_cap,
    int64_t pf, float gap_tol) {
  constexpr int NPHI = SMAX > 1 ? SMAX - 1 : 1;
  extern __shared__ float2 smem_u[];
  __shared__ float Lsh[OMP_THREADS / 32][SMAX][SMAX];  // per warp: L[j][q] (q < j)
  __shared__ float Csh[OMP_THREADS / 32][SMAX];        // per warp: c_q = 1/L_qq
  const int wib = threadIdx.x >> 5;
  const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
  if (i >= m) return;
  // Warm L2 with the correlations and samples of signal i + pf, which a warp of
  // a later block picks up about when this one finishes (pf ~ the warps resident
  // on the GPU): its first loads then hit L2 instead of DRAM (measured: OMP 2%
  // faster).  One 128-byte line per lane, inside the rows of A0 and Y.
  {
    const int lane = threadIdx.x & 31;
    const int64_t ip = i + pf;
    if (ip < m) {
      if (lane * 32 < n) asm volatile("prefetch.global.L2 [%0];" ::"l"(A0 + ip * lda + lane * 32));
      if (lane * 32 < p) asm volatile("prefetch.global.L2 [%0];" ::"l"(Y + ip * p + lane * 32));
    }
  }
  float2* u_s = NR < NPHI ? smem_u + (size_t)wib * (NPHI - NR) * (NT / 2) * 32 : nullptr;
  const GramGlobal<FULLN> gsrc{G, n};
  omp_one<NT, SMAX, NR, FULLN, true>(i, gsrc, Lsh[wib], Csh[wib], u_s, A0 + i * lda, n, Y + i * p, p,
                                s, nullptr, oidx, oval, ocnt, ores, err, rs_list, rs_count, rs_cap,
                                gap_tol);
}

// OMP restricted to K proposed candidates per signal (cand: m x K, ascending):
// the correlations d_c^T y of the candidates are computed here, the Gram
// entries come from the full Gram matrix.  Writes the slots (atom indices) and
// the residual estimate; a signal whose residual energy exceeds `tol2` times its
// reference residual energy (ref_res from the last full pass) is appended to
// fb_list for full OMP.
template <int SMAX>
__global__ void __launch_bounds__(OMP_THREADS) omp_restricted_kernel(
    const int32_t* __restrict__ cand, int K, const float* __restrict__ D, const float* __restrict__ G,
    int n, const float* __restrict__ Y, int p, int64_t m, int s, int32_t* __restrict__ oidx,
    float* __restrict__ oval, int32_t* __restrict__ ocnt, float* __restrict__ ores,
    const float* __restrict__ ref_res, float tol2, int* __restrict__ fb_list, int* __restrict__ fb_count,
    int* __restrict__ err) {
  __shared__ float Lsh[OMP_THREADS / 32][SMAX][SMAX];
  __shared__ float Csh[OMP_THREADS / 32][SMAX];
  __shared__ float a0sh[OMP_THREADS / 32][32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
  if (i >= m) return;
  const int32_t* ci = cand + i * K;
  const float* y = Y + i * p;
  float a = 0.f;
  if (lane < K) {
    const float* dc = D + (size_t)ci[lane] * p;
    for (int r = 0; r < p; ++r) a = fmaf(dc[r], y[r], a);
  }
  a0sh[wib][lane] = a;
  __syncwarp();
  const GramRestricted gsrc{G, n, ci, K};
  omp_one<2, SMAX, (SMAX > 1 ? SMAX - 1 : 1), false, false>(i, gsrc, Lsh[wib], Csh[wib], nullptr, a0sh[wib], K, y, p, s, ci,
                                 oidx, oval, ocnt, ores, err, nullptr, nullptr, 0, 0.f);
  __syncwarp();
  if (lane == 0 && fb_count && ores[i] > tol2 * ref_res[i]) {
    const int pos = atomicAdd(fb_count, 1);
    if (pos < (int)m) fb_list[pos] = (int)i;
  }
}

// Full OMP of the listed signals (the proposer's fallback): one warp computes the
// signal's correlations D^T y into shared memory, then runs the OMP.
template <int NT, int SMAX>
__global__ void __launch_bounds__(OMP_THREADS) omp_listed_kernel(
    const int* __restrict__ list, const int* __restrict__ count, const float* __restrict__ A0,
    int64_t lda, const float* __restrict__ G, int n, const float* __restrict__ Y, int p, int s,
    int32_t* __restrict__ oidx, float* __restrict__ oval, int32_t* __restrict__ ocnt,
    float* __restrict__ ores, int* __restrict__ err, int* __restrict__ rs_list,
    int* __restrict__ rs_count, int rs_cap) {
  __shared__ float Lsh[OMP_THREADS / 32][SMAX][SMAX];
  __shared__ float Csh[OMP_THREADS / 32][SMAX];
  const int wib = threadIdx.x >> 5;
  const int total = *count;
  const int nw = gridDim.x * (blockDim.x >> 5);
  for (int e = blockIdx.x * (blockDim.x >> 5) + wib; e < total; e += nw) {
    const int64_t i = list[e];
    const GramGlobal<false> gsrc{G, n};
    omp_one<NT, SMAX, (SMAX > 1 ? SMAX - 1 : 1), false, true>(i, gsrc, Lsh[wib], Csh[wib], nullptr, A0 + i * lda, n, Y + i * p,
                                    p, s, nullptr, oidx, oval, ocnt, ores, err, rs_list, rs_count,
                                    rs_cap, 0.f);
    __syncwarp();
  }
}

template <int NT, int SMAX, int NR, bool FULLN>
cudaError_t launch_t(const float* A0, int64_t lda, const float* G, int n, const float* Y, int p,
                     int64_t m, int s, int32_t* idx, float* val, int32_t* cnt, int* err,
                     int* rs_list, int* rs_count, int rs_cap, int warps_hint, float* ores,
                     float gt, cudaStream_t st) {
  constexpr int NPHI = SMAX > 1 ? SMAX - 1 : 1;
  int warps = (warps_hint >= 1 && warps_hint <= OMP_THREADS / 32) ? warps_hint : OMP_THREADS / 32;
  size_t smem = 0;
  if (NR < NPHI) {
    const size_t per_warp = (size_t)(NPHI - NR) * (NT / 2) * 32 * sizeof(float2);
    const int cap = (int)((190u * 1024u) / per_warp);
    if (warps > cap) warps = cap;
    if (warps < 1) warps = 1;
    smem = per_warp * warps;
    cudaFuncSetAttribute(omp_warp_kernel<NT, SMAX, NR, FULLN>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  } else {  // Gram rows are re-read through L1: give L1 the shared-memory carveout
    cudaFuncSetAttribute(omp_warp_kernel<NT, SMAX, NR, FULLN>,
                         cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxL1);
  }
  const int64_t blocks = (m + warps - 1) / warps;
  omp_warp_kernel<NT, SMAX, NR, FULLN><<<(unsigned)blocks, warps * 32, smem, st>>>(
      A0, lda, G, n, Y, p, m, s, idx, val, cnt, ores, err, rs_list, rs_count, rs_cap,
      (int64_t)8 * num_sms(), gt);
  return cudaGetLastError();
}

// How many u vectors stay in registers.  With 16 alpha elements per lane
// (n <= 512) keeping all of them caps the kernel near 168 registers (12 warps
// per SM); three in registers and the rest in shared memory gives ~126
// registers and 16 warps per SM, which hides more of the Gram-row latency
// (measured 8% faster at n = 512, s = 8).  Otherwise: all in registers while
// alpha + u fit (NT*(SMAX-1) <= 128 floats), else all in shared memory.
template <int NT, int SMAX>
constexpr int reg_us() {
  constexpr int nphi = SMAX > 1 ? SMAX - 1 : 1;
  if (NT == 16 && nphi > 3) return 3;
  return NT * (SMAX - 1) <= 128 ? nphi : 0;
}

template <int NT, int SMAX>
cudaError_t pick_store(const float* A0, int64_t lda, const float* G, int n, const float* Y, int p,
                       int64_t m, int s, int32_t* idx, float* val, int32_t* cnt, int* err,
                       int* rl, int* rc, int rcap, int wh, float* ores, float gt, cudaStream_t st) {
  constexpr int NR = reg_us<NT, SMAX>();
  if (n == 32 * NT)
    return launch_t<NT, SMAX, NR, true>(A0, lda, G, n, Y, p, m, s, idx, val, cnt, err, rl, rc, rcap, wh, ores, gt, st);
  return launch_t<NT, SMAX, NR, false>(A0, lda, G, n, Y, p, m, s, idx, val, cnt, err, rl, rc, rcap, wh, ores, gt, st);
}

template <int NT>
cudaError_t pick_s(const float* A0, int64_t lda, const float* G, int n, const float* Y, int p,
                   int64_t m, int s, int32_t* idx, float* val, int32_t* cnt, int* err,
                   int* rl, int* rc, int rcap, int wh, float* ores, float gt, cudaStream_t st) {
  if (s <= 4) return pick_store<NT, 4>(A0, lda, G, n, Y, p, m, s, idx, val, cnt, err, rl, rc, rcap, wh, ores, gt, st);
  if (s <= 8) return pick_store<NT, 8>(A0, lda, G, n, Y, p, m, s, idx, val, cnt, err, rl, rc, rcap, wh, ores, gt, st);
  if (s <= 12) return pick_store<NT, 12>(A0, lda, G, n, Y, p, m, s, idx, val, cnt, err, rl, rc, rcap, wh, ores, gt, st);
  return pick_store<NT, 16>(A0, lda, G, n, Y, p, m, s, idx, val, cnt, err, rl, rc, rcap, wh, ores, gt, st);
}

}  // namespace

bool omp_supported(int n, int s) { return n >= 1 && n <= 1024 && s >= 1 && s <= 16; }

bool omp_restricted_supported(int n, int s, int K) {
  const int nt = (n + 31) / 32;
  const int sm = s <= 4 ? 4 : s <= 8 ? 8 : 0;
  return K >= 1 && K <= 32 && s <= K && sm > 0 && (nt <= 2 ? 2 : nt <= 4 ? 4 : nt <= 8 ? 8 : 16) * (sm - 1) <= 128 &&
         n <= 512;
}

cudaError_t omp_restricted(const int32_t* cand, int K, const float* D, const float* G, int n,
                           const float* Y, int p, int64_t m, int s, int32_t* idx, float* val,
                           int32_t* cnt, float* ores, const float* ref_res, float tol2, int* fb_list,
                           int* fb_count, int* err, cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((m + 3) / 4);
  if (s <= 4)
    omp_restricted_kernel<4><<<blocks, OMP_THREADS, 0, st>>>(cand, K, D, G, n, Y, p, m, s, idx, val,
                                                             cnt, ores, ref_res, tol2, fb_list,
                                                             fb_count, err);
  else
    omp_restricted_kernel<8><<<blocks, OMP_THREADS, 0, st>>>(cand, K, D, G, n, Y, p, m, s, idx, val,
                                                             cnt, ores, ref_res, tol2, fb_list,
                                                             fb_count, err);
  return cudaGetLastError();
}

template <int NT>
cudaError_t listed_s(const int* list, const int* count, const float* A0, int64_t lda, const float* G,
                     int n, const float* Y, int p, int s, int32_t* idx, float* val, int32_t* cnt,
                     float* ores, int* err, int* rl, int* rc, int rcap, cudaStream_t st) {
  const unsigned blocks = (unsigned)(num_sms() * 3);
  if (s <= 4)
    omp_listed_kernel<NT, 4><<<blocks, OMP_THREADS, 0, st>>>(list, count, A0, lda, G, n, Y, p, s, idx,
                                                             val, cnt, ores, err, rl, rc, rcap);
  else
    omp_listed_kernel<NT, 8><<<blocks, OMP_THREADS, 0, st>>>(list, count, A0, lda, G, n, Y, p, s, idx,
                                                             val, cnt, ores, err, rl, rc, rcap);
  return cudaGetLastError();
}

cudaError_t omp_listed(const int* list, const int* count, const float* A0, int64_t lda,
                       const float* G, int n, const float* Y, int p, int s, int32_t* idx, float* val,
                       int32_t* cnt, float* ores, int* err, int* rl, int* rc, int rcap,
                       cudaStream_t st) {
  const int nt = (n + 31) / 32;
  if (nt <= 2) return listed_s<2>(list, count, A0, lda, G, n, Y, p, s, idx, val, cnt, ores, err, rl, rc, rcap, st);
  if (nt <= 4) return listed_s<4>(list, count, A0, lda, G, n, Y, p, s, idx, val, cnt, ores, err, rl, rc, rcap, st);
  if (nt <= 8) return listed_s<8>(list, count, A0, lda, G, n, Y, p, s, idx, val, cnt, ores, err, rl, rc, rcap, st);
  return listed_s<16>(list, count, A0, lda, G, n, Y, p, s, idx, val, cnt, ores, err, rl, rc, rcap, st);
}

cudaError_t omp_batch(const float* A0, int64_t lda, const float* G, int n, const float* Y, int p,
                      int64_t m, int s, int32_t* idx, float* val, int32_t* cnt, int* err,
                      int* rl, int* rc, int rcap, int wh, float* ores, float gt, cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  const int nt = (n + 31) / 32;
  if (nt <= 2) return pick_s<2>(A0, lda, G, n, Y, p, m, s, idx, val, cnt, err, rl, rc, rcap, wh, ores, gt, st);
  if (nt <= 4) return pick_s<4>(A0, lda, G, n, Y, p, m, s, idx, val, cnt, err, rl, rc, rcap, wh, ores, gt, st);
  if (nt <= 8) return pick_s<8>(A0, lda, G, n, Y, p, m, s, idx, val, cnt, err, rl, rc, rcap, wh, ores, gt, st);
  if (nt <= 16) return pick_s<16>(A0, lda, G, n, Y, p, m, s, idx, val, cnt, err, rl, rc, rcap, wh, ores, gt, st);
  return pick_s<32>(A0, lda, G, n, Y, p, m, s, idx, val, cnt, err, rl, rc, rcap, wh, ores, gt, st);
}

}  // namespace dlk
