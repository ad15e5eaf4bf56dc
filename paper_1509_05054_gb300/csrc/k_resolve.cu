// Re-solve of the signals the FP32 OMP cannot decide: a Cholesky pivot below
// 1e-6 (dominated by FP32 rounding), or, for long supports, a step whose top
// two |correlations| lie inside the FP32 error of alpha.  One warp per listed
// signal redoes its whole OMP (Algorithm 1 step 1) so that every decision and
// the coefficients are those of the FP64 Batch-OMP:
//
//   * the residual r = y - D_I gamma is kept in FP64 (p values), with gamma
//     from the FP64 Cholesky factor of G[I,I] (entries d_q^T d_sel taken in
//     FP64 from the FP32 atoms, which FP64 holds exactly), alpha0_I = D_I^T y
//     in FP64 and the forward/back substitutions in FP64;
//   * each step's correlations alpha = alpha0 - G[:, I] gamma are taken in
//     FP32, fresh every step (no rounding carries over from step to step), from
//     alpha0 (the FP32 product of the coding pass, or, after reduced-precision
//     correlations, D^T y taken here in FP32), the FP32 Gram rows of the
//     selected atoms (copied to shared memory as atoms are selected) and gamma
//     rounded to FP32.  With alpha0 within c ||y|| dmax and the Gram entries
//     within c dmax^2 of exact, c = max(4.5e-6, (p + 2) 2^-24) (split-TF32
//     products: three 2^-22 terms and FP32 sums; or FP32 sums of p products;
//     measured 2.2e-7 and 4.7e-7 at p = 64), alpha is within
//     E = (c + 1.5e-6) dmax (||y|| + dmax sum |gamma_q|) of exact, so
//     the exact argmax lies among the atoms within 2E of the FP32 maximum; when
//     more than one atom is there, each one's correlation d_j^T r is recomputed
//     in FP64 and the largest is taken (lowest index on ties), as the FP64
//     oracle decides;
//   * the stop rules are the FP64 ones: pivot <= 1e-12, residual energy
//     <= 1e-14 ||y||^2, max |alpha| = 0.
//
// FP64 runs at a small fraction of the FP32 rate on this GPU, so the FP64 work
// is kept to O(k p) per step (the Cholesky row, alpha0 of the new atom, the
// residual and the few candidates); the O(n p) and O(n k) products stay FP32.
#include "dl_internal.cuh"

#include <math.h>

namespace dlk {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int RS_PMAX = 128;     // largest p (4 rows per lane)
constexpr int RS_RL = RS_PMAX / 32;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

// One warp per CTA; dynamic shared memory: the Gram rows of the selected atoms
// (s x n floats; at the start also the 32-atom tiles of D when alpha0 is taken
// here), alpha0 (n), |alpha| of the current step (n), y (p).
__global__ void __launch_bounds__(32) resolve_kernel(
    const float* __restrict__ Y, int p, const float* __restrict__ D, const float* __restrict__ G,
    const float* __restrict__ A0, int64_t lda, int n, int s, const int* __restrict__ list,
    const int* __restrict__ count, int cap, int32_t* __restrict__ oidx, float* __restrict__ oval,
    int32_t* __restrict__ ocnt) {
  __shared__ double L[DL_RESOLVE_SMAX][DL_RESOLVE_SMAX];
  __shared__ double Z[DL_RESOLVE_SMAX];   // z = L^-1 alpha0_I
  __shared__ double Gm[DL_RESOLVE_SMAX];  // gamma
  __shared__ float g32[DL_RESOLVE_SMAX];  // gamma rounded to FP32
  __shared__ int I[DL_RESOLVE_SMAX];
  extern __shared__ float sh[];
  const int lane = threadIdx.x;
  const int pitch = p | 1;  // odd row pitch: lane-per-atom tile reads hit distinct banks
  const size_t grows = (size_t)s * n > (size_t)32 * pitch ? (size_t)s * n : (size_t)32 * pitch;
  float* Gs = sh;              // row q: G[I_q][:]
  float* a0 = sh + grows;      // alpha0 (NaN once selected)
  float* al = a0 + n;          // |alpha| of the step
  float* ys = al + n;          // y
  int total = *count;
  if (total > cap) total = cap;
  if ((int)blockIdx.x >= total) return;  // nothing listed for this warp (the usual case)

  // largest atom norm (the error bound scales with it)
  float dmax2 = 0.f;
  for (int j = lane; j < n; j += 32) dmax2 = fmaxf(dmax2, __ldg(G + (size_t)j * n + j));
  const double dmax =
      sqrt((double)__uint_as_float(__reduce_max_sync(FULL, __float_as_uint(dmax2))) * 1.0001);
  // relative error of alpha0 and of the Gram entries (split TF32, or FP32 sums of p
  // products), plus the FP32 sums over the selected atoms
  const double cerr = fmax(4.5e-6, (p + 2) * 0x1p-24) + 1.5e-6;

  for (int e = blockIdx.x; e < total; e += gridDim.x) {
    const int64_t i = list[e];
    const float* y = Y + i * p;
    // the residual r (FP64), lane holds rows lane + 32 u
    double yv[RS_RL], rv[RS_RL];
    double yy = 0.0;
#pragma unroll
    for (int u = 0; u < RS_RL; ++u) {
      const int r = lane + 32 * u;
      yv[u] = r < p ? (double)y[r] : 0.0;
      rv[u] = yv[u];
      yy = fma(yv[u], yv[u], yy);
      if (r < p) ys[r] = y[r];
    }
    yy = warp_sum_d(yy);
    __syncwarp();
    if (A0) {  // FP32 correlations of the coding pass
      for (int j = lane; j < n; j += 32) a0[j] = __ldg(A0 + i * lda + j);
    } else {   // alpha0 = D^T y in FP32, 32-atom tiles of D staged in shared memory
      for (int j0 = 0; j0 < n; j0 += 32) {
        const int na = min(32, n - j0);
#pragma unroll 8
        for (int q = lane; q < na * p; q += 32) Gs[(q / p) * pitch + q % p] = D[(size_t)j0 * p + q];
        __syncwarp();
        if (lane < na) {
          float a = 0.f;
          for (int r = 0; r < p; ++r) a = fmaf(Gs[lane * pitch + r], ys[r], a);
          a0[j0 + lane] = a;
        }
        __syncwarp();
      }
    }
    __syncwarp();
    const double ynorm = sqrt(yy);
    double rr = yy;
    double gsum = 0.0;  // sum |gamma_q|
    int k = 0;
    for (int step = 0; step < s; ++step) {
      // ---- FP32 correlations alpha = alpha0 - G[:, I] gamma (selected: NaN)
      float best = 0.f;
      for (int j = lane; j < n; j += 32) {
        float a = a0[j];
        for (int q = 0; q < k; ++q) a = fmaf(-Gs[(size_t)q * n + j], g32[q], a);
        a = fabsf(a);
        al[j] = a;
        best = fmaxf(best, a);  // NaN ignored
      }
      best = __uint_as_float(__reduce_max_sync(FULL, __float_as_uint(best)));
      __syncwarp();
      if (!(best > 0.f)) break;
      // ---- the exact argmax among the atoms within 2E of the FP32 maximum
      const double E = cerr * dmax * (ynorm + dmax * gsum);
      const float lo = (float)((double)best - 2.0 * E) * (1.f - 0x1p-22f);
      int sel = n;
      double bestv = -1.0;
      for (int j0 = 0; j0 < n; j0 += 32) {
        const int j = j0 + lane;
        unsigned ball = __ballot_sync(FULL, j < n && al[j] >= lo);
        while (ball) {
          const int jc = j0 + __ffs(ball) - 1;
          ball &= ball - 1;
          double a = 0.0;
#pragma unroll
          for (int u = 0; u < RS_RL; ++u) {
            const int r = lane + 32 * u;
            if (r < p) a = fma((double)__ldg(D + (size_t)jc * p + r), rv[u], a);
          }
          a = fabs(warp_sum_d(a));
          if (a > bestv) {  // ascending jc: ties keep the lower index
            bestv = a;
            sel = jc;
          }
        }
      }
      if (sel >= n || !(bestv > 0.0)) break;
      // ---- FP64 Cholesky row: w = L^-1 G[I, sel], delta = G[sel, sel] - w.w
      const float* dsel = D + (size_t)sel * p;
      double ds[RS_RL];
      double gss = 0.0, a0s = 0.0;  // d_sel^T d_sel, d_sel^T y
#pragma unroll
      for (int u = 0; u < RS_RL; ++u) {
        const int r = lane + 32 * u;
        ds[u] = r < p ? (double)__ldg(dsel + r) : 0.0;
        gss = fma(ds[u], ds[u], gss);
        a0s = fma(ds[u], yv[u], a0s);
      }
      gss = warp_sum_d(gss);
      a0s = warp_sum_d(a0s);
      double w = 0.0, wsq = 0.0, wz = 0.0;  // lane q keeps w_q
      for (int q = 0; q < k; ++q) {
        const float* dq = D + (size_t)I[q] * p;
        double g = 0.0;
#pragma unroll
        for (int u = 0; u < RS_RL; ++u) {
          const int r = lane + 32 * u;
          if (r < p) g = fma((double)__ldg(dq + r), ds[u], g);
        }
        double acc = warp_sum_d(g);  // d_{I_q}^T d_sel
        for (int t = 0; t < q; ++t) acc -= L[q][t] * __shfl_sync(FULL, w, t);
        const double wq = acc / L[q][q];
        if (lane == q) w = wq;
        wsq = fma(wq, wq, wsq);
        wz = fma(wq, Z[q], wz);
      }
      const double delta = gss - wsq;
      if (delta <= 1e-12) break;
      const double lkk = sqrt(delta);
      const double zk = (a0s - wz) / lkk;
      __syncwarp();
      if (lane < k) L[k][lane] = w;
      if (lane == 0) {
        L[k][k] = lkk;
        Z[k] = zk;
        I[k] = sel;
        a0[sel] = __int_as_float(0x7fc00000);  // masked from now on
      }
      for (int j = lane; j < n; j += 32) Gs[(size_t)k * n + j] = __ldg(G + (size_t)sel * n + j);
      __syncwarp();
      k = step + 1;
      rr -= zk * zk;
      // ---- gamma = L^-T z and r = y - D_I gamma
      if (lane == 0) {
        for (int q = k - 1; q >= 0; --q) {
          double a = Z[q];
          for (int t = q + 1; t < k; ++t) a -= L[t][q] * Gm[t];
          Gm[q] = a / L[q][q];
        }
      }
      __syncwarp();
      if (lane < k) g32[lane] = (float)Gm[lane];
      gsum = 0.0;
      for (int q = 0; q < k; ++q) gsum += fabs(Gm[q]);
#pragma unroll
      for (int u = 0; u < RS_RL; ++u) {
        const int r = lane + 32 * u;
        double v = yv[u];
        if (r < p) {
#pragma unroll 4
          for (int q = 0; q < k; ++q) v = fma(-(double)__ldg(D + (size_t)I[q] * p + r), Gm[q], v);
        }
        rv[u] = v;
      }
      __syncwarp();
      if (rr <= 1e-14 * yy) break;
    }
    __syncwarp();
    // ---- write the support in ascending atom order with gamma
    if (lane < k) {
      int rank = 0;
      for (int q = 0; q < k; ++q) rank += I[q] < I[lane] ? 1 : 0;
      oidx[i * s + rank] = I[lane];
      oval[i * s + rank] = (float)Gm[lane];
    } else if (lane < s) {
      oidx[i * s + lane] = -1;
      oval[i * s + lane] = 0.f;
    }
    if (lane == 0) ocnt[i] = k;
    __syncwarp();
  }
}

}  // namespace

cudaError_t omp_resolve64(const float* Y, int p, const float* D, const float* G, const float* A0,
                          int64_t lda, int n, int s, const int* list, const int* count, int cap,
                          int32_t* idx, float* val, int32_t* cnt, cudaStream_t st) {
  if (p < 1 || p > RS_PMAX || s < 1 || s > DL_RESOLVE_SMAX) return cudaErrorInvalidValue;
  const size_t grows =
      (size_t)s * n > (size_t)32 * (p | 1) ? (size_t)s * n : (size_t)32 * (p | 1);
  const size_t smem = (grows + 2 * (size_t)n + p) * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(resolve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  resolve_kernel<<<DL_RESOLVE_WARPS, 32, smem, st>>>(Y, p, D, G, A0, lda, n, s, list, count, cap,
                                                     idx, val, cnt);
  return cudaGetLastError();
}

}  // namespace dlk
