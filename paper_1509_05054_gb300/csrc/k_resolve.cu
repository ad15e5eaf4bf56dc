// FP64 re-solve of the signals whose FP32 OMP met a Cholesky pivot below 1e-6.
//
// In FP32 a pivot delta = G_ss - ||w||^2 below ~1e-6 is dominated by rounding,
// so the FP32 kernel stops such a signal and appends it to a list.  Here one
// warp per listed signal redoes its whole OMP (Algorithm 1 step 1) in FP64 from
// D and y: correlations, Gram entries d_j^T d_sel computed on the fly, exact
// argmax with the lowest index on ties, the Gram-Schmidt form of the Cholesky
// update, and the FP64 stop rules (pivot <= 1e-12, residual <= 1e-14 ||y||^2).
// The per-warp vectors live in a global scratch area (the path is rare, so its
// speed is secondary).
#include "dl_internal.cuh"

#include <math.h>

namespace dlk {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int RS_THREADS = 128;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

__global__ void __launch_bounds__(RS_THREADS) resolve_kernel(
    const float* __restrict__ Y, int p, const float* __restrict__ D, int n, int s,
    const int* __restrict__ list, const int* __restrict__ count, int cap, double* __restrict__ scratch,
    int32_t* __restrict__ oidx, float* __restrict__ oval, int32_t* __restrict__ ocnt) {
  __shared__ double Lsh[RS_THREADS / 32][DL_RESOLVE_SMAX][DL_RESOLVE_SMAX];
  __shared__ double Csh[RS_THREADS / 32][DL_RESOLVE_SMAX];
  __shared__ double Zsh[RS_THREADS / 32][DL_RESOLVE_SMAX];
  __shared__ int Ish[RS_THREADS / 32][DL_RESOLVE_SMAX];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int gw = blockIdx.x * (RS_THREADS / 32) + wib;
  const int nwarps = gridDim.x * (RS_THREADS / 32);
  double* alpha = scratch + (size_t)gw * (DL_RESOLVE_SMAX + 1) * n;  // alpha, then u_0..u_{s-2}
  double(&L)[DL_RESOLVE_SMAX][DL_RESOLVE_SMAX] = Lsh[wib];
  double(&C)[DL_RESOLVE_SMAX] = Csh[wib];
  double(&Z)[DL_RESOLVE_SMAX] = Zsh[wib];
  int(&I)[DL_RESOLVE_SMAX] = Ish[wib];
  int total = *count;
  if (total > cap) total = cap;

  for (int e = gw; e < total; e += nwarps) {
    const int64_t i = list[e];
    const float* y = Y + i * p;
    double yy = 0.0;
    for (int r = lane; r < p; r += 32) yy += (double)y[r] * (double)y[r];
    yy = warp_sum_d(yy);
    for (int j = lane; j < n; j += 32) {
      double a = 0.0;
      for (int r = 0; r < p; ++r) a += (double)D[(size_t)j * p + r] * (double)y[r];
      alpha[j] = a;
    }
    __syncwarp();
    double rr = yy;
    int k = 0;
    for (int step = 0; step < s; ++step) {
      // exact argmax |alpha| over unselected atoms (NaN = selected), lowest index on ties
      double bv = -1.0;
      int bj = n;
      for (int j = lane; j < n; j += 32) {
        const double v = fabs(alpha[j]);
        if (v > bv) {
          bv = v;
          bj = j;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(FULL, bv, o);
        const int oj = __shfl_xor_sync(FULL, bj, o);
        if (ov > bv || (ov == bv && oj < bj)) {
          bv = ov;
          bj = oj;
        }
      }
      if (!(bv > 0.0) || bj >= n) break;
      const int sel = bj;
      const float* dsel = D + (size_t)sel * p;
      // w_q = c_q u_q[sel], delta = d_sel.d_sel - ||w||^2
      double gss = 0.0;
      for (int r = lane; r < p; r += 32) gss += (double)dsel[r] * (double)dsel[r];
      gss = warp_sum_d(gss);
      double wsq = 0.0;
      for (int q = 0; q < step; ++q) {
        const double w = C[q] * alpha[(size_t)(q + 1) * n + sel];
        wsq += w * w;
        if (lane == 0) L[step][q] = w;
      }
      const double delta = gss - wsq;
      if (delta <= 1e-12) break;
      const double c = 1.0 / sqrt(delta);
      const double z = alpha[sel] * c;
      __syncwarp();
      if (lane == 0) {
        C[step] = c;
        Z[step] = z;
        I[step] = sel;
        L[step][step] = 1.0 / c;
      }
      __syncwarp();
      // u_step = G[:, sel] - sum_q (w_q c_q) u_q ;  alpha -= z c u_step
      double* ustep = alpha + (size_t)(step + 1) * n;
      for (int j = lane; j < n; j += 32) {
        double g = 0.0;
        const float* dj = D + (size_t)j * p;
        for (int r = 0; r < p; ++r) g += (double)dj[r] * (double)dsel[r];
        for (int q = 0; q < step; ++q) g -= L[step][q] * C[q] * alpha[(size_t)(q + 1) * n + j];
        if (step + 1 < DL_RESOLVE_SMAX) ustep[j] = g;
        alpha[j] = (j == sel) ? __longlong_as_double(0x7ff8000000000000ll) : alpha[j] - z * c * g;
      }
      __syncwarp();
      rr -= z * z;
      k = step + 1;
      if (rr <= 1e-14 * yy) break;
    }
    // back substitution L^T gamma = z, then ascending order
    if (lane == 0) {
      double gam[DL_RESOLVE_SMAX];
      for (int q = k - 1; q >= 0; --q) {
        double a = Z[q];
        for (int r = q + 1; r < k; ++r) a -= L[r][q] * gam[r];
        gam[q] = a / L[q][q];
      }
      for (int a = 1; a < k; ++a) {  // insertion sort by atom
        const int ti = I[a];
        const double tv = gam[a];
        int b = a - 1;
        while (b >= 0 && I[b] > ti) {
          I[b + 1] = I[b];
          gam[b + 1] = gam[b];
          --b;
        }
        I[b + 1] = ti;
        gam[b + 1] = tv;
      }
      for (int t = 0; t < s; ++t) {
        oidx[i * s + t] = t < k ? I[t] : -1;
        oval[i * s + t] = t < k ? (float)gam[t] : 0.f;
      }
      ocnt[i] = k;
    }
    __syncwarp();
  }
}

}  // namespace

cudaError_t omp_resolve64(const float* Y, int p, const float* D, int n, int s, const int* list,
                          const int* count, int cap, double* scratch, int32_t* idx, float* val,
                          int32_t* cnt, cudaStream_t st) {
  resolve_kernel<<<DL_RESOLVE_WARPS / (RS_THREADS / 32), RS_THREADS, 0, st>>>(
      Y, p, D, n, s, list, count, cap, scratch, idx, val, cnt);
  return cudaGetLastError();
}

}  // namespace dlk
