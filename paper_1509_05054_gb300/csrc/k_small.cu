// Whole DL iterations of small problems, one CTA per problem (Algorithm 1 for
// each problem of a batch, all its iterations in one launch).
//
// A batch of many small problems (the dictionary-recovery experiment of
// Section 4.1: p = 20, n = 50, m = 1500, s <= 5, 200 problems per batch) is
// bound by launch and graph-node throughput when each problem runs the
// large-problem kernels.  Here one CTA of 32 warps holds its problem's
// dictionary, Gram matrix and U = E X^T in shared memory and runs every stage
// of every iteration itself:
//   1. G = D^T D (FP32) from the shared-memory atoms;
//   2. OMP, one warp per signal (omp_one, the same Gram-Schmidt Batch-OMP as the
//      large-problem kernels, Gram rows from shared memory); a signal whose
//      Cholesky pivot falls below 1e-6 is redone by the same warp in FP64 with
//      the oracle's stop rules;
//   3. e_i = y_i - D x_i, U = E X^T and r_j = ||x_j||^2 by shared-memory
//      reductions (X_prev for P-NSGK, Eq. 7), ||E||^2 and ||Y||^2;
//   4. the atom update (Eq. 5): d_j' = (U_j + r_j d_j) / ||.||, c_j = d_j^T d_j';
//   5. the row update x' = e^T d' + c x (AK-SVD; SGK and P-NSGK keep X) and
//      ||Y - D'X'||^2;
//   6. the RMSE pair of the iteration, D = D'.
// After the last iteration it writes D and X (CSC).  p <= 32, n <= 64, s <= 8,
// group size n.
#include "dl_internal.cuh"
#include "omp_common.cuh"
#include "omp_one.cuh"

#include <math.h>

namespace dlk {
namespace {

using namespace omp;

constexpr int SM_THREADS = 1024;
constexpr int SM_WARPS = SM_THREADS / 32;

// Gram rows from the problem's Gram matrix in shared memory (row pitch n).
struct GramShared {
  const float* G;
  int n;
  template <int NV>
  __device__ __forceinline__ void row(int sel, int lane, float2 (&out)[NV]) const {
    const float* Gr = G + sel * n;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const int j0 = 64 * v + lane, j1 = j0 + 32;
      out[v].x = j0 < n ? Gr[j0] : 0.f;
      out[v].y = j1 < n ? Gr[j1] : 0.f;
    }
  }
  __device__ __forceinline__ float diag(int sel) const { return G[sel * n + sel]; }
};

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

// Per-warp FP64 scratch of the re-solve.
struct Omp64Scratch {
  double L[kSmallS][kSmallS];
  double Z[kSmallS];
  double Gm[kSmallS];
  int I[kSmallS];
};

// FP64 Batch-OMP of signal i by one warp, with the oracle's decisions and stop
// rules (pivot <= 1e-12, residual energy <= 1e-14 ||y||^2, max |alpha| = 0):
// exact correlations of the FP64 residual each step (lane l: atoms l, l + 32),
// Cholesky row from FP64 dot products of the FP32 atoms, lowest index on ties.
// Lane r holds row r of y and of the residual (p <= 32).
__device__ void omp64_small(const float* Ds, int pitch, int n, int p, int s,
                            const float* __restrict__ y, Omp64Scratch& w64, int64_t i,
                            int32_t* __restrict__ oidx, float* __restrict__ oval,
                            int32_t* __restrict__ ocnt) {
  const int lane = threadIdx.x & 31;
  const double yr = lane < p ? (double)y[lane] : 0.0;
  double rv = yr;
  const double yy = warp_sum_d(yr * yr);
  double rr = yy;
  int k = 0;
  for (int step = 0; step < s; ++step) {
    double a[2] = {0.0, 0.0};
    for (int r = 0; r < p; ++r) {
      const double rb = __shfl_sync(FULL, rv, r);
      if (lane < n) a[0] = fma((double)Ds[lane * pitch + r], rb, a[0]);
      if (lane + 32 < n) a[1] = fma((double)Ds[(lane + 32) * pitch + r], rb, a[1]);
    }
    double bv = -1.0;
    int bi = n;
    for (int h = 0; h < 2; ++h) {
      const int j = lane + 32 * h;
      bool taken = j >= n;
      for (int q = 0; q < k; ++q) taken |= w64.I[q] == j;
      const double v = taken ? -1.0 : fabs(a[h]);
      if (v > bv) {
        bv = v;
        bi = j;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(FULL, bv, o);
      const int oi = __shfl_xor_sync(FULL, bi, o);
      if (ov > bv || (ov == bv && oi < bi)) {
        bv = ov;
        bi = oi;
      }
    }
    if (!(bv > 0.0) || bi >= n) break;
    const int sel = bi;
    double gq = 0.0;  // lane q < k: d_{I_q}^T d_sel
    if (lane < k)
      for (int r = 0; r < p; ++r)
        gq = fma((double)Ds[w64.I[lane] * pitch + r], (double)Ds[sel * pitch + r], gq);
    const double ds = lane < p ? (double)Ds[sel * pitch + lane] : 0.0;
    const double gss = warp_sum_d(ds * ds), a0s = warp_sum_d(ds * yr);
    double wmine = 0.0, wsq = 0.0, wz = 0.0;
    for (int q = 0; q < k; ++q) {
      double acc = __shfl_sync(FULL, gq, q);
      for (int t = 0; t < q; ++t) acc -= w64.L[q][t] * __shfl_sync(FULL, wmine, t);
      const double wq = acc / w64.L[q][q];
      if (lane == q) wmine = wq;
      wsq = fma(wq, wq, wsq);
      wz = fma(wq, w64.Z[q], wz);
    }
    const double delta = gss - wsq;
    if (delta <= 1e-12) break;
    const double lkk = sqrt(delta), zk = (a0s - wz) / lkk;
    __syncwarp();
    if (lane < k) w64.L[k][lane] = wmine;
    if (lane == 0) {
      w64.L[k][k] = lkk;
      w64.Z[k] = zk;
      w64.I[k] = sel;
    }
    __syncwarp();
    k = step + 1;
    rr -= zk * zk;
    if (lane == 0)  // gamma = L^-T z
      for (int q = k - 1; q >= 0; --q) {
        double acc = w64.Z[q];
        for (int t = q + 1; t < k; ++t) acc -= w64.L[t][q] * w64.Gm[t];
        w64.Gm[q] = acc / w64.L[q][q];
      }
    __syncwarp();
    rv = yr;
    if (lane < p)
      for (int q = 0; q < k; ++q) rv = fma(-(double)Ds[w64.I[q] * pitch + lane], w64.Gm[q], rv);
    if (rr <= 1e-14 * yy) break;
  }
  __syncwarp();
  if (lane < k) {  // ascending atom order
    int rank = 0;
    for (int q = 0; q < k; ++q) rank += w64.I[q] < w64.I[lane] ? 1 : 0;
    oidx[i * s + rank] = w64.I[lane];
    oval[i * s + rank] = (float)w64.Gm[lane];
  } else if (lane < s) {
    oidx[i * s + lane] = -1;
    oval[i * s + lane] = 0.f;
  }
  if (lane == 0) ocnt[i] = k;
  __syncwarp();
}

// Block-wide sums of three doubles; valid on thread 0.
__device__ void block_sum3(double& a, double& b, double& c, double (*red)[3]) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  a = warp_sum_d(a);
  b = warp_sum_d(b);
  c = warp_sum_d(c);
  __syncthreads();
  if (lane == 0) {
    red[w][0] = a;
    red[w][1] = b;
    red[w][2] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    a = b = c = 0.0;
    for (int q = 0; q < SM_WARPS; ++q) {
      a += red[q][0];
      b += red[q][1];
      c += red[q][2];
    }
  }
  __syncthreads();
}

// Shared memory of one CTA (floats unless noted); pitch of D rows = p | 1 (odd:
// the lane-per-atom reads of the correlations hit distinct banks).
struct SmallSmem {
  int pitch, n;
  size_t ds, dn, g, u, r, c, a0, lf, cf, w64, total;
  __host__ __device__ SmallSmem(int p_, int n_) : pitch(p_ | 1), n(n_) {
    ds = 0;
    dn = ds + (size_t)n * pitch;
    g = dn + (size_t)n * pitch;
    u = g + (size_t)n * n;
    r = u + (size_t)n * pitch;
    c = r + n;
    a0 = c + n;
    lf = a0 + (size_t)SM_WARPS * kSmallN;
    cf = lf + (size_t)SM_WARPS * kSmallS * kSmallS;
    w64 = (cf + (size_t)SM_WARPS * kSmallS + 1) / 2 * 2;  // 8-byte aligned
    total = w64 * sizeof(float) + (size_t)SM_WARPS * sizeof(Omp64Scratch);
  }
};

__global__ void __launch_bounds__(SM_THREADS) small_dl_kernel(const SmallProblem* __restrict__ probs,
                                                              int iters, int rule,
                                                              int* __restrict__ err) {
  extern __shared__ float smem[];
  __shared__ double red[SM_WARPS][3];
  __shared__ int rs_cnt[SM_WARPS];
  __shared__ int rs_one[SM_WARPS];
  const SmallProblem P = probs[blockIdx.x];
  const int p = P.p, n = P.n, s = P.s;
  const int64_t m = P.m;
  const SmallSmem lay(p, n);
  const int pitch = lay.pitch;
  float* Ds = smem + lay.ds;  // atoms (current)
  float* Dn = smem + lay.dn;  // updated atoms
  float* G = smem + lay.g;
  float* U = smem + lay.u;    // U_j at U + j * pitch, rows r < p
  float* R = smem + lay.r;
  float* Cc = smem + lay.c;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* a0w = smem + lay.a0 + warp * kSmallN;
  float(&Lw)[kSmallS][kSmallS] =
      *(float(*)[kSmallS][kSmallS])(smem + lay.lf + warp * kSmallS * kSmallS);
  float(&Cw)[kSmallS] = *(float(*)[kSmallS])(smem + lay.cf + warp * kSmallS);
  Omp64Scratch& w64 = ((Omp64Scratch*)(smem + lay.w64))[warp];
  const bool nsgk = rule == 2, sgk = rule != 0;

  for (int q = threadIdx.x; q < n * p; q += SM_THREADS) Ds[(q / p) * pitch + q % p] = P.D[q];
  __syncthreads();
  for (int it = 0; it < iters; ++it) {
    // ---- 1. Gram matrix
    for (int q = threadIdx.x; q < n * n; q += SM_THREADS) {
      const int j = q / n, k = q - j * n;
      float a = 0.f;
      for (int r = 0; r < p; ++r) a = fmaf(Ds[j * pitch + r], Ds[k * pitch + r], a);
      G[q] = a;
    }
    for (int q = threadIdx.x; q < n * pitch + n; q += SM_THREADS) U[q] = 0.f;  // U, then R
    __syncthreads();
    // ---- 2. sparse coding, one warp per signal
    const GramShared gsrc{G, n};
    for (int64_t i = warp; i < m; i += SM_WARPS) {
      const float* y = P.Y + i * p;
      const float yv = lane < p ? y[lane] : 0.f;
      float a[2] = {0.f, 0.f};
      for (int r = 0; r < p; ++r) {
        const float yr = __shfl_sync(FULL, yv, r);
        if (lane < n) a[0] = fmaf(Ds[lane * pitch + r], yr, a[0]);
        if (lane + 32 < n) a[1] = fmaf(Ds[(lane + 32) * pitch + r], yr, a[1]);
      }
      a0w[lane] = a[0];
      a0w[lane + 32] = a[1];
      if (lane == 0) rs_cnt[warp] = 0;
      __syncwarp();
      omp_one<2, kSmallS, kSmallS - 1, false, false>(i, gsrc, Lw, Cw, nullptr, a0w, n, y, p, s,
                                                     nullptr, P.sidx, P.sval, P.scnt, nullptr, err,
                                                     &rs_one[warp], &rs_cnt[warp], 1, 0.f);
      __syncwarp();
      if (rs_cnt[warp] > 0)  // a pivot below 1e-6: redo the signal in FP64
        omp64_small(Ds, pitch, n, p, s, y, w64, i, P.sidx, P.sval, P.scnt);
      __syncwarp();
    }
    __syncthreads();
    // ---- 3. errors, U = E X^T and r (X_prev's slots for P-NSGK once there is one)
    const bool prev = nsgk && *P.pvalid != 0;
    const int32_t* aidx = prev ? P.pidx : P.sidx;
    const float* aval = prev ? P.pval : P.sval;
    const int32_t* acnt = prev ? P.pcnt : P.scnt;
    double ee = 0.0, yy = 0.0, e2 = 0.0;
    for (int64_t i = warp; i < m; i += SM_WARPS) {
      const float yv = lane < p ? P.Y[i * p + lane] : 0.f;
      const int c = P.scnt[i];
      const int jt = lane < c ? P.sidx[i * s + lane] : 0;
      const float xt = lane < c ? P.sval[i * s + lane] : 0.f;
      float e = yv;
      for (int t = 0; t < c; ++t) {
        const int j = __shfl_sync(FULL, jt, t);
        const float x = __shfl_sync(FULL, xt, t);
        if (lane < p) e = fmaf(-x, Ds[j * pitch + lane], e);
      }
      ee += (double)(e * e);
      yy += (double)(yv * yv);
      const int ca = acnt[i];
      const int ja = lane < ca ? aidx[i * s + lane] : 0;
      const float xa = lane < ca ? aval[i * s + lane] : 0.f;
      for (int t = 0; t < ca; ++t) {
        const int j = __shfl_sync(FULL, ja, t);
        const float x = __shfl_sync(FULL, xa, t);
        if (lane < p) atomicAdd(&U[j * pitch + lane], x * e);
        if (lane == 0) atomicAdd(&R[j], x * x);
      }
    }
    __syncthreads();
    // ---- 4. atom update, one warp per atom
    for (int j = warp; j < n; j += SM_WARPS) {
      const float d = lane < p ? Ds[j * pitch + lane] : 0.f;
      const float v = lane < p ? fmaf(R[j], d, U[j * pitch + lane]) : 0.f;
      const float vv = warp_sum(v * v);
      if (vv > 0.f) {
        const float dn = v * (1.0f / sqrtf(vv));
        const float cj = warp_sum(d * dn);
        if (lane < p) Dn[j * pitch + lane] = dn;
        if (lane == 0) Cc[j] = cj;
      } else {  // unused atom (or F x^T = 0): kept
        if (lane < p) Dn[j * pitch + lane] = d;
        if (lane == 0) Cc[j] = 1.f;
      }
    }
    __syncthreads();
    // ---- 5. row update and the error with the updated atoms
    for (int64_t i = warp; i < m; i += SM_WARPS) {
      const float yv = lane < p ? P.Y[i * p + lane] : 0.f;
      const int c = P.scnt[i];
      const int jt = lane < c ? P.sidx[i * s + lane] : 0;
      const float xt = lane < c ? P.sval[i * s + lane] : 0.f;
      float e = yv;
      for (int t = 0; t < c; ++t) {
        const int j = __shfl_sync(FULL, jt, t);
        const float x = __shfl_sync(FULL, xt, t);
        if (lane < p) e = fmaf(-x, Ds[j * pitch + lane], e);
      }
      float r2 = yv, xnew = xt;
      for (int t = 0; t < c; ++t) {
        const int j = __shfl_sync(FULL, jt, t);
        const float x = __shfl_sync(FULL, xt, t);
        const float dn = lane < p ? Dn[j * pitch + lane] : 0.f;
        const float xn = sgk ? x : fmaf(Cc[j], x, warp_sum(e * dn));
        if (lane == t) xnew = xn;
        r2 = fmaf(-xn, dn, r2);
      }
      if (lane < p) e2 += (double)(r2 * r2);
      if (lane < c) P.sval[i * s + lane] = xnew;
    }
    block_sum3(ee, yy, e2, red);
    if (threadIdx.x == 0) {
      P.rmse[2 * it] = yy > 0.0 ? sqrt(ee / yy) : 0.0;
      P.rmse[2 * it + 1] = yy > 0.0 ? sqrt(e2 / yy) : 0.0;
      if (!isfinite(ee) || !isfinite(yy)) atomicOr(err, ERR_NONFINITE);
    }
    // ---- 6. D = D'; this X becomes P-NSGK's previous representation
    for (int q = threadIdx.x; q < n * pitch; q += SM_THREADS) Ds[q] = Dn[q];
    if (nsgk) {
      for (int64_t q = threadIdx.x; q < m * s; q += SM_THREADS) {
        P.pidx[q] = P.sidx[q];
        P.pval[q] = P.sval[q];
      }
      for (int64_t q = threadIdx.x; q < m; q += SM_THREADS) P.pcnt[q] = P.scnt[q];
      __syncthreads();
      if (threadIdx.x == 0) *P.pvalid = 1;
    }
    __syncthreads();
  }

  // ---- the final D and X (CSC: colptr = exclusive scan of the counts)
  for (int q = threadIdx.x; q < n * p; q += SM_THREADS) P.D[q] = Ds[(q / p) * pitch + q % p];
  __shared__ int64_t wsum[SM_WARPS];
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < m; base += SM_THREADS) {
    const int64_t i = base + threadIdx.x;
    const int64_t v = i < m ? P.scnt[i] : 0;
    int64_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t t = __shfl_up_sync(FULL, inc, o);
      if (lane >= o) inc += t;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
      int64_t x = wsum[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t t = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += t;
      }
      wsum[lane] = x;
    }
    __syncthreads();
    const int64_t start = carry + (warp > 0 ? wsum[warp - 1] : 0) + inc - v;
    if (i < m) {
      P.colptr[i] = start;
      for (int t = 0; t < (int)v; ++t) {
        P.rowidx[start + t] = P.sidx[i * s + t];
        P.cval[start + t] = P.sval[i * s + t];
      }
    }
    __syncthreads();
    if (threadIdx.x == SM_THREADS - 1) carry = start + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) P.colptr[m] = carry;
}

}  // namespace

bool small_supported(int p, int n, int s) {
  return p >= 1 && p <= kSmallP && n >= 1 && n <= kSmallN && s >= 1 && s <= kSmallS && s <= n;
}

cudaError_t small_dl(const SmallProblem* probs, int count, int iters, int rule, int* err,
                     cudaStream_t st) {
  if (count <= 0 || iters <= 0) return cudaSuccess;
  const size_t smem = SmallSmem(kSmallP, kSmallN).total;  // the largest layout
  cudaError_t e = cudaFuncSetAttribute(small_dl_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  small_dl_kernel<<<count, SM_THREADS, smem, st>>>(probs, iters, rule, err);
  return cudaGetLastError();
}

}  // namespace dlk
