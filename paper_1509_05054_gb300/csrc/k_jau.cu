// Jacobi atom update in the AK-SVD form with full parallelism (PAK-SVD,
// group size n; Section 3, Eq. 3 and Eq. 5; Algorithm 2 with step 4 replaced
// by Eq. 5).  With E = Y - D X formed once:
//   F_j x_j^T = E_{I_j} x_{j,I_j}^T + ||x_{j,I_j}||^2 d_j  =  U_j + r_j d_j
//   d_j'      = (U_j + r_j d_j) / ||U_j + r_j d_j||
//   x_{j,i}'  = F^T d_j' = e_i^T d_j' + (d_j^T d_j') x_{j,i}      for i in I_j
// U = E X^T (p x n) and r_j = ||x_j||^2 are accumulated signal by signal (the
// support sets I_j are never materialised), then every atom is updated by one
// warp, then every signal recomputes its error and its coefficients.
//
// The passes over the signals give each signal eight lanes (four signals per
// warp).  With p % 4 == 0 and 16-byte aligned Y and D they move float4 rows
// and pass A adds x e_i into 16 copies of U with vector reductions in L2
// (red.v4.f32); otherwise pass A keeps per-CTA copies of U (shared memory when
// they fit).  The copies are summed in a fixed order.  The energy partial sums are reduced in a
// fixed order.
#include "dl_internal.cuh"

#include <math.h>

namespace dlk {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int ACC_THREADS = 1024;
constexpr int ROW_THREADS = 256;
constexpr int ACC4_THREADS = 256;
constexpr int kMaxAtoms = 1024;  // largest n the library accepts

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

// Block-wide sum of a double; result valid on thread 0.
__device__ double block_sum_d(double v, double* scratch) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum_d(v);
  __syncthreads();
  if (lane == 0) scratch[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int q = 0; q < nw; ++q) r += scratch[q];
  return r;
}

// Pass A: e_i = y_i - D x_i; U[:, j] += x_{j,i} e_i; r_j += x_{j,i}^2;
// partial ||E||^2 and ||Y||^2.  Eight lanes per signal (four signals per warp):
// lane g of group q holds rows g + 8((t + q) mod RL), t < RL (p <= 8*RL); the
// rotation by q puts the four groups' shared-memory atomics on distinct banks.
// Support slots t and t + 8 live on group lane t % 8.
template <int RL, bool SMEM>
__global__ void __launch_bounds__(ACC_THREADS, 1) accum_kernel(
    const float* __restrict__ Y, int p, int64_t m, const float* __restrict__ D, int n, int s,
    const int32_t* __restrict__ idx, const float* __restrict__ val, const int32_t* __restrict__ cnt,
    float* __restrict__ Upart, double* __restrict__ epart, int* __restrict__ err) {
  extern __shared__ float sh[];
  __shared__ double red[ACC_THREADS / 32];
  const int lane = threadIdx.x & 31;
  const int g = lane & 7, gbase = lane & ~7;
  const int q = (threadIdx.x >> 3) & 3;
  int row[RL];
#pragma unroll
  for (int t = 0; t < RL; ++t) row[t] = g + 8 * ((t + q) % RL);
  const int np = n * p;
  float* U = SMEM ? sh : Upart;  // atom-major: U[j*p + r]; then r_j at U[np + j]
  if (SMEM) {
    for (int q = threadIdx.x; q < np + n; q += blockDim.x) U[q] = 0.f;
    __syncthreads();
  }
  float ee = 0.f, yy = 0.f;
  const int64_t groups = (int64_t)gridDim.x * (blockDim.x >> 3);
  const int64_t g0 = (int64_t)blockIdx.x * (blockDim.x >> 3) + (threadIdx.x >> 3);
  // every lane of a warp loops the same number of times (shuffles stay converged)
  const int64_t trips = (m + groups - 1) / groups;
  for (int64_t k = 0; k < trips; ++k) {
    const int64_t i = g0 + k * groups;
    const bool live = i < m;
    float e[RL];
#pragma unroll
    for (int t = 0; t < RL; ++t) {
      const int r = row[t];
      e[t] = (live && r < p) ? Y[i * p + r] : 0.f;
      yy = fmaf(e[t], e[t], yy);
    }
    const int c = live ? cnt[i] : 0;
    const int j0 = (g < c) ? idx[i * s + g] : 0;
    const float x0 = (g < c) ? val[i * s + g] : 0.f;
    const int j1 = (g + 8 < c) ? idx[i * s + g + 8] : 0;
    const float x1 = (g + 8 < c) ? val[i * s + g + 8] : 0.f;
    const int cmax = __reduce_max_sync(0xffffffffu, (unsigned)c);
    for (int t = 0; t < cmax; ++t) {
      const int jj = __shfl_sync(0xffffffffu, t < 8 ? j0 : j1, gbase + (t & 7));
      const float xx = __shfl_sync(0xffffffffu, t < 8 ? x0 : x1, gbase + (t & 7));
      if (t < c) {
#pragma unroll
        for (int u = 0; u < RL; ++u) {
          const int r = row[u];
          if (r < p) e[u] = fmaf(-xx, __ldg(D + (size_t)jj * p + r), e[u]);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < RL; ++u) ee = fmaf(e[u], e[u], ee);
    for (int t = 0; t < cmax; ++t) {
      const int jj = __shfl_sync(0xffffffffu, t < 8 ? j0 : j1, gbase + (t & 7));
      const float xx = __shfl_sync(0xffffffffu, t < 8 ? x0 : x1, gbase + (t & 7));
      if (t < c) {
#pragma unroll
        for (int u = 0; u < RL; ++u) {
          const int r = row[u];
          if (r < p) atomicAdd(&U[(size_t)jj * p + r], xx * e[u]);
        }
        if (g == 0) atomicAdd(&U[np + jj], xx * xx);
      }
    }
  }
  if (!isfinite(ee) || !isfinite(yy)) atomicOr(err, ERR_NONFINITE);
  if (SMEM) {
    __syncthreads();
    float* out = Upart + (size_t)blockIdx.x * (np + n);
    for (int q = threadIdx.x; q < np + n; q += blockDim.x) out[q] = U[q];
  }
  const double see = block_sum_d((double)ee, red);
  const double syy = block_sum_d((double)yy, red);
  if (threadIdx.x == 0) {
    epart[2 * blockIdx.x] = see;
    epart[2 * blockIdx.x + 1] = syy;
  }
}

// ---- float4 forms (p % 4 == 0, Y and D 16-byte aligned) ----
// Eight lanes per signal; lane g holds the float4 vectors v = g + 8k (rows
// 4v..4v+3), k < RV, p <= 32 RV.  The support loops are unrolled to SMAX.

__device__ __forceinline__ void red_add_v4(float* addr, float4 v) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(v.x), "f"(v.y),
               "f"(v.z), "f"(v.w)
               : "memory");
}
__device__ __forceinline__ float4 f4_fma(float a, float4 b, float4 c) {
  return make_float4(fmaf(a, b.x, c.x), fmaf(a, b.y, c.y), fmaf(a, b.z, c.z), fmaf(a, b.w, c.w));
}
__device__ __forceinline__ float f4_dot(float4 a, float4 b, float acc) {
  return fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, fmaf(a.w, b.w, acc))));
}

// Pass A, float4 form: CTA b adds x_{j,i} e_i into copy b mod kUCopies of U
// (zeroed, p x n atom-major, then r at + n p) by vector reductions in L2
// (native FP32 adds); r_j is summed per CTA in shared memory and added once per
// CTA.  Spreading the reductions over several copies keeps the L2 lines of
// frequently used atoms from serialising them; the copies are then summed in a
// fixed order.
// NS (P-NSGK, Eq. 7): the error is that of Z = Y + D0 Xp - D0 X against the
// current atoms and the previous representations Xp, e = y - D0 x + (D0 - D) xp
// (D0: the dictionary the iteration started from; equal to D before any group
// has moved), and U, r are accumulated over Xp's supports and values.  *pvalid
// == 0 means there are no previous representations yet: Xp = X.
template <int RV, int SMAX, bool NS>
__global__ void __launch_bounds__(ACC4_THREADS, 4) accum4_kernel(
    const float* __restrict__ Y, int p, int64_t m, const float* __restrict__ D, int n, int s,
    const int32_t* __restrict__ idx, const float* __restrict__ val, const int32_t* __restrict__ cnt,
    float* __restrict__ U, double* __restrict__ epart, int* __restrict__ err, int a0, int a1,
    int energies, const float* __restrict__ D0, const int32_t* __restrict__ pidx,
    const float* __restrict__ pval, const int32_t* __restrict__ pcnt,
    const int* __restrict__ pvalid, int moved) {
  __shared__ float rsh[kMaxAtoms];
  __shared__ double red[ACC4_THREADS / 32];
  for (int j = threadIdx.x; j < n; j += blockDim.x) rsh[j] = 0.f;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int g = lane & 7, gbase = lane & ~7;
  const int pv = p >> 2;
  const float4* __restrict__ Y4 = (const float4*)Y;
  const float4* __restrict__ D4 = (const float4*)(NS ? D0 : D);
  const float4* __restrict__ Dc4 = (const float4*)D;
  const bool have_prev = NS && *pvalid != 0;
  const int32_t* __restrict__ sidx = have_prev ? pidx : idx;
  const float* __restrict__ sval = have_prev ? pval : val;
  const int32_t* __restrict__ scnt = have_prev ? pcnt : cnt;
  float* __restrict__ Uc = U + (size_t)(blockIdx.x % kUCopies) * jau_ulen(p, n);
  float ee = 0.f, yy = 0.f;
  const int64_t groups = (int64_t)gridDim.x * (blockDim.x >> 3);
  const int64_t g0 = (int64_t)blockIdx.x * (blockDim.x >> 3) + (threadIdx.x >> 3);
  const int64_t trips = (m + groups - 1) / groups;
  for (int64_t k = 0; k < trips; ++k) {
    const int64_t i = g0 + k * groups;
    const bool live = i < m;
    float4 e[RV];
#pragma unroll
    for (int q = 0; q < RV; ++q) {
      const int v = g + 8 * q;
      e[q] = (live && v < pv) ? Y4[i * pv + v] : make_float4(0.f, 0.f, 0.f, 0.f);
      yy = f4_dot(e[q], e[q], yy);
    }
    const int c = live ? cnt[i] : 0;
    const int j0 = (g < c) ? idx[i * s + g] : 0;
    const float x0 = (g < c) ? val[i * s + g] : 0.f;
    const int j1 = (SMAX > 8 && g + 8 < c) ? idx[i * s + g + 8] : 0;
    const float x1 = (SMAX > 8 && g + 8 < c) ? val[i * s + g + 8] : 0.f;
    const int cmax = __reduce_max_sync(FULL, (unsigned)c);
#pragma unroll
    for (int t = 0; t < SMAX; ++t) {
      if (t >= cmax) break;
      const int jj = __shfl_sync(FULL, t < 8 ? j0 : j1, gbase + (t & 7));
      const float xx = __shfl_sync(FULL, t < 8 ? x0 : x1, gbase + (t & 7));
      if (t < c) {
#pragma unroll
        for (int q = 0; q < RV; ++q) {
          const int v = g + 8 * q;
          if (v < pv) e[q] = f4_fma(-xx, __ldg(D4 + (size_t)jj * pv + v), e[q]);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < RV; ++q) ee = f4_dot(e[q], e[q], ee);
    // the slots whose contributions are accumulated: X, or Xp for P-NSGK
    int sc = c, sj0 = j0, sj1 = j1, scmax = cmax;
    float sx0 = x0, sx1 = x1;
    if (NS) {
      sc = live ? scnt[i] : 0;
      sj0 = (g < sc) ? sidx[i * s + g] : 0;
      sx0 = (g < sc) ? sval[i * s + g] : 0.f;
      sj1 = (SMAX > 8 && g + 8 < sc) ? sidx[i * s + g + 8] : 0;
      sx1 = (SMAX > 8 && g + 8 < sc) ? sval[i * s + g + 8] : 0.f;
      scmax = __reduce_max_sync(FULL, (unsigned)sc);
      if (moved) {  // e += (D0 - D) xp for the atoms earlier groups have moved
#pragma unroll
        for (int t = 0; t < SMAX; ++t) {
          if (t >= scmax) break;
          const int jj = __shfl_sync(FULL, t < 8 ? sj0 : sj1, gbase + (t & 7));
          const float xx = __shfl_sync(FULL, t < 8 ? sx0 : sx1, gbase + (t & 7));
          if (t < sc) {
#pragma unroll
            for (int q = 0; q < RV; ++q) {
              const int v = g + 8 * q;
              if (v < pv) {
                e[q] = f4_fma(xx, __ldg(D4 + (size_t)jj * pv + v), e[q]);
                e[q] = f4_fma(-xx, __ldg(Dc4 + (size_t)jj * pv + v), e[q]);
              }
            }
          }
        }
      }
    }
#pragma unroll
    for (int t = 0; t < SMAX; ++t) {
      if (t >= scmax) break;
      const int jj = __shfl_sync(FULL, t < 8 ? sj0 : sj1, gbase + (t & 7));
      const float xx = __shfl_sync(FULL, t < 8 ? sx0 : sx1, gbase + (t & 7));
      if (t < sc && jj >= a0 && jj < a1) {
#pragma unroll
        for (int q = 0; q < RV; ++q) {
          const int v = g + 8 * q;
          if (v < pv)
            red_add_v4(Uc + ((size_t)jj * pv + v) * 4,
                       make_float4(xx * e[q].x, xx * e[q].y, xx * e[q].z, xx * e[q].w));
        }
        if (g == 0) atomicAdd(&rsh[jj], xx * xx);
      }
    }
  }
  if (!isfinite(ee) || !isfinite(yy)) atomicOr(err, ERR_NONFINITE);
  __syncthreads();
  const size_t np = (size_t)n * p;
  for (int j = threadIdx.x; j < n; j += blockDim.x)
    if (rsh[j] != 0.f) atomicAdd(Uc + np + j, rsh[j]);
  const double see = block_sum_d((double)ee, red);
  const double syy = block_sum_d((double)yy, red);
  if (threadIdx.x == 0 && energies) {
    epart[2 * blockIdx.x] = see;
    epart[2 * blockIdx.x + 1] = syy;
  }
}

// ---- Pass A, deterministic form ---------------------------------------------
// U_j = sum_{i in I_j} x_{j,i} e_i and r_j = sum x_{j,i}^2 summed in an order
// fixed by the signal and slot indices, so that every run gives the same bits
// (float4 rows, p <= 128, n <= 1024, s <= 16).  CTA b owns a contiguous range
// of signals (at most DET_R):
//   1. eight lanes per signal form e_i into shared memory (as accum4_kernel),
//      and the (atom, x) pair of every accumulated slot, numbered k = signal x
//      s + slot within the range; counts per atom;
//   2. the pairs are bucketed by atom (exclusive scan of the counts, then
//      positions inside each bucket from shared-memory counters);
//   3. each bucket is put in ascending k order (ranks by comparison, one warp
//      per bucket), which fixes the order whatever the counters handed out;
//   4. one warp per atom sums x e_i and x^2 over its bucket in that order and
//      writes the range's U_j and r_j as slice b (zeros for atoms the range
//      does not use).
// The slices are then summed in slice order (reduce4_kernel).
constexpr int DET_THREADS = 1024;

int det_range(int p, int n, int s) {  // signals per CTA within 200 KB of shared memory
  const size_t per = sizeof(float) * (size_t)p + (size_t)s * (4 + 4 + 4 + 4);
  const size_t fixed = sizeof(int) * (3 * (size_t)n + 1) + 64;
  const size_t cap = 200u * 1024u;
  return fixed >= cap ? 0 : (int)((cap - fixed) / per);
}
size_t det_smem_bytes(int p, int n, int s, int R) {
  return sizeof(float) * (size_t)R * p + (size_t)R * s * (4 + 4 + 4 + 4) +
         sizeof(int) * (3 * (size_t)n + 1) + 64;
}

template <int RV, int SMAX, bool NS>
__global__ void __launch_bounds__(DET_THREADS, 1) accum_det_kernel(
    const float* __restrict__ Y, int p, int64_t m, int64_t R, const float* __restrict__ D, int n,
    int s, const int32_t* __restrict__ idx, const float* __restrict__ val,
    const int32_t* __restrict__ cnt, float* __restrict__ Upart, size_t len,
    double* __restrict__ epart, int* __restrict__ err, int a0, int a1, int energies,
    const float* __restrict__ D0, const int32_t* __restrict__ pidx, const float* __restrict__ pval,
    const int32_t* __restrict__ pcnt, const int* __restrict__ pvalid, int moved) {
  extern __shared__ float dsh[];
  __shared__ double red[DET_THREADS / 32];
  const int64_t lo = (int64_t)blockIdx.x * R;
  const int64_t hi = lo + R < m ? lo + R : m;
  const int nr = (int)(hi > lo ? hi - lo : 0);  // signals of this range
  const int npair = nr * s;
  float* Es = dsh;                                   // [R][p]
  int* pa = (int*)(Es + (size_t)R * p);              // [R s] atom of pair k (-1: none)
  float* px = (float*)(pa + (size_t)R * s);          // [R s] x of pair k
  int* bk = (int*)(px + (size_t)R * s);              // [R s] bucketed: k
  float* bx = (float*)(bk + (size_t)R * s);          // [R s] bucketed: x
  int* cntA = (int*)(bx + (size_t)R * s);            // [n] pairs per atom
  int* off = cntA + n;                               // [n + 1] bucket starts
  int* fill = off + n + 1;                           // [n]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane & 7, gbase = lane & ~7;
  const int pv = p >> 2;
  for (int a = threadIdx.x; a < n; a += DET_THREADS) {
    cntA[a] = 0;
    fill[a] = 0;
  }
  __syncthreads();
  const float4* __restrict__ Y4 = (const float4*)Y;
  const float4* __restrict__ D4 = (const float4*)(NS ? D0 : D);
  const float4* __restrict__ Dc4 = (const float4*)D;
  const bool have_prev = NS && *pvalid != 0;
  const int32_t* __restrict__ sidx = have_prev ? pidx : idx;
  const float* __restrict__ sval = have_prev ? pval : val;
  const int32_t* __restrict__ scnt = have_prev ? pcnt : cnt;
  float ee = 0.f, yy = 0.f;
  // ---- 1. errors and pairs
  for (int sl = threadIdx.x >> 3; sl < ((nr + 3) & ~3); sl += DET_THREADS / 8) {
    const int64_t i = lo + sl;
    const bool live = sl < nr;
    float4 e[RV];
#pragma unroll
    for (int q = 0; q < RV; ++q) {
      const int v = g + 8 * q;
      e[q] = (live && v < pv) ? Y4[i * pv + v] : make_float4(0.f, 0.f, 0.f, 0.f);
      yy = f4_dot(e[q], e[q], yy);
    }
    const int c = live ? cnt[i] : 0;
    const int j0 = (g < c) ? idx[i * s + g] : 0;
    const float x0 = (g < c) ? val[i * s + g] : 0.f;
    const int j1 = (SMAX > 8 && g + 8 < c) ? idx[i * s + g + 8] : 0;
    const float x1 = (SMAX > 8 && g + 8 < c) ? val[i * s + g + 8] : 0.f;
    const int cmax = __reduce_max_sync(FULL, (unsigned)c);
#pragma unroll
    for (int t = 0; t < SMAX; ++t) {
      if (t >= cmax) break;
      const int jj = __shfl_sync(FULL, t < 8 ? j0 : j1, gbase + (t & 7));
      const float xx = __shfl_sync(FULL, t < 8 ? x0 : x1, gbase + (t & 7));
      if (t < c) {
#pragma unroll
        for (int q = 0; q < RV; ++q) {
          const int v = g + 8 * q;
          if (v < pv) e[q] = f4_fma(-xx, __ldg(D4 + (size_t)jj * pv + v), e[q]);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < RV; ++q) ee = f4_dot(e[q], e[q], ee);
    int sc = c, sj0 = j0, sj1 = j1;
    float sx0 = x0, sx1 = x1;
    if (NS) {
      sc = live ? scnt[i] : 0;
      sj0 = (g < sc) ? sidx[i * s + g] : 0;
      sx0 = (g < sc) ? sval[i * s + g] : 0.f;
      sj1 = (SMAX > 8 && g + 8 < sc) ? sidx[i * s + g + 8] : 0;
      sx1 = (SMAX > 8 && g + 8 < sc) ? sval[i * s + g + 8] : 0.f;
      const int scmax = __reduce_max_sync(FULL, (unsigned)sc);
      if (moved) {  // e += (D0 - D) xp for the atoms earlier groups have moved
#pragma unroll
        for (int t = 0; t < SMAX; ++t) {
          if (t >= scmax) break;
          const int jj = __shfl_sync(FULL, t < 8 ? sj0 : sj1, gbase + (t & 7));
          const float xx = __shfl_sync(FULL, t < 8 ? sx0 : sx1, gbase + (t & 7));
          if (t < sc) {
#pragma unroll
            for (int q = 0; q < RV; ++q) {
              const int v = g + 8 * q;
              if (v < pv) {
                e[q] = f4_fma(xx, __ldg(D4 + (size_t)jj * pv + v), e[q]);
                e[q] = f4_fma(-xx, __ldg(Dc4 + (size_t)jj * pv + v), e[q]);
              }
            }
          }
        }
      }
    }
    if (live) {
#pragma unroll
      for (int q = 0; q < RV; ++q) {
        const int v = g + 8 * q;
        if (v < pv) *(float4*)(Es + (size_t)sl * p + 4 * v) = e[q];
      }
      if (g < s) {
        const bool ok = g < sc && sj0 >= a0 && sj0 < a1;
        pa[sl * s + g] = ok ? sj0 : -1;
        px[sl * s + g] = sx0;
        if (ok) atomicAdd(&cntA[sj0], 1);
      }
      if (SMAX > 8 && g + 8 < s) {
        const bool ok = g + 8 < sc && sj1 >= a0 && sj1 < a1;
        pa[sl * s + g + 8] = ok ? sj1 : -1;
        px[sl * s + g + 8] = sx1;
        if (ok) atomicAdd(&cntA[sj1], 1);
      }
    }
  }
  if (!isfinite(ee) || !isfinite(yy)) atomicOr(err, ERR_NONFINITE);
  __syncthreads();
  // ---- 2. buckets: exclusive scan of the counts (n <= 1024), then positions
  {
    const int a = threadIdx.x;
    const int v = a < n ? cntA[a] : 0;
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(FULL, inc, o);
      if (lane >= o) inc += t;
    }
    __shared__ int wsum[32];
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
      int x = wsum[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += t;
      }
      wsum[lane] = x;
    }
    __syncthreads();
    const int ex = (warp > 0 ? wsum[warp - 1] : 0) + inc - v;
    if (a < n) off[a] = ex;
    if (a == n - 1) off[n] = ex + v;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < npair; k += DET_THREADS) {
    const int a = pa[k];
    if (a >= 0) {
      const int pos = off[a] + atomicAdd(&fill[a], 1);
      bk[pos] = k;
      bx[pos] = px[k];
    }
  }
  __syncthreads();
  // ---- 3. and 4. one warp per atom: order the bucket by k, then sum over it
  float* out = Upart + (size_t)blockIdx.x * len;
  const size_t np = (size_t)n * p;
  for (int a = warp; a < n; a += DET_THREADS / 32) {
    const int b0 = off[a], L = off[a + 1] - b0;
    for (int q0 = 0; q0 < L; q0 += 32) {  // rank of each pair by k among the bucket's pairs
      const int q = q0 + lane;
      const int kq = q < L ? bk[b0 + q] : 0x7fffffff;
      const float xq = q < L ? bx[b0 + q] : 0.f;
      int rank = 0;
      for (int r0 = 0; r0 < L; r0 += 32) {
        const int kr = r0 + lane < L ? bk[b0 + r0 + lane] : 0x7fffffff;
#pragma unroll 8
        for (int j = 0; j < 32; ++j) rank += __shfl_sync(FULL, kr, j) < kq ? 1 : 0;
      }
      __syncwarp();
      if (q < L) {  // park at the final position in the pair arrays (free after step 2)
        pa[b0 + rank] = kq;
        px[b0 + rank] = xq;
      }
      __syncwarp();
    }
    __syncwarp();
    constexpr int RU = RV;  // rows lane + 32 u of U_j, u < ceil(p / 32) <= RV
    float ac[RU];
#pragma unroll
    for (int u = 0; u < RU; ++u) ac[u] = 0.f;
    float rx = 0.f;
    for (int q = 0; q < L; ++q) {
      const int k = pa[b0 + q];
      const float xx = px[b0 + q];
      const float* er = Es + (size_t)(k / s) * p;
#pragma unroll
      for (int u = 0; u < RU; ++u) {
        const int r = lane + 32 * u;
        if (r < p) ac[u] = fmaf(xx, er[r], ac[u]);
      }
      rx = fmaf(xx, xx, rx);
    }
#pragma unroll
    for (int u = 0; u < RU; ++u) {
      const int r = lane + 32 * u;
      if (r < p) out[(size_t)a * p + r] = ac[u];
    }
    if (lane == 0) out[np + a] = rx;
  }
  for (size_t q = np + n + threadIdx.x; q < len; q += DET_THREADS) out[q] = 0.f;
  const double see = block_sum_d((double)ee, red);
  const double syy = block_sum_d((double)yy, red);
  if (threadIdx.x == 0 && energies) {
    epart[2 * blockIdx.x] = see;
    epart[2 * blockIdx.x + 1] = syy;
  }
}

// Pass B, float4 form: e = y - D x; x_t' = e.d'_{j_t} + c_{j_t} x_t for all t
// (independent dot products), then y - D' x'.  GROUP: only slots whose atom is
// in [a0, a1) are updated; the others keep x_t and their current atom in the
// residual.  sgk: the coefficients stay (x' = x; SGK rule, Eq. 6).
template <int RV, int SMAX, bool GROUP>
__global__ void __launch_bounds__(ROW_THREADS, 4) rows4_kernel(
    const float* __restrict__ Y, int p, int64_t m, const float* __restrict__ D,
    const float* __restrict__ Dn, const float* __restrict__ C, int s,
    const int32_t* __restrict__ idx, float* __restrict__ val, const int32_t* __restrict__ cnt,
    const int64_t* __restrict__ colptr, int32_t* __restrict__ csc_rowidx,
    float* __restrict__ csc_val, double* __restrict__ epart, int a0, int a1, int sgk) {
  __shared__ double red[ROW_THREADS / 32];
  const int lane = threadIdx.x & 31;
  const int g = lane & 7, gbase = lane & ~7;
  const int pv = p >> 2;
  const float4* __restrict__ Y4 = (const float4*)Y;
  const float4* __restrict__ D4 = (const float4*)D;
  const float4* __restrict__ N4 = (const float4*)Dn;
  (void)a0;
  (void)a1;
  float e2 = 0.f;
  const int64_t groups = (int64_t)gridDim.x * (blockDim.x >> 3);
  const int64_t g0 = (int64_t)blockIdx.x * (blockDim.x >> 3) + (threadIdx.x >> 3);
  const int64_t trips = (m + groups - 1) / groups;
  for (int64_t k = 0; k < trips; ++k) {
    const int64_t i = g0 + k * groups;
    const bool live = i < m;
    {  // warm L2 with the next trip's signal: its samples, slots, count and column start
      const int64_t inx = i + groups;
      if (inx < m) {
        const char* a = nullptr;
        if (g < 2 * RV && 128 * g < 4 * p) a = (const char*)(Y + inx * p) + 128 * g;
        else if (g == 6) a = (const char*)(idx + inx * s);
        else if (g == 7) a = (const char*)(val + inx * s);
        if (a) asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
      }
    }
    float4 y[RV], e[RV];
#pragma unroll
    for (int q = 0; q < RV; ++q) {
      const int v = g + 8 * q;
      y[q] = (live && v < pv) ? Y4[i * pv + v] : make_float4(0.f, 0.f, 0.f, 0.f);
      e[q] = y[q];
    }
    const int c = live ? cnt[i] : 0;
    const int j0 = (g < c) ? idx[i * s + g] : 0;
    const float x0 = (g < c) ? val[i * s + g] : 0.f;
    const int j1 = (SMAX > 8 && g + 8 < c) ? idx[i * s + g + 8] : 0;
    const float x1 = (SMAX > 8 && g + 8 < c) ? val[i * s + g + 8] : 0.f;
    const int cmax = __reduce_max_sync(FULL, (unsigned)c);
#pragma unroll
    for (int t = 0; t < SMAX; ++t) {
      if (t >= cmax) break;
      const int jj = __shfl_sync(FULL, t < 8 ? j0 : j1, gbase + (t & 7));
      const float xx = __shfl_sync(FULL, t < 8 ? x0 : x1, gbase + (t & 7));
      if (t < c) {
        const bool other = GROUP && (jj < a0 || jj >= a1);  // stays: also in the final residual
#pragma unroll
        for (int q = 0; q < RV; ++q) {
          const int v = g + 8 * q;
          if (v < pv) {
            const float4 d = __ldg(D4 + (size_t)jj * pv + v);
            e[q] = f4_fma(-xx, d, e[q]);
            if (other) y[q] = f4_fma(-xx, d, y[q]);
          }
        }
      }
    }
    float xn[SMAX];
#pragma unroll
    for (int t = 0; t < SMAX; ++t) {
      xn[t] = 0.f;
      if (t >= cmax) break;
      const int jj = __shfl_sync(FULL, t < 8 ? j0 : j1, gbase + (t & 7));
      const float xx = __shfl_sync(FULL, t < 8 ? x0 : x1, gbase + (t & 7));
      const bool upd = t < c && (!GROUP || (jj >= a0 && jj < a1));
      float dot = 0.f;
      float4 dn[RV];
#pragma unroll
      for (int q = 0; q < RV; ++q) {
        const int v = g + 8 * q;
        dn[q] = (upd && v < pv) ? __ldg(N4 + (size_t)jj * pv + v) : make_float4(0.f, 0.f, 0.f, 0.f);
        dot = f4_dot(e[q], dn[q], dot);
      }
      dot += __shfl_xor_sync(FULL, dot, 4);
      dot += __shfl_xor_sync(FULL, dot, 2);
      dot += __shfl_xor_sync(FULL, dot, 1);
      xn[t] = upd && !sgk ? fmaf(__ldg(C + jj), xx, dot) : (t < c ? xx : 0.f);
      // residual with the updated atoms, y - D' x', from the same rows of D'
#pragma unroll
      for (int q = 0; q < RV; ++q) y[q] = f4_fma(upd ? -xn[t] : 0.f, dn[q], y[q]);
    }
#pragma unroll
    for (int q = 0; q < RV; ++q) e2 = f4_dot(y[q], y[q], e2);
    // lane g writes slots g and g + 8
    float nx0 = 0.f, nx1 = 0.f;
#pragma unroll
    for (int t = 0; t < SMAX; ++t) {
      if (t == g) nx0 = xn[t];
      if (t == g + 8) nx1 = xn[t];
    }
    if (g < c) {
      val[i * s + g] = nx0;
      if (csc_val) {
        const int64_t o = colptr[i] + g;
        if (csc_rowidx) csc_rowidx[o] = j0;
        csc_val[o] = nx0;
      }
    }
    if (SMAX > 8 && g + 8 < c) {
      val[i * s + g + 8] = nx1;
      if (csc_val) {
        const int64_t o = colptr[i] + g + 8;
        if (csc_rowidx) csc_rowidx[o] = j1;
        csc_val[o] = nx1;
      }
    }
  }
  const double se = block_sum_d((double)e2, red);
  if (threadIdx.x == 0) epart[blockIdx.x] = se;
}

// U = sum of the partial slices, float4 columns (len % 4 == 0): 8 slice
// groups per column in a CTA of 256 threads, then the 8 group sums in order
// (deterministic).
__global__ void __launch_bounds__(256) reduce4_kernel(const float4* __restrict__ Upart, int nslices,
                                                      int len4, float4* __restrict__ U) {
  __shared__ float4 part[8][32];
  const int tx = threadIdx.x & 31, gs = threadIdx.x >> 5;
  const int c = blockIdx.x * 32 + tx;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  if (c < len4) {
#pragma unroll 4
    for (int b = gs; b < nslices; b += 8) {
      const float4 v = Upart[(size_t)b * len4 + c];
      acc.x += v.x;
      acc.y += v.y;
      acc.z += v.z;
      acc.w += v.w;
    }
  }
  part[gs][tx] = acc;
  __syncthreads();
  if (gs == 0 && c < len4) {
    float4 t = part[0][tx];
#pragma unroll
    for (int q = 1; q < 8; ++q) {
      t.x += part[q][tx].x;
      t.y += part[q][tx].y;
      t.z += part[q][tx].z;
      t.w += part[q][tx].w;
    }
    U[c] = t;
  }
}

// U[q] = sum over partial slices in slice order (deterministic).
__global__ void reduce_kernel(const float* __restrict__ Upart, int nslices, int len,
                              float* __restrict__ U) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= len) return;
  float acc = 0.f;
  for (int b = 0; b < nslices; ++b) acc += Upart[(size_t)b * len + q];
  U[q] = acc;
}

// One warp per atom: v = U_j + r_j d_j; d' = v/||v|| (d kept if v = 0); c = d^T d'.
template <int PL>
// Atoms a0 <= j < a1.
__global__ void atoms_kernel(const float* __restrict__ D, int p, int n, const float* __restrict__ U,
                             float* __restrict__ Dn, float* __restrict__ C, int a0, int a1) {
  const int lane = threadIdx.x & 31;
  const int j = a0 + blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j >= a1) return;
  const float rj = U[(size_t)n * p + j];
  float d[PL], v[PL];
  float vv = 0.f;
#pragma unroll
  for (int u = 0; u < PL; ++u) {
    const int r = lane + 32 * u;
    d[u] = (r < p) ? D[(size_t)j * p + r] : 0.f;
    v[u] = (r < p) ? fmaf(rj, d[u], U[(size_t)j * p + r]) : 0.f;
    vv = fmaf(v[u], v[u], vv);
  }
  vv = warp_sum(vv);
  if (vv > 0.f) {
    const float inv = 1.0f / sqrtf(vv);
    float c = 0.f;
#pragma unroll
    for (int u = 0; u < PL; ++u) {
      const int r = lane + 32 * u;
      v[u] *= inv;
      c = fmaf(d[u], v[u], c);
      if (r < p) Dn[(size_t)j * p + r] = v[u];
    }
    c = warp_sum(c);
    if (lane == 0) C[j] = c;
  } else {
#pragma unroll
    for (int u = 0; u < PL; ++u) {
      const int r = lane + 32 * u;
      if (r < p) Dn[(size_t)j * p + r] = d[u];
    }
    if (lane == 0) C[j] = 1.f;
  }
}

// Pass B: per signal, e = y - D x (old atoms), x_t' = e.d'_{j_t} + c_{j_t} x_t,
// then ||y - D' x'||^2.  Writes the slots and, optionally, the CSC arrays.
// Eight lanes per signal (four signals per warp), as in pass A.
template <int RL>
__global__ void __launch_bounds__(ROW_THREADS) rows_kernel(
    const float* __restrict__ Y, int p, int64_t m, const float* __restrict__ D,
    const float* __restrict__ Dn, const float* __restrict__ C, int s,
    const int32_t* __restrict__ idx, float* __restrict__ val, const int32_t* __restrict__ cnt,
    const int64_t* __restrict__ colptr, int32_t* __restrict__ csc_rowidx,
    float* __restrict__ csc_val, double* __restrict__ epart, int sgk) {
  __shared__ double red[ROW_THREADS / 32];
  const int lane = threadIdx.x & 31;
  const int g = lane & 7, gbase = lane & ~7;
  float e2 = 0.f;
  const int64_t groups = (int64_t)gridDim.x * (blockDim.x >> 3);
  const int64_t g0 = (int64_t)blockIdx.x * (blockDim.x >> 3) + (threadIdx.x >> 3);
  const int64_t trips = (m + groups - 1) / groups;
  for (int64_t k = 0; k < trips; ++k) {
    const int64_t i = g0 + k * groups;
    const bool live = i < m;
    float y[RL], e[RL];
#pragma unroll
    for (int u = 0; u < RL; ++u) {
      const int r = g + 8 * u;
      y[u] = (live && r < p) ? Y[i * p + r] : 0.f;
      e[u] = y[u];
    }
    const int c = live ? cnt[i] : 0;
    const int j0 = (g < c) ? idx[i * s + g] : 0;
    const float x0 = (g < c) ? val[i * s + g] : 0.f;
    const int j1 = (g + 8 < c) ? idx[i * s + g + 8] : 0;
    const float x1 = (g + 8 < c) ? val[i * s + g + 8] : 0.f;
    const int cmax = __reduce_max_sync(0xffffffffu, (unsigned)c);
    for (int t = 0; t < cmax; ++t) {
      const int jj = __shfl_sync(0xffffffffu, t < 8 ? j0 : j1, gbase + (t & 7));
      const float xx = __shfl_sync(0xffffffffu, t < 8 ? x0 : x1, gbase + (t & 7));
      if (t < c) {
#pragma unroll
        for (int u = 0; u < RL; ++u) {
          const int r = g + 8 * u;
          if (r < p) e[u] = fmaf(-xx, __ldg(D + (size_t)jj * p + r), e[u]);
        }
      }
    }
    float nx0 = 0.f, nx1 = 0.f;  // x_t' for the slots held by this lane
    for (int t = 0; t < cmax; ++t) {
      const int jj = __shfl_sync(0xffffffffu, t < 8 ? j0 : j1, gbase + (t & 7));
      const float xx = __shfl_sync(0xffffffffu, t < 8 ? x0 : x1, gbase + (t & 7));
      float dot = 0.f;
      if (t < c) {
#pragma unroll
        for (int u = 0; u < RL; ++u) {
          const int r = g + 8 * u;
          if (r < p) dot = fmaf(e[u], __ldg(Dn + (size_t)jj * p + r), dot);
        }
      }
      dot += __shfl_xor_sync(0xffffffffu, dot, 4);
      dot += __shfl_xor_sync(0xffffffffu, dot, 2);
      dot += __shfl_xor_sync(0xffffffffu, dot, 1);
      if (t < c) {
        const float xn = sgk ? xx : fmaf(__ldg(C + jj), xx, dot);
        if (g == (t & 7)) {
          if (t < 8) nx0 = xn;
          else nx1 = xn;
        }
        // residual with the updated atoms: y - D' x'
#pragma unroll
        for (int u = 0; u < RL; ++u) {
          const int r = g + 8 * u;
          if (r < p) y[u] = fmaf(-xn, __ldg(Dn + (size_t)jj * p + r), y[u]);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < RL; ++u) e2 = fmaf(y[u], y[u], e2);
    if (g < c) {
      val[i * s + g] = nx0;
      if (csc_val) {
        const int64_t o = colptr[i] + g;
        if (csc_rowidx) csc_rowidx[o] = j0;
        csc_val[o] = nx0;
      }
    }
    if (g + 8 < c) {
      val[i * s + g + 8] = nx1;
      if (csc_val) {
        const int64_t o = colptr[i] + g + 8;
        if (csc_rowidx) csc_rowidx[o] = j1;
        csc_val[o] = nx1;
      }
    }
  }
  const double se = block_sum_d((double)e2, red);
  if (threadIdx.x == 0) epart[blockIdx.x] = se;
}

// One block: strided partial sums in a fixed order, then a fixed-order tree.
constexpr int FIN_THREADS = 256;
// Block 0: the RMSE before and after the update from the partial sums; the
// other blocks copy the updated atoms Dn into D.
__global__ void __launch_bounds__(FIN_THREADS) finalize_kernel(
    const double* __restrict__ epa, int na, const double* __restrict__ epb, int nb,
    double* __restrict__ rmse, int* __restrict__ iter, const float* __restrict__ Dn,
    float* __restrict__ D, int64_t np) {
  __shared__ double red[FIN_THREADS / 32];
  if (blockIdx.x > 0) {
    const int64_t stride = (int64_t)(gridDim.x - 1) * blockDim.x;
    for (int64_t q = (int64_t)(blockIdx.x - 1) * blockDim.x + threadIdx.x; q < np; q += stride)
      D[q] = Dn[q];
    return;
  }
  double ee = 0.0, yy = 0.0, e2 = 0.0;
  for (int b = threadIdx.x; b < na; b += FIN_THREADS) {
    ee += epa[2 * b];
    yy += epa[2 * b + 1];
  }
  for (int b = threadIdx.x; b < nb; b += FIN_THREADS) e2 += epb[b];
  ee = block_sum_d(ee, red);
  yy = block_sum_d(yy, red);
  e2 = block_sum_d(e2, red);
  if (threadIdx.x == 0) {
    const int it = *iter;
    rmse[2 * it] = yy > 0.0 ? sqrt(ee / yy) : 0.0;
    rmse[2 * it + 1] = yy > 0.0 ? sqrt(e2 / yy) : 0.0;
    *iter = it + 1;
  }
}

// ---- CSC helpers ------------------------------------------------------------------
constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_PER_THREAD = 4;
constexpr int SCAN_CHUNK = SCAN_THREADS * SCAN_PER_THREAD;

__global__ void __launch_bounds__(SCAN_THREADS) scan_sum_kernel(const int32_t* __restrict__ cnt,
                                                                 int64_t m, int64_t* __restrict__ bsum) {
  __shared__ double red[SCAN_THREADS / 32];
  const int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK + (int64_t)threadIdx.x * SCAN_PER_THREAD;
  int64_t loc = 0;
#pragma unroll
  for (int u = 0; u < SCAN_PER_THREAD; ++u)
    if (base + u < m) loc += cnt[base + u];
  const double tot = block_sum_d((double)loc, red);
  if (threadIdx.x == 0) bsum[blockIdx.x] = (int64_t)tot;
}

__global__ void __launch_bounds__(SCAN_THREADS) scan_write_kernel(const int32_t* __restrict__ cnt,
                                                                   int64_t m,
                                                                   const int64_t* __restrict__ bsum,
                                                                   int64_t* __restrict__ colptr) {
  __shared__ int64_t wsum[SCAN_THREADS / 32];
  __shared__ int64_t boff;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    int64_t o = 0;
    for (unsigned b = 0; b < blockIdx.x; ++b) o += bsum[b];
    boff = o;
  }
  const int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK + (int64_t)threadIdx.x * SCAN_PER_THREAD;
  int64_t v[SCAN_PER_THREAD];
  int64_t loc = 0;
#pragma unroll
  for (int u = 0; u < SCAN_PER_THREAD; ++u) {
    v[u] = (base + u < m) ? cnt[base + u] : 0;
    loc += v[u];
  }
  // inclusive warp scan of loc
  int64_t inc = loc;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t nb = __shfl_up_sync(FULL, inc, o);
    if (lane >= o) inc += nb;
  }
  if (lane == 31) wsum[w] = inc;
  __syncthreads();
  if (w == 0) {
    int64_t x = (lane < SCAN_THREADS / 32) ? wsum[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t nb = __shfl_up_sync(FULL, x, o);
      if (lane >= o) x += nb;
    }
    if (lane < SCAN_THREADS / 32) wsum[lane] = x;  // inclusive over warps
  }
  __syncthreads();
  int64_t run = boff + (w > 0 ? wsum[w - 1] : 0) + (inc - loc);
#pragma unroll
  for (int u = 0; u < SCAN_PER_THREAD; ++u) {
    if (base + u < m) colptr[base + u] = run;
    run += v[u];
    if (base + u == m - 1) colptr[m] = run;
  }
}

__global__ void slots_to_csc_kernel(const int32_t* __restrict__ idx, const float* __restrict__ val,
                                    const int32_t* __restrict__ cnt, int64_t m, int s,
                                    const int64_t* __restrict__ colptr, int32_t* __restrict__ rowidx,
                                    float* __restrict__ cval) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= m * s) return;
  const int64_t i = g / s;
  const int t = (int)(g - i * s);
  if (t < cnt[i]) {
    rowidx[colptr[i] + t] = idx[g];
    if (cval) cval[colptr[i] + t] = val[g];
  }
}

__global__ void csc_to_slots_kernel(const int64_t* __restrict__ colptr,
                                    const int32_t* __restrict__ rowidx, const float* __restrict__ cval,
                                    int64_t m, int n, int s, int32_t* __restrict__ idx,
                                    float* __restrict__ val, int32_t* __restrict__ cnt,
                                    int* __restrict__ err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int64_t a = colptr[i], b = colptr[i + 1];
  int c = (int)(b - a);
  bool ok = (b >= a) && (c <= s) && (a >= 0) && (b <= m * (int64_t)s);
  for (int t = 0; ok && t < c; ++t) {
    const int j = rowidx[a + t];
    if (j < 0 || j >= n || (t > 0 && j <= rowidx[a + t - 1])) ok = false;
  }
  if (!ok) {
    atomicOr(err, ERR_CSC);
    c = 0;
  }
  for (int t = 0; t < s; ++t) {
    idx[i * s + t] = (t < c) ? rowidx[a + t] : -1;
    val[i * s + t] = (t < c) ? cval[a + t] : 0.f;
  }
  cnt[i] = c;
}

cudaError_t reduce_slices(float* Upart, int nslices, int len, float* U, cudaStream_t st) {
  if (len % 4 == 0)
    reduce4_kernel<<<(len / 4 + 31) / 32, 256, 0, st>>>((const float4*)Upart, nslices, len / 4,
                                                         (float4*)U);
  else
    reduce_kernel<<<(len + 255) / 256, 256, 0, st>>>(Upart, nslices, len, U);
  return cudaGetLastError();
}

template <int PL>
cudaError_t accum_t(const float* Y, int p, int64_t m, const float* D, int n, int s,
                    const int32_t* idx, const float* val, const int32_t* cnt, const JauWork& w,
                    int* err, cudaStream_t st) {
  const size_t smem = jau_accum_smem(p, n);
  if (smem > 0) {
    cudaFuncSetAttribute(accum_kernel<PL, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    accum_kernel<PL, true><<<w.nb_accum, ACC_THREADS, smem, st>>>(Y, p, m, D, n, s, idx, val, cnt,
                                                                  w.Upart, w.epart_a, err);
  } else {
    cudaMemsetAsync(w.Upart, 0, sizeof(float) * ((size_t)n * p + n), st);
    accum_kernel<PL, false><<<w.nb_accum, ACC_THREADS, 0, st>>>(Y, p, m, D, n, s, idx, val, cnt,
                                                                w.Upart, w.epart_a, err);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return reduce_slices(w.Upart, smem > 0 ? w.nb_accum : 1, n * p + n, w.U, st);
}

}  // namespace

int num_sms() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

size_t jau_accum_smem(int p, int n) {
  const size_t bytes = sizeof(float) * ((size_t)n * p + n);
  return bytes <= 200u * 1024u ? bytes : 0;
}
int jau_accum_blocks(int p, int n, int mult) {
  // float4 form: 4 (8) CTAs of 256 threads per SM
  if (p % 4 == 0) return (mult >= 2 ? 8 : 4) * num_sms();
  // the shared-memory form runs 1 CTA per SM unless two partial slices fit on one SM
  if (jau_accum_smem(p, n) > 0)
    return (mult >= 2 && jau_accum_smem(p, n) <= 100u * 1024u) ? 2 * num_sms() : num_sms();
  return (mult >= 2 ? 8 : 4) * num_sms();
}
int jau_accum_blocks_max(int p, int n) {
  return (p % 4 != 0 && jau_accum_smem(p, n) > 0) ? 2 * num_sms() : 8 * num_sms();
}
bool jau_vec4(int p, const float* Y, const float* D) {
  return p % 4 == 0 && ((uintptr_t)Y % 16) == 0 && ((uintptr_t)D % 16) == 0;
}
int jau_launches(int p, const float* Y, const float* D) {
  // accumulate + slice/copy reduction + atoms + rows + finalize
  (void)p;
  (void)Y;
  (void)D;
  return 5;
}
int jau_row_blocks(int per_sm) { return (per_sm == 2 || per_sm == 8 ? per_sm : 4) * num_sms(); }
int jau_row_blocks_max() { return 8 * num_sms(); }

bool jau_det_supported(int p, int n, int s, const float* Y, const float* D) {
  return (Y || D ? jau_vec4(p, Y, D) : p % 4 == 0) && p <= 128 && n <= 1024 && s <= 16 &&
         det_range(p, n, s) >= 64;
}
// CTAs of the deterministic pass A for m signals: at least one per SM, each range
// within the shared-memory budget
int64_t jau_det_ranges(int64_t m, int p, int n, int s) {
  const int64_t R = det_range(p, n, s);
  int64_t nb = R > 0 ? (m + R - 1) / R : 1;
  const int64_t floor_nb = 2 * (int64_t)num_sms();
  if (nb < floor_nb) nb = floor_nb;
  return nb;
}

cudaError_t jau_accumulate_det(const float* Y, int p, int64_t m, const float* D, int n, int s,
                               const int32_t* idx, const float* val, const int32_t* cnt,
                               const JauWork& w, int* err, cudaStream_t st) {
  const int nb = w.nb_accum;
  const int64_t R = (m + nb - 1) / nb;
  const size_t len = jau_ulen(p, n);
  const size_t smem = det_smem_bytes(p, n, s, (int)R);
  const int a0 = w.a0, a1 = w.a1 > 0 ? w.a1 : n;
  cudaError_t e = cudaSuccess;
#define DL_ACCD(RV, SM)                                                                        \
  do {                                                                                         \
    if (w.nsgk) {                                                                              \
      e = cudaFuncSetAttribute(accum_det_kernel<RV, SM, true>,                                 \
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);        \
      if (e == cudaSuccess)                                                                    \
        accum_det_kernel<RV, SM, true><<<nb, DET_THREADS, smem, st>>>(                         \
            Y, p, m, R, D, n, s, idx, val, cnt, w.Upart, len, w.epart_a, err, a0, a1,          \
            (int)w.energies, w.D0, w.pidx, w.pval, w.pcnt, w.pvalid, w.a0 > 0 ? 1 : 0);        \
    } else {                                                                                   \
      e = cudaFuncSetAttribute(accum_det_kernel<RV, SM, false>,                                \
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);        \
      if (e == cudaSuccess)                                                                    \
        accum_det_kernel<RV, SM, false><<<nb, DET_THREADS, smem, st>>>(                        \
            Y, p, m, R, D, n, s, idx, val, cnt, w.Upart, len, w.epart_a, err, a0, a1,          \
            (int)w.energies, D, idx, val, cnt, nullptr, 0);                                    \
    }                                                                                          \
  } while (0)
#define DL_ACCD_S(RV) \
  if (s <= 8) DL_ACCD(RV, 8); else DL_ACCD(RV, 16)
  if (p <= 32) { DL_ACCD_S(1); }
  else if (p <= 64) { DL_ACCD_S(2); }
  else if (p <= 96) { DL_ACCD_S(3); }
  else { DL_ACCD_S(4); }
#undef DL_ACCD_S
#undef DL_ACCD
  if (e != cudaSuccess) return e;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return reduce_slices(w.Upart, nb, (int)len, w.U, st);
}

cudaError_t jau_accumulate(const float* Y, int p, int64_t m, const float* D, int n, int s,
                           const int32_t* idx, const float* val, const int32_t* cnt,
                           const JauWork& w, int* err, cudaStream_t st) {
  if (w.det && jau_det_supported(p, n, s, Y, D))
    return jau_accumulate_det(Y, p, m, D, n, s, idx, val, cnt, w, err, st);
  if (jau_vec4(p, Y, D)) {
    const size_t len = jau_ulen(p, n);
    cudaError_t e = cudaMemsetAsync(w.Upart, 0, sizeof(float) * len * kUCopies, st);
    if (e != cudaSuccess) return e;
#define DL_ACC4(RV, SM)                                                                  \
  do {                                                                                       \
    if (w.nsgk)                                                                              \
      accum4_kernel<RV, SM, true><<<w.nb_accum, ACC4_THREADS, 0, st>>>(                     \
          Y, p, m, D, n, s, idx, val, cnt, w.Upart, w.epart_a, err, w.a0, w.a1 > 0 ? w.a1 : n, \
          (int)w.energies, w.D0, w.pidx, w.pval, w.pcnt, w.pvalid, w.a0 > 0 ? 1 : 0);         \
    else                                                                                     \
      accum4_kernel<RV, SM, false><<<w.nb_accum, ACC4_THREADS, 0, st>>>(                    \
          Y, p, m, D, n, s, idx, val, cnt, w.Upart, w.epart_a, err, w.a0, w.a1 > 0 ? w.a1 : n, \
          (int)w.energies, D, idx, val, cnt, nullptr, 0);                                     \
  } while (0)
#define DL_ACC4_S(RV) \
  if (s <= 8) DL_ACC4(RV, 8); else DL_ACC4(RV, 16)
    if (p <= 32) { DL_ACC4_S(1); }
    else if (p <= 64) { DL_ACC4_S(2); }
    else if (p <= 96) { DL_ACC4_S(3); }
    else { DL_ACC4_S(4); }
#undef DL_ACC4_S
#undef DL_ACC4
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return reduce_slices(w.Upart, kUCopies, (int)len, w.U, st);
  }
  if (p % 4 == 0) {
    // unaligned operands: scalar form with global atomics and w.nb_accum CTAs
    cudaError_t e = cudaMemsetAsync(w.Upart, 0, sizeof(float) * ((size_t)n * p + n), st);
    if (e != cudaSuccess) return e;
#define DL_ACCG(PL)                                                                          \
  accum_kernel<PL, false><<<w.nb_accum, ACC_THREADS, 0, st>>>(Y, p, m, D, n, s, idx, val, cnt, \
                                                              w.Upart, w.epart_a, err)
    if (p <= 32) DL_ACCG(4);
    else if (p <= 64) DL_ACCG(8);
    else if (p <= 96) DL_ACCG(12);
    else DL_ACCG(16);
#undef DL_ACCG
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int len = n * p + n;
    reduce_kernel<<<(len + 255) / 256, 256, 0, st>>>(w.Upart, 1, len, w.U);
    return cudaGetLastError();
  }
  if (p <= 32) return accum_t<4>(Y, p, m, D, n, s, idx, val, cnt, w, err, st);
  if (p <= 64) return accum_t<8>(Y, p, m, D, n, s, idx, val, cnt, w, err, st);
  if (p <= 96) return accum_t<12>(Y, p, m, D, n, s, idx, val, cnt, w, err, st);
  return accum_t<16>(Y, p, m, D, n, s, idx, val, cnt, w, err, st);
}

cudaError_t jau_atoms(const float* D, int p, int n, const JauWork& w, cudaStream_t st) {
  const int a0 = w.a0, a1 = w.a1 > 0 ? w.a1 : n;
  const int blocks = (a1 - a0 + 7) / 8;
  if (blocks <= 0) return cudaSuccess;
  if (p <= 32) atoms_kernel<1><<<blocks, 256, 0, st>>>(D, p, n, w.U, w.Dn, w.C, a0, a1);
  else if (p <= 64) atoms_kernel<2><<<blocks, 256, 0, st>>>(D, p, n, w.U, w.Dn, w.C, a0, a1);
  else if (p <= 96) atoms_kernel<3><<<blocks, 256, 0, st>>>(D, p, n, w.U, w.Dn, w.C, a0, a1);
  else atoms_kernel<4><<<blocks, 256, 0, st>>>(D, p, n, w.U, w.Dn, w.C, a0, a1);
  return cudaGetLastError();
}

cudaError_t jau_rows(const float* Y, int p, int64_t m, const float* D, int n, int s,
                     const int32_t* idx, float* val, const int32_t* cnt, const JauWork& w,
                     const int64_t* colptr, int32_t* csc_rowidx, float* csc_val, cudaStream_t st) {
  const int nb = w.nb_row;
  const int a1 = w.a1 > 0 ? w.a1 : n;
  const bool grouped = w.a0 > 0 || a1 < n;
#define DL_ROWS(PL)                                                                              \
  rows_kernel<PL><<<nb, ROW_THREADS, 0, st>>>(Y, p, m, D, w.Dn, w.C, s, idx, val, cnt, colptr, \
                                              csc_rowidx, csc_val, w.epart_b, (int)w.sgk)
  if (jau_vec4(p, Y, D)) {
#define DL_ROWS4(RV, SM)                                                                         \
  do {                                                                                         \
    if (grouped)                                                                               \
      rows4_kernel<RV, SM, true><<<nb, ROW_THREADS, 0, st>>>(Y, p, m, D, w.Dn, w.C, s, idx, val, \
                                                             cnt, colptr, csc_rowidx, csc_val,  \
                                                             w.epart_b, w.a0, a1, (int)w.sgk);  \
    else                                                                                       \
      rows4_kernel<RV, SM, false><<<nb, ROW_THREADS, 0, st>>>(Y, p, m, D, w.Dn, w.C, s, idx,    \
                                                              val, cnt, colptr, csc_rowidx,     \
                                                              csc_val, w.epart_b, 0, n,         \
                                                              (int)w.sgk);                      \
  } while (0)
#define DL_ROWS4_S(RV) \
  if (s <= 8) DL_ROWS4(RV, 8); else DL_ROWS4(RV, 16)
    if (p <= 32) { DL_ROWS4_S(1); }
    else if (p <= 64) { DL_ROWS4_S(2); }
    else if (p <= 96) { DL_ROWS4_S(3); }
    else { DL_ROWS4_S(4); }
#undef DL_ROWS4_S
#undef DL_ROWS4
    return cudaGetLastError();
  }
  if (p <= 32) DL_ROWS(4);
  else if (p <= 64) DL_ROWS(8);
  else if (p <= 96) DL_ROWS(12);
  else DL_ROWS(16);
#undef DL_ROWS
  return cudaGetLastError();
}

cudaError_t jau_finalize(const JauWork& w, double* rmse_out, int* iter, float* D, int n, int p,
                         cudaStream_t st) {
  const int64_t np = (int64_t)n * p;
  int64_t cb = (np + FIN_THREADS - 1) / FIN_THREADS;
  if (cb > 64) cb = 64;
  finalize_kernel<<<(unsigned)(1 + cb), FIN_THREADS, 0, st>>>(w.epart_a, w.nb_accum, w.epart_b,
                                                              w.nb_row, rmse_out, iter, w.Dn, D, np);
  return cudaGetLastError();
}

int64_t scan_blocks(int64_t m) { return (m + SCAN_CHUNK - 1) / SCAN_CHUNK; }

cudaError_t counts_to_colptr(const int32_t* cnt, int64_t m, int64_t* bsum, int64_t* colptr,
                             cudaStream_t st) {
  if (m <= 0) {
    cudaMemsetAsync(colptr, 0, sizeof(int64_t), st);
    return cudaGetLastError();
  }
  const unsigned nb = (unsigned)scan_blocks(m);
  scan_sum_kernel<<<nb, SCAN_THREADS, 0, st>>>(cnt, m, bsum);
  scan_write_kernel<<<nb, SCAN_THREADS, 0, st>>>(cnt, m, bsum, colptr);
  return cudaGetLastError();
}

cudaError_t slots_to_csc(const int32_t* idx, const float* val, const int32_t* cnt, int64_t m,
                         int s, const int64_t* colptr, int32_t* rowidx, float* cval,
                         cudaStream_t st) {
  const int64_t tot = m * s;
  if (tot <= 0) return cudaSuccess;
  slots_to_csc_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(idx, val, cnt, m, s, colptr,
                                                                     rowidx, cval);
  return cudaGetLastError();
}

cudaError_t csc_to_slots(const int64_t* colptr, const int32_t* rowidx, const float* cval,
                         int64_t m, int n, int s, int32_t* idx, float* val, int32_t* cnt,
                         int* err, cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  csc_to_slots_kernel<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(colptr, rowidx, cval, m, n, s,
                                                                   idx, val, cnt, err);
  return cudaGetLastError();
}

}  // namespace dlk
