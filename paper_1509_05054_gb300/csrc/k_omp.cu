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

#include <math.h>

namespace dlk {
namespace {

using namespace omp;
constexpr int OMP_THREADS = 128;

// On the lane owning atom sel = 32*tsel + lane: read alpha[tsel] and mask it
// (NaN), and read u_q[tsel] for q < step.  Executed by one lane; the dense
// switch becomes an indexed branch instead of a select over all NT registers
// on every lane.
template <int NT, int NPHI>
struct Take {
  template <typename UAt>
  __device__ __forceinline__ static float run(float2 (&alpha)[NT / 2], UAt u_at, int tsel, int step,
                                              float (&ul)[NPHI], float qnan) {
    float out = 0.f;
#define DL_TAKE_CASE(T)                                     \
  case T:                                                   \
    if constexpr (T < NT) {                                 \
      constexpr int TT = T < NT ? T : 0;                    \
      if constexpr (TT & 1) {                               \
        out = alpha[TT >> 1].y;                             \
        alpha[TT >> 1].y = qnan;                            \
      } else {                                              \
        out = alpha[TT >> 1].x;                             \
        alpha[TT >> 1].x = qnan;                            \
      }                                                     \
      _Pragma("unroll") for (int q = 0; q < NPHI; ++q)      \
        if (q < step) ul[q] = u_at(q, TT);                  \
    }                                                       \
    break;
    switch (tsel) {
      DL_TAKE_CASE(0) DL_TAKE_CASE(1) DL_TAKE_CASE(2) DL_TAKE_CASE(3) DL_TAKE_CASE(4)
      DL_TAKE_CASE(5) DL_TAKE_CASE(6) DL_TAKE_CASE(7) DL_TAKE_CASE(8) DL_TAKE_CASE(9)
      DL_TAKE_CASE(10) DL_TAKE_CASE(11) DL_TAKE_CASE(12) DL_TAKE_CASE(13) DL_TAKE_CASE(14)
      DL_TAKE_CASE(15) DL_TAKE_CASE(16) DL_TAKE_CASE(17) DL_TAKE_CASE(18) DL_TAKE_CASE(19)
      DL_TAKE_CASE(20) DL_TAKE_CASE(21) DL_TAKE_CASE(22) DL_TAKE_CASE(23) DL_TAKE_CASE(24)
      DL_TAKE_CASE(25) DL_TAKE_CASE(26) DL_TAKE_CASE(27) DL_TAKE_CASE(28) DL_TAKE_CASE(29)
      DL_TAKE_CASE(30) DL_TAKE_CASE(31)
      default: break;
    }
#undef DL_TAKE_CASE
    return out;
  }
};

// Gram rows from global memory (L2): pair v of lane l = (G[sel][64v+l], G[sel][64v+32+l]).
template <bool FULLN>
struct GramGlobal {
  const float* __restrict__ G;
  int n;
  template <int NV>
  __device__ __forceinline__ void row(int sel, int lane, float2 (&out)[NV]) const {
    const float* __restrict__ Gr = G + (size_t)sel * n;  // row sel == column sel (G symmetric)
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const int j0 = 64 * v + lane, j1 = j0 + 32;
      out[v].x = (FULLN || j0 < n) ? __ldg(Gr + j0) : 0.f;
      out[v].y = (FULLN || j1 < n) ? __ldg(Gr + j1) : 0.f;
    }
  }
  __device__ __forceinline__ float diag(int sel) const { return __ldg(G + (size_t)sel * n + sel); }
};

// Gram entries among K candidate atoms cand[0..K) (ascending) of one signal:
// element j of "row" sel is G[cand[j]][cand[sel]]; lane l holds candidate l.
struct GramRestricted {
  const float* __restrict__ G;
  int n;
  const int32_t* __restrict__ cand;
  int K;
  template <int NV>
  __device__ __forceinline__ void row(int sel, int lane, float2 (&out)[NV]) const {
    const int as = cand[sel];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const int j0 = 64 * v + lane, j1 = j0 + 32;
      out[v].x = j0 < K ? __ldg(G + (size_t)cand[j0] * n + as) : 0.f;
      out[v].y = j1 < K ? __ldg(G + (size_t)cand[j1] * n + as) : 0.f;
    }
  }
  __device__ __forceinline__ float diag(int sel) const {
    const int as = cand[sel];
    return __ldg(G + (size_t)as * n + as);
  }
};

// One signal, one warp: the whole OMP of signal i (see the file header).
// a0row: its correlations (element j, j < n; in global memory when A0G, else in
// shared memory); y: the signal (global memory); L, C: this warp's
// shared-memory Cholesky rows and 1/L_qq; u_q for q < NR live in registers,
// the others in u_s (this warp's shared-memory slice).
// Outputs slots i*s.. (atom index = idxmap[j] when idxmap is given), the count,
// and the residual-energy estimate ||y||^2 - sum z^2 in ores[i] when given.
// Long supports (SMAX >= 12, s > 8): a step whose top two |alpha| lie closer than
// gap_tol ||y|| is a decision FP32 cannot be trusted with -- the accumulated
// rounding of alpha over many steps is of that size -- so the signal is handed
// to the re-solve (rs_list), which takes the FP64 decisions, and its FP32 run
// stops there.
template <int NT, int SMAX, int NR, bool FULLN, bool A0G, class GSrc>
__device__ __forceinline__ void omp_one(
    int64_t i, const GSrc& gsrc, float (&L)[SMAX][SMAX], float (&C)[SMAX], float2* u_s,
    const float* __restrict__ a0row, int n, const float* __restrict__ y, int p, int s,
    const int32_t* __restrict__ idxmap, int32_t* __restrict__ oidx, float* __restrict__ oval,
    int32_t* __restrict__ ocnt, float* __restrict__ ores, int* __restrict__ err,
    int* __restrict__ rs_list, int* __restrict__ rs_count, int rs_cap, float gap_tol) {
  static_assert(NT >= 2 && NT % 2 == 0, "alpha is held in float2 pairs");
  constexpr int NV = NT / 2;
  constexpr int NPHI = SMAX > 1 ? SMAX - 1 : 1;
  constexpr int TB = tbits<NT>();
  constexpr unsigned TMASK = (1u << TB) - 1u;
  constexpr unsigned VMASK = 0x7FFFFFFFu & ~TMASK;

  static_assert(NR >= 0 && NR <= NPHI, "register u vectors");
  const int lane = threadIdx.x & 31;
  float2 u_r[NR > 0 ? NR : 1][NV];
#define UV(q, v) \
  (*((q) >= NR ? &u_s[(((q) - NR) * NV + (v)) * 32 + lane] : &u_r[(q) < NR ? (q) : 0][(v)]))

  // ||y||^2 for the residual stop rule and the non-finite check
  float yy = 0.f;
  for (int r = lane; r < p; r += 32) {
    const float v = ld_stream(y + r);
    yy = fmaf(v, v, yy);
  }
  yy = warp_sum(yy);
  const bool finite_in = isfinite(yy);  // a non-finite D shows up as a non-finite pivot
  if (!finite_in && lane == 0) atomicOr(err, ERR_NONFINITE);

  const float qnan = __int_as_float(0x7fc00000);
  float2 alpha[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const int j0 = 64 * v + lane, j1 = j0 + 32;
    alpha[v].x = (FULLN || j0 < n) ? (A0G ? ld_stream(a0row + j0) : a0row[j0]) : qnan;
    alpha[v].y = (FULLN || j1 < n) ? (A0G ? ld_stream(a0row + j1) : a0row[j1]) : qnan;
  }

  float negaw[SMAX];  // -(w_q c_q), broadcast to all lanes
#pragma unroll
  for (int q = 0; q < SMAX; ++q) negaw[q] = 0.f;
  float invLdiag = 0.f;  // lane j: c_j = 1 / L_jj
  float myz = 0.f;       // lane j: z_j
  int myI = -1;          // lane j: I_j
  float rr = yy;
  int k = 0;

#pragma unroll
  for (int step = 0; step < SMAX; ++step) {
    if (step >= s || !finite_in) break;
    // ---- argmax |alpha| over unselected atoms (see key_max); lowest lane on ties
    const float kmax = keys_max<NT>(alpha, VMASK);
    const unsigned kbits = __reduce_max_sync(FULL, __float_as_uint(kmax));
    if ((kbits & VMASK) == 0u) break;  // max |alpha| = 0
    const unsigned ball = __ballot_sync(FULL, __float_as_uint(kmax) == kbits);
    const int lsel = __ffs(ball) - 1;
    const int tsel = NT - 1 - (int)(kbits & TMASK);
    const int sel = 32 * tsel + lsel;
    // issue the Gram loads early: the diagonal first (the pivot needs it before
    // the row is used), then the row (needed unless this is the last step)
    const bool need_u = (step + 1 < s) && (step + 1 < SMAX);
    const float gss = gsrc.diag(sel);
    if (need_u) {
      float2 grow[NV];
      gsrc.template row<NV>(sel, lane, grow);
#pragma unroll
      for (int v = 0; v < NV; ++v) UV(step < NPHI ? step : 0, v) = grow[v];
    }

    // alpha[sel] (exact, signed), its masking, and u_q[sel] on the owning lane
    float amine = 0.f;
    float ul[NPHI];
#pragma unroll
    for (int q = 0; q < NPHI; ++q) ul[q] = 0.f;
    if (lane == lsel) {
      auto u_at = [&](int q, int t) -> float {
        const float2 pr = UV(q, t >> 1);
        return (t & 1) ? pr.y : pr.x;
      };
      amine = Take<NT, NPHI>::run(alpha, u_at, tsel, step, ul, qnan);
    }
    const float asel = __shfl_sync(FULL, amine, lsel);
    if constexpr (SMAX >= 12) {
      if (gap_tol > 0.f && rs_count) {
        // second largest |alpha| (the winner is masked now), full precision
        float top2 = 0.f;
#pragma unroll
        for (int v = 0; v < NV; ++v) top2 = fmaxf(top2, fmaxf(fabsf(alpha[v].x), fabsf(alpha[v].y)));
        top2 = __uint_as_float(__reduce_max_sync(FULL, __float_as_uint(top2)));
        if (fabsf(asel) - top2 < gap_tol * sqrtf(yy)) {
          if (lane == 0) {
            const int pos = atomicAdd(rs_count, 1);
            if (pos < rs_cap) rs_list[pos] = (int)i;
          }
          break;
        }
      }
    }
    float wsq = 0.f;
#pragma unroll
    for (int q = 0; q < SMAX - 1; ++q) {
      if (q >= step) break;
      const float cq = C[q];
      const float wq = __shfl_sync(FULL, ul[q], lsel) * cq;  // w_q = c_q u_q[sel]
      wsq = fmaf(wq, wq, wsq);
      negaw[q] = -wq * cq;
      if (lane == q) L[step][q] = wq;
    }
    const float delta = gss - wsq;
    if (!(delta > kPivotMin)) {
      if (lane == 0) {
        if (!isfinite(delta)) atomicOr(err, ERR_NONFINITE);
        if (rs_count) {  // rounding dominates this pivot: redo the signal in FP64
          const int pos = atomicAdd(rs_count, 1);
          if (pos < rs_cap) rs_list[pos] = (int)i;
        }
      }
      break;
    }
    // c_k = 1 / L_kk: rsqrtf refined by one Newton-Raphson step, y + y (1 - d y^2) / 2
    float ck = rsqrtf(delta);
    ck = fmaf(0.5f * ck, fmaf(-delta * ck, ck, 1.0f), ck);
    const float zk = asel * ck;
    if (lane == step) {
      invLdiag = ck;
      myz = zk;
      myI = sel;
    }
    if (lane == 0) C[step] = ck;
    rr = fmaf(-zk, zk, rr);
    k = step + 1;

    // ---- u_k and alpha update, two elements per packed FMA
    if (need_u) {
      const float nz = -zk * ck;
      const float2 nz2 = make_float2(nz, nz);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        float2 g = UV(step < NPHI ? step : 0, v);
#pragma unroll
        for (int q = 0; q < SMAX - 1; ++q) {
          if (q >= step) break;
          g = __ffma2_rn(make_float2(negaw[q], negaw[q]), UV(q, v), g);
        }
        UV(step < NPHI ? step : 0, v) = g;
        alpha[v] = __ffma2_rn(nz2, g, alpha[v]);
      }
    }
    __syncwarp();  // row `step` of L and c_step (shared memory) are read later
    if (rr <= kResidRel * yy) break;
  }
#undef UV
  __syncwarp();

  // ---- back substitution L^T gamma = z
  float gam = 0.f, acc2 = 0.f;
#pragma unroll
  for (int q = SMAX - 1; q >= 0; --q) {
    if (q < k) {
      const float gl = (myz - acc2) * invLdiag;  // valid on lane q
      const float gq = __shfl_sync(FULL, gl, q);
      if (lane == q) gam = gq;
      if (lane < q) acc2 = fmaf(L[q][lane], gq, acc2);
    }
  }

  // ---- write the support in ascending atom order
  int rank = 0;
#pragma unroll
  for (int q = 0; q < SMAX; ++q) {
    if (q < k) {
      const int Iq = __shfl_sync(FULL, myI, q);
      rank += (Iq < myI) ? 1 : 0;
    }
  }
  const int64_t base = i * s;
  if (lane < k) {
    oidx[base + rank] = idxmap ? idxmap[myI] : myI;
    oval[base + rank] = gam;
  } else if (lane < s) {
    oidx[base + lane] = -1;
    oval[base + lane] = 0.f;
  }
  if (lane == 0) {
    ocnt[i] = k;
    if (ores) ores[i] = rr;
  }

}

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
