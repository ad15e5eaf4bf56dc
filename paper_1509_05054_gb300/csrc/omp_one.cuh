// The one-warp-per-signal Batch-OMP (omp_one) and its Gram-row sources, shared
// by the OMP kernels of k_omp.cu and the small-problem kernel of k_small.cu.
// Internal to the library.  See k_omp.cu for the arithmetic.
#pragma once

#include "dl_internal.cuh"
#include "omp_common.cuh"

#include <math.h>

namespace dlk {
namespace {

using namespace omp;

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

}  // namespace
}  // namespace dlk
