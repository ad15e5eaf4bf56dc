// Batch-OMP sparse coding with the per-signal vectors of the progressive
// Cholesky held in tensor memory (Algorithm 1 step 1; the Batch-OMP of the
// OMP-Box tool named in Section 4, in the Gram-Schmidt form of k_omp.cu).
//
// One warp per signal, as in omp_warp_kernel: lane l holds alpha[32t + l]
// (t < NT) in registers.  What differs is where the vectors u_q (q < s - 1)
// live.  They are the bulk of a signal's state (s - 1 vectors of n floats) and,
// held in registers and shared memory, they cap the kernel at 16 warps per SM
// and leave L1 little room for the Gram rows every step reads.  Here they go
// to TMEM, which the tensor cores use and this kernel otherwise would not:
// a persistent CTA of 4Q warps allocates all 512 TMEM columns, and warp w (TMEM
// lanes 32 (w mod 4) .. + 31, slot w / 4) owns 512/Q of its quadrant's
// columns: u_q[32t + l] sits in TMEM lane 32 (w mod 4) + l, column
// slot * (512/Q) + 16 q + t.  A whole u_q moves between TMEM and registers in
// one tcgen05.ld/st of 16 columns; the vectors that do not fit (Q > 4) stay in
// shared memory.  Reading u_q[sel] for the Cholesky row is one single-column
// tcgen05.ld by the warp and a shuffle from the owning lane.
//
// The arithmetic, and so every result, is identical to omp_warp_kernel's.
#include "dl_internal.cuh"
#include "omp_common.cuh"
#include "tc_ptx.cuh"

#include <math.h>

namespace dlk {
namespace {

using namespace omp;

// ---- TMEM access (32 lanes x 32-bit columns, this warp's quadrant)
__device__ __forceinline__ void tm_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
// Completion of this thread's TMEM loads; the registers are tied to the wait so
// that no use of them is scheduled before it.
__device__ __forceinline__ void tm_wait_ld16(uint32_t (&r)[16]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                 "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                 "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
               :
               : "memory");
}
__device__ __forceinline__ uint32_t tm_ld1(uint32_t taddr) {
  uint32_t r;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r) : "r"(taddr));
  return r;
}
// Completion of the single-column loads of the first K entries of r (K <= 7),
// with exactly those registers tied to the wait.
#define DL_TMW_OPS1 "+r"(r[0])
#define DL_TMW_OPS2 DL_TMW_OPS1, "+r"(r[1])
#define DL_TMW_OPS3 DL_TMW_OPS2, "+r"(r[2])
#define DL_TMW_OPS4 DL_TMW_OPS3, "+r"(r[3])
#define DL_TMW_OPS5 DL_TMW_OPS4, "+r"(r[4])
#define DL_TMW_OPS6 DL_TMW_OPS5, "+r"(r[5])
#define DL_TMW_OPS7 DL_TMW_OPS6, "+r"(r[6])
template <int K, int N>
__device__ __forceinline__ void tm_wait_ld(uint32_t (&r)[N]) {
  static_assert(K <= N && K <= 7, "tied registers");
  if constexpr (K == 0) asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
  else if constexpr (K == 1) asm volatile("tcgen05.wait::ld.sync.aligned;" : DL_TMW_OPS1 :: "memory");
  else if constexpr (K == 2) asm volatile("tcgen05.wait::ld.sync.aligned;" : DL_TMW_OPS2 :: "memory");
  else if constexpr (K == 3) asm volatile("tcgen05.wait::ld.sync.aligned;" : DL_TMW_OPS3 :: "memory");
  else if constexpr (K == 4) asm volatile("tcgen05.wait::ld.sync.aligned;" : DL_TMW_OPS4 :: "memory");
  else if constexpr (K == 5) asm volatile("tcgen05.wait::ld.sync.aligned;" : DL_TMW_OPS5 :: "memory");
  else if constexpr (K == 6) asm volatile("tcgen05.wait::ld.sync.aligned;" : DL_TMW_OPS6 :: "memory");
  else asm volatile("tcgen05.wait::ld.sync.aligned;" : DL_TMW_OPS7 :: "memory");
}
// The same with K known after unrolling (a switch the compiler folds).
template <int N>
__device__ __forceinline__ void tm_wait_ld_k(int k, uint32_t (&r)[N]) {
  switch (k) {
    case 0: tm_wait_ld<0>(r); break;
    case 1: tm_wait_ld<1 <= N ? 1 : 0>(r); break;
    case 2: tm_wait_ld<2 <= N ? 2 : 0>(r); break;
    case 3: tm_wait_ld<3 <= N ? 3 : 0>(r); break;
    case 4: tm_wait_ld<4 <= N ? 4 : 0>(r); break;
    case 5: tm_wait_ld<5 <= N ? 5 : 0>(r); break;
    case 6: tm_wait_ld<6 <= N ? 6 : 0>(r); break;
    default: tm_wait_ld<7 <= N ? 7 : 0>(r); break;
  }
}
#undef DL_TMW_OPS7
#undef DL_TMW_OPS6
#undef DL_TMW_OPS5
#undef DL_TMW_OPS4
#undef DL_TMW_OPS3
#undef DL_TMW_OPS2
#undef DL_TMW_OPS1
__device__ __forceinline__ void tm_st16(uint32_t taddr, const float2 (&v)[8]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
      "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
      "r"(__float_as_uint(v[0].x)), "r"(__float_as_uint(v[0].y)), "r"(__float_as_uint(v[1].x)),
      "r"(__float_as_uint(v[1].y)), "r"(__float_as_uint(v[2].x)), "r"(__float_as_uint(v[2].y)),
      "r"(__float_as_uint(v[3].x)), "r"(__float_as_uint(v[3].y)), "r"(__float_as_uint(v[4].x)),
      "r"(__float_as_uint(v[4].y)), "r"(__float_as_uint(v[5].x)), "r"(__float_as_uint(v[5].y)),
      "r"(__float_as_uint(v[6].x)), "r"(__float_as_uint(v[6].y)), "r"(__float_as_uint(v[7].x)),
      "r"(__float_as_uint(v[7].y))
      : "memory");
}
__device__ __forceinline__ void tm_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// One correlation of the signal's alpha0 row: FP32, or BF16 (the bits of a
// uint16_t, the BF16 mixed-precision form), widened to FP32.  Read once, not
// allocated in L1 (it leaves L1 to the Gram rows).
__device__ __forceinline__ float ld_a0(const float* p) { return ld_stream(p); }
__device__ __forceinline__ float ld_a0(const uint16_t* p) {
  unsigned short h;
  asm("ld.global.nc.L1::no_allocate.u16 %0, [%1];" : "=h"(h) : "l"(p));
  return __uint_as_float((uint32_t)h << 16);
}

// alpha[tsel] on the owning lane, masked to NaN (selected); an indexed branch
// executed by one lane.
template <int NT>
__device__ __forceinline__ float take_alpha(float2 (&alpha)[NT / 2], int tsel, float qnan) {
  float out = 0.f;
#define DL_TAKE_CASE(T)                 \
  case T:                               \
    if constexpr (T < NT) {             \
      constexpr int TT = T < NT ? T : 0; \
      if constexpr (TT & 1) {           \
        out = alpha[TT >> 1].y;         \
        alpha[TT >> 1].y = qnan;        \
      } else {                          \
        out = alpha[TT >> 1].x;         \
        alpha[TT >> 1].x = qnan;        \
      }                                 \
    }                                   \
    break;
  switch (tsel) {
    DL_TAKE_CASE(0) DL_TAKE_CASE(1) DL_TAKE_CASE(2) DL_TAKE_CASE(3) DL_TAKE_CASE(4)
    DL_TAKE_CASE(5) DL_TAKE_CASE(6) DL_TAKE_CASE(7) DL_TAKE_CASE(8) DL_TAKE_CASE(9)
    DL_TAKE_CASE(10) DL_TAKE_CASE(11) DL_TAKE_CASE(12) DL_TAKE_CASE(13) DL_TAKE_CASE(14)
    DL_TAKE_CASE(15)
    default: break;
  }
#undef DL_TAKE_CASE
  return out;
}

// The OMP of signal i by one warp; see omp_one in k_omp.cu for the steps.
// tcol: TMEM address of this warp's first column (its quadrant's lane field
// set); u_q for q < NTM at tcol + 16 q, the others in u_s (shared memory).
template <int NT, int SMAX, int NTM, typename AT>
__device__ __forceinline__ void omp_one_tm(
    int64_t i, const float* __restrict__ G, int n, float (&L)[SMAX][SMAX], float2* u_s,
    uint32_t tcol, const AT* __restrict__ a0row, const float* __restrict__ y, int p, int s,
    int32_t* __restrict__ oidx, float* __restrict__ oval, int32_t* __restrict__ ocnt,
    int* __restrict__ err, int* __restrict__ rs_list, int* __restrict__ rs_count, int rs_cap) {
  static_assert(NT == 16, "alpha layout of this kernel: n = 512");
  constexpr int NV = NT / 2;
  constexpr int NPHI = SMAX - 1;
  constexpr int TB = tbits<NT>();
  constexpr unsigned TMASK = (1u << TB) - 1u;
  constexpr unsigned VMASK = 0x7FFFFFFFu & ~TMASK;
  static_assert(NTM >= 1 && NTM <= NPHI, "u vectors in TMEM");
  const int lane = threadIdx.x & 31;
#define US(q, v) (u_s[(((q) - NTM) * NV + (v)) * 32 + lane])

  float yy = 0.f;
  for (int r = lane; r < p; r += 32) {
    const float v = ld_stream(y + r);
    yy = fmaf(v, v, yy);
  }
  yy = warp_sum(yy);
  const bool finite_in = isfinite(yy);
  if (!finite_in && lane == 0) atomicOr(err, ERR_NONFINITE);

  const float qnan = __int_as_float(0x7fc00000);
  float2 alpha[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    alpha[v].x = ld_a0(a0row + 64 * v + lane);
    alpha[v].y = ld_a0(a0row + 64 * v + 32 + lane);
  }

  float cq[SMAX];     // c_q = 1 / L_qq, uniform
  float negaw[SMAX];  // -(w_q c_q), uniform
#pragma unroll
  for (int q = 0; q < SMAX; ++q) {
    cq[q] = 0.f;
    negaw[q] = 0.f;
  }
  float invLdiag = 0.f;  // lane j: c_j
  float myz = 0.f;       // lane j: z_j
  int myI = -1;          // lane j: I_j
  float rr = yy;
  int k = 0;

#pragma unroll
  for (int step = 0; step < SMAX; ++step) {
    if (step >= s || !finite_in) break;
    const float kmax = keys_max<NT>(alpha, VMASK);
    const unsigned kbits = __reduce_max_sync(FULL, __float_as_uint(kmax));
    if ((kbits & VMASK) == 0u) break;
    const unsigned ball = __ballot_sync(FULL, __float_as_uint(kmax) == kbits);
    const int lsel = __ffs(ball) - 1;
    const int tsel = NT - 1 - (int)(kbits & TMASK);
    const int sel = 32 * tsel + lsel;
    const bool need_u = (step + 1 < s) && (step + 1 < SMAX);
    const float gss = __ldg(G + (size_t)sel * n + sel);
    float2 g[NV];
    if (need_u) {
      const float* __restrict__ Gr = G + (size_t)sel * n;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        g[v].x = __ldg(Gr + 64 * v + lane);
        g[v].y = __ldg(Gr + 64 * v + 32 + lane);
      }
    }
    // u_q[sel], q < step: single TMEM columns (then the owning lane's value), or
    // shared memory (read directly from the owning lane's slot)
    float ul[NPHI];
    {
      constexpr int NL = NPHI < 7 ? NPHI : 7;
      const int KL = step < NTM ? step : NTM;  // single columns to load
      uint32_t tv[NL];
      if (step > 0) tm_wait_st();  // u_{step-1} was just stored
#pragma unroll
      for (int q = 0; q < NL; ++q)
        if (q < KL) tv[q] = tm_ld1(tcol + 16 * q + tsel);
      if (KL > 0) tm_wait_ld_k(KL < NL ? KL : NL, tv);
#pragma unroll
      for (int q = 0; q < NPHI; ++q) {
        ul[q] = 0.f;
        if (q < step) {
          if (q < NTM) {
            ul[q] = __shfl_sync(FULL, __uint_as_float(tv[q < NL ? q : 0]), lsel);
          } else {
            const float2 pr = u_s[((q - NTM) * NV + (tsel >> 1)) * 32 + lsel];
            ul[q] = (tsel & 1) ? pr.y : pr.x;
          }
        }
      }
    }
    float amine = 0.f;
    if (lane == lsel) amine = take_alpha<NT>(alpha, tsel, qnan);
    const float asel = __shfl_sync(FULL, amine, lsel);
    float wsq = 0.f;
#pragma unroll
    for (int q = 0; q < SMAX - 1; ++q) {
      if (q >= step) break;
      const float wq = ul[q] * cq[q];  // w_q = c_q u_q[sel]
      wsq = fmaf(wq, wq, wsq);
      negaw[q] = -wq * cq[q];
      if (lane == q) L[step][q] = wq;
    }
    const float delta = gss - wsq;
    if (!(delta > kPivotMin)) {
      if (lane == 0) {
        if (!isfinite(delta)) atomicOr(err, ERR_NONFINITE);
        if (rs_count) {
          const int pos = atomicAdd(rs_count, 1);
          if (pos < rs_cap) rs_list[pos] = (int)i;
        }
      }
      break;
    }
    float ck = rsqrtf(delta);
    ck = fmaf(0.5f * ck, fmaf(-delta * ck, ck, 1.0f), ck);
    const float zk = asel * ck;
    if (lane == step) {
      invLdiag = ck;
      myz = zk;
      myI = sel;
    }
    cq[step] = ck;
    rr = fmaf(-zk, zk, rr);
    k = step + 1;

    if (need_u) {
      // u_step = G[:, sel] + sum_q negaw_q u_q
#pragma unroll
      for (int q = 0; q < SMAX - 1; ++q) {
        if (q >= step) break;
        const float2 nw = make_float2(negaw[q], negaw[q]);
        if (q < NTM) {
          uint32_t r[16];
          tm_ld16(tcol + 16 * q, r);
          tm_wait_ld16(r);
#pragma unroll
          for (int v = 0; v < NV; ++v)
            g[v] = __ffma2_rn(nw, make_float2(__uint_as_float(r[2 * v]), __uint_as_float(r[2 * v + 1])), g[v]);
        } else {
#pragma unroll
          for (int v = 0; v < NV; ++v) g[v] = __ffma2_rn(nw, US(q, v), g[v]);
        }
      }
      if (step < NTM) {
        tm_st16(tcol + 16 * step, g);
      } else if (step < NPHI) {
#pragma unroll
        for (int v = 0; v < NV; ++v) US(step < NPHI ? step : NTM, v) = g[v];
      }
      const float nz = -zk * ck;
      const float2 nz2 = make_float2(nz, nz);
#pragma unroll
      for (int v = 0; v < NV; ++v) alpha[v] = __ffma2_rn(nz2, g[v], alpha[v]);
    }
    __syncwarp();
    if (rr <= kResidRel * yy) break;
  }
#undef US
  tm_wait_st();
  __syncwarp();

  // back substitution L^T gamma = z
  float gam = 0.f, acc2 = 0.f;
#pragma unroll
  for (int q = SMAX - 1; q >= 0; --q) {
    if (q < k) {
      const float gl = (myz - acc2) * invLdiag;
      const float gq = __shfl_sync(FULL, gl, q);
      if (lane == q) gam = gq;
      if (lane < q) acc2 = fmaf(L[q][lane], gq, acc2);
    }
  }
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
    oidx[base + rank] = myI;
    oval[base + rank] = gam;
  } else if (lane < s) {
    oidx[base + lane] = -1;
    oval[base + lane] = 0.f;
  }
  if (lane == 0) ocnt[i] = k;
  __syncwarp();
}

// Persistent: one CTA of 4Q warps per SM; warp w of CTA b codes signals
// b * 4Q + w + t * gridDim.x * 4Q.
template <int NT, int SMAX, int Q, typename AT>
__global__ void __launch_bounds__(Q * 128, 1) omp_tm_kernel(
    const AT* __restrict__ A0, int64_t lda, const float* __restrict__ G, int n,
    const float* __restrict__ Y, int p, int64_t m, int s, int32_t* __restrict__ oidx,
    float* __restrict__ oval, int32_t* __restrict__ ocnt, int* __restrict__ err,
    int* __restrict__ rs_list, int* __restrict__ rs_count, int rs_cap, int64_t pf) {
  constexpr int W = 4 * Q;
  constexpr int COLS = (512 / Q) / 16 * 16;  // columns per warp
  constexpr int NTM = (COLS / 16) < (SMAX - 1) ? (COLS / 16) : (SMAX - 1);
  constexpr int NSH = (SMAX - 1) - NTM;       // u vectors in shared memory
  extern __shared__ float2 smem_u[];
  __shared__ float Lsh[W][SMAX][SMAX];
  __shared__ uint32_t tbase_sh;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     tc::smem_u32(&tbase_sh)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tbase = tbase_sh;
  const uint32_t tcol = tbase + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)((warp >> 2) * COLS);
  float2* u_s = NSH > 0 ? smem_u + (size_t)warp * NSH * (NT / 2) * 32 : nullptr;
  const int64_t stride = (int64_t)gridDim.x * W;
  for (int64_t i = (int64_t)blockIdx.x * W + warp; i < m; i += stride) {
    const int64_t ip = i + pf;
    if (ip < m) {  // warm L2 with a later signal's correlations and samples
      constexpr int per_line = 128 / (int)sizeof(AT);  // correlations per 128-byte line
      if (lane * per_line < n)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(A0 + ip * lda + lane * per_line));
      if (lane * 32 < p) asm volatile("prefetch.global.L2 [%0];" ::"l"(Y + ip * p + lane * 32));
    }
    omp_one_tm<NT, SMAX, NTM, AT>(i, G, n, Lsh[warp], u_s, tcol, A0 + i * lda, Y + i * p, p, s, oidx,
                              oval, ocnt, err, rs_list, rs_count, rs_cap);
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(512)
                 : "memory");
}

template <int Q, typename AT>
cudaError_t launch_tm(const AT* A0, int64_t lda, const float* G, int n, const float* Y, int p,
                      int64_t m, int s, int32_t* idx, float* val, int32_t* cnt, int* err, int* rl,
                      int* rc, int rcap, cudaStream_t st) {
  constexpr int NT = 16, SMAX = 8, W = 4 * Q;
  constexpr int COLS = (512 / Q) / 16 * 16;
  constexpr int NTM = (COLS / 16) < (SMAX - 1) ? (COLS / 16) : (SMAX - 1);
  constexpr int NSH = (SMAX - 1) - NTM;
  const size_t smem = (size_t)W * NSH * (NT / 2) * 32 * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(omp_tm_kernel<NT, SMAX, Q, AT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t need = (m + W - 1) / W;
  const int grid = (int)(need < num_sms() ? need : num_sms());
  omp_tm_kernel<NT, SMAX, Q, AT><<<grid, W * 32, smem, st>>>(A0, lda, G, n, Y, p, m, s, idx, val, cnt,
                                                          err, rl, rc, rcap,
                                                          (int64_t)grid * W * 2);
  return cudaGetLastError();
}

}  // namespace

bool omp_tm_supported(int n, int s) { return n == 512 && s >= 5 && s <= 8; }

cudaError_t omp_batch_tm(int q, const void* A0, bool a0_bf16, int64_t lda, const float* G, int n,
                         const float* Y, int p, int64_t m, int s, int32_t* idx, float* val,
                         int32_t* cnt, int* err, int* rl, int* rc, int rcap, cudaStream_t st) {
  if (!omp_tm_supported(n, s)) return cudaErrorInvalidValue;
  if (m <= 0) return cudaSuccess;
#define DL_TM(QQ)                                                                                  \
  return a0_bf16 ? launch_tm<QQ>((const uint16_t*)A0, lda, G, n, Y, p, m, s, idx, val, cnt, err, rl, \
                                 rc, rcap, st)                                                     \
                 : launch_tm<QQ>((const float*)A0, lda, G, n, Y, p, m, s, idx, val, cnt, err, rl,   \
                                 rc, rcap, st)
  switch (q) {
    case 4: DL_TM(4);
    case 6: DL_TM(6);
    default: DL_TM(5);
  }
#undef DL_TM
}

}  // namespace dlk
