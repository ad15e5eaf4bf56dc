// Residual-form OMP sparse coding on the tensor cores, correlations included
// (Algorithm 1 step 1: the OMP of every signal with the current dictionary).
//
// Batch-OMP (k_omp.cu, k_omp_tm.cu) updates alpha = D^T r from alpha0 = D^T y
// and Gram rows, one warp per signal: per step a reduction over n correlations
// spread over 32 lanes, a gathered Gram row and s packed FMAs per element, all
// on the CUDA cores (about 2,300 warp instructions per signal at n = 512,
// s = 8), after alpha0 itself made a round trip through HBM.  Here the
// correlations of every step are recomputed from the residual instead,
// alpha^(k) = D^T r^(k), as one dense product per 128-signal tile:
//
//   * D (n <= 512 atoms, p <= 64) sits in shared memory for the whole kernel as
//     two FP16 parts, D 2^eD = Dh + Dl (22 significant bits); the residuals of a
//     tile are split the same way, r 2^er = Rh + Rl, and tcgen05.mma (kind::f16,
//     FP32 accumulation in TMEM) forms Rl Dh^T + Rh Dl^T + Rh Dh^T: 128 signals x
//     up to 512 atoms, one signal per TMEM lane.  The dropped Rl Dl^T term and
//     the FP16 roundings leave an error of about 2^-21 ||r|| ||d_j|| per
//     correlation -- the accuracy class of FP32 Batch-OMP.  alpha0 is step 0 of
//     the same product and never leaves the chip.  The BF16 form (BF) keeps
//     the top and bottom 16 bits of each FP32 value of D 2^eD instead: the top
//     plane (D truncated to BF16) and the residual rounded to BF16 give one
//     kind::f16 product per step; both planes together give FP32 D exactly.
//   * Two threads per signal ("halves", the same lane of two warps) read its
//     TMEM row (tcgen05.ld 32x32b, its lane), each half 128 of every
//     accumulator unit's 256 columns, and take the argmax of |alpha| with the
//     lowest index among equal values (16-column keys as in omp_common.cuh,
//     chunks in ascending order; the halves' bests are exchanged through
//     shared memory).  Each half holds 32 of the residual's 64 elements and
//     computes its part of alpha_sel = d_sel^T r in FP32 from D's
//     shared-memory planes (hi + lo, 22 significant bits; exact FP32 D in the
//     BF16 form).  The lead half
//     extends B = L^-1 (the inverse Cholesky factor of G_I, Gram entries from
//     G) and writes the step's coefficient changes; both halves then update
//     their elements of r^(k+1) = r^(k) - D_I (gamma^(k+1) - gamma^(k)) in FP32
//     in one rolled loop over the selected atoms (one copy of that code, not
//     one per step, keeps the kernel small enough for the instruction cache).
//     The stop rules and the FP64 re-solve hand-off are those of Batch-OMP:
//     max |alpha| = 0, residual energy <= kResidRel ||y||^2, a Cholesky pivot
//     below kPivotMin (the signal goes to omp_resolve64).
//   * A persistent CTA per SM keeps two tiles in flight (slots): while the
//     owners of one slot sweep and update, the tensor core computes the other
//     slot's correlations.  TMEM holds two 256-column accumulator units; a step
//     of a 512-atom problem uses both (the sweep of the first overlaps the MMAs
//     of the second), a step with n <= 256 uses one, alternating.
//
// Warp roles (512 threads, four warps per SM sub-partition, so up to 128
// registers a thread): warps 0-7 hold slot 0, warps 8-15 slot 1; within a
// slot, warps 0-3 are the lead halves and warps 4-7 the other halves of the
// same 128 signals (warp w reads TMEM lanes 32 (w mod 4) ..).  Thread 0 of a
// slot's first warp issues the slot's MMAs once the slot's eight warps have
// written their residuals (a named barrier per slot); the two warps of a
// signal quad meet at a named barrier of their own for each exchange.
// mbarriers: tfull[u] (tcgen05.commit -> owners) and
// tempty[u] (owners -> the next use of accumulator unit u).  The uses of the
// units follow one fixed order (round, step, slot, unit); before waiting for
// its own tfull phase an owner waits for the unit's previous use to have been
// read, which makes every parity wait unambiguous.  Every wait is bounded
// (about 2 s); a timeout sets ERR_TIMEOUT and the kernel unwinds and frees its
// TMEM.
#include "dl_internal.cuh"
#include "omp_common.cuh"
#include "tc_ptx.cuh"

#include <cuda_fp16.h>
#include <math.h>

namespace dlk {
namespace {

using namespace tc;

constexpr int RT_M = 128;                 // signals per tile = TMEM lanes
constexpr int RT_N = 256;                 // atoms per MMA = TMEM columns per unit
constexpr int RT_ROWB = 128;              // bytes of one FP16 row, p <= 64 padded
constexpr int RT_NMAX = 2 * RT_N;         // atoms
constexpr int RT_PMAX = 64;
constexpr int RT_NS = 2;                  // tiles in flight
constexpr int RT_HALVES = 2;              // threads per signal
constexpr int RT_OWNER_WARPS = 4 * RT_NS * RT_HALVES;
constexpr int RT_THREADS = 32 * RT_OWNER_WARPS;
constexpr int RT_SIGS = RT_M * RT_NS;     // signals in flight per CTA
constexpr int RT_SMAX = 8;
constexpr int RT_PH = RT_PMAX / RT_HALVES;  // residual elements a thread holds
// kind::f16: D F32 (bits 4-5 = 1), A and B F16 (format 0), K-major, N = 256, M = 128
constexpr uint32_t RT_IDESC =
    (1u << 4) | ((uint32_t)(RT_N >> 3) << 17) | ((uint32_t)(RT_M >> 4) << 24);
// the same with A and B BF16 (the BF16 form: one product of BF16 operands)
constexpr uint32_t RT_IDESC_BF = RT_IDESC | (1u << 7) | (1u << 10);

enum { RB_TFULL = 0, RB_TEMPTY = 2, RB_COUNT = 4 };

// Shared memory (offsets from a 1024-byte aligned base).
struct RtSmem {
  static constexpr size_t dh = 0;                                   // Dh rows, 128-byte swizzle
  static constexpr size_t dl = dh + (size_t)RT_NMAX * RT_ROWB;      // Dl rows
  static constexpr size_t a = dl + (size_t)RT_NMAX * RT_ROWB;       // per slot: Rh, Rl
  static constexpr size_t a_part = (size_t)RT_M * RT_ROWB;          // 16 KB
  static constexpr size_t a_slot = 2 * a_part;
  static constexpr size_t bars = a + RT_NS * a_slot;
  static constexpr size_t misc = bars + 8 * RB_COUNT;               // tmem slot, fail, max|D|
  // per signal (element q at q * RT_SIGS + signal): I (u16), dg and gamma
  static constexpr size_t is = misc + 64;
  static constexpr size_t dg = is + (size_t)RT_SMAX * RT_SIGS * 2;
  static constexpr size_t gm = dg + (size_t)RT_SMAX * RT_SIGS * 4;
  static constexpr size_t xch = gm + (size_t)RT_SMAX * RT_SIGS * 4;  // per signal and half
  static constexpr size_t dyn = xch + (size_t)RT_SIGS * RT_HALVES * 20 + 1024;
};
static_assert(RtSmem::dyn <= 232448, "shared memory of one CTA");

// Byte offset of 16-byte unit g (FP16 elements 8g .. 8g+7) of row r in a
// K-major tile with the 128-byte swizzle (8-row groups of 1024 bytes).
__device__ __forceinline__ uint32_t sw_off(int r, int g) {
  return (uint32_t)(r * RT_ROWB + ((g ^ (r & 7)) << 4));
}

// 16 consecutive TMEM columns of this warp's lanes, without the wait.
__device__ __forceinline__ void tm_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tm_wait16(uint32_t (&r)[16]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                 "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                 "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
               :
               : "memory");
}

// Two FP32 values as packed FP16 (round to nearest), v0 in the low half.
__device__ __forceinline__ uint32_t pack_f16x2(float v0, float v1) {
  uint32_t d;
  asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(v1), "f"(v0));
  return d;
}
// Split 2^e-scaled FP32 values into FP16 parts: v = hi + lo + O(2^-22 |v|).
// hi = v rounded to 11 significant bits (Veltkamp's splitting with 2^13 + 1),
// lo = v - hi exactly; both then convert to FP16 without further rounding
// (|v| < 2^14, so hi is a normal FP16 number unless |v| < 2^-14).
__device__ __forceinline__ void split2(float v0, float v1, uint32_t& hi, uint32_t& lo) {
  const float c0 = __fmul_rn(v0, 8193.f), c1 = __fmul_rn(v1, 8193.f);
  const float h0 = __fsub_rn(c0, __fsub_rn(c0, v0)), h1 = __fsub_rn(c1, __fsub_rn(c1, v1));
  hi = pack_f16x2(h0, h1);
  lo = pack_f16x2(__fsub_rn(v0, h0), __fsub_rn(v1, h1));
}

// Power of two 2^e as a float, e clamped to the normal range.
__device__ __forceinline__ float pow2i(int e) {
  e = e < -120 ? -120 : (e > 120 ? 120 : e);
  return __int_as_float((127 + e) << 23);
}

// Argmax key of 16 columns: |alpha| with the low 4 mantissa bits replaced by
// (15 - t), so the float maximum of the keys is the largest |alpha| and, among
// values equal to within 2^-19 relative, the lowest column t.  Two interleaved
// running maxima keep few keys live at once.
__device__ __forceinline__ float chunk_key(const uint32_t* v) {
  auto key = [&](int t) { return __uint_as_float((v[t] & 0x7FFFFFF0u) | (uint32_t)(15 - t)); };
  float m = omp::fmax3(key(0), key(1), key(2));
  float q = omp::fmax3(key(3), key(4), key(5));
  m = omp::fmax3(m, key(6), key(7));
  q = omp::fmax3(q, key(8), key(9));
  m = omp::fmax3(m, key(10), key(11));
  q = omp::fmax3(q, key(12), key(13));
  m = omp::fmax3(m, key(14), key(15));
  return fmaxf(m, q);
}

// Position of B_qj (j <= q) in the packed lower triangle.
__host__ __device__ constexpr int tri(int q, int j) { return q * (q + 1) / 2 + j; }

// One signal's OMP state as its two threads ("halves") hold it.  Half hf
// holds the 16-byte units g = 2u + hf (u < 4) of the residual, elements 8g ..
// 8g+7.  Half 0 (the lead) also holds B and the stop rule's energies and runs
// the Cholesky step; it writes the step's atom, the coefficient changes and
// gamma to the signal's column of a shared-memory scratch (element q at
// q * RT_SIGS + signal), from which both halves update their residual
// elements in one rolled loop (one copy of that code, not one per step, keeps
// the kernel small enough for the instruction cache).
struct Owner {
  float2 r[RT_PH / 2];        // this half of r^(k), FP32 pairs (packed FMAs), zero past p
  float B[RT_SMAX * (RT_SMAX + 1) / 2];  // lead: B = L^-1, lower triangle by rows (L L^T = G_I)
  float yy;                   // lead: ||y||^2
  float rr;                   // lead: ||y||^2 - sum z_q^2 (the stop rule's residual energy)
  float rn;                   // ||r||^2 of the stored residual (its FP16 scale)
  int k;                      // lead: atoms selected
  bool active;                // still selecting
};

// (hi + lo) of two FP16 pairs as FP32: the two halves of word hw and of word
// lw, the low halves first.  Exact: lo is the remainder of hi, so the sum has
// at most 24 significant bits.  hi is converted, lo is added in the same
// instruction (the mixed-precision add with an FP16 and an FP32 operand).
__device__ __forceinline__ float2 hl_sum(uint32_t hw, uint32_t lw) {
  float2 d;
  asm("{\n\t.reg .f16 h0, h1, l0, l1;\n\t.reg .f32 f0, f1;\n\t"
      "mov.b32 {h0, h1}, %2;\n\tmov.b32 {l0, l1}, %3;\n\t"
      "cvt.f32.f16 f0, h0;\n\tcvt.f32.f16 f1, h1;\n\t"
      "add.f32.f16 %0, l0, f0;\n\tadd.f32.f16 %1, l1, f1;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "r"(hw), "r"(lw));
  return d;
}

// Unit g of row j of D from the shared-memory planes (elements 8g .. 8g+7) as
// FP32 pairs, D_j 2^eD.  FP32 form: the FP16 parts, hi + lo.  BF16 form (BF):
// the top and bottom 16 bits of each FP32 value, put back together exactly by
// one byte permute per value (the top plane is D truncated to BF16, the
// MMA's operand).
template <bool BF>
__device__ __forceinline__ void row_unit(const uint8_t* Dh, const uint8_t* Dl, int j, int g,
                                         float2 (&d)[4]) {
  const uint4 a = *reinterpret_cast<const uint4*>(Dh + sw_off(j, g));
  const uint4 b = *reinterpret_cast<const uint4*>(Dl + sw_off(j, g));
  if constexpr (BF) {
    d[0] = make_float2(__uint_as_float(__byte_perm(b.x, a.x, 0x5410)),
                       __uint_as_float(__byte_perm(b.x, a.x, 0x7632)));
    d[1] = make_float2(__uint_as_float(__byte_perm(b.y, a.y, 0x5410)),
                       __uint_as_float(__byte_perm(b.y, a.y, 0x7632)));
    d[2] = make_float2(__uint_as_float(__byte_perm(b.z, a.z, 0x5410)),
                       __uint_as_float(__byte_perm(b.z, a.z, 0x7632)));
    d[3] = make_float2(__uint_as_float(__byte_perm(b.w, a.w, 0x5410)),
                       __uint_as_float(__byte_perm(b.w, a.w, 0x7632)));
  } else {
    d[0] = hl_sum(a.x, b.x);
    d[1] = hl_sum(a.y, b.y);
    d[2] = hl_sum(a.z, b.z);
    d[3] = hl_sum(a.w, b.w);
  }
}

// Step STEP of one signal after the argmax chose atom sel and alpha_sel =
// d_sel^T r^(k) is known (Batch-OMP's progressive Cholesky in the
// inverse-factor form), run by the lead:
//   w = B g with g_q = G[I_q][sel] (the new row of L), delta = G[sel][sel] - ||w||^2;
//   c = 1/sqrt(delta), z = alpha_sel c; row STEP of B: B_kj = -c sum_{q>=j} w_q B_qj,
//   B_kk = c; dg = z B_k,: (the change of gamma), gamma += dg.
// Writes I_STEP = sel, dg and gamma to the signal's scratch column.  Returns
// true when the residual is to be updated (r -= D_I dg) for a further step.  A
// pivot delta <= kPivotMin stops the signal and lists it for the FP64
// re-solve, as in omp_one.
template <int STEP>
__device__ __forceinline__ bool owner_chol(Owner& o, int sel, float asel, float gss,
                                           const float (&g)[RT_SMAX], uint16_t* Is, float* dgs,
                                           float* gms, int s, int64_t i, int* __restrict__ err,
                                           int* __restrict__ rs_list, int* __restrict__ rs_count,
                                           int rs_cap) {
  float w[STEP > 0 ? STEP : 1];
  float wsq = 0.f;
#pragma unroll
  for (int q = 0; q < STEP; ++q) {
    float acc = 0.f;
#pragma unroll
    for (int j = 0; j <= q; ++j) acc = fmaf(o.B[tri(q, j)], g[j], acc);
    w[q] = acc;
    wsq = fmaf(acc, acc, wsq);
  }
  const float delta = gss - wsq;
  if (!(delta > kPivotMin)) {
    if (!isfinite(delta)) atomicOr(err, ERR_NONFINITE);
    if (rs_count) {  // rounding dominates this pivot: redo the signal in FP64
      const int pos = atomicAdd(rs_count, 1);
      if (pos < rs_cap) rs_list[pos] = (int)i;
    }
    o.active = false;
    return false;
  }
  // c = 1 / L_kk: rsqrtf refined by one Newton-Raphson step, y + y (1 - d y^2) / 2
  float c = rsqrtf(delta);
  c = fmaf(0.5f * c, fmaf(-delta * c, c, 1.0f), c);
  const float z = asel * c;
#pragma unroll
  for (int j = 0; j < STEP; ++j) {
    float acc = 0.f;
#pragma unroll
    for (int q = j; q < STEP; ++q) acc = fmaf(w[q], o.B[tri(q, j)], acc);
    o.B[tri(STEP, j)] = -c * acc;
    const float dg = z * o.B[tri(STEP, j)];
    dgs[j * RT_SIGS] = dg;
    gms[j * RT_SIGS] += dg;
  }
  o.B[tri(STEP, STEP)] = c;
  dgs[STEP * RT_SIGS] = z * c;
  gms[STEP * RT_SIGS] = z * c;
  Is[STEP * RT_SIGS] = (uint16_t)sel;
  o.k = STEP + 1;
  o.rr = fmaf(-z, z, o.rr);
  if (STEP + 1 >= s || STEP + 1 >= RT_SMAX || o.rr <= kResidRel * o.yy) {
    o.active = false;  // complete
    return false;
  }
  return true;
}

// This half's part of d_j^T r for atom j, from the shared-memory planes (D =
// (hi + lo) 2^-eD, exact to about 2^-22 relative, or exact in the BF16 form;
// no global-memory latency on the step's chain), in units of 2^-eD.
template <bool BF>
__device__ __forceinline__ float owner_dot(const Owner& o, int j, int hf, const uint8_t* Dh,
                                           const uint8_t* Dl) {
  float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
#pragma unroll
  for (int u = 0; u < RT_PH / 8; ++u) {
    float2 d[4];
    row_unit<BF>(Dh, Dl, j, 2 * u + hf, d);
    a0 = __ffma2_rn(o.r[4 * u], d[0], a0);
    a1 = __ffma2_rn(o.r[4 * u + 1], d[1], a1);
    a0 = __ffma2_rn(o.r[4 * u + 2], d[2], a0);
    a1 = __ffma2_rn(o.r[4 * u + 3], d[3], a1);
  }
  return (a0.x + a0.y) + (a1.x + a1.y);
}

// This half's part of ||r||^2, packed.
__device__ __forceinline__ float owner_norm2(const Owner& o) {
  float2 n = make_float2(0.f, 0.f);
#pragma unroll
  for (int e = 0; e < RT_PH / 2; ++e) n = __ffma2_rn(o.r[e], o.r[e], n);
  return n.x + n.y;
}

// r^(k+1) = r^(k) - sum_{j <= step} dg_j d_{I_j} on this half's elements (atoms
// from the shared-memory parts, scaled back by 2^-eD); returns this half's part
// of ||r^(k+1)||^2.  One rolled loop over atoms; packed FP32x2 multiply-adds.
template <bool BF>
__device__ __forceinline__ float owner_update(Owner& o, int step, int hf, const uint16_t* Is,
                                              const float* dgs, const uint8_t* Dh,
                                              const uint8_t* Dl, float dsc) {
#pragma unroll 1
  for (int j = 0; j <= step; ++j) {
    const int a = Is[j * RT_SIGS];
    const float nd = -dgs[j * RT_SIGS] * dsc;
    const float2 nd2 = make_float2(nd, nd);
#pragma unroll
    for (int u = 0; u < RT_PH / 8; ++u) {
      float2 d[4];
      row_unit<BF>(Dh, Dl, a, 2 * u + hf, d);
#pragma unroll
      for (int e = 0; e < 4; ++e) o.r[4 * u + e] = __ffma2_rn(nd2, d[e], o.r[4 * u + e]);
    }
  }
  return owner_norm2(o);
}

// Two FP32 values as packed BF16 (round to nearest), v0 in the low half.
__device__ __forceinline__ uint32_t pack_bf16x2(float v0, float v1) {
  uint32_t u;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(u) : "f"(v1), "f"(v0));
  return u;
}

// This half of the signal's residual into row `row` of the slot's K-major
// tiles.  FP32 form: as FP16 parts in the two tiles, scaled by 2^er with
// ||r|| 2^er < 2^14 (o.rn: the whole residual's ||r||^2).  BF16 form: rounded
// to BF16 in the first tile.
template <bool BF>
__device__ __forceinline__ void owner_store(const Owner& o, int hf, uint8_t* Ah, uint8_t* Al,
                                            int row) {
  if constexpr (BF) {
#pragma unroll
    for (int u = 0; u < RT_PH / 8; ++u) {
      uint32_t h[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) h[e] = pack_bf16x2(o.r[4 * u + e].x, o.r[4 * u + e].y);
      *reinterpret_cast<uint4*>(Ah + sw_off(row, 2 * u + hf)) = make_uint4(h[0], h[1], h[2], h[3]);
    }
    return;
  }
  int E = 0;
  frexpf(sqrtf(o.rn), &E);
  const float sc = o.rn > 0.f ? pow2i(14 - E) : 1.f;
  const float2 sc2 = make_float2(sc, sc), m1 = make_float2(-1.f, -1.f);
  const float2 k2 = make_float2(8193.f, 8193.f);
#pragma unroll
  for (int u = 0; u < RT_PH / 8; ++u) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      // split2 with packed operations: c = 8193 v, hi = c - (c - v), lo = v - hi
      // (each subtraction one FMA with -1: a single rounding, as __fsub_rn)
      const float2 v = __fmul2_rn(o.r[4 * u + e], sc2);
      const float2 c = __fmul2_rn(v, k2);
      const float2 hi = __ffma2_rn(__ffma2_rn(v, m1, c), m1, c);
      const float2 lo = __ffma2_rn(hi, m1, v);
      h[e] = pack_f16x2(hi.x, hi.y);
      l[e] = pack_f16x2(lo.x, lo.y);
    }
    const int g = 2 * u + hf;
    *reinterpret_cast<uint4*>(Ah + sw_off(row, g)) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(Al + sw_off(row, g)) = make_uint4(l[0], l[1], l[2], l[3]);
  }
}

// The signal's support in ascending atom order (slots i*s ..), -1 padding, and its count.
__device__ __forceinline__ void owner_write(const Owner& o, const uint16_t* Is, const float* gms,
                                            int64_t i, int s, int32_t* __restrict__ oidx,
                                            float* __restrict__ oval, int32_t* __restrict__ ocnt) {
  const int64_t base = i * s;
  int I[RT_SMAX];
#pragma unroll
  for (int q = 0; q < RT_SMAX; ++q) I[q] = q < o.k ? (int)Is[q * RT_SIGS] : 0;
#pragma unroll
  for (int q = 0; q < RT_SMAX; ++q) {
    if (q < o.k) {
      int rank = 0;
#pragma unroll
      for (int t = 0; t < RT_SMAX; ++t) rank += (t < o.k && I[t] < I[q]) ? 1 : 0;
      oidx[base + rank] = I[q];
      oval[base + rank] = gms[q * RT_SIGS];
    } else if (q < s) {
      oidx[base + q] = -1;
      oval[base + q] = 0.f;
    }
  }
  ocnt[i] = o.k;
}

// Bounded wait that also gives up as soon as another thread has recorded a
// failure; a timeout records one.
__device__ __forceinline__ bool wait_or_fail(uint64_t* bar, uint32_t parity, volatile int* fail) {
  const uint64_t t0 = gtimer();
  while (!mbar_try_wait(bar, parity)) {
    if (*fail) return false;
    if (gtimer() - t0 > kWaitNs) {
      *fail = 1;
      return false;
    }
  }
  return true;
}

// This half's sweep of one accumulator unit: its 128 columns (atoms 256 h +
// 128 hf ..) as eight 16-column chunks in ascending order, keeping the running
// best key and its chunk (global chunk index; the lowest chunk wins equal
// keys).  Warp-collective: every lane executes it.
__device__ __forceinline__ void sweep_half(uint32_t ta, int h, int hf, float& best, int& bc) {
  constexpr int NC = RT_N / RT_HALVES / 16;
  const int cb = 16 * h + NC * hf;
  // tcgen05.wait::ld waits for all of the thread's loads: the next chunk's
  // load is issued before the current chunk's keys and waited for after them
  uint32_t va[16], vb[16];
  tm_ld16(ta, va);
  tm_wait16(va);
#pragma unroll
  for (int c = 0; c < NC; c += 2) {
    tm_ld16(ta + 16 * (c + 1), vb);
    const float k0 = chunk_key(va);
    if (k0 > best) { best = k0; bc = cb + c; }
    tm_wait16(vb);
    if (c + 2 < NC) tm_ld16(ta + 16 * (c + 2), va);
    const float k1 = chunk_key(vb);
    if (k1 > best) { best = k1; bc = cb + c + 1; }
    if (c + 2 < NC) tm_wait16(va);
  }
}

// Pair exchange record of one half of a signal.
struct Xch {
  float key;   // best argmax key of the half's columns (-2: failed wait)
  int chunk;   // its chunk
  float dot;   // half 1: its part of d_sel^T r; both: their parts of ||y||^2
  float nrm;   // the half's part of ||r^(k+1)||^2
  int more;    // lead: the Cholesky step's outcome (1: update and go on)
};

template <bool BF>
__global__ void __launch_bounds__(RT_THREADS, 1)
    romp_kernel(const float* __restrict__ Y, int64_t m, int p, const float* __restrict__ D, int n,
                const float* __restrict__ G, int s, int32_t* __restrict__ oidx,
                float* __restrict__ oval, int32_t* __restrict__ ocnt, int* __restrict__ err,
                int* __restrict__ rs_list, int* __restrict__ rs_count, int rs_cap) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(base + RtSmem::bars);
  uint32_t* tmem_slot = (uint32_t*)(base + RtSmem::misc);
  volatile int* fail = (volatile int*)(tmem_slot + 1);
  unsigned* dmax = (unsigned*)(tmem_slot + 2);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nh = n > RT_N ? 2 : 1;
  const int64_t ntiles = (m + RT_M - 1) / RT_M;
  const int64_t grid = gridDim.x, b = blockIdx.x;
  const int64_t ntb = b < ntiles ? (ntiles - 1 - b) / grid + 1 : 0;  // tiles of this CTA
  const int rounds = (int)((ntb + RT_NS - 1) / RT_NS);

  if (threadIdx.x == 0) {
    *fail = 0;
    *dmax = 0u;
    for (int u = 0; u < 2; ++u) {
      mbar_init(&bars[RB_TFULL + u], 1);
      mbar_init(&bars[RB_TEMPTY + u], 4 * RT_HALVES);  // the slot's warps
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(2 * RT_N)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  __syncthreads();

  // ---- D 2^eD as FP16 parts, rows padded with zeros to 256 nh atoms x 64
  {
    float mx = 0.f;
    for (int e = threadIdx.x; e < n * p; e += RT_THREADS) mx = fmaxf(mx, fabsf(__ldg(D + e)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(omp::FULL, mx, o));
    if (lane == 0) atomicMax(dmax, __float_as_uint(mx));  // non-negative floats order as integers
  }
  __syncthreads();
  float dsc = 1.f;  // 2^-eD
  {
    const float dm = __uint_as_float(*dmax);
    int E = 0;
    frexpf(dm, &E);
    const bool scaled = dm > 0.f && isfinite(dm);
    const float sc = scaled ? pow2i(14 - E) : 1.f;  // max |D| 2^eD < 2^14
    dsc = scaled ? pow2i(E - 14) : 1.f;
    for (int u = threadIdx.x; u < nh * RT_N * 8; u += RT_THREADS) {
      const int j = u >> 3, g = u & 7;
      float v[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int c = 8 * g + e;
        v[e] = (j < n && c < p) ? __ldg(D + (size_t)j * p + c) * sc : 0.f;
      }
      uint32_t h[4], l[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        if constexpr (BF) {  // top / bottom 16 bits of each FP32 value
          const uint32_t b0 = __float_as_uint(v[2 * e]), b1 = __float_as_uint(v[2 * e + 1]);
          h[e] = __byte_perm(b0, b1, 0x7632);
          l[e] = __byte_perm(b0, b1, 0x5410);
        } else {
          split2(v[2 * e], v[2 * e + 1], h[e], l[e]);
        }
      }
      *reinterpret_cast<uint4*>(base + RtSmem::dh + sw_off(j, g)) = make_uint4(h[0], h[1], h[2], h[3]);
      *reinterpret_cast<uint4*>(base + RtSmem::dl + sw_off(j, g)) = make_uint4(l[0], l[1], l[2], l[3]);
    }
  }
  fence_async_smem();  // generic-proxy writes -> the tensor core's reads
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  {
    // ---------------- owners: two threads (halves) per signal ----------------
    const int sl = warp >> 3, hf = (warp >> 2) & 1, quad = warp & 3, row = quad * 32 + lane;
    const bool issuer = hf == 0 && quad == 0 && lane == 0;
    const bool lead = hf == 0;  // the half that runs the Cholesky step and writes the results
    const int pair_bar = 1 + RT_NS + sl * 4 + quad;  // the quad's two warps
    const int sig = sl * RT_M + row;                 // the signal's scratch column
    const uint32_t tl = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(hf * (RT_N / 2));
    uint8_t* Ah = base + RtSmem::a + sl * RtSmem::a_slot;
    uint8_t* Al = Ah + RtSmem::a_part;
    const uint8_t* Dh = base + RtSmem::dh;
    const uint8_t* Dl = base + RtSmem::dl;
    uint16_t* Is = (uint16_t*)(base + RtSmem::is) + sig;
    float* dgs = (float*)(base + RtSmem::dg) + sig;
    float* gms = (float*)(base + RtSmem::gm) + sig;
    Xch* xme = (Xch*)(base + RtSmem::xch) + sig * RT_HALVES + hf;
    const Xch* xpa = (const Xch*)(base + RtSmem::xch) + sig * RT_HALVES + (hf ^ 1);
    // Per step the halves meet at the slot barrier and at four pair barriers:
    // X1 (argmax keys), X2 (half 1's part of alpha_sel), X4 (the lead's
    // Cholesky outcome) and X3 (the parts of ||r||^2).  An exchange field is
    // rewritten only after a barrier that the reader passes after reading it.
    // After a failed wait (*fail set) the loops still run to their end with the
    // work skipped, so that the warps of a slot and the two halves of a signal
    // always meet at the same named barriers.
    for (int j = 0; j < rounds; ++j) {
      const int64_t v = (int64_t)j * RT_NS + sl;
      if (v >= ntb) break;  // this slot has no tile in the CTA's last round (slot-uniform)
      const int aj = (int)(ntb - (int64_t)j * RT_NS < RT_NS ? ntb - (int64_t)j * RT_NS : RT_NS);
      const int64_t i = (b + v * grid) * RT_M + row;
      Owner o;
      o.active = i < m;
      o.k = 0;
      {
        const float* yp = Y + (size_t)(o.active ? i : 0) * p;
#pragma unroll
        for (int u = 0; u < RT_PH / 8; ++u) {
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            const int c = 8 * (2 * u + hf) + 4 * q;
            const float4 t = (o.active && c < p) ? __ldg(reinterpret_cast<const float4*>(yp + c))
                                                 : make_float4(0.f, 0.f, 0.f, 0.f);
            o.r[4 * u + 2 * q] = make_float2(t.x, t.y);
            o.r[4 * u + 2 * q + 1] = make_float2(t.z, t.w);
          }
        }
      }
      if (lead) {
#pragma unroll
        for (int q = 0; q < RT_SMAX; ++q) gms[q * RT_SIGS] = 0.f;
      }
      {  // ||y||^2: the halves' parts (a sum of two terms: the same in both halves),
         // through the dot fields, which were last read before the previous X4
        const float mine = owner_norm2(o);
        xme->dot = mine;
        asm volatile("bar.sync %0, %1;" ::"r"(pair_bar), "r"(64) : "memory");
        o.yy = o.rr = o.rn = mine + xpa->dot;
      }
      if (!isfinite(o.yy)) {
        if (lead) atomicOr(err, ERR_NONFINITE);
        o.active = false;
#pragma unroll
        for (int e = 0; e < RT_PH / 2; ++e) o.r[e] = make_float2(0.f, 0.f);
        o.rn = 0.f;
      }
      for (int step = 0; step < s; ++step) {
        if (step == 0 || o.active) owner_store<BF>(o, hf, Ah, Al, row);
        fence_async_smem();  // the residual rows -> the tensor core's reads
        asm volatile("bar.sync %0, %1;" ::"r"(1 + sl), "r"(32 * 4 * RT_HALVES) : "memory");
        const int u = j * s * RT_NS + step * aj + sl;  // this use's place in the fixed order
        if (issuer && !*fail) {
          const uint64_t dhd = sw128_desc(base + RtSmem::dh), dld = sw128_desc(base + RtSmem::dl);
          const uint64_t ahd = sw128_desc(Ah), ald = sw128_desc(Al);
          for (int h = 0; h < nh; ++h) {
            const int hc = u * nh + h, unit = hc & 1;
            if (hc >= 2 && !wait_or_fail(&bars[RB_TEMPTY + unit], (uint32_t)(((hc >> 1) - 1) & 1), fail))
              break;
            tc_fence_after();
            const uint32_t dcol = tmem + (uint32_t)(unit * RT_N);
            const uint64_t boff = (uint64_t)((h * RT_N * RT_ROWB) >> 4);
            const uint64_t bh = dhd + boff, bl = dld + boff;
            if constexpr (BF) {  // one product of BF16 operands
#pragma unroll
              for (int kk = 0; kk < 4; ++kk)  // 16 elements = 32 bytes of K per MMA
                mma_f16(dcol, ahd + (uint64_t)(2 * kk), bh + (uint64_t)(2 * kk), RT_IDESC_BF,
                        kk > 0 ? 1u : 0u);
            } else {
              // the two correction products first, then the leading one
#pragma unroll
              for (int kk = 0; kk < 4; ++kk)  // 16 FP16 = 32 bytes of K per MMA
                mma_f16(dcol, ald + (uint64_t)(2 * kk), bh + (uint64_t)(2 * kk), RT_IDESC,
                        kk > 0 ? 1u : 0u);
#pragma unroll
              for (int kk = 0; kk < 4; ++kk)
                mma_f16(dcol, ahd + (uint64_t)(2 * kk), bl + (uint64_t)(2 * kk), RT_IDESC, 1u);
#pragma unroll
              for (int kk = 0; kk < 4; ++kk)
                mma_f16(dcol, ahd + (uint64_t)(2 * kk), bh + (uint64_t)(2 * kk), RT_IDESC, 1u);
            }
            mma_commit(&bars[RB_TFULL + unit]);
          }
        }
        __syncwarp();
        float best = -1.f;
        int bc = 0;
        bool good = true;
        for (int h = 0; h < nh; ++h) {
          const int hc = u * nh + h, unit = hc & 1;
          bool w = good && !*fail;
          if (w && hc >= 2) w = wait_or_fail(&bars[RB_TEMPTY + unit], (uint32_t)(((hc >> 1) - 1) & 1), fail);
          if (w) w = wait_or_fail(&bars[RB_TFULL + unit], (uint32_t)((hc >> 1) & 1), fail);
          good = __all_sync(omp::FULL, w);
          if (!good) continue;
          tc_fence_after();
          sweep_half(tl + (uint32_t)(unit * RT_N), h, hf, best, bc);
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&bars[RB_TEMPTY + unit]);
        }
        // X1: the halves' best keys; equal keys go to the lower chunk
        xme->key = good ? best : -2.f;
        xme->chunk = bc;
        asm volatile("bar.sync %0, %1;" ::"r"(pair_bar), "r"(64) : "memory");
        {
          const float pk = xpa->key;
          const int pc = xpa->chunk;
          good = good && pk > -1.5f;
          if (pk > best || (pk == best && pc < bc)) {
            best = pk;
            bc = pc;
          }
        }
        bool pick = good && o.active;
        int sel = 0;
        if (pick) {
          const uint32_t kb = __float_as_uint(best);
          sel = 16 * bc + 15 - (int)(kb & 15u);
          if ((kb & 0x7FFFFFF0u) == 0u || sel >= n) {
            o.active = false;  // max |alpha| = 0
            pick = false;
          }
        }
        float gss = 0.f, dpart = 0.f;
        float g[RT_SMAX];
        if (pick) {
          if (lead) {  // the Gram entries first: their latency overlaps the dot product
            gss = __ldg(G + (size_t)sel * n + sel);
#pragma unroll
            for (int q = 0; q < RT_SMAX; ++q)
              g[q] = q < step ? __ldg(G + (size_t)Is[q * RT_SIGS] * n + sel) : 0.f;
          }
          dpart = owner_dot<BF>(o, sel, hf, Dh, Dl);
        }
        // X2: half 1's part of alpha_sel to the lead
        if (!lead) xme->dot = dpart;
        asm volatile("bar.sync %0, %1;" ::"r"(pair_bar), "r"(64) : "memory");
        bool more = false;
        if (pick && lead) {
          const float asel = (dpart + xpa->dot) * dsc;
          switch (step) {
#define DL_ROMP_STEP(S)                                                                    \
  case S:                                                                                  \
    more = owner_chol<S>(o, sel, asel, gss, g, Is, dgs, gms, s, i, err, rs_list, rs_count, \
                         rs_cap);                                                          \
    break;
            DL_ROMP_STEP(0) DL_ROMP_STEP(1) DL_ROMP_STEP(2) DL_ROMP_STEP(3)
            DL_ROMP_STEP(4) DL_ROMP_STEP(5) DL_ROMP_STEP(6) DL_ROMP_STEP(7)
#undef DL_ROMP_STEP
            default: break;
          }
          xme->more = more ? 1 : 0;
        }
        // X4: the lead's Cholesky outcome (and its scratch writes) to half 1
        asm volatile("bar.sync %0, %1;" ::"r"(pair_bar), "r"(64) : "memory");
        if (pick && !lead) {
          more = xpa->more != 0;
          o.active = more;
        }
        float npart = 0.f;
        if (more) npart = owner_update<BF>(o, step, hf, Is, dgs, Dh, Dl, dsc);
        if (!good) o.active = false;
        // X3: ||r^(k+1)||^2 from the halves' parts
        xme->nrm = npart;
        asm volatile("bar.sync %0, %1;" ::"r"(pair_bar), "r"(64) : "memory");
        if (more) o.rn = npart + xpa->nrm;
      }
      if (lead && !*fail && i < m) owner_write(o, Is, gms, i, s, oidx, oval, ocnt);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * RT_N)
                 : "memory");
  }
  if (threadIdx.x == 0 && *fail) atomicOr(err, ERR_TIMEOUT);
}

}  // namespace

int64_t omp_res_round_signals() { return (int64_t)num_sms() * RT_NS * RT_M; }

bool omp_res_supported(int p, int n, int s, const float* Y, const float* D) {
  return p >= 4 && p <= RT_PMAX && p % 4 == 0 && n >= 1 && n <= RT_NMAX && s >= 1 &&
         s <= RT_SMAX && s <= n && ((uintptr_t)Y % 16) == 0 && ((uintptr_t)D % 16) == 0;
}

cudaError_t omp_res(const float* Y, int64_t m, int p, const float* D, int n, const float* G, int s,
                    int32_t* idx, float* val, int32_t* cnt, int* err, int* rs_list, int* rs_count,
                    int rs_cap, bool bf16, cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  auto kern = bf16 ? romp_kernel<true> : romp_kernel<false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)RtSmem::dyn);
  if (e != cudaSuccess) return e;
  const int64_t ntiles = (m + RT_M - 1) / RT_M;
  const int grid = (int)(ntiles < num_sms() ? ntiles : num_sms());
  kern<<<grid, RT_THREADS, RtSmem::dyn, st>>>(Y, m, p, D, n, G, s, idx, val, cnt, err, rs_list,
                                              rs_count, rs_cap);
  return cudaGetLastError();
}

}  // namespace dlk
