// C ABI of the library (include/dl_gb300.h): argument validation, workspace,
// host staging, and the per-iteration launch sequence (captured once into a
// CUDA graph and replayed).
#include "../../include/dl_gb300.h"
#include "dl_internal.cuh"

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

// The learned support proposer (MLP p -> hidden -> hidden -> n, BF16 weights
// with FP32 masters and Adam state; see k_mlp.cu).
struct dl_proposer {
  int dev = 0, p = 0, pk = 0, n = 0, hidden = 0;
  int64_t bmax = 0;        // rows per training batch
  int64_t ichunk = 0;      // rows per inference chunk (activations stay in L2)
  cudaStream_t st = nullptr;
  float* w[6] = {};        // W1 (hidden x pk), b1, W2 (hidden x hidden), b2, W3 (n x hidden), b3
  float* g[6] = {};        // gradients of the last training step
  float* am[6] = {};       // Adam first moments
  float* av[6] = {};       // Adam second moments
  int64_t wlen[6] = {};
  void* wb[3] = {};        // BF16 copies of W1, W2, W3
  void* wt[2] = {};        // BF16 transposes of W2 (hidden x hidden) and W3 (hidden x n)
  // activations (bmax rows)
  void* X = nullptr;       // BF16 bmax x pk
  float* A1 = nullptr;     // FP32 pre-activations (training)
  float* A2 = nullptr;
  void* H1 = nullptr;      // BF16 activations
  void* H2 = nullptr;
  float* Z = nullptr;      // FP32 logits (training)
  void* Zb = nullptr;      // BF16 logits (inference)
  int32_t* sup = nullptr;  // gathered supports of the batch (bmax x 16)
  // backward scratch (BF16)
  void *dZ = nullptr, *dZt = nullptr, *H2t = nullptr, *dA2 = nullptr, *dA2t = nullptr, *H1t = nullptr,
       *dA1 = nullptr, *dA1t = nullptr, *Xt = nullptr;
  double* loss = nullptr;
  int* err = nullptr;
  int step = 0;
};

struct dl_ctx {
  int dev = 0;
  int p = 0, n = 0, s_max = 0, precision = 0;
  int64_t m_max = 0;
  cudaStream_t st = nullptr;
  int64_t lda = 0;  // row stride of the correlation matrix A0 (floats)
  // workspace
  float* G = nullptr;
  float* A0 = nullptr;
  int jau_kernels = 5;   // kernel launches of the last enqueued JAU update
  int ntilde = 0;        // group size of the atom update (0 or n: all atoms at once)
  int rule = DL_RULE_AKSVD;  // atom update rule
  // P-NSGK: the representations of the previous iteration (slots), a device
  // flag telling whether they exist yet, and the dictionary an iteration starts from
  int32_t* pidx = nullptr;
  float* pval = nullptr;
  int32_t* pcnt = nullptr;
  int* pvalid = nullptr;
  float* D0 = nullptr;
  int omp_kernels[2] = {5, 5};  // ... of the last enqueued coding pass (plain, learned)
  float* Dhi = nullptr;  // TF32 head / tail of D for the tensor-core correlations
  float* Dlo = nullptr;
  // reduced-precision correlations (precision DL_BF16 / DL_FP8)
  int lp_kind = 0;        // 0 = FP32 path, dlk::LP_BF16, dlk::LP_E4M3
  void* Ylp = nullptr;    // m_max x lp_row_elems, converted once per call
  float* Ysc = nullptr;   // per-signal inverse scales (E4M3)
  void* Dlp = nullptr;    // n x lp_row_elems, converted per iteration
  float* Dsc = nullptr;   // per-atom inverse scales (E4M3)
  // FP64 re-solve of signals whose FP32 pivot fell below 1e-6
  int* rs_list = nullptr;
  int* rs_count = nullptr;
  int64_t rs_flagged = 0;  // total flagged (read back at synchronising calls)
  // learned proposer attached (dl_attach_proposer)
  dl_proposer* prop = nullptr;
  int prop_K = 0, prop_full_every = 10;
  float prop_tol2 = 1.0201f;
  int64_t prop_counter = 0;
  float* rr_ref = nullptr;   // residual energy of the last full OMP of each signal
  float* rr_L = nullptr;     // residual energy of the restricted OMP
  int* fb_list = nullptr;
  int* fb_count = nullptr;
  int32_t* cand = nullptr;   // m_max x K
  void* Ybf = nullptr;       // m_max x pk BF16 copy of Y for the proposer
  bool learned_now = false;  // the iteration being enqueued uses the proposer
  bool prop_corr = false;    // network-free proposer: the K largest |D^T y| (no MLP)
  bool a0_bf16 = false;      // the coding pass stores alpha0 in BF16 (BF16 form, TMEM OMP)
  cudaGraphExec_t gexec_learned = nullptr;
  int32_t* sidx = nullptr;
  float* sval = nullptr;
  int32_t* scnt = nullptr;
  int64_t* bsum = nullptr;
  int* err = nullptr;
  int* iter = nullptr;
  double* rmse = nullptr;
  int rmse_cap = 0;  // iterations
  dlk::JauWork jw{};
  // host staging (lazily allocated)
  float* hY = nullptr;
  float* hD = nullptr;
  int64_t* hcolptr = nullptr;
  int32_t* hrowidx = nullptr;
  float* hval = nullptr;
  // graph cache for one DL iteration
  cudaGraphExec_t gexec = nullptr;
  const void* gkey[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  int64_t gkey_m = -1;
  int gkey_s = -1;
  int gkey_seen = 0;
  int gkey_seen_l = 0;
  // graph of one whole host-buffer call (upload of D, the staged iteration with
  // its upload of Y, downloads of D and X), keyed by the host pointers, m, s and
  // every setting that changes what is enqueued
  cudaGraphExec_t hgexec = nullptr;
  const void* hkey[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  int64_t hkey_m = -1;
  int hkey_s = -1;
  int64_t hsig[11] = {};
  int hseen = 0;
  int hg_kernels = 0;
  int64_t launches = 0;
  // launch shapes (chosen by dl_autotune; defaults otherwise)
  int cfg_omp_warps = 4;  // warps per CTA of the OMP kernel
  int cfg_omp_tm = 5;     // warps per TMEM quadrant of the TMEM-resident OMP kernel (0: off)
  int cfg_omp_res = 1;    // residual-form OMP with per-step tensor-core correlations (0: off)
  int last_omp = -1;      // the coding kernel of the last pass (dl_last_omp_kernel)
  int deterministic = 0;  // pass A with a fixed summation order (dl_set_deterministic)
  int cfg_acc_mult = 1;   // accumulation CTAs: 1x or 2x the base count
  int cfg_row_per_sm = 4; // row-update CTAs per SM
  int cfg_corr_tc = 1;    // tensor-core correlations when the shape allows
  // side stream: the colptr scan overlaps the first pass of the atom update
  cudaStream_t st2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_join2 = nullptr;
  int scan_kernels = 2;  // side-stream kernels of the last iteration (colptr scan, rowidx)
  // host-buffer calls: the signals arrive in chunks on the side stream
  static constexpr int kChunks = 3;
  cudaEvent_t ev_chunk[kChunks] = {};
  // optional per-phase timing with CUDA events recorded on the context's stream
  bool prof = false;
  cudaEvent_t ev[9] = {};
  double phase_ms[8] = {};
  int64_t phase_count = 0;
};

namespace {

constexpr int kKernelsScan = 2;      // colptr scan

void free_ctx(dl_ctx* c) {
  if (!c) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(c->dev);
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->gexec_learned) cudaGraphExecDestroy(c->gexec_learned);
  if (c->hgexec) cudaGraphExecDestroy(c->hgexec);
  for (void* q : {(void*)c->rr_ref, (void*)c->rr_L, (void*)c->fb_list, (void*)c->fb_count,
                  (void*)c->cand, c->Ybf})
    if (q) cudaFree(q);
  for (cudaEvent_t e : c->ev)
    if (e) cudaEventDestroy(e);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  for (cudaEvent_t e : c->ev_chunk)
    if (e) cudaEventDestroy(e);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->ev_join2) cudaEventDestroy(c->ev_join2);
  if (c->st2) cudaStreamDestroy(c->st2);
  void* ptrs[] = {c->G, c->A0, c->Dhi, c->Dlo, c->Ylp, c->Ysc, c->Dlp, c->Dsc, c->rs_list,
                  c->rs_count, c->sidx, c->sval, c->scnt, c->bsum, c->err, c->iter, c->rmse,
                  c->jw.Upart, c->jw.U, c->jw.epart_a, c->jw.epart_b, c->jw.Dn, c->jw.C,
                  c->hY, c->hD, c->hcolptr, c->hrowidx, c->hval, c->pidx, c->pval, c->pcnt,
                  c->pvalid, c->D0};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  cudaSetDevice(prev);
  delete c;
}

template <typename T>
bool dalloc(T** out, size_t count) {
  if (count == 0) count = 1;
  return cudaMalloc((void**)out, sizeof(T) * count) == cudaSuccess;
}

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return DL_OK;
  if (e == cudaErrorMemoryAllocation) return DL_ENOMEM;
  return DL_ECUDA;
}

#define DL_CHECK(expr)                   \
  do {                                   \
    cudaError_t e_ = (expr);             \
    if (e_ != cudaSuccess) return cuda_status(e_); \
  } while (0)

struct DevGuard {
  int prev = 0;
  explicit DevGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DevGuard() {
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != prev) cudaSetDevice(prev);
  }
};

// 1 = device (or managed) memory, 0 = host memory, -1 = null
int ptr_kind(const void* p) {
  if (!p) return -1;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) ? 1 : 0;
}

// Read and clear the device error word; returns a status.
int take_device_error(dl_ctx* c) {
  int h = 0;
  DL_CHECK(cudaMemcpyAsync(&h, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  DL_CHECK(cudaStreamSynchronize(c->st));
  if (h) DL_CHECK(cudaMemsetAsync(c->err, 0, sizeof(int), c->st));
  if (h & dlk::ERR_CSC) return DL_EINVAL;
  if (h & dlk::ERR_NONFINITE) return DL_ENUMERIC;
  if (h & dlk::ERR_TIMEOUT) return DL_ETIMEOUT;
  return DL_OK;
}

int ensure_rmse(dl_ctx* c, int iters) {
  if (iters <= c->rmse_cap) return DL_OK;
  DL_CHECK(cudaStreamSynchronize(c->st));
  if (c->rmse) cudaFree(c->rmse);
  c->rmse = nullptr;
  c->rmse_cap = 0;
  int cap = iters < 64 ? 64 : iters;
  if (!dalloc(&c->rmse, (size_t)2 * cap)) return DL_ENOMEM;
  c->rmse_cap = cap;
  return DL_OK;
}

int ensure_staging(dl_ctx* c) {
  if (c->hY) return DL_OK;
  const size_t m = (size_t)c->m_max;
  if (!dalloc(&c->hY, m * c->p) || !dalloc(&c->hD, (size_t)c->n * c->p) ||
      !dalloc(&c->hcolptr, m + 1) || !dalloc(&c->hrowidx, m * c->s_max) ||
      !dalloc(&c->hval, m * c->s_max))
    return DL_ENOMEM;
  return DL_OK;
}

// Phase boundaries for optional timing: 0 gram | 1 correlations | 2 omp | 3 colptr scan |
// 4 accumulate+reduce | 5 atoms | 6 rows | 7 finalize+copy | 8
// Inside stream capture the record becomes an external event node of the graph.
void mark(dl_ctx* c, int k) {
  if (!c->prof) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(c->st, &cs);
  if (cs == cudaStreamCaptureStatusActive)
    cudaEventRecordWithFlags(c->ev[k], c->st, cudaEventRecordExternal);
  else
    cudaEventRecord(c->ev[k], c->st);
}

// ---- enqueue helpers (no synchronisation) --------------------------------------
// The tensor-core path needs p % 4 == 0, p <= 64, n <= 1024 and 16-byte aligned operands;
// other shapes use the FP32 CUDA-core GEMM.
bool tc_ok(dl_ctx* c, const float* Y, const float* D) {
  if (getenv("DL_FORCE_SIMT_GEMM") || !c->cfg_corr_tc) return false;
  return dlk::corr_tc_supported(Y, c->p, c->n, c->lda) &&
         dlk::corr_tc_supported(D, c->p, c->n, c->n);
}

cudaError_t enq_gram(dl_ctx* c, const float* D, bool tc) {
  if (!tc) return dlk::gemm_nt_simt(D, c->n, D, c->n, c->p, c->G, c->n, c->st);
  cudaError_t e = dlk::split_tf32(D, (int64_t)c->n * c->p, c->Dhi, c->Dlo, c->st);
  if (e != cudaSuccess) return e;
  return dlk::corr_tf32x3(D, c->n, c->Dhi, c->Dlo, c->n, c->p, c->G, c->n, c->err, c->st);
}

bool lp_ok(dl_ctx* c) { return c->lp_kind != 0 && dlk::corr_lp_supported(c->lp_kind, c->p, c->n, c->lda); }

// BF16 correlations straight from FP32 Y (converted on chip by the pipelined kernel).
bool lp_ws(dl_ctx* c, const float* Y) {
  return lp_ok(c) && c->lp_kind == dlk::LP_BF16 &&
         dlk::corr_bf16_ws_supported(Y, c->p, c->n, c->lda);
}

// Y converted to the reduced-precision format (once per call, before any iteration),
// unless the correlation kernel reads it in FP32.
bool needs_y_conversion(dl_ctx* c, const float* Y) { return lp_ok(c) && !lp_ws(c, Y); }
cudaError_t enq_convert_y(dl_ctx* c, const float* Y, int64_t m) {
  if (!needs_y_conversion(c, Y)) return cudaSuccess;
  return dlk::to_lowp(c->lp_kind, Y, m, c->p, c->Ylp, c->Ysc, c->st);
}

cudaError_t enq_corr(dl_ctx* c, const float* Y, int64_t m, const float* D, bool tc) {
  if (lp_ok(c)) {
    cudaError_t e = dlk::to_lowp(c->lp_kind, D, c->n, c->p, c->Dlp, c->Dsc, c->st);
    if (e != cudaSuccess) return e;
    if (lp_ws(c, Y))
      return dlk::corr_bf16_ws(Y, m, c->Dlp, c->n, c->p, c->A0, c->a0_bf16, c->lda, c->err, c->st);
    return dlk::corr_lp(c->lp_kind, c->Ylp, m, c->Ysc, c->Dlp, c->Dsc, c->n, c->p, c->A0, c->lda,
                        c->err, c->st);
  }
  if (!tc) return dlk::gemm_nt_simt(Y, m, D, c->n, c->p, c->A0, c->lda, c->st);
  return dlk::corr_tf32x3(Y, m, c->Dhi, c->Dlo, c->n, c->p, c->A0, c->lda, c->err, c->st);
}

cudaError_t enq_proposer_forward(dl_proposer* P, const void* Xbf, int64_t m, int K, int32_t* cand,
                                 cudaStream_t st);
int64_t proposer_chunks(dl_proposer* P, int64_t m);
// A support proposer is attached: the learned one or the network-free one.
bool has_prop(const dl_ctx* c) { return c->prop != nullptr || c->prop_corr; }

// Sparse coding with the learned proposer: top-K candidates from the MLP,
// OMP restricted to them, full OMP for the signals whose residual energy
// exceeds tol2 times the one of their last full OMP.
cudaError_t enq_omp_learned(dl_ctx* c, const float* Y, int64_t m, const float* D, int s, bool tc) {
  cudaError_t e;
  c->last_omp = 3;
  if (c->prop_corr) {
    // network-free proposer: the correlations of all signals first, then the K
    // largest |alpha0| of each
    c->omp_kernels[1] = (tc ? 2 : 1) /* Gram */ + (lp_ok(c) ? 2 : 1) /* correlations */ +
                        1 /* top-K */ + 3 /* restricted, listed, re-solve */;
    if ((e = enq_corr(c, Y, m, D, tc)) != cudaSuccess) return e;
    if ((e = dlk::topk_abs(c->A0, c->lda, m, c->n, c->prop_K, c->cand, c->st)) != cudaSuccess)
      return e;
  } else {
    c->omp_kernels[1] = (tc ? 2 : 1) /* Gram */ + 4 * (int)proposer_chunks(c->prop, m) /* 3 GEMMs +
        top-K per chunk */ + 3 /* restricted, listed, re-solve */ + (lp_ok(c) ? 2 : 1) /* correlations */;
    e = enq_proposer_forward(c->prop, c->Ybf, m, c->prop_K, c->cand, c->st);
    if (e != cudaSuccess) return e;
  }
  mark(c, 2);
  if ((e = cudaMemsetAsync(c->fb_count, 0, sizeof(int), c->st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(c->rs_count, 0, sizeof(int), c->st)) != cudaSuccess) return e;
  e = dlk::omp_restricted(c->cand, c->prop_K, D, c->G, c->n, Y, c->p, m, s, c->sidx, c->sval,
                          c->scnt, c->rr_L, c->rr_ref, c->prop_tol2, c->fb_list, c->fb_count, c->err,
                          c->st);
  if (e != cudaSuccess) return e;
  // the fallback signals read their correlations from the tensor-core product of all signals
  if (!c->prop_corr && (e = enq_corr(c, Y, m, D, tc)) != cudaSuccess) return e;
  e = dlk::omp_listed(c->fb_list, c->fb_count, c->A0, c->lda, c->G, c->n, Y, c->p, s, c->sidx,
                      c->sval, c->scnt, c->rr_ref, c->err, c->rs_list, c->rs_count, (int)c->m_max,
                      c->st);
  if (e != cudaSuccess) return e;
  e = dlk::omp_resolve64(Y, c->p, D, c->G, lp_ok(c) ? nullptr : c->A0, c->lda, c->n, s,
                         c->rs_list, c->rs_count, (int)c->m_max, c->sidx, c->sval, c->scnt, c->st);
  mark(c, 3);
  return e;
}

// The residual-form OMP (correlations of every step on the tensor cores, no
// alpha0 pass) codes a plain FP32 or BF16 call without a proposer when it is
// supported and, in the automatic mode, when n > 256 and the call has at least
// three quarters of one round of tiles (both slots of most SMs busy): at
// n = 256, or with about one tile per SM (p = 64, n = 512, m = 20000: 96
// against 90 us for Gram, correlations and the TMEM Batch-OMP), the Batch-OMP
// forms are as fast or faster.  Mode 2 (DL_OMP_RES=2) takes it for every
// supported call.  The E4M3 form keeps its alpha0 pass.
bool use_res(dl_ctx* c, const float* Y, const float* D, int s, int64_t m) {
  if (!c->cfg_omp_res || has_prop(c) || c->precision == DL_FP8 ||
      !dlk::omp_res_supported(c->p, c->n, s, Y, D))
    return false;
  return c->cfg_omp_res == 2 || (c->n > 256 && 4 * m >= 3 * dlk::omp_res_round_signals());
}

cudaError_t enq_omp_res(dl_ctx* c, const float* Y, int64_t m, const float* D, int s) {
  c->a0_bf16 = false;
  mark(c, 0);
  cudaError_t e = dlk::gram_simt(D, c->n, c->p, c->G, c->st);  // G for the Cholesky rows
  if (e != cudaSuccess) return e;
  mark(c, 1);
  mark(c, 2);
  if ((e = cudaMemsetAsync(c->rs_count, 0, sizeof(int), c->st)) != cudaSuccess) return e;
  c->last_omp = 2;
  e = dlk::omp_res(Y, m, c->p, D, c->n, c->G, s, c->sidx, c->sval, c->scnt, c->err, c->rs_list,
                   c->rs_count, (int)c->m_max, c->precision == DL_BF16, c->st);
  if (e != cudaSuccess) return e;
  e = dlk::omp_resolve64(Y, c->p, D, c->G, nullptr, c->lda, c->n, s, c->rs_list, c->rs_count,
                         (int)c->m_max, c->sidx, c->sval, c->scnt, c->st);
  c->omp_kernels[0] = 3;  // Gram, OMP, FP64 re-solve
  mark(c, 3);
  return e;
}

cudaError_t enq_omp(dl_ctx* c, const float* Y, int64_t m, const float* D, int s) {
  if (use_res(c, Y, D, s, m)) return enq_omp_res(c, Y, m, D, s);
  const bool tc = tc_ok(c, Y, D);
  const bool learned = has_prop(c) && c->learned_now;
  // BF16 form: alpha0 is only as accurate as BF16 anyway, so it is stored in BF16
  // (half the write) when the TMEM OMP reads it
  c->a0_bf16 = lp_ws(c, Y) && c->cfg_omp_tm && !has_prop(c) && dlk::omp_tm_supported(c->n, s);
  mark(c, 0);
  cudaError_t e;
  if (tc && !learned && !lp_ok(c)) {
    // one launch computes the Gram matrix and the correlations of all signals
    if ((e = dlk::split_tf32(D, (int64_t)c->n * c->p, c->Dhi, c->Dlo, c->st)) != cudaSuccess) return e;
    mark(c, 1);
    e = dlk::corr_tf32x3_pair(Y, m, c->A0, c->lda, D, c->n, c->G, c->n, c->Dhi, c->Dlo, c->n, c->p,
                              c->err, c->st);
    if (e != cudaSuccess) return e;
    c->omp_kernels[0] = 2 /* split, products */ + 2 /* OMP, FP64 re-solve */;
  } else {
    if ((e = enq_gram(c, D, tc)) != cudaSuccess) return e;
    mark(c, 1);
    if (learned) return enq_omp_learned(c, Y, m, D, s, tc);
    if ((e = enq_corr(c, Y, m, D, tc)) != cudaSuccess) return e;
    c->omp_kernels[0] = (tc ? 2 : 1) + (lp_ok(c) ? 2 : 1) + 2;
  }
  mark(c, 2);
  e = cudaMemsetAsync(c->rs_count, 0, sizeof(int), c->st);
  if (e != cudaSuccess) return e;
  const bool tm = c->cfg_omp_tm && !has_prop(c) && dlk::omp_tm_supported(c->n, s);
  c->last_omp = tm ? 1 : 0;
  if (tm)
    e = dlk::omp_batch_tm(c->cfg_omp_tm, c->A0, c->a0_bf16, c->lda, c->G, c->n, Y, c->p, m, s, c->sidx, c->sval,
                          c->scnt, c->err, c->rs_list, c->rs_count, (int)c->m_max, c->st);
  else
    e = dlk::omp_batch(c->A0, c->lda, c->G, c->n, Y, c->p, m, s, c->sidx, c->sval, c->scnt, c->err,
                       c->rs_list, c->rs_count, (int)c->m_max, c->cfg_omp_warps,
                       has_prop(c) ? c->rr_ref : nullptr, lp_ok(c) ? 0.f : dlk::kGapTol, c->st);
  if (e != cudaSuccess) return e;
  e = dlk::omp_resolve64(Y, c->p, D, c->G, lp_ok(c) ? nullptr : c->A0, c->lda, c->n, s,
                         c->rs_list, c->rs_count, (int)c->m_max, c->sidx, c->sval, c->scnt, c->st);
  mark(c, 3);
  return e;
}

// join: when given, colptr is produced on the side stream and the row pass waits for it.
// Group size in effect: groups of ntilde consecutive atoms, updated one group
// after another (Algorithm 1 steps 2-5); ntilde = n is the Jacobi form.
int group_size(dl_ctx* c) { return c->ntilde > 0 && c->ntilde < c->n ? c->ntilde : c->n; }

// join: when given, colptr is produced on the side stream and the row pass waits for it.
cudaError_t enq_jau(dl_ctx* c, const float* Y, int64_t m, float* D, int s, const int64_t* colptr,
                    int32_t* rowidx_out, float* val_out, cudaEvent_t join) {
  c->jw.det = c->deterministic && dlk::jau_det_supported(c->p, c->n, s, Y, D);
  c->jw.nb_accum = c->jw.det ? (int)dlk::jau_det_ranges(m, c->p, c->n, s)
                             : dlk::jau_accum_blocks(c->p, c->n, c->cfg_acc_mult);
  c->jw.nb_row = dlk::jau_row_blocks(c->cfg_row_per_sm);
  const int nt = group_size(c);
  const int ngroups = (c->n + nt - 1) / nt;
  const bool nsgk = c->rule == DL_RULE_NSGK;
  c->jw.nsgk = nsgk;
  c->jw.pidx = c->pidx;
  c->jw.pval = c->pval;
  c->jw.pcnt = c->pcnt;
  c->jw.pvalid = c->pvalid;
  c->jw.D0 = c->D0;
  cudaError_t e0;
  if (nsgk && (e0 = cudaMemcpyAsync(c->D0, D, sizeof(float) * (size_t)c->n * c->p,
                                    cudaMemcpyDeviceToDevice, c->st)) != cudaSuccess)
    return e0;
  // (groups need the float4 passes; the entry points check this before enqueuing)
  c->jau_kernels = (dlk::jau_launches(c->p, Y, D) - 1) * ngroups + 1;
  mark(c, 4);
  cudaError_t e = cudaSuccess;
  for (int a0 = 0; a0 < c->n; a0 += nt) {
    const int a1 = a0 + nt < c->n ? a0 + nt : c->n;
    c->jw.a0 = ngroups == 1 ? 0 : a0;
    c->jw.a1 = ngroups == 1 ? 0 : a1;
    c->jw.energies = a0 == 0;  // the error of the coding pass, before any atom moves
    c->jw.sgk = c->rule != DL_RULE_AKSVD;  // SGK and P-NSGK leave the coefficients
    e = dlk::jau_accumulate(Y, c->p, m, D, c->n, s, c->sidx, c->sval, c->scnt, c->jw, c->err,
                            c->st);
    if (e != cudaSuccess) break;
    if (a0 == 0) mark(c, 5);
    if ((e = dlk::jau_atoms(D, c->p, c->n, c->jw, c->st)) != cudaSuccess) break;
    if (a0 == 0) {
      mark(c, 6);
      if (join && (e = cudaStreamWaitEvent(c->st, join, 0)) != cudaSuccess) break;
    }
    e = dlk::jau_rows(Y, c->p, m, D, c->n, s, c->sidx, c->sval, c->scnt, c->jw, colptr,
                      rowidx_out, val_out, c->st);
    if (e != cudaSuccess) break;
    // the next group works from the atoms updated so far
    if (a1 < c->n)
      e = cudaMemcpyAsync(D + (size_t)a0 * c->p, c->jw.Dn + (size_t)a0 * c->p,
                          sizeof(float) * (size_t)(a1 - a0) * c->p, cudaMemcpyDeviceToDevice,
                          c->st);
    if (e != cudaSuccess) break;
  }
  c->jw.a0 = c->jw.a1 = 0;
  c->jw.energies = true;
  c->jw.nsgk = false;
  if (e != cudaSuccess) return e;
  if (nsgk) {  // this iteration's representations are the next one's previous ones
    const size_t ms = (size_t)m * s;
    if ((e = cudaMemcpyAsync(c->pidx, c->sidx, sizeof(int32_t) * ms, cudaMemcpyDeviceToDevice,
                             c->st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(c->pval, c->sval, sizeof(float) * ms, cudaMemcpyDeviceToDevice,
                             c->st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(c->pcnt, c->scnt, sizeof(int32_t) * (size_t)m,
                             cudaMemcpyDeviceToDevice, c->st)) != cudaSuccess ||
        (e = cudaMemsetAsync(c->pvalid, 1, sizeof(int), c->st)) != cudaSuccess)
      return e;
  }
  mark(c, 7);
  e = dlk::jau_finalize(c->jw, c->rmse, c->iter, D, c->n, c->p, c->st);
  mark(c, 8);
  return e;
}

// Whether a call with host buffers overlaps the upload of Y with the first
// iteration's coding pass: the residual-form OMP (FP32 or BF16) or the plain
// FP32 tensor-core correlations, at least kChunks x 128 signals.
bool staged_ok(dl_ctx* c, const float* dY, const float* dD, int64_t m, int s) {
  if (has_prop(c) || m < (int64_t)dl_ctx::kChunks * 128) return false;
  return use_res(c, dY, dD, s, m) || (!lp_ok(c) && tc_ok(c, dY, dD));
}

// Piece q of the staged coding pass covers signals [off[q], off[q+1]).  Each
// piece is kGrow times the one before it: uploading a signal takes about a
// third of the time its correlations and OMP take (p=64, n=512: ~1.3 against
// ~3.9 ns), so piece q+1 arrives while piece q is being coded and only the
// first, small piece is waited for.  Boundaries are multiples of 128 signals
// (row tiles); trailing pieces may be empty.
constexpr double kGrow = 2.5;
void staged_pieces(int64_t m, int64_t (&off)[dl_ctx::kChunks + 1]) {
  double w = 1.0, total = 0.0;
  for (int q = 0; q < dl_ctx::kChunks; ++q, w *= kGrow) total += w;
  double acc = 0.0;
  w = 1.0;
  off[0] = 0;
  for (int q = 0; q < dl_ctx::kChunks; ++q, w *= kGrow) {
    acc += w;
    int64_t b = q + 1 == dl_ctx::kChunks ? m : ((int64_t)(m * (acc / total)) + 127) / 128 * 128;
    if (b > m) b = m;
    if (b < off[q]) b = off[q];
    off[q + 1] = b;
  }
}

// The coding pass with Y still on the host: Y is copied in kChunks pieces on the
// side stream, and the correlations (the Gram matrix with the first piece), the
// OMP and the FP64 re-solve of each piece start as soon as it has arrived.
// dY is the device staging buffer the pieces go to.  Returns the kernel count.
// The staged coding pass of the residual-form OMP: the Gram matrix first (it
// needs no signal), then Y in two pieces; the first holds one full round of the
// OMP kernel's tiles (all SMs, both slots), so that only its upload is waited
// for and splitting adds no partial round.
cudaError_t enq_omp_res_staged(dl_ctx* c, const float* hostY, const float* dY, int64_t m,
                               const float* D, int s, int* kernels) {
  const int64_t p = c->p;
  int64_t offs[3] = {0, std::min(m, dlk::omp_res_round_signals()), m};
  cudaError_t e;
  c->a0_bf16 = false;
  c->last_omp = 2;
  mark(c, 0);
  if ((e = dlk::gram_simt(D, c->n, c->p, c->G, c->st)) != cudaSuccess) return e;
  int k = 1;
  mark(c, 1);
  if ((e = cudaEventRecord(c->ev_fork, c->st)) != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(c->st2, c->ev_fork, 0)) != cudaSuccess) return e;
  for (int q = 0; q < 2; ++q) {
    const int64_t off = offs[q], mk = offs[q + 1] - offs[q];
    if (mk <= 0) continue;
    e = cudaMemcpyAsync((float*)dY + off * p, hostY + off * p, sizeof(float) * (size_t)(mk * p),
                        cudaMemcpyHostToDevice, c->st2);
    if (e != cudaSuccess) return e;
    if ((e = cudaEventRecord(c->ev_chunk[q], c->st2)) != cudaSuccess) return e;
  }
  mark(c, 2);
  for (int q = 0; q < 2; ++q) {
    const int64_t off = offs[q], mk = offs[q + 1] - offs[q];
    if (mk <= 0) continue;
    const float* Yq = dY + off * p;
    if ((e = cudaStreamWaitEvent(c->st, c->ev_chunk[q], 0)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(c->rs_count, 0, sizeof(int), c->st)) != cudaSuccess) return e;
    e = dlk::omp_res(Yq, mk, c->p, D, c->n, c->G, s, c->sidx + off * s, c->sval + off * s,
                     c->scnt + off, c->err, c->rs_list, c->rs_count, (int)c->m_max,
                     c->precision == DL_BF16, c->st);
    if (e != cudaSuccess) return e;
    e = dlk::omp_resolve64(Yq, c->p, D, c->G, nullptr, c->lda, c->n, s, c->rs_list, c->rs_count,
                           (int)c->m_max, c->sidx + off * s, c->sval + off * s, c->scnt + off,
                           c->st);
    if (e != cudaSuccess) return e;
    k += 2;
  }
  mark(c, 3);
  *kernels = k;
  return cudaSuccess;
}

cudaError_t enq_omp_staged(dl_ctx* c, const float* hostY, const float* dY, int64_t m,
                           const float* D, int s, int* kernels) {
  if (use_res(c, dY, D, s, m)) return enq_omp_res_staged(c, hostY, dY, m, D, s, kernels);
  const int64_t p = c->p;
  int64_t offs[dl_ctx::kChunks + 1];
  staged_pieces(m, offs);
  cudaError_t e;
  int k = 0;
  mark(c, 0);
  if ((e = dlk::split_tf32(D, (int64_t)c->n * c->p, c->Dhi, c->Dlo, c->st)) != cudaSuccess) return e;
  ++k;
  mark(c, 1);
  if ((e = cudaEventRecord(c->ev_fork, c->st)) != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(c->st2, c->ev_fork, 0)) != cudaSuccess) return e;
  for (int q = 0; q < dl_ctx::kChunks; ++q) {
    const int64_t off = offs[q], mk = offs[q + 1] - offs[q];
    if (mk <= 0) continue;
    e = cudaMemcpyAsync((float*)dY + off * p, hostY + off * p, sizeof(float) * (size_t)(mk * p),
                        cudaMemcpyHostToDevice, c->st2);
    if (e != cudaSuccess) return e;
    if ((e = cudaEventRecord(c->ev_chunk[q], c->st2)) != cudaSuccess) return e;
  }
  mark(c, 2);
  bool first = true;
  for (int q = 0; q < dl_ctx::kChunks; ++q) {
    const int64_t off = offs[q], mk = offs[q + 1] - offs[q];
    if (mk <= 0) continue;
    const float* Yq = dY + off * p;
    float* Aq = c->A0 + off * c->lda;
    if ((e = cudaStreamWaitEvent(c->st, c->ev_chunk[q], 0)) != cudaSuccess) return e;
    e = first ? dlk::corr_tf32x3_pair(Yq, mk, Aq, c->lda, D, c->n, c->G, c->n, c->Dhi, c->Dlo,
                                       c->n, c->p, c->err, c->st)
               : dlk::corr_tf32x3(Yq, mk, c->Dhi, c->Dlo, c->n, c->p, Aq, c->lda, c->err, c->st);
    if (e != cudaSuccess) return e;
    first = false;
    if ((e = cudaMemsetAsync(c->rs_count, 0, sizeof(int), c->st)) != cudaSuccess) return e;
    if (c->cfg_omp_tm && dlk::omp_tm_supported(c->n, s))
      e = dlk::omp_batch_tm(c->cfg_omp_tm, Aq, false, c->lda, c->G, c->n, Yq, c->p, mk, s, c->sidx + off * s,
                            c->sval + off * s, c->scnt + off, c->err, c->rs_list, c->rs_count,
                            (int)c->m_max, c->st);
    else
      e = dlk::omp_batch(Aq, c->lda, c->G, c->n, Yq, c->p, mk, s, c->sidx + off * s,
                         c->sval + off * s, c->scnt + off, c->err, c->rs_list, c->rs_count,
                         (int)c->m_max, c->cfg_omp_warps, nullptr, dlk::kGapTol, c->st);
    if (e != cudaSuccess) return e;
    e = dlk::omp_resolve64(Yq, c->p, D, c->G, Aq, c->lda, c->n, s, c->rs_list, c->rs_count,
                           (int)c->m_max, c->sidx + off * s, c->sval + off * s, c->scnt + off,
                           c->st);
    if (e != cudaSuccess) return e;
    k += 3;
  }
  mark(c, 3);
  c->last_omp = c->cfg_omp_tm && dlk::omp_tm_supported(c->n, s) ? 1 : 0;
  *kernels = k;
  return cudaSuccess;
}

// hostY: when given, Y is uploaded into the staging buffer Y by the coding pass
// itself (enq_omp_staged); staged_kernels then receives that pass's kernel count.
// The side stream scans the counts into colptr while the atom update starts and
// then writes the CSC row indices from the coding pass's slots (the supports do
// not change in the atom update; the row pass writes only the values); with
// colptr_dl / rowidx_dl (page-locked host buffers) it also downloads both there,
// under the atom update.
cudaError_t enq_iteration(dl_ctx* c, const float* Y, int64_t m, float* D, int s, int64_t* colptr,
                          int32_t* rowidx, float* val, const float* hostY = nullptr,
                          int* staged_kernels = nullptr, int64_t* colptr_dl = nullptr,
                          int32_t* rowidx_dl = nullptr) {
  cudaError_t e = hostY ? enq_omp_staged(c, hostY, Y, m, D, s, staged_kernels)
                        : enq_omp(c, Y, m, D, s);
  if (e != cudaSuccess) return e;
  if ((e = cudaEventRecord(c->ev_fork, c->st)) != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(c->st2, c->ev_fork, 0)) != cudaSuccess) return e;
  e = dlk::counts_to_colptr(c->scnt, m, c->bsum, colptr, c->st2);
  if (e != cudaSuccess) return e;
  if ((e = cudaEventRecord(c->ev_join, c->st2)) != cudaSuccess) return e;  // the row pass's colptr
  c->scan_kernels = 2;
  const bool side_rowidx = rowidx != nullptr && m > 0;
  if (side_rowidx) {
    if ((e = dlk::slots_to_csc(c->sidx, nullptr, c->scnt, m, s, colptr, rowidx, nullptr,
                               c->st2)) != cudaSuccess)
      return e;
    c->scan_kernels = 3;
    if (colptr_dl && (e = cudaMemcpyAsync(colptr_dl, colptr, sizeof(int64_t) * (size_t)(m + 1),
                                          cudaMemcpyDeviceToHost, c->st2)) != cudaSuccess)
      return e;
    if (rowidx_dl && (e = cudaMemcpyAsync(rowidx_dl, rowidx, sizeof(int32_t) * (size_t)m * s,
                                          cudaMemcpyDeviceToHost, c->st2)) != cudaSuccess)
      return e;
    if ((e = cudaEventRecord(c->ev_join2, c->st2)) != cudaSuccess) return e;
  }
  e = enq_jau(c, Y, m, D, s, colptr, side_rowidx ? nullptr : rowidx, val, c->ev_join);
  if (e != cudaSuccess) return e;
  if (side_rowidx) e = cudaStreamWaitEvent(c->st, c->ev_join2, 0);
  return e;
}

// Kernels one DL iteration enqueues (the claim behind dl_kernel_launches).
// The counts are recorded when the pass is enqueued (eagerly or into a graph).
int64_t kernels_per_iteration(dl_ctx* c, bool learned) {
  return c->omp_kernels[learned ? 1 : 0] + c->scan_kernels + c->jau_kernels;
}

int check_common(dl_ctx* c, int64_t m) {
  if (!c) return DL_EINVAL;
  if (m < 0 || m > c->m_max) return DL_EINVAL;
  return DL_OK;
}

// Page-locked host memory (the only host memory a captured copy may use).
bool pinned_host(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

// One whole host-buffer call of one iteration: D uploaded, the staged
// iteration (Y uploaded in pieces under the coding pass), D and X downloaded.
cudaError_t enq_host_call(dl_ctx* c, const float* Y, int64_t m, float* D, int s,
                          int64_t* colptr, int32_t* rowidx, float* val, int* kernels) {
  cudaError_t e;
  const size_t np = (size_t)c->n * c->p, ms = (size_t)m * s;
  if ((e = cudaMemcpyAsync(c->hD, D, sizeof(float) * np, cudaMemcpyHostToDevice, c->st)) !=
          cudaSuccess ||
      (e = cudaMemsetAsync(c->iter, 0, sizeof(int), c->st)) != cudaSuccess)
    return e;
  int ko = 0;
  // colptr and the row indices go down on the side stream under the atom update
  if ((e = enq_iteration(c, c->hY, m, c->hD, s, c->hcolptr, c->hrowidx, c->hval, Y, &ko, colptr,
                         rowidx)) != cudaSuccess)
    return e;
  *kernels = ko + c->scan_kernels + c->jau_kernels;
  // all s*m entries (the caller's capacity), so no synchronisation is needed to learn nnz
  if ((e = cudaMemcpyAsync(D, c->hD, sizeof(float) * np, cudaMemcpyDeviceToHost, c->st)) !=
          cudaSuccess ||
      (e = cudaMemcpyAsync(val, c->hval, sizeof(float) * ms, cudaMemcpyDeviceToHost, c->st)) !=
          cudaSuccess)
    return e;
  return cudaSuccess;
}

// dl_iterate with host buffers, one iteration, staged upload, page-locked
// buffers: the first call with a key runs eagerly, the next ones replay a
// graph of the whole call (the host then only launches it).
int host_call_graphed(dl_ctx* c, const float* Y, int64_t m, float* D, int s, int64_t* colptr,
                      int32_t* rowidx, float* val, double* rmse) {
  // (the caller has matched the host buffers against hkey)
  if (c->gkey[0] != (const void*)c->hY)
    c->gkey_m = -1;  // a later call with device buffers starts from a fresh key
  const int64_t sig[11] = {m, s, c->rule, c->ntilde, c->cfg_omp_warps, c->cfg_acc_mult,
                           c->cfg_row_per_sm, c->cfg_corr_tc, (int64_t)(intptr_t)c->st,
                           (int64_t)(intptr_t)c->prop + (c->prop_corr ? 1 : 0), c->deterministic};
  if (memcmp(sig, c->hsig, sizeof(sig)) != 0) {
    if (c->hgexec) cudaGraphExecDestroy(c->hgexec);
    c->hgexec = nullptr;
    c->hseen = 0;
    memcpy(c->hsig, sig, sizeof(sig));
  }
  if (c->hseen >= 1 && !c->hgexec) {
    cudaGraph_t graph = nullptr;
    int k = 0;
    DL_CHECK(cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = enq_host_call(c, Y, m, D, s, colptr, rowidx, val, &k);
    cudaError_t e2 = cudaStreamEndCapture(c->st, &graph);
    if (e != cudaSuccess) return cuda_status(e);
    if (e2 != cudaSuccess) return cuda_status(e2);
    e = cudaGraphInstantiate(&c->hgexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      c->hgexec = nullptr;
      return cuda_status(e);
    }
    c->hg_kernels = k;
  }
  if (c->hgexec) {
    DL_CHECK(cudaGraphLaunch(c->hgexec, c->st));
    c->launches += c->hg_kernels;
  } else {
    int k = 0;
    DL_CHECK(enq_host_call(c, Y, m, D, s, colptr, rowidx, val, &k));
    c->launches += k;
    c->hseen++;
  }
  if (rmse)
    DL_CHECK(cudaMemcpyAsync(rmse, c->rmse, sizeof(double) * 2, cudaMemcpyDeviceToHost, c->st));
  return take_device_error(c);
}

}  // namespace

extern "C" {

const char* dl_strerror(int status) {
  switch (status) {
    case DL_OK: return "success";
    case DL_EINVAL: return "invalid argument (sizes, pointers, or CSC content)";
    case DL_ECUDA: return "CUDA runtime error";
    case DL_ENUMERIC: return "non-finite value met in the inputs";
    case DL_ETIMEOUT: return "a bounded device-side wait timed out";
    case DL_ENOMEM: return "device memory allocation failed";
    case DL_ENOTIMPL: return "not implemented in this build";
    default: return "unknown status";
  }
}

int dl_init(dl_ctx** out, int p, int n, int64_t m_max, int s_max, int precision, void* stream) {
  if (!out) return DL_EINVAL;
  if (p < 1 || p > DL_MAX_P || n < 1 || n > DL_MAX_N || m_max < 1 || s_max < 1 ||
      s_max > DL_MAX_S || s_max > p || s_max > n)
    return DL_EINVAL;
  if (precision != DL_FP32 && precision != DL_BF16 && precision != DL_FP8) return DL_EINVAL;
  dl_ctx* c = new dl_ctx();
  cudaGetDevice(&c->dev);
  c->p = p;
  c->n = n;
  c->m_max = m_max;
  c->s_max = s_max;
  c->precision = precision;
  c->st = (cudaStream_t)stream;
  c->lda = ((int64_t)n + 31) / 32 * 32;
  if (const char* v = getenv("DL_OMP_TM")) c->cfg_omp_tm = atoi(v);  // 0 (off), 4, 5 or 6
  if (const char* v = getenv("DL_OMP_RES")) c->cfg_omp_res = atoi(v);  // 0 off, 1 on, 2 any n
  const size_t mm = (size_t)m_max;
  c->jw.nb_accum = dlk::jau_accum_blocks_max(p, n);
  // the deterministic pass A writes one slice of U and one energy partial per range of signals
  const bool det = dlk::jau_det_supported(p, n, s_max, nullptr, nullptr);
  const int64_t nbd = det ? dlk::jau_det_ranges(m_max, p, n, s_max) : 0;
  if (nbd > c->jw.nb_accum) c->jw.nb_accum = (int)nbd;
  c->jw.nb_row = dlk::jau_row_blocks_max();
  const size_t ulen = dlk::jau_ulen(p, n);
  size_t nslices = dlk::jau_accum_smem(p, n) > 0 ? (size_t)c->jw.nb_accum : 1;
  if (nslices < (size_t)dlk::kUCopies) nslices = dlk::kUCopies;
  if (nslices < (size_t)nbd) nslices = (size_t)nbd;
  bool ok = dalloc(&c->G, (size_t)n * n) && dalloc(&c->A0, mm * c->lda) &&
            dalloc(&c->sidx, mm * s_max) && dalloc(&c->sval, mm * s_max) &&
            dalloc(&c->scnt, mm) && dalloc(&c->bsum, (size_t)dlk::scan_blocks(m_max) + 1) &&
            dalloc(&c->err, 1) && dalloc(&c->iter, 1) && dalloc(&c->jw.Upart, nslices * ulen) &&
            dalloc(&c->jw.U, ulen) && dalloc(&c->jw.epart_a, (size_t)2 * c->jw.nb_accum) &&
            dalloc(&c->jw.epart_b, (size_t)c->jw.nb_row) && dalloc(&c->jw.Dn, (size_t)n * p) &&
            dalloc(&c->jw.C, (size_t)n) && dalloc(&c->Dhi, (size_t)n * p) &&
            dalloc(&c->Dlo, (size_t)n * p) && dalloc(&c->rs_list, mm) && dalloc(&c->rs_count, 1);
  ok = ok && cudaStreamCreateWithFlags(&c->st2, cudaStreamNonBlocking) == cudaSuccess &&
       cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
       cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) == cudaSuccess &&
       cudaEventCreateWithFlags(&c->ev_join2, cudaEventDisableTiming) == cudaSuccess;
  for (cudaEvent_t& e : c->ev_chunk)
    ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
  if (ok && precision != DL_FP32) {
    c->lp_kind = precision == DL_BF16 ? dlk::LP_BF16 : dlk::LP_E4M3;
    const size_t esz = precision == DL_BF16 ? 2 : 1;
    const size_t ld = (size_t)dlk::lp_row_elems(c->lp_kind, p);
    ok = dalloc((uint8_t**)&c->Ylp, mm * ld * esz) && dalloc(&c->Ysc, mm) &&
         dalloc((uint8_t**)&c->Dlp, (size_t)n * ld * esz) && dalloc(&c->Dsc, (size_t)n + 16);
  }
  if (!ok) {
    cudaGetLastError();
    free_ctx(c);
    return DL_ENOMEM;
  }
  if (ensure_rmse(c, 64) != DL_OK || cudaMemset(c->err, 0, sizeof(int)) != cudaSuccess ||
      cudaMemset(c->iter, 0, sizeof(int)) != cudaSuccess) {
    free_ctx(c);
    return DL_ECUDA;
  }
  *out = c;
  return DL_OK;
}

int dl_set_stream(dl_ctx* c, void* stream) {
  if (!c) return DL_EINVAL;
  if ((cudaStream_t)stream != c->st) {
    c->st = (cudaStream_t)stream;
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
    c->gkey_seen = 0;
  }
  return DL_OK;
}

int dl_destroy(dl_ctx* c) {
  free_ctx(c);
  return DL_OK;
}

int dl_sync(dl_ctx* c) {
  if (!c) return DL_EINVAL;
  DevGuard g(c->dev);
  return take_device_error(c);
}

int64_t dl_kernel_launches(dl_ctx* c) { return c ? c->launches : 0; }

int dl_check_bounded_wait(dl_ctx* c) {
  if (!c) return DL_EINVAL;
  DevGuard g(c->dev);
  if (int rc = take_device_error(c)) return rc;  // report an earlier error first
  DL_CHECK(dlk::bounded_wait_check(c->err, c->st));
  c->launches += 1;
  return take_device_error(c);
}

int dl_fp32_probe(int packed, int64_t iters, float* out, double* flops, void* stream) {
  if (!out || !flops || iters < 1) return DL_EINVAL;
  DL_CHECK(dlk::ffma_probe(packed, iters, out, flops, (cudaStream_t)stream));
  return DL_OK;
}

int dl_set_group_size(dl_ctx* c, int ntilde) {
  if (!c || ntilde < 1 || ntilde > c->n) return DL_EINVAL;
  if (ntilde != c->ntilde) c->gkey_m = -1;  // captured iterations no longer apply
  c->ntilde = ntilde;
  return DL_OK;
}

int dl_set_deterministic(dl_ctx* c, int on) {
  if (!c) return DL_EINVAL;
  on = on ? 1 : 0;
  if (on != c->deterministic) c->gkey_m = -1;  // captured iterations no longer apply
  c->deterministic = on;
  return DL_OK;
}

int dl_set_update_rule(dl_ctx* c, int rule) {
  if (!c || (rule != DL_RULE_AKSVD && rule != DL_RULE_SGK && rule != DL_RULE_NSGK))
    return DL_EINVAL;
  DevGuard g(c->dev);
  if (rule == DL_RULE_NSGK) {
    const size_t ms = (size_t)c->m_max * c->s_max;
    if (!c->pvalid && !(dalloc(&c->pidx, ms) && dalloc(&c->pval, ms) &&
                        dalloc(&c->pcnt, (size_t)c->m_max) && dalloc(&c->pvalid, 1) &&
                        dalloc(&c->D0, (size_t)c->n * c->p))) {
      cudaGetLastError();
      return DL_ENOMEM;
    }
    // the first P-NSGK iteration has no previous representations
    DL_CHECK(cudaMemsetAsync(c->pvalid, 0, sizeof(int), c->st));
  }
  if (rule != c->rule) c->gkey_m = -1;  // captured iterations no longer apply
  c->rule = rule;
  return DL_OK;
}

int dl_set_profiling(dl_ctx* c, int on) {
  if (!c) return DL_EINVAL;
  DevGuard g(c->dev);
  const bool want = on != 0;
  if (want && !c->ev[0])
    for (cudaEvent_t& e : c->ev) DL_CHECK(cudaEventCreate(&e));
  if (want != c->prof) {
    c->prof = want;
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
    c->gkey_seen = 0;
  }
  for (double& x : c->phase_ms) x = 0.0;
  c->phase_count = 0;
  return DL_OK;
}

int dl_phase_times(dl_ctx* c, double* ms, int max_phases) {
  if (!c || !ms || max_phases < 0) return DL_EINVAL;
  const int k = max_phases < 8 ? max_phases : 8;
  for (int q = 0; q < k; ++q) ms[q] = c->phase_count ? c->phase_ms[q] / c->phase_count : 0.0;
  return 8;
}

int dl_gram(dl_ctx* c, const float* D, float* G) {
  if (!c || !D || !G || ptr_kind(D) != 1 || ptr_kind(G) != 1) return DL_EINVAL;
  DevGuard g(c->dev);
  const bool tc = tc_ok(c, D, D);
  DL_CHECK(enq_gram(c, D, tc));
  DL_CHECK(cudaMemcpyAsync(G, c->G, sizeof(float) * (size_t)c->n * c->n, cudaMemcpyDeviceToDevice, c->st));
  c->launches += tc ? 2 : 1;
  return DL_OK;
}

int dl_correlate(dl_ctx* c, const float* Y, int64_t m, const float* D, float* A) {
  int rc = check_common(c, m);
  if (rc) return rc;
  if (!Y || !D || !A || ptr_kind(Y) != 1 || ptr_kind(D) != 1 || ptr_kind(A) != 1) return DL_EINVAL;
  DevGuard g(c->dev);
  const bool tc = tc_ok(c, Y, D);
  c->a0_bf16 = false;  // the caller's A is FP32
  if (tc) DL_CHECK(dlk::split_tf32(D, (int64_t)c->n * c->p, c->Dhi, c->Dlo, c->st));
  DL_CHECK(enq_convert_y(c, Y, m));
  DL_CHECK(enq_corr(c, Y, m, D, tc));
  if (m > 0)
    DL_CHECK(cudaMemcpy2DAsync(A, sizeof(float) * c->n, c->A0, sizeof(float) * c->lda,
                               sizeof(float) * c->n, (size_t)m, cudaMemcpyDeviceToDevice, c->st));
  c->launches += tc ? 2 : 1;
  return DL_OK;
}

int64_t dl_last_resolved(dl_ctx* c) {
  if (!c) return DL_EINVAL;
  DevGuard g(c->dev);
  int h = 0;
  if (cudaMemcpyAsync(&h, c->rs_count, sizeof(int), cudaMemcpyDeviceToHost, c->st) != cudaSuccess ||
      cudaStreamSynchronize(c->st) != cudaSuccess)
    return DL_ECUDA;
  return h;
}

int dl_uses_tensor_cores(dl_ctx* c) {
  if (!c) return DL_EINVAL;
  return dlk::corr_tc_supported(nullptr, c->p, c->n, c->lda) ? 1 : 0;
}

int omp_code(dl_ctx* c, const float* Y, int64_t m, const float* D, int s, int64_t* colptr,
             int32_t* rowidx, float* val) {
  int rc = check_common(c, m);
  if (rc) return rc;
  if (s < 1 || s > c->s_max || !Y || !D || !colptr || !rowidx || !val) return DL_EINVAL;
  const int kind = ptr_kind(Y);
  if (ptr_kind(D) != kind || ptr_kind(colptr) != kind || ptr_kind(rowidx) != kind ||
      ptr_kind(val) != kind)
    return DL_EINVAL;
  DevGuard g(c->dev);
  const float *dY = Y, *dD = D;
  int64_t* dcp = colptr;
  int32_t* dri = rowidx;
  float* dv = val;
  if (kind == 0) {
    if ((rc = ensure_staging(c))) return rc;
    DL_CHECK(cudaMemcpyAsync(c->hY, Y, sizeof(float) * (size_t)m * c->p, cudaMemcpyHostToDevice, c->st));
    DL_CHECK(cudaMemcpyAsync(c->hD, D, sizeof(float) * (size_t)c->n * c->p, cudaMemcpyHostToDevice, c->st));
    dY = c->hY;
    dD = c->hD;
    dcp = c->hcolptr;
    dri = c->hrowidx;
    dv = c->hval;
  }
  DL_CHECK(enq_convert_y(c, dY, m));
  if (needs_y_conversion(c, dY)) c->launches += 1;
  c->learned_now = false;
  DL_CHECK(enq_omp(c, dY, m, dD, s));
  DL_CHECK(dlk::counts_to_colptr(c->scnt, m, c->bsum, dcp, c->st));
  DL_CHECK(dlk::slots_to_csc(c->sidx, c->sval, c->scnt, m, s, dcp, dri, dv, c->st));
  c->launches += c->omp_kernels[0] + kKernelsScan + 1;
  if (kind == 0) {
    // all s*m entries (the caller's capacity), so no synchronisation is needed to learn nnz;
    // entries past colptr[m] are unspecified
    DL_CHECK(cudaMemcpyAsync(colptr, dcp, sizeof(int64_t) * (size_t)(m + 1), cudaMemcpyDeviceToHost, c->st));
    DL_CHECK(cudaMemcpyAsync(rowidx, dri, sizeof(int32_t) * (size_t)m * s, cudaMemcpyDeviceToHost, c->st));
    DL_CHECK(cudaMemcpyAsync(val, dv, sizeof(float) * (size_t)m * s, cudaMemcpyDeviceToHost, c->st));
    return take_device_error(c);
  }
  return DL_OK;
}

int jau_update(dl_ctx* c, const float* Y, int64_t m, float* D, const int64_t* colptr,
               const int32_t* rowidx, float* val, double* rmse2) {
  int rc = check_common(c, m);
  if (rc) return rc;
  if (!Y || !D || !colptr || !rowidx || !val) return DL_EINVAL;
  const int kind = ptr_kind(Y);
  if (ptr_kind(D) != kind || ptr_kind(colptr) != kind || ptr_kind(rowidx) != kind ||
      ptr_kind(val) != kind)
    return DL_EINVAL;
  if ((group_size(c) < c->n || c->rule == DL_RULE_NSGK) &&
      (c->p % 4 != 0 || (kind == 1 && !dlk::jau_vec4(c->p, Y, D))))
    return DL_ENOTIMPL;
  DevGuard g(c->dev);
  const int s = c->s_max;
  const float* dY = Y;
  float* dD = D;
  const int64_t* dcp = colptr;
  const int32_t* dri = rowidx;
  float* dv = val;
  int64_t nnz = 0;
  if (kind == 0) {
    nnz = colptr[m];
    if (nnz < 0 || nnz > m * (int64_t)s || colptr[0] != 0) return DL_EINVAL;
    if ((rc = ensure_staging(c))) return rc;
    DL_CHECK(cudaMemcpyAsync(c->hY, Y, sizeof(float) * (size_t)m * c->p, cudaMemcpyHostToDevice, c->st));
    DL_CHECK(cudaMemcpyAsync(c->hD, D, sizeof(float) * (size_t)c->n * c->p, cudaMemcpyHostToDevice, c->st));
    DL_CHECK(cudaMemcpyAsync(c->hcolptr, colptr, sizeof(int64_t) * (size_t)(m + 1), cudaMemcpyHostToDevice, c->st));
    DL_CHECK(cudaMemcpyAsync(c->hrowidx, rowidx, sizeof(int32_t) * (size_t)nnz, cudaMemcpyHostToDevice, c->st));
    DL_CHECK(cudaMemcpyAsync(c->hval, val, sizeof(float) * (size_t)nnz, cudaMemcpyHostToDevice, c->st));
    dY = c->hY;
    dD = c->hD;
    dcp = c->hcolptr;
    dri = c->hrowidx;
    dv = c->hval;
  }
  DL_CHECK(cudaMemsetAsync(c->iter, 0, sizeof(int), c->st));
  DL_CHECK(dlk::csc_to_slots(dcp, dri, dv, m, c->n, s, c->sidx, c->sval, c->scnt, c->err, c->st));
  DL_CHECK(enq_jau(c, dY, m, dD, s, dcp, nullptr, dv, nullptr));
  c->launches += 1 + c->jau_kernels;
  if (kind == 0) {
    DL_CHECK(cudaMemcpyAsync(D, dD, sizeof(float) * (size_t)c->n * c->p, cudaMemcpyDeviceToHost, c->st));
    DL_CHECK(cudaMemcpyAsync(val, dv, sizeof(float) * (size_t)nnz, cudaMemcpyDeviceToHost, c->st));
  }
  if (rmse2) DL_CHECK(cudaMemcpyAsync(rmse2, c->rmse, sizeof(double) * 2, cudaMemcpyDeviceToHost, c->st));
  if (kind == 0 || rmse2) return take_device_error(c);
  return DL_OK;
}

int dl_iterate(dl_ctx* c, const float* Y, int64_t m, float* D, int s, int iters, int64_t* colptr,
               int32_t* rowidx, float* val, double* rmse) {
  int rc = check_common(c, m);
  if (rc) return rc;
  if (s < 1 || s > c->s_max || iters < 0 || !Y || !D || !colptr || !rowidx || !val)
    return DL_EINVAL;
  const int kind = ptr_kind(Y);
  if (ptr_kind(D) != kind || ptr_kind(colptr) != kind || ptr_kind(rowidx) != kind ||
      ptr_kind(val) != kind)
    return DL_EINVAL;
  if (iters == 0) return DL_OK;
  if (kind == 1 && (group_size(c) < c->n || c->rule == DL_RULE_NSGK) &&
      !dlk::jau_vec4(c->p, Y, D))
    return DL_ENOTIMPL;
  DevGuard g(c->dev);
  if ((rc = ensure_rmse(c, iters))) return rc;
  const float* dY = Y;
  float* dD = D;
  int64_t* dcp = colptr;
  int32_t* dri = rowidx;
  float* dv = val;
  bool staged = false;
  if (kind == 0) {
    if ((rc = ensure_staging(c))) return rc;
    dY = c->hY;
    dD = c->hD;
    dcp = c->hcolptr;
    dri = c->hrowidx;
    dv = c->hval;
    staged = staged_ok(c, dY, dD, m, s);
    if ((group_size(c) < c->n || c->rule == DL_RULE_NSGK) && !dlk::jau_vec4(c->p, dY, dD))
      return DL_ENOTIMPL;
    const void* hk[5] = {Y, D, colptr, rowidx, val};
    if (memcmp(hk, c->hkey, sizeof(hk)) != 0 || m != c->hkey_m || s != c->hkey_s) {
      // other host buffers: the stored P-NSGK representations do not apply (the
      // staging buffers stay the same, so the device key cannot tell), and a
      // graph of the previous buffers' call is stale
      if (c->pvalid) DL_CHECK(cudaMemsetAsync(c->pvalid, 0, sizeof(int), c->st));
      if (c->hgexec) cudaGraphExecDestroy(c->hgexec);
      c->hgexec = nullptr;
      c->hseen = 0;
      memcpy(c->hkey, hk, sizeof(hk));
      c->hkey_m = m;
      c->hkey_s = s;
    }
    if (staged && iters == 1 && !c->prof && c->st && pinned_host(Y) && pinned_host(D) &&
        pinned_host(colptr) && pinned_host(rowidx) && pinned_host(val))
      return host_call_graphed(c, Y, m, D, s, colptr, rowidx, val, rmse);
    if (!staged)
      DL_CHECK(cudaMemcpyAsync(c->hY, Y, sizeof(float) * (size_t)m * c->p, cudaMemcpyHostToDevice, c->st));
    DL_CHECK(cudaMemcpyAsync(c->hD, D, sizeof(float) * (size_t)c->n * c->p, cudaMemcpyHostToDevice, c->st));
  }
  DL_CHECK(cudaMemsetAsync(c->iter, 0, sizeof(int), c->st));
  const void* key[5] = {dY, dD, dcp, dri, dv};
  const bool same = c->gkey_m == m && c->gkey_s == s && memcmp(key, c->gkey, sizeof(key)) == 0;
  if (!same) {
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
    if (c->gexec_learned) cudaGraphExecDestroy(c->gexec_learned);
    c->gexec_learned = nullptr;
    c->gkey_seen_l = 0;
    memcpy(c->gkey, key, sizeof(key));
    c->gkey_m = m;
    c->gkey_s = s;
    c->gkey_seen = 0;
    // other signals or sizes: the stored P-NSGK representations do not apply
    if (c->pvalid) DL_CHECK(cudaMemsetAsync(c->pvalid, 0, sizeof(int), c->st));
    if (kind == 1) c->hkey[0] = nullptr;  // nor to a later host-buffer call
  }
  const bool can_graph = c->st != nullptr && m > 0;
  DL_CHECK(enq_convert_y(c, dY, m));
  if (c->prop) DL_CHECK(dlk::to_lowp(dlk::LP_BF16, dY, m, c->p, c->Ybf, nullptr, c->st));
  c->launches += (needs_y_conversion(c, dY) ? 1 : 0) + (c->prop ? 1 : 0);  // per-call conversions of Y
  for (int it = 0; it < iters; ++it) {
    const bool learned = has_prop(c) && (c->prop_counter % c->prop_full_every) != 0;
    c->learned_now = learned;
    cudaGraphExec_t& gx = learned ? c->gexec_learned : c->gexec;
    int& seen = learned ? c->gkey_seen_l : c->gkey_seen;
    if (staged && it == 0) {
      // first iteration of a host-buffer call: upload overlapped with the coding pass
      int ko = 0;
      DL_CHECK(enq_iteration(c, dY, m, dD, s, dcp, dri, dv, Y, &ko));
      c->launches += ko + c->scan_kernels + c->jau_kernels;
      if (c->prof) {
        DL_CHECK(cudaStreamSynchronize(c->st));
        for (int k = 0; k < 8; ++k) {
          float ms = 0.f;
          DL_CHECK(cudaEventElapsedTime(&ms, c->ev[k], c->ev[k + 1]));
          c->phase_ms[k] += ms;
        }
        c->phase_count++;
      }
      continue;
    }
    if (can_graph && seen >= 1 && !gx) {
      cudaGraph_t graph = nullptr;
      DL_CHECK(cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal));
      cudaError_t e = enq_iteration(c, dY, m, dD, s, dcp, dri, dv);
      cudaError_t e2 = cudaStreamEndCapture(c->st, &graph);
      if (e != cudaSuccess) return cuda_status(e);
      if (e2 != cudaSuccess) return cuda_status(e2);
      e = cudaGraphInstantiate(&gx, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) {
        gx = nullptr;
        return cuda_status(e);
      }
    }
    if (gx) {
      DL_CHECK(cudaGraphLaunch(gx, c->st));
    } else {
      DL_CHECK(enq_iteration(c, dY, m, dD, s, dcp, dri, dv));
      seen++;
    }
    c->launches += kernels_per_iteration(c, learned);
    if (has_prop(c)) c->prop_counter++;
    c->learned_now = false;
    if (c->prof) {
      DL_CHECK(cudaStreamSynchronize(c->st));
      for (int k = 0; k < 8; ++k) {
        float ms = 0.f;
        DL_CHECK(cudaEventElapsedTime(&ms, c->ev[k], c->ev[k + 1]));
        c->phase_ms[k] += ms;
      }
      c->phase_count++;
    }
  }
  if (kind == 0) {
    DL_CHECK(cudaMemcpyAsync(D, dD, sizeof(float) * (size_t)c->n * c->p, cudaMemcpyDeviceToHost, c->st));
    // all s*m entries (the caller's capacity), so no synchronisation is needed to learn nnz;
    // entries past colptr[m] are unspecified
    DL_CHECK(cudaMemcpyAsync(colptr, dcp, sizeof(int64_t) * (size_t)(m + 1), cudaMemcpyDeviceToHost, c->st));
    DL_CHECK(cudaMemcpyAsync(rowidx, dri, sizeof(int32_t) * (size_t)m * s, cudaMemcpyDeviceToHost, c->st));
    DL_CHECK(cudaMemcpyAsync(val, dv, sizeof(float) * (size_t)m * s, cudaMemcpyDeviceToHost, c->st));
  }
  if (rmse)
    DL_CHECK(cudaMemcpyAsync(rmse, c->rmse, sizeof(double) * 2 * (size_t)iters,
                             cudaMemcpyDeviceToHost, c->st));
  if (kind == 0 || rmse) return take_device_error(c);
  return DL_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------
// Autotuner: coordinate search over the launch shapes of one context, timing one
// DL iteration per candidate (median of 3, CUDA events) from a scratch copy of D.

namespace {

float time_iteration(dl_ctx* c, const float* Y, int64_t m, const float* D, float* Dtmp, int s,
                     int64_t* cp, int32_t* ri, float* v, cudaEvent_t e0, cudaEvent_t e1) {
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    cudaMemcpyAsync(Dtmp, D, sizeof(float) * (size_t)c->n * c->p, cudaMemcpyDeviceToDevice, c->st);
    cudaMemsetAsync(c->iter, 0, sizeof(int), c->st);
    cudaEventRecord(e0, c->st);
    if (enq_iteration(c, Y, m, Dtmp, s, cp, ri, v) != cudaSuccess) return 1e30f;
    cudaEventRecord(e1, c->st);
    if (cudaEventSynchronize(e1) != cudaSuccess) return 1e30f;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  return best;
}

}  // namespace

extern "C" int dl_autotune(dl_ctx* c, const float* Y, int64_t m, const float* D, int s) {
  int rc = check_common(c, m);
  if (rc) return rc;
  if (m < 1 || s < 1 || s > c->s_max || ptr_kind(Y) != 1 || ptr_kind(D) != 1) return DL_EINVAL;
  DevGuard g(c->dev);
  float* Dtmp = nullptr;
  int64_t* cp = nullptr;
  int32_t* ri = nullptr;
  float* v = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (!dalloc(&Dtmp, (size_t)c->n * c->p) || !dalloc(&cp, (size_t)m + 1) ||
      !dalloc(&ri, (size_t)m * s) || !dalloc(&v, (size_t)m * s) ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaFree(Dtmp); cudaFree(cp); cudaFree(ri); cudaFree(v);
    return DL_ENOMEM;
  }
  rc = enq_convert_y(c, Y, m) == cudaSuccess ? DL_OK : DL_ECUDA;
  const bool prof = c->prof;
  c->prof = false;
  int* knobs[4] = {&c->cfg_corr_tc, &c->cfg_omp_warps, &c->cfg_acc_mult, &c->cfg_row_per_sm};
  const int choices[4][3] = {{1, 0, -1}, {4, 2, 1}, {1, 2, -1}, {4, 2, 8}};
  time_iteration(c, Y, m, D, Dtmp, s, cp, ri, v, e0, e1);  // warm-up
  float best = time_iteration(c, Y, m, D, Dtmp, s, cp, ri, v, e0, e1);
  for (int k = 0; k < 4 && rc == DL_OK; ++k) {
    const int keep = *knobs[k];
    int arg = keep;
    for (int q = 0; q < 3; ++q) {
      const int cand = choices[k][q];
      if (cand < 0 || cand == keep) continue;
      if (k == 0 && !dlk::corr_tc_supported(Y, c->p, c->n, c->lda)) continue;
      *knobs[k] = cand;
      const float t = time_iteration(c, Y, m, D, Dtmp, s, cp, ri, v, e0, e1);
      if (t < best) {
        best = t;
        arg = cand;
      }
    }
    *knobs[k] = arg;
  }
  if (cudaStreamSynchronize(c->st) != cudaSuccess) rc = DL_ECUDA;
  c->prof = prof;
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  c->gexec = nullptr;
  c->gkey_seen = 0;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(Dtmp); cudaFree(cp); cudaFree(ri); cudaFree(v);
  cudaMemset(c->err, 0, sizeof(int));
  return rc;
}

extern "C" int dl_last_omp_kernel(dl_ctx* c, int* kind) {
  if (!c || !kind) return DL_EINVAL;
  *kind = c->last_omp;
  return DL_OK;
}

extern "C" int dl_get_config(dl_ctx* c, int* cfg4) {
  if (!c || !cfg4) return DL_EINVAL;
  cfg4[0] = c->cfg_corr_tc;
  cfg4[1] = c->cfg_omp_warps;
  cfg4[2] = c->cfg_acc_mult;
  cfg4[3] = c->cfg_row_per_sm;
  return DL_OK;
}

// ---------------------------------------------------------------------------------
// Batches of independent problems: one context per problem, all problems'
// iterations captured into one CUDA graph with one branch (stream) per problem.

struct dl_batch {
  int count = 0;
  int dev = 0;
  cudaStream_t main = nullptr;
  std::vector<dl_problem> probs;
  std::vector<dl_ctx*> ctxs;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> joins;
  cudaEvent_t fork = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int graph_iters = -1;
  // small problems (dlk::small_supported, FP32): all iterations of all problems in one
  // launch of dlk::small_dl, one CTA per problem
  bool small = false;
  int rule = DL_RULE_AKSVD;
  int ntilde = 0;                              // group size set on the batch (0: n)
  std::vector<dlk::SmallProblem> sp;           // host copies of the descriptors
  dlk::SmallProblem* d_sp = nullptr;           // device descriptors
  void* sbuf = nullptr;                        // slots, previous slots, counts, flags
  double* srmse = nullptr;                     // count x 2 x srmse_iters
  int srmse_iters = 0;
  int* serr = nullptr;
  int64_t small_launches = 0;
};

namespace {

void free_batch(dl_batch* b) {
  if (!b) return;
  DevGuard g(b->dev);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  for (dl_ctx* c : b->ctxs) free_ctx(c);
  for (cudaStream_t st : b->streams) cudaStreamDestroy(st);
  for (cudaEvent_t e : b->joins) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  for (void* q : {(void*)b->d_sp, b->sbuf, (void*)b->srmse, (void*)b->serr})
    if (q) cudaFree(q);
  delete b;
}

// The small-problem path: every problem small enough for one CTA.  Its slot
// buffers live in one allocation.
int setup_small(dl_batch* b) {
  for (const dl_problem& q : b->probs)
    if (!dlk::small_supported(q.p, q.n, q.s)) return DL_OK;  // not eligible: graph path
  size_t words = 0;
  for (const dl_problem& q : b->probs) words += (size_t)4 * q.m * q.s + 2 * (size_t)q.m + 4;
  if (!dalloc((int**)&b->sbuf, words) || !dalloc(&b->d_sp, (size_t)b->count) ||
      !dalloc(&b->serr, 1))
    return DL_ENOMEM;
  DL_CHECK(cudaMemset(b->sbuf, 0, sizeof(int) * words));
  DL_CHECK(cudaMemset(b->serr, 0, sizeof(int)));
  int* w = (int*)b->sbuf;
  for (const dl_problem& q : b->probs) {
    dlk::SmallProblem sp{};
    const size_t ms = (size_t)q.m * q.s;
    sp.Y = q.Y;
    sp.D = q.D;
    sp.p = q.p;
    sp.n = q.n;
    sp.s = q.s;
    sp.m = q.m;
    sp.sidx = w;
    sp.sval = (float*)(w + ms);
    sp.pidx = w + 2 * ms;
    sp.pval = (float*)(w + 3 * ms);
    sp.scnt = w + 4 * ms;
    sp.pcnt = w + 4 * ms + q.m;
    sp.pvalid = w + 4 * ms + 2 * q.m;
    sp.colptr = q.colptr;
    sp.rowidx = q.rowidx;
    sp.cval = q.val;
    w += 4 * ms + 2 * (size_t)q.m + 4;
    b->sp.push_back(sp);
  }
  b->small = true;
  return DL_OK;
}

bool small_active(const dl_batch* b) {
  if (!b->small) return false;
  for (const dl_problem& q : b->probs)
    if (b->ntilde > 0 && b->ntilde < q.n) return false;  // groups: the graph path
  return true;
}

int iterate_small(dl_batch* b, int iters, double* rmse) {
  if (iters > b->srmse_iters) {  // per problem 2 x srmse_iters doubles
    DL_CHECK(cudaStreamSynchronize(b->main));
    if (b->srmse) cudaFree(b->srmse);
    b->srmse = nullptr;
    b->srmse_iters = 0;
    if (!dalloc(&b->srmse, (size_t)b->count * 2 * iters)) return DL_ENOMEM;
    b->srmse_iters = iters;
    for (int k = 0; k < b->count; ++k) b->sp[k].rmse = b->srmse + (size_t)k * 2 * iters;
    // a copy from pageable memory has read the host array when the call returns
    DL_CHECK(cudaMemcpyAsync(b->d_sp, b->sp.data(), sizeof(dlk::SmallProblem) * b->count,
                             cudaMemcpyHostToDevice, b->main));
  }
  DL_CHECK(dlk::small_dl(b->d_sp, b->count, iters, b->rule, b->serr, b->main));
  b->small_launches += 1;
  if (rmse) {
    DL_CHECK(cudaStreamSynchronize(b->main));
    const size_t per = (size_t)2 * b->srmse_iters;
    std::vector<double> h((size_t)b->count * per);
    DL_CHECK(cudaMemcpy(h.data(), b->srmse, sizeof(double) * h.size(), cudaMemcpyDeviceToHost));
    for (int k = 0; k < b->count; ++k)
      std::copy(h.begin() + k * per, h.begin() + k * per + 2 * iters, rmse + (size_t)k * 2 * iters);
    int e = 0;
    DL_CHECK(cudaMemcpy(&e, b->serr, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) {
      DL_CHECK(cudaMemset(b->serr, 0, sizeof(int)));
      return DL_ENUMERIC;
    }
  }
  return DL_OK;
}

cudaError_t enq_batch(dl_batch* b, int iters) {
  cudaError_t e = cudaEventRecord(b->fork, b->main);
  if (e != cudaSuccess) return e;
  for (int k = 0; k < b->count; ++k) {
    dl_ctx* c = b->ctxs[k];
    const dl_problem& q = b->probs[k];
    if ((e = cudaStreamWaitEvent(c->st, b->fork, 0)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(c->iter, 0, sizeof(int), c->st)) != cudaSuccess) return e;
    if ((e = enq_convert_y(c, q.Y, q.m)) != cudaSuccess) return e;
    for (int it = 0; it < iters; ++it)
      if ((e = enq_iteration(c, q.Y, q.m, q.D, q.s, q.colptr, q.rowidx, q.val)) != cudaSuccess)
        return e;
    if ((e = cudaEventRecord(b->joins[k], c->st)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(b->main, b->joins[k], 0)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

extern "C" int dl_batch_create(dl_batch** out, const dl_problem* problems, int count, int precision,
                               int autotune, void* stream) {
  if (!out || !problems || count < 1) return DL_EINVAL;
  for (int k = 0; k < count; ++k) {
    const dl_problem& q = problems[k];
    if (q.m < 1 || !q.Y || !q.D || !q.colptr || !q.rowidx || !q.val || ptr_kind(q.Y) != 1 ||
        ptr_kind(q.D) != 1 || ptr_kind(q.colptr) != 1 || ptr_kind(q.rowidx) != 1 ||
        ptr_kind(q.val) != 1)
      return DL_EINVAL;
  }
  dl_batch* b = new dl_batch();
  cudaGetDevice(&b->dev);
  b->count = count;
  b->main = (cudaStream_t)stream;
  b->probs.assign(problems, problems + count);
  if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) {
    free_batch(b);
    return DL_ECUDA;
  }
  for (int k = 0; k < count; ++k) {
    const dl_problem& q = problems[k];
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
      free_batch(b);
      return DL_ECUDA;
    }
    b->streams.push_back(st);
    b->joins.push_back(ev);
    dl_ctx* c = nullptr;
    const int rc = dl_init(&c, q.p, q.n, q.m, q.s, precision, st);
    if (rc != DL_OK) {
      free_batch(b);
      return rc;
    }
    b->ctxs.push_back(c);
  }
  // one eager iteration per problem (sets kernel attributes outside any capture), then tune
  for (int k = 0; k < count; ++k) {
    dl_ctx* c = b->ctxs[k];
    const dl_problem& q = b->probs[k];
    int rc = autotune ? dl_autotune(c, q.Y, q.m, q.D, q.s) : DL_OK;
    if (rc == DL_OK && !autotune) {
      float* Dtmp = nullptr;
      if (!dalloc(&Dtmp, (size_t)c->n * c->p)) rc = DL_ENOMEM;
      if (rc == DL_OK && (cudaMemcpyAsync(Dtmp, q.D, sizeof(float) * (size_t)c->n * c->p,
                                          cudaMemcpyDeviceToDevice, c->st) != cudaSuccess ||
                          enq_convert_y(c, q.Y, q.m) != cudaSuccess ||
                          enq_iteration(c, q.Y, q.m, Dtmp, q.s, q.colptr, q.rowidx, q.val) !=
                              cudaSuccess ||
                          cudaStreamSynchronize(c->st) != cudaSuccess))
        rc = DL_ECUDA;
      cudaFree(Dtmp);
    }
    if (rc != DL_OK) {
      free_batch(b);
      return rc;
    }
  }
  if (precision == DL_FP32 && setup_small(b) != DL_OK) {
    free_batch(b);
    return DL_ENOMEM;
  }
  *out = b;
  return DL_OK;
}

extern "C" int dl_batch_iterate(dl_batch* b, int iters, double* rmse) {
  if (!b || iters < 0) return DL_EINVAL;
  if (iters == 0) return DL_OK;
  DevGuard g(b->dev);
  if (small_active(b)) return iterate_small(b, iters, rmse);
  for (int k = 0; k < b->count; ++k) {
    dl_ctx* c = b->ctxs[k];
    if ((group_size(c) < c->n || c->rule == DL_RULE_NSGK) &&
        !dlk::jau_vec4(c->p, b->probs[k].Y, b->probs[k].D))
      return DL_ENOTIMPL;
    if (int rc = ensure_rmse(c, iters)) return rc;
  }
  if (!b->gexec || b->graph_iters != iters) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
    if (!b->main) return DL_EINVAL;  // capture needs a non-default stream
    cudaGraph_t graph = nullptr;
    DL_CHECK(cudaStreamBeginCapture(b->main, cudaStreamCaptureModeThreadLocal));
    const cudaError_t e = enq_batch(b, iters);
    const cudaError_t e2 = cudaStreamEndCapture(b->main, &graph);
    if (e != cudaSuccess) return cuda_status(e);
    if (e2 != cudaSuccess) return cuda_status(e2);
    const cudaError_t e3 = cudaGraphInstantiate(&b->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e3 != cudaSuccess) {
      b->gexec = nullptr;
      return cuda_status(e3);
    }
    b->graph_iters = iters;
  }
  DL_CHECK(cudaGraphLaunch(b->gexec, b->main));
  for (dl_ctx* c : b->ctxs) c->launches += (int64_t)iters * (c->omp_kernels[0] + c->scan_kernels + c->jau_kernels);
  if (rmse) {
    DL_CHECK(cudaStreamSynchronize(b->main));
    for (int k = 0; k < b->count; ++k)
      DL_CHECK(cudaMemcpy(rmse + (size_t)k * 2 * iters, b->ctxs[k]->rmse, sizeof(double) * 2 * iters,
                          cudaMemcpyDeviceToHost));
    for (dl_ctx* c : b->ctxs)
      if (int rc = take_device_error(c)) return rc;
  }
  return DL_OK;
}

extern "C" int dl_batch_set_update_rule(dl_batch* b, int rule) {
  if (!b) return DL_EINVAL;
  for (dl_ctx* c : b->ctxs)
    if (int rc = dl_set_update_rule(c, rule)) return rc;
  b->rule = rule;
  if (b->small) {  // the stored representations are dropped
    DevGuard g(b->dev);
    DL_CHECK(cudaStreamSynchronize(b->main));
    for (const dlk::SmallProblem& q : b->sp) DL_CHECK(cudaMemset(q.pvalid, 0, sizeof(int)));
  }
  for (dl_ctx* c : b->ctxs) DL_CHECK(cudaStreamSynchronize(c->st));  // the flag resets
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  b->gexec = nullptr;
  return DL_OK;
}

extern "C" int dl_batch_set_group_size(dl_batch* b, int ntilde) {
  if (!b) return DL_EINVAL;
  for (dl_ctx* c : b->ctxs)
    if (ntilde < 1 || ntilde > c->n) return DL_EINVAL;
  for (dl_ctx* c : b->ctxs) dl_set_group_size(c, ntilde);
  b->ntilde = ntilde;
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  b->gexec = nullptr;
  return DL_OK;
}

extern "C" int dl_batch_destroy(dl_batch* b) {
  free_batch(b);
  return DL_OK;
}

extern "C" int64_t dl_batch_kernel_launches(dl_batch* b) {
  if (!b) return 0;
  int64_t t = b->small_launches;
  for (dl_ctx* c : b->ctxs) t += c->launches;
  return t;
}

extern "C" int dl_batch_config(dl_batch* b, int k, int* cfg4) {
  if (!b || k < 0 || k >= b->count) return DL_EINVAL;
  return dl_get_config(b->ctxs[k], cfg4);
}

// ---------------------------------------------------------------------------------
// Learned support proposer: MLP p -> hidden -> hidden -> n with GELU and sigmoid
// outputs, BCE-with-logits on multi-hot OMP supports, Adam; top-K candidates.

namespace {

constexpr int kPropMaxS = 16;  // support slots gathered per training row

void free_proposer(dl_proposer* P) {
  if (!P) return;
  DevGuard g(P->dev);
  for (int k = 0; k < 6; ++k)
    for (void* q : {(void*)P->w[k], (void*)P->g[k], (void*)P->am[k], (void*)P->av[k]})
      if (q) cudaFree(q);
  for (void* q : {P->wb[0], P->wb[1], P->wb[2], P->wt[0], P->wt[1], P->X, (void*)P->A1,
                  (void*)P->A2, P->H1, P->H2, (void*)P->Z, P->Zb, (void*)P->sup, P->dZ, P->dZt,
                  P->H2t, P->dA2, P->dA2t, P->H1t, P->dA1, P->dA1t, P->Xt, (void*)P->loss,
                  (void*)P->err})
    if (q) cudaFree(q);
  delete P;
}

int64_t proposer_chunks(dl_proposer* P, int64_t m) { return P ? (m + P->ichunk - 1) / P->ichunk : 0; }

// rows of Y (FP32, p wide; selected by idx when given) -> BF16 rows pk wide, and
// their support slots (-1 padded to kPropMaxS) when sup is given.
__global__ void gather_rows_kernel(const float* __restrict__ Y, int p, int pk,
                                   const int64_t* __restrict__ idx, int64_t B,
                                   const int32_t* __restrict__ sup_in, int s,
                                   __nv_bfloat16* __restrict__ X, int32_t* __restrict__ sup_out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= B * pk) return;
  const int64_t b = e / pk;
  const int c = (int)(e - b * pk);
  const int64_t r = idx ? idx[b] : b;
  X[e] = __float2bfloat16_rn(c < p ? Y[r * p + c] : 0.f);
  if (sup_in && c < kPropMaxS) sup_out[b * kPropMaxS + c] = c < s ? sup_in[r * s + c] : -1;
}

cudaError_t enq_forward_chunk(dl_proposer* P, const void* X, int64_t B, bool train) {
  const int h = P->hidden;
  cudaError_t e = dlk::mlp_gemm(X, B, P->wb[0], h, P->pk, dlk::MLP_EPI_GELU_FWD, P->w[1], nullptr, 0,
                                train ? P->A1 : nullptr, P->H1, h, P->err, P->st);
  if (e != cudaSuccess) return e;
  e = dlk::mlp_gemm(P->H1, B, P->wb[1], h, h, dlk::MLP_EPI_GELU_FWD, P->w[3], nullptr, 0,
                    train ? P->A2 : nullptr, P->H2, h, P->err, P->st);
  if (e != cudaSuccess) return e;
  return dlk::mlp_gemm(P->H2, B, P->wb[2], P->n, h, train ? dlk::MLP_EPI_F32 : dlk::MLP_EPI_BF16,
                       P->w[5], nullptr, 0, train ? P->Z : nullptr, train ? nullptr : P->Zb, P->n,
                       P->err, P->st);
}

// Logits/top-K of m signals already converted to BF16 rows (pk wide), in chunks
// of bmax rows whose activations stay in L2.
cudaError_t enq_proposer_forward(dl_proposer* P, const void* Xbf, int64_t m, int K, int32_t* cand,
                                 cudaStream_t st) {
  P->st = st;
  for (int64_t r0 = 0; r0 < m; r0 += P->ichunk) {
    const int64_t B = m - r0 < P->ichunk ? m - r0 : P->ichunk;
    const void* X = (const __nv_bfloat16*)Xbf + r0 * P->pk;
    cudaError_t e = enq_forward_chunk(P, X, B, false);
    if (e != cudaSuccess) return e;
    if ((e = dlk::mlp_topk(P->Zb, B, P->n, K, cand + r0 * K, st)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// One training step on B gathered rows already in P->X / P->sup.
cudaError_t enq_train_step(dl_proposer* P, int64_t B, float lr) {
  const int h = P->hidden, n = P->n;
  cudaError_t e = enq_forward_chunk(P, P->X, B, true);
  if (e != cudaSuccess) return e;
  if ((e = dlk::mlp_bce_grad(P->Z, B, n, P->sup, kPropMaxS, P->dZ, P->loss, P->st))) return e;
  // layer 3
  if ((e = dlk::mlp_transpose(P->dZ, B, n, P->dZt, P->st))) return e;
  if ((e = dlk::mlp_transpose(P->H2, B, h, P->H2t, P->st))) return e;
  if ((e = dlk::mlp_gemm(P->dZt, n, P->H2t, h, (int)B, dlk::MLP_EPI_F32, nullptr, nullptr, 0, P->g[4],
                         nullptr, h, P->err, P->st)))
    return e;
  if ((e = dlk::mlp_colsum(P->dZ, B, n, P->g[5], P->st))) return e;
  if ((e = dlk::mlp_transpose(P->wb[2], n, h, P->wt[1], P->st))) return e;
  if ((e = dlk::mlp_gemm(P->dZ, B, P->wt[1], h, n, dlk::MLP_EPI_GELU_BWD, nullptr, P->A2, h, nullptr,
                         P->dA2, h, P->err, P->st)))
    return e;
  // layer 2
  if ((e = dlk::mlp_transpose(P->dA2, B, h, P->dA2t, P->st))) return e;
  if ((e = dlk::mlp_transpose(P->H1, B, h, P->H1t, P->st))) return e;
  if ((e = dlk::mlp_gemm(P->dA2t, h, P->H1t, h, (int)B, dlk::MLP_EPI_F32, nullptr, nullptr, 0, P->g[2],
                         nullptr, h, P->err, P->st)))
    return e;
  if ((e = dlk::mlp_colsum(P->dA2, B, h, P->g[3], P->st))) return e;
  if ((e = dlk::mlp_transpose(P->wb[1], h, h, P->wt[0], P->st))) return e;
  if ((e = dlk::mlp_gemm(P->dA2, B, P->wt[0], h, h, dlk::MLP_EPI_GELU_BWD, nullptr, P->A1, h, nullptr,
                         P->dA1, h, P->err, P->st)))
    return e;
  // layer 1
  if ((e = dlk::mlp_transpose(P->dA1, B, h, P->dA1t, P->st))) return e;
  if ((e = dlk::mlp_transpose(P->X, B, P->pk, P->Xt, P->st))) return e;
  if ((e = dlk::mlp_gemm(P->dA1t, h, P->Xt, P->pk, (int)B, dlk::MLP_EPI_F32, nullptr, nullptr, 0,
                         P->g[0], nullptr, P->pk, P->err, P->st)))
    return e;
  if ((e = dlk::mlp_colsum(P->dA1, B, h, P->g[1], P->st))) return e;
  if (lr > 0.f) {
    ++P->step;
    for (int k = 0; k < 6; ++k)
      if ((e = dlk::mlp_adam(P->w[k], P->g[k], P->am[k], P->av[k], P->wlen[k], lr, P->step,
                             (k % 2 == 0) ? P->wb[k / 2] : nullptr, P->st)))
        return e;
  }
  return cudaSuccess;
}

}  // namespace

extern "C" int dl_proposer_create(dl_proposer** out, int p, int n, int hidden, int64_t batch,
                                  void* stream) {
  if (!out || p < 1 || p > DL_MAX_P || n < 64 || n > DL_MAX_N || n % 64 || hidden < 64 ||
      hidden % 64 || batch < 64 || batch % 64 || !dlk::mlp_gemm_supported())
    return DL_EINVAL;
  dl_proposer* P = new dl_proposer();
  cudaGetDevice(&P->dev);
  P->p = p;
  P->pk = (p + 63) / 64 * 64;
  P->n = n;
  P->hidden = hidden;
  P->bmax = batch;
  P->ichunk = batch > 16384 ? batch : 16384;
  P->st = (cudaStream_t)stream;
  const int64_t h = hidden, B = batch, BI = P->ichunk;
  const int64_t lens[6] = {h * P->pk, h, h * h, h, (int64_t)n * h, n};
  bool ok = true;
  for (int k = 0; k < 6 && ok; ++k) {
    P->wlen[k] = lens[k];
    ok = dalloc(&P->w[k], lens[k]) && dalloc(&P->g[k], lens[k]) && dalloc(&P->am[k], lens[k]) &&
         dalloc(&P->av[k], lens[k]);
    if (ok) ok = cudaMemset(P->w[k], 0, lens[k] * 4) == cudaSuccess &&
                 cudaMemset(P->am[k], 0, lens[k] * 4) == cudaSuccess &&
                 cudaMemset(P->av[k], 0, lens[k] * 4) == cudaSuccess;
  }
  const size_t b2 = 2;  // BF16 bytes
  ok = ok && dalloc((uint8_t**)&P->wb[0], lens[0] * b2) && dalloc((uint8_t**)&P->wb[1], lens[2] * b2) &&
       dalloc((uint8_t**)&P->wb[2], lens[4] * b2) && dalloc((uint8_t**)&P->wt[0], lens[2] * b2) &&
       dalloc((uint8_t**)&P->wt[1], lens[4] * b2) && dalloc((uint8_t**)&P->X, B * P->pk * b2) &&
       dalloc(&P->A1, B * h) && dalloc(&P->A2, B * h) && dalloc((uint8_t**)&P->H1, BI * h * b2) &&
       dalloc((uint8_t**)&P->H2, BI * h * b2) && dalloc(&P->Z, B * n) &&
       dalloc((uint8_t**)&P->Zb, BI * n * b2) && dalloc(&P->sup, B * kPropMaxS) &&
       dalloc((uint8_t**)&P->dZ, B * n * b2) && dalloc((uint8_t**)&P->dZt, B * n * b2) &&
       dalloc((uint8_t**)&P->H2t, B * h * b2) && dalloc((uint8_t**)&P->dA2, B * h * b2) &&
       dalloc((uint8_t**)&P->dA2t, B * h * b2) && dalloc((uint8_t**)&P->H1t, B * h * b2) &&
       dalloc((uint8_t**)&P->dA1, B * h * b2) && dalloc((uint8_t**)&P->dA1t, B * h * b2) &&
       dalloc((uint8_t**)&P->Xt, B * P->pk * b2) && dalloc(&P->loss, 1) && dalloc(&P->err, 1) &&
       cudaMemset(P->err, 0, sizeof(int)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_proposer(P);
    return DL_ENOMEM;
  }
  *out = P;
  return DL_OK;
}

extern "C" int dl_proposer_destroy(dl_proposer* P) {
  free_proposer(P);
  return DL_OK;
}

extern "C" int dl_proposer_set_weights(dl_proposer* P, const float* W1, const float* b1,
                                       const float* W2, const float* b2, const float* W3,
                                       const float* b3) {
  if (!P || !W1 || !b1 || !W2 || !b2 || !W3 || !b3) return DL_EINVAL;
  DevGuard g(P->dev);
  // W1 arrives hidden x p; store it hidden x pk with zero padding
  DL_CHECK(cudaMemsetAsync(P->w[0], 0, P->wlen[0] * 4, P->st));
  DL_CHECK(cudaMemcpy2DAsync(P->w[0], (size_t)P->pk * 4, W1, (size_t)P->p * 4, (size_t)P->p * 4,
                             (size_t)P->hidden, cudaMemcpyHostToDevice, P->st));
  const float* src[6] = {nullptr, b1, W2, b2, W3, b3};
  for (int k = 1; k < 6; ++k)
    DL_CHECK(cudaMemcpyAsync(P->w[k], src[k], P->wlen[k] * 4, cudaMemcpyHostToDevice, P->st));
  for (int k = 0; k < 3; ++k) DL_CHECK(dlk::mlp_to_bf16(P->w[2 * k], P->wlen[2 * k], P->wb[k], P->st));
  for (int k = 0; k < 6; ++k) {
    DL_CHECK(cudaMemsetAsync(P->am[k], 0, P->wlen[k] * 4, P->st));
    DL_CHECK(cudaMemsetAsync(P->av[k], 0, P->wlen[k] * 4, P->st));
  }
  P->step = 0;
  DL_CHECK(cudaStreamSynchronize(P->st));
  return DL_OK;
}

// which = 0: weights, 1: gradients of the last training step (host FP32, W1 hidden x p).
extern "C" int dl_proposer_get(dl_proposer* P, int which, float* W1, float* b1, float* W2, float* b2,
                               float* W3, float* b3) {
  if (!P || (which != 0 && which != 1) || !W1 || !b1 || !W2 || !b2 || !W3 || !b3) return DL_EINVAL;
  DevGuard g(P->dev);
  float** src = which ? P->g : P->w;
  DL_CHECK(cudaStreamSynchronize(P->st));
  DL_CHECK(cudaMemcpy2D(W1, (size_t)P->p * 4, src[0], (size_t)P->pk * 4, (size_t)P->p * 4,
                        (size_t)P->hidden, cudaMemcpyDeviceToHost));
  float* dst[6] = {nullptr, b1, W2, b2, W3, b3};
  for (int k = 1; k < 6; ++k)
    DL_CHECK(cudaMemcpy(dst[k], src[k], P->wlen[k] * 4, cudaMemcpyDeviceToHost));
  return DL_OK;
}

extern "C" int dl_proposer_train(dl_proposer* P, const float* Y, int64_t m, const int32_t* sup, int s,
                                 const int64_t* perm, int64_t batch, float lr, double* mean_loss) {
  if (!P || !Y || !sup || m < 1 || s < 1 || s > kPropMaxS || batch < 64 || batch > P->bmax ||
      batch % 64 || ptr_kind(Y) != 1 || ptr_kind(sup) != 1 || (perm && ptr_kind(perm) != 1))
    return DL_EINVAL;
  DevGuard g(P->dev);
  DL_CHECK(cudaMemsetAsync(P->loss, 0, sizeof(double), P->st));
  int64_t steps = 0;
  for (int64_t r0 = 0; r0 + batch <= m; r0 += batch, ++steps) {
    const int64_t tot = batch * P->pk;
    gather_rows_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, P->st>>>(
        perm ? Y : Y + r0 * P->p, P->p, P->pk, perm ? perm + r0 : nullptr, batch, perm ? sup : sup + r0 * s,
        s, (__nv_bfloat16*)P->X, P->sup);
    DL_CHECK(cudaGetLastError());
    DL_CHECK(enq_train_step(P, batch, lr));
  }
  if (steps == 0) return DL_EINVAL;
  if (mean_loss) {
    double h = 0.0;
    DL_CHECK(cudaMemcpyAsync(&h, P->loss, sizeof(double), cudaMemcpyDeviceToHost, P->st));
    DL_CHECK(cudaStreamSynchronize(P->st));
    *mean_loss = h / (double)steps;
  }
  int herr = 0;
  DL_CHECK(cudaMemcpy(&herr, P->err, sizeof(int), cudaMemcpyDeviceToHost));
  return herr ? DL_ETIMEOUT : DL_OK;
}

extern "C" int dl_proposer_forward(dl_proposer* P, const float* Y, int64_t m, float* logits,
                                   int32_t* cand, int K) {
  if (!P || !Y || m < 1 || ptr_kind(Y) != 1 || (!logits && !cand) || (cand && (K < 1 || K > 32)))
    return DL_EINVAL;
  DevGuard g(P->dev);
  for (int64_t r0 = 0; r0 < m; r0 += P->bmax) {
    const int64_t B = m - r0 < P->bmax ? m - r0 : P->bmax;
    const int64_t tot = B * P->pk;
    gather_rows_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, P->st>>>(
        Y + r0 * P->p, P->p, P->pk, nullptr, B, nullptr, 0, (__nv_bfloat16*)P->X, nullptr);
    DL_CHECK(cudaGetLastError());
    if (logits) {
      DL_CHECK(enq_forward_chunk(P, P->X, B, true));
      DL_CHECK(cudaMemcpyAsync(logits + r0 * P->n, P->Z, sizeof(float) * B * P->n,
                               cudaMemcpyDeviceToDevice, P->st));
    }
    if (cand) {
      DL_CHECK(enq_forward_chunk(P, P->X, B, false));
      DL_CHECK(dlk::mlp_topk(P->Zb, B, P->n, K, cand + r0 * K, P->st));
    }
  }
  DL_CHECK(cudaStreamSynchronize(P->st));
  return DL_OK;
}

// Attach the learned proposer P, or (P null, corr) the network-free one.
static int attach_proposer(dl_ctx* c, dl_proposer* P, bool corr, int K, int full_every, double tol) {
  if (!c) return DL_EINVAL;
  DevGuard g(c->dev);
  if (!P && !corr) {
    c->prop = nullptr;
    c->prop_corr = false;
    return DL_OK;
  }
  if ((P && (P->p != c->p || P->n != c->n)) || K < c->s_max || K > 32 || full_every < 1 ||
      tol < 0 || !dlk::omp_restricted_supported(c->n, c->s_max, K))
    return DL_EINVAL;
  const size_t mm = (size_t)c->m_max;
  if (!c->rr_ref) {
    if (!dalloc(&c->rr_ref, mm) || !dalloc(&c->rr_L, mm) || !dalloc(&c->fb_list, mm) ||
        !dalloc(&c->fb_count, 1))
      return DL_ENOMEM;
    DL_CHECK(cudaMemset(c->fb_count, 0, sizeof(int)));
  }
  if (P && !c->Ybf && !dalloc((uint8_t**)&c->Ybf, mm * P->pk * 2)) return DL_ENOMEM;
  if (c->cand) cudaFree(c->cand);
  c->cand = nullptr;
  if (!dalloc(&c->cand, mm * K)) return DL_ENOMEM;
  c->prop = P;
  c->prop_corr = corr && !P;
  c->prop_K = K;
  c->prop_full_every = full_every;
  c->prop_tol2 = (float)((1.0 + tol) * (1.0 + tol));
  c->prop_counter = 0;
  if (c->gexec_learned) cudaGraphExecDestroy(c->gexec_learned);
  c->gexec_learned = nullptr;
  c->gkey_seen_l = 0;
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  c->gexec = nullptr;
  c->gkey_seen = 0;
  return DL_OK;
}

extern "C" int dl_attach_proposer(dl_ctx* c, dl_proposer* P, int K, int full_every, double tol) {
  return attach_proposer(c, P, false, K, full_every, tol);
}

extern "C" int dl_attach_correlation_proposer(dl_ctx* c, int K, int full_every, double tol) {
  return attach_proposer(c, nullptr, true, K, full_every, tol);
}

extern "C" int64_t dl_last_fallbacks(dl_ctx* c) {
  if (!c || !c->fb_count) return c ? 0 : DL_EINVAL;
  DevGuard g(c->dev);
  int h = 0;
  if (cudaMemcpyAsync(&h, c->fb_count, sizeof(int), cudaMemcpyDeviceToHost, c->st) != cudaSuccess ||
      cudaStreamSynchronize(c->st) != cudaSuccess)
    return DL_ECUDA;
  return h;
}
