// Internal declarations shared by the library's translation units.
// Nothing here is part of the public C ABI (include/dl_gb300.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dlk {

// Device-side error word bits (read back by the host at synchronisation).
enum : int {
  ERR_NONFINITE = 1,  // NaN/Inf met in Y or D
  ERR_CSC = 2,        // caller CSC column with > s_max entries or atom index out of range
  ERR_TIMEOUT = 4,    // a bounded device wait gave up
};

constexpr float kPivotMin = 1e-6f;     // Cholesky pivot delta below this: dependent atom, stop
constexpr float kResidRel = 1e-6f;     // residual energy below this * ||y||^2: stop
// Long supports (s > 8): a top-two |alpha| gap below kGapTol ||y|| sends the
// signal to the re-solve, which takes the FP64 decisions.  The FP32
// error of alpha after up to 16 steps -- split-TF32 correlations (~2^-22
// relative per product) plus the rounding of the progressive Cholesky updates --
// stays below 1e-6 ||y|| on unit atoms; the tolerance keeps a factor of 4.
constexpr float kGapTol = 4e-6f;

// ---- correlations and Gram --------------------------------------------------
// C[i*ldc + j] = sum_r A[i*p + r] * B[j*p + r]  for i < rows_a, j < rows_b (FP32, CUDA cores)
cudaError_t gemm_nt_simt(const float* A, int64_t rows_a, const float* B, int rows_b, int p, float* C,
                         int64_t ldc, cudaStream_t st);
// G = D D^T (n x n, exactly symmetric), FP32 on the CUDA cores in one short launch.
cudaError_t gram_simt(const float* D, int n, int p, float* G, cudaStream_t st);

// FP32-accurate C = A B^T on tcgen05 tensor cores (split TF32, see k_corr_tc.cu).
// B is given pre-split (B = Bhi + Blo).  Requires corr_tc_supported().
bool corr_tc_supported(const float* A, int p, int n, int64_t ldc);
cudaError_t split_tf32(const float* B, int64_t count, float* hi, float* lo, cudaStream_t st);
cudaError_t corr_tf32x3(const float* A, int64_t rows_a, const float* Bhi, const float* Blo, int n,
                        int p, float* C, int64_t ldc, int* err, cudaStream_t st);
// Two products with the same B in one launch: C0 = A0 B^T and C1 = A1 B^T (A1 may be null).
cudaError_t corr_tf32x3_pair(const float* A0, int64_t rows0, float* C0, int64_t ldc0,
                             const float* A1, int64_t rows1, float* C1, int64_t ldc1,
                             const float* Bhi, const float* Blo, int n, int p, int* err,
                             cudaStream_t st);

// Diagnostic: a wait on an mbarrier nothing arrives at, bounded as in the
// tensor-core kernels; sets ERR_TIMEOUT in *err after about 2 s.
cudaError_t bounded_wait_check(int* err, cudaStream_t st);
// FP32 multiply-add throughput probe (k_diag.cu): launches 4 CTAs per SM running
// independent FMA chains; *flops receives the FLOP count of the launch.
cudaError_t ffma_probe(int packed, int64_t iters, float* out, double* flops, cudaStream_t st);

// Reduced-precision correlations (k_corr_lp.cu): operands converted to padded
// row-major BF16 or E4M3 (+ inverse row scales) buffers, then tcgen05 MMAs.
enum : int { LP_BF16 = 1, LP_E4M3 = 2 };
int lp_row_elems(int kind, int p);  // padded row length in elements
bool corr_lp_supported(int kind, int p, int n, int64_t ldc);
cudaError_t to_lowp(int kind, const float* src, int64_t rows, int p, void* dst, float* inv_scale,
                    cudaStream_t st);
// BF16 correlations of FP32 signals, persistent and pipelined (k_corr_lp.cu): Y is
// converted to BF16 on chip; Dbf = D converted by to_lowp(LP_BF16).  p <= 64, p % 4 == 0.
bool corr_bf16_ws_supported(const float* Y, int p, int n, int64_t ldc);
// C: FP32, or (out_bf16) BF16 rows of ldc elements.
cudaError_t corr_bf16_ws(const float* Y, int64_t rows, const void* Dbf, int n, int p, void* C,
                         bool out_bf16, int64_t ldc, int* err, cudaStream_t st);
cudaError_t corr_lp(int kind, const void* A, int64_t rows_a, const float* a_inv_scale,
                    const void* B, const float* b_inv_scale, int n, int p, float* C, int64_t ldc,
                    int* err, cudaStream_t st);

// ---- OMP ----------------------------------------------------------------------

// Batch-OMP of m signals from their correlations A0 (row i = D^T y_i, stride lda) and G = D^T D.
// Writes s slots per signal (atoms ascending, unused slots idx = -1) and the count.
// Signals stopped by a pivot below kPivotMin, and (s > 8, gap_tol > 0) signals with a
// top-two gap below gap_tol ||y|| at some step, are appended to rs_list (if given) for
// the FP64 re-solve.
cudaError_t omp_batch(const float* A0, int64_t lda, const float* G, int n, const float* Y, int p,
                      int64_t m, int s, int32_t* idx, float* val, int32_t* cnt, int* err,
                      int* rs_list, int* rs_count, int rs_cap, int warps_per_block,
                      float* ores, float gap_tol, cudaStream_t st);

// The same Batch-OMP with the progressive-Cholesky vectors in tensor memory
// (k_omp_tm.cu): persistent CTAs of 4q warps (q = 4, 5, 6).  n = 512, 5 <= s <= 8.
// Residual-form OMP with the correlations of every step on the tensor cores
// (alpha^(k) = D^T r^(k) from FP16 hi/lo parts of D and r, or with bf16 from
// BF16 operands, FP32 accumulation; one persistent CTA per SM, two 128-signal
// tiles in flight); no alpha0 input.  alpha_sel, the Cholesky factor and the
// residual are FP32 in both forms.
// p % 4 == 0, p <= 64, n <= 512, s <= 8, Y and D 16-byte aligned.  Signals with
// a pivot below kPivotMin are listed for omp_resolve64.
bool omp_res_supported(int p, int n, int s, const float* Y, const float* D);
int64_t omp_res_round_signals();  // signals of one round of tiles (all SMs, all slots)
cudaError_t omp_res(const float* Y, int64_t m, int p, const float* D, int n, const float* G, int s,
                    int32_t* idx, float* val, int32_t* cnt, int* err, int* rs_list, int* rs_count,
                    int rs_cap, bool bf16, cudaStream_t st);
bool omp_tm_supported(int n, int s);
// A0: FP32 rows, or BF16 rows (a0_bf16) of lda elements.
cudaError_t omp_batch_tm(int q, const void* A0, bool a0_bf16, int64_t lda, const float* G, int n,
                         const float* Y, int p, int64_t m, int s, int32_t* idx, float* val,
                         int32_t* cnt, int* err, int* rs_list, int* rs_count, int rs_cap,
                         cudaStream_t st);

// ---- whole DL iterations of small problems, one CTA per problem (k_small.cu) ----
// Problems with p <= 32, n <= 64, s <= 8 and group size n: a batch runs all its
// problems' iterations in one launch.
struct SmallProblem {
  const float* Y;        // m x p
  float* D;              // n x p (in/out)
  int p, n, s;
  int64_t m;
  int32_t* sidx;         // m x s slots of the current X
  float* sval;
  int32_t* scnt;
  int32_t* pidx;         // m x s slots of the previous X (P-NSGK)
  float* pval;
  int32_t* pcnt;
  int* pvalid;           // the previous X exists
  double* rmse;          // 2 per iteration
  int64_t* colptr;       // CSC of the final X
  int32_t* rowidx;
  float* cval;
};
constexpr int kSmallP = 32, kSmallN = 64, kSmallS = 8;
bool small_supported(int p, int n, int s);
cudaError_t small_dl(const SmallProblem* probs, int count, int iters, int rule, int* err,
                     cudaStream_t st);

// OMP restricted to K ascending candidates per signal (the learned proposer's
// path) and the full-OMP fallback of listed signals.  ores: residual-energy
// estimate per signal; ref_res/tol2: fallback when ores > tol2 * ref_res.
bool omp_restricted_supported(int n, int s, int K);
cudaError_t omp_restricted(const int32_t* cand, int K, const float* D, const float* G, int n,
                           const float* Y, int p, int64_t m, int s, int32_t* idx, float* val,
                           int32_t* cnt, float* ores, const float* ref_res, float tol2, int* fb_list,
                           int* fb_count, int* err, cudaStream_t st);
cudaError_t omp_listed(const int* list, const int* count, const float* A0, int64_t lda,
                       const float* G, int n, const float* Y, int p, int s, int32_t* idx, float* val,
                       int32_t* cnt, float* ores, int* err, int* rl, int* rc, int rcap,
                       cudaStream_t st);

// ---- learned proposer (k_mlp.cu) ----------------------------------------------
enum : int { MLP_EPI_BF16 = 0, MLP_EPI_F32 = 1, MLP_EPI_GELU_FWD = 2, MLP_EPI_GELU_BWD = 3 };
bool mlp_gemm_supported();
// C[M x N] = A[M x K] B[N x K]^T, BF16 row-major operands (K % 64 == 0), epilogue op.
cudaError_t mlp_gemm(const void* A, int64_t M, const void* B, int N, int K, int op, const float* bias,
                     const float* aux, int64_t ldaux, float* out_f32, void* out_bf16, int64_t ldc,
                     int* err, cudaStream_t st);
cudaError_t mlp_transpose(const void* in, int64_t R, int64_t C, void* out, cudaStream_t st);
cudaError_t mlp_to_bf16(const float* in, int64_t count, void* out, cudaStream_t st);
cudaError_t mlp_bce_grad(const float* z, int64_t B, int n, const int32_t* sup, int s, void* dz,
                         double* loss, cudaStream_t st);
cudaError_t mlp_colsum(const void* in, int64_t R, int C, float* out, cudaStream_t st);
cudaError_t mlp_adam(float* w, const float* g, float* m, float* v, int64_t count, float lr, int t,
                     void* wbf, cudaStream_t st);
cudaError_t mlp_topk(const void* z, int64_t m, int n, int K, int32_t* cand, cudaStream_t st);
// The K largest |A[i][j]| of each row (row i at A + i * lda), indices ascending.
cudaError_t topk_abs(const float* A, int64_t lda, int64_t m, int n, int K, int32_t* cand,
                     cudaStream_t st);

// Re-solve (k_resolve.cu) of the listed signals with the FP64 Batch-OMP's decisions and
// coefficients (FP64 residual and Cholesky factor, FP32 correlations with an exact check of
// the atoms within their error bound), overwriting their slots.  G: the FP32 Gram matrix;
// A0 (row i = FP32 D^T y_i, stride lda) or null to take D^T y here.  p <= 128, s <= 16.
constexpr int DL_RESOLVE_SMAX = 16;
constexpr int DL_RESOLVE_WARPS = 608;  // CTAs of one warp
cudaError_t omp_resolve64(const float* Y, int p, const float* D, const float* G, const float* A0,
                          int64_t lda, int n, int s, const int* list, const int* count, int cap,
                          int32_t* idx, float* val, int32_t* cnt, cudaStream_t st);
bool omp_supported(int n, int s);

// ---- JAU / PAK-SVD (group size n) ---------------------------------------------
struct JauWork {
  float* Upart;     // [nb_accum][n*p + n] per-CTA partial U = E X^T and r = row energies
  float* U;         // [n*p + n] reduced
  double* epart_a;  // [nb_accum][2]  (||E||^2, ||Y||^2) partials
  double* epart_b;  // [nb_row]       ||Y - D'X'||^2 partials
  float* Dn;        // [n*p] updated atoms
  float* C;         // [n]   d_j^T d_j'
  int nb_accum;
  int nb_row;
  // group of atoms [a0, a1) being updated (a1 = 0: all n, the Jacobi form); the
  // float4 passes then accumulate and update only slots of the group, and
  // energies selects whether pass A writes the (||E||^2, ||Y||^2) partials
  int a0 = 0, a1 = 0;
  bool energies = true;
  // SGK rule (Eq. 6, P-SGK): atoms as in AK-SVD, coefficients left as they are
  bool sgk = false;
  // P-NSGK (Eq. 7, float4 form): previous representations (slots), whether they
  // exist yet (device flag), and the dictionary the iteration started from
  bool nsgk = false;
  const int32_t* pidx = nullptr;
  const float* pval = nullptr;
  const int32_t* pcnt = nullptr;
  const int* pvalid = nullptr;
  const float* D0 = nullptr;
  // pass A in its deterministic form (jau_det_supported): nb_accum ranges of signals,
  // one slice of Upart each
  bool det = false;
};
// Grid sizes: mult selects 1x/2x the base CTA count of the accumulation pass
// and 2/4/8 CTAs per SM for the row pass; *_max give the partial-buffer sizes.
constexpr int kUCopies = 16;  // copies of U the float4 accumulation spreads its L2 reductions over
// Floats per copy of U (n p atom sums, then n row energies), padded to a
// multiple of 4 so that every copy, and with p % 4 == 0 every atom row in it,
// starts on a 16-byte boundary for the float4 reductions; U and each slice of
// the partial buffer are allocated with this length.
__host__ __device__ inline size_t jau_ulen(int p, int n) { return ((size_t)n * p + n + 3) / 4 * 4; }
int jau_accum_blocks(int p, int n, int mult);
int jau_accum_blocks_max(int p, int n);
int jau_row_blocks(int per_sm);
int jau_row_blocks_max();
size_t jau_accum_smem(int p, int n);
// float4 passes (p % 4 == 0, Y and D 16-byte aligned); kernel launches of the JAU passes.
bool jau_vec4(int p, const float* Y, const float* D);
// Pass A with a fixed summation order, bitwise reproducible (float4 rows, p <= 128,
// n <= 1024, s <= 16, a range of signals per CTA in shared memory); its CTA count.
bool jau_det_supported(int p, int n, int s, const float* Y, const float* D);
int64_t jau_det_ranges(int64_t m, int p, int n, int s);
int jau_launches(int p, const float* Y, const float* D);

cudaError_t jau_accumulate(const float* Y, int p, int64_t m, const float* D, int n, int s,
                           const int32_t* idx, const float* val, const int32_t* cnt,
                           const JauWork& w, int* err, cudaStream_t st);
cudaError_t jau_atoms(const float* D, int p, int n, const JauWork& w, cudaStream_t st);
// x' = E^T d' + c x per slot; writes slots (val) and, when csc_val != nullptr, the CSC arrays.
cudaError_t jau_rows(const float* Y, int p, int64_t m, const float* D, int n, int s,
                     const int32_t* idx, float* val, const int32_t* cnt, const JauWork& w,
                     const int64_t* colptr, int32_t* csc_rowidx, float* csc_val, cudaStream_t st);
// rmse_out[2*(*iter)] / [2*(*iter)+1] from the partials, then ++*iter (device counter).
// RMSE before/after into rmse_out[2*iter..], iter += 1, and D = Dn (updated atoms).
cudaError_t jau_finalize(const JauWork& w, double* rmse_out, int* iter, float* D, int n, int p,
                         cudaStream_t st);

// ---- CSC <-> slots --------------------------------------------------------------
int64_t scan_blocks(int64_t m);
cudaError_t counts_to_colptr(const int32_t* cnt, int64_t m, int64_t* bsum, int64_t* colptr,
                             cudaStream_t st);
cudaError_t slots_to_csc(const int32_t* idx, const float* val, const int32_t* cnt, int64_t m,
                         int s, const int64_t* colptr, int32_t* rowidx, float* cval,
                         cudaStream_t st);
cudaError_t csc_to_slots(const int64_t* colptr, const int32_t* rowidx, const float* cval,
                         int64_t m, int n, int s, int32_t* idx, float* val, int32_t* cnt,
                         int* err, cudaStream_t st);

int num_sms();

}  // namespace dlk
