/*
 * dl_gb300.h -- C ABI of the GB300 (sm_103a) dictionary-learning library.
 *
 * The library implements one dictionary-learning (DL) iteration of
 * Irofti & Dumitrescu, "Overcomplete Dictionary Learning with Jacobi Atom
 * Updates" (arXiv 1509.05054): OMP sparse coding of every signal (Algorithm 1,
 * step 1; Batch-OMP Cholesky form of the OMP-Box tool cited in Section 4)
 * followed by the Jacobi atom update in its AK-SVD form with full parallelism,
 * PAK-SVD with group size n (Section 3, Eq. 3 and Eq. 5, Algorithm 2 with
 * step 4 replaced by Eq. 5).
 *
 * Problem statement (Section 1, Eq. 1): signals Y (p x m), dictionary D
 * (p x n) with unit-norm columns, sparsity s; find D and an s-sparse X
 * (n x m, at most s nonzeros per column) minimising ||Y - D X||_F.
 *
 * Layouts (all single precision unless stated):
 *   Y       p x m, column-major: signal i occupies Y[i*p .. i*p+p).
 *   D       p x n, column-major: atom j occupies D[j*p .. j*p+p).
 *   X       n x m compressed sparse column (CSC): colptr[m+1] int64 with
 *           colptr[0] = 0, rowidx[] int32 atom indices, val[] float
 *           coefficients; column i holds entries colptr[i] .. colptr[i+1]-1,
 *           at most s of them, atom indices strictly ascending.  The caller
 *           sizes rowidx/val for s*m entries.
 *
 * Memory: every array argument is owned by the caller.  Either all array
 * arguments of one call are device pointers (cudaMalloc, or torch tensors on
 * the context's GPU), or all are host pointers (pageable or pinned); in the
 * host case the call stages them through device buffers owned by the context
 * and copies results back before returning (all s*m entries of rowidx/val;
 * those past colptr[m] are unspecified).  A dl_iterate of one iteration with
 * page-locked host buffers on a stream of its own (not the legacy default
 * stream) is run eagerly the first time and, from the second call with the
 * same buffers, sizes and settings, by replaying a CUDA graph of the whole call
 * (uploads, iteration, downloads); host buffers that change between calls are
 * new signals for P-NSGK (no previous representations).  `rmse` outputs are
 * always host memory.  The context owns only its workspace (Gram matrix,
 * correlations, per-signal slots, partial sums, staging buffers).
 *
 * Streams: work is enqueued on the context's stream (set by dl_init or
 * dl_set_stream) and is asynchronous for device pointers unless a host `rmse`
 * array is requested, in which case the call synchronises the stream before
 * returning.  Calls on one context must not overlap from several host
 * threads.
 *
 * Errors: every entry point returns DL_OK (0) or a negative status.  Argument
 * errors (DL_EINVAL) are detected before anything is enqueued and leave all
 * outputs untouched.  DL_ECUDA reports a CUDA runtime error.  DL_ENUMERIC is
 * reported at the next synchronisation when a kernel met a non-finite input
 * (NaN/Inf in Y or D).  dl_strerror() gives a one-line description.
 */
#ifndef DL_GB300_H
#define DL_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dl_ctx dl_ctx;

/* status codes */
#define DL_OK 0
#define DL_EINVAL (-1)
#define DL_ECUDA (-2)
#define DL_ENUMERIC (-3)
#define DL_ETIMEOUT (-4)
#define DL_ENOMEM (-5)
#define DL_ENOTIMPL (-6)

/* arithmetic of the correlations D^T Y (the Gram D^T D stays FP32-accurate) */
#define DL_FP32 0 /* FP32-accurate (split-TF32 tensor cores, FP32 accumulation) */
#define DL_BF16 1 /* BF16 operands, FP32 accumulation */
#define DL_FP8 2  /* E4M3 operands with per-atom and per-signal scales, FP32 accumulation */

/* compiled limits */
#define DL_MAX_P 128
#define DL_MAX_N 1024
#define DL_MAX_S 16

/*
 * dl_init -- create a context for problems with signal length p, n atoms, up
 * to m_max signals and sparsity up to s_max (Section 1, Eq. 1).
 *   out        receives the new context (unchanged on error).
 *   p          1 <= p <= DL_MAX_P.
 *   n          1 <= n <= DL_MAX_N.
 *   m_max      1 <= m_max; workspace is sized for m_max signals
 *              (about m_max * (4n + 8 s_max + 16) bytes plus O(n^2 + 152 n p)).
 *   s_max      1 <= s_max <= min(p, n, DL_MAX_S).
 *   precision  DL_FP32, DL_BF16 or DL_FP8: the arithmetic of the correlations
 *              D^T Y (mixed precision: BF16, or E4M3 with each atom and each
 *              signal scaled so its largest entry maps to 448, accumulated in
 *              FP32 on the tensor cores).  The Gram D^T D, the OMP loop, the
 *              Cholesky and coefficient solves stay FP32 in every mode; a
 *              signal whose Cholesky pivot falls below 1e-6 is redone in FP64
 *              (see dl_last_resolved).  Shapes the reduced-precision kernel
 *              does not cover (BF16 p > 128, E4M3 p > 256, n > 512) use the
 *              FP32 path.
 *   stream     a cudaStream_t (NULL = the legacy default stream).
 * The context binds to the CUDA device current at the call.
 * Returns DL_OK, DL_EINVAL, DL_ENOMEM or DL_ECUDA.
 */
int dl_init(dl_ctx** out, int p, int n, int64_t m_max, int s_max, int precision, void* stream);

/* dl_set_stream -- enqueue subsequent work of ctx on `stream` (cudaStream_t). */
int dl_set_stream(dl_ctx* ctx, void* stream);

/* dl_destroy -- free the context's workspace; NULL is accepted. */
int dl_destroy(dl_ctx* ctx);

/* dl_strerror -- static one-line description of a status code. */
const char* dl_strerror(int status);

/*
 * omp_code -- sparse coding stage (Algorithm 1, step 1): for every signal y_i
 * (column i of Y), greedy OMP selects at most s atoms of D and the
 * least-squares coefficients on them.  Batch-OMP form: alpha0 = D^T y,
 * G = D^T D; at each of s steps the atom with the largest |alpha_j| among the
 * unselected ones is added (lowest index on ties), the Cholesky factor of
 * G[I,I] grows by one row, and alpha is the correlation of the new residual.
 * A column stops early (fewer than s entries) when max|alpha| is 0, when the
 * new Cholesky pivot is below 1e-6 (numerically dependent atom), or when the
 * residual energy is below 1e-6 ||y||^2.
 *   Y       p x m signals;  m <= m_max of the context.
 *   D       p x n dictionary (unit-norm columns expected; other columns are
 *           accepted and selection then uses the raw correlations d_j^T r).
 *   s       1 <= s <= s_max.
 *   colptr, rowidx, val   X output in CSC form (see the layout notes above).
 * Returns DL_OK, DL_EINVAL, DL_ECUDA or DL_ENUMERIC.
 */
int omp_code(dl_ctx* ctx, const float* Y, int64_t m, const float* D, int s, int64_t* colptr,
             int32_t* rowidx, float* val);

/*
 * jau_update -- atom-update stage of one DL iteration, Jacobi form with full
 * parallelism (PAK-SVD with group size n; Section 3, Eq. 3 and Eq. 5): with
 * E = Y - D X formed once from the input D and X, every atom j used by some
 * signal becomes
 *     d_j' = F x^T / ||F x^T||,  F = E_{I_j} + d_j x_{j,I_j}
 *          ~ E_{I_j} x_{j,I_j}^T + ||x_{j,I_j}||^2 d_j,
 * and its row of X becomes x_{j,I_j}' = F^T d_j' = E_{I_j}^T d_j' +
 * (d_j^T d_j') x_{j,I_j}.  Atoms no signal uses (or whose F x^T is zero) are
 * left unchanged.  The support of X is not changed.
 *   Y       p x m signals.
 *   D       p x n dictionary, updated in place.
 *   colptr, rowidx   X support (CSC, read only; at most s_max per column).
 *   val     X coefficients, updated in place.
 *   rmse2   NULL, or host double[2] receiving ||Y - D X||_F / ||Y||_F before
 *           and after the update (the call then synchronises).
 * Returns DL_OK, DL_EINVAL, DL_ECUDA or DL_ENUMERIC.
 */
int jau_update(dl_ctx* ctx, const float* Y, int64_t m, float* D, const int64_t* colptr,
               const int32_t* rowidx, float* val, double* rmse2);

/*
 * dl_iterate -- `iters` full DL iterations (Algorithm 1 with group size n):
 * omp_code with the current D, then jau_update.  D is updated in place; X
 * (CSC) holds the representation of the last iteration after its atom update.
 *   rmse    NULL, or host double[2*iters]: rmse[2k] = ||Y - D X||_F/||Y||_F
 *           right after sparse coding of iteration k, rmse[2k+1] the same at
 *           the end of iteration k (updated D and X, as Section 4.2 computes
 *           the error at the end of a PAK-SVD iteration).
 * Returns DL_OK, DL_EINVAL, DL_ECUDA or DL_ENUMERIC.
 */
int dl_iterate(dl_ctx* ctx, const float* Y, int64_t m, float* D, int s, int iters,
               int64_t* colptr, int32_t* rowidx, float* val, double* rmse);

/*
 * dl_check_bounded_wait -- failure-path check of the tensor-core kernels: one
 * GPU thread waits on a barrier that nothing ever completes, through the same
 * bounded wait (about 2 s of the GPU's global timer) every mbarrier wait of
 * the library uses, gives up, and flags a timeout in the context's device
 * error word.  No fault and no hang: the context stays usable.  The paper has
 * no counterpart (failure detection of this implementation).  Blocks for about
 * 2 s on the context's stream.  Returns DL_ETIMEOUT when the wait gave up as
 * designed, an earlier pending error of the context (DL_EINVAL, DL_ENUMERIC,
 * DL_ETIMEOUT) if there was one, DL_EINVAL for a null context or DL_ECUDA.
 */
int dl_check_bounded_wait(dl_ctx* ctx);

/*
 * dl_fp32_probe -- measurement aid for the FP32 CUDA-core roofline of the
 * sparse-coding kernel (the OMP greedy loop of Algorithm 1 step 1 is bound by
 * FP32 multiply-adds).  The paper has no counterpart.  Enqueues on `stream`
 * one launch of 4 CTAs x 256 threads per SM, each thread running 8
 * independent chains of float2 multiply-adds `iters` times (packed FFMA2 when
 * `packed` != 0, else scalar FFMA), and writes its FLOP count (FMA = 2) to
 * *flops (host).  The caller times the launch (CUDA events on `stream`);
 * FLOP / time is the SM array's FP32 multiply-add rate at the running clock.
 * `out` is a device buffer of 4 * 256 * (SM count) floats that the kernel
 * never writes in practice (it keeps the chains live).  Returns DL_OK,
 * DL_EINVAL (null pointers, iters < 1) or DL_ECUDA.
 */
int dl_fp32_probe(int packed, int64_t iters, float* out, double* flops, void* stream);

/*
 * dl_set_group_size -- group size ntilde of the atom-update stage (Algorithm 1
 * steps 2-5, Section 3): the atoms are updated in groups of ntilde consecutive
 * atoms [k*ntilde, (k+1)*ntilde), one group after another; the atoms of one
 * group are updated from the same error E = Y - D X (Eq. 3, Eq. 5), which for
 * later groups already includes the atoms and coefficients updated by the
 * earlier ones.  ntilde = n (the default) is the fully parallel Jacobi form
 * PAK-SVD; ntilde = 1 the sequential Gauss-Seidel form AK-SVD.  A group size
 * below n costs one pass over the signals per group and needs the float4 data
 * path (p % 4 == 0, Y and D 16-byte aligned): jau_update and dl_iterate return
 * DL_ENOTIMPL otherwise.  Applies to later jau_update / dl_iterate calls.
 * Returns DL_OK, or DL_EINVAL unless 1 <= ntilde <= n.
 */
int dl_set_group_size(dl_ctx* ctx, int ntilde);

/*
 * dl_set_deterministic -- the order in which the atom-update stage sums
 * U = E X^T and r_j = ||x_j||^2 (Eq. 3, Eq. 5: F x_j^T = U_j + r_j d_j).  The
 * paper fixes no order; floating-point sums depend on it.
 *   on = 0 (default): every signal adds its contributions x_{j,i} e_i into
 *          copies of U in L2 by float vector reductions; the order of those
 *          additions varies from run to run, so D and X are reproducible to
 *          rounding, not bit for bit.
 *   on = 1: the contributions are summed in an order fixed by the signal and
 *          slot indices (per range of signals, each atom's pairs sorted by
 *          signal and slot; then the ranges in order), so repeated runs give
 *          bit-identical D, X and RMSE values.  Slower (about 2x the
 *          accumulation time at p = 64, n = 512, s = 8).  Needs the float4 data
 *          path (p % 4 == 0, Y and D 16-byte aligned; other shapes keep the
 *          default order).
 * Applies to later jau_update / dl_iterate calls.  Returns DL_OK or DL_EINVAL
 * (null context).
 */
int dl_set_deterministic(dl_ctx* ctx, int on);

/*
 * dl_set_update_rule -- how the atom-update stage treats each atom j of a group
 * (Section 3; F = E_{I_j} + d_j x_{j,I_j}, Eq. 3):
 *   DL_RULE_AKSVD (default)  d_j = F x^T / ||F x^T||, then x_{j,I_j} = F^T d_j
 *                            (one power step, Eq. 5: PAK-SVD / AK-SVD);
 *   DL_RULE_SGK              d_j = F x^T / (x x^T), normalised, coefficients
 *                            unchanged (Eq. 6 and Algorithm 2: P-SGK / SGK);
 *   DL_RULE_NSGK             P-NSGK (Eq. 7): the SGK update with Y replaced by
 *                            Z = Y + D X_prev - D X and the representations
 *                            taken from X_prev, the X the previous iteration
 *                            ended with (stored by the context).  The first
 *                            P-NSGK iteration after this call, or after a
 *                            dl_iterate on other signals or sizes, has no
 *                            X_prev and uses its own X (it is then P-SGK).
 *                            Needs the float4 data path like group sizes < n
 *                            (DL_ENOTIMPL otherwise) and allocates the stored
 *                            representations on first use (DL_ENOMEM).
 * AK-SVD and SGK give the same atom direction; SGK and P-NSGK leave X as the
 * coding pass made it.  Applies to later jau_update / dl_iterate calls.
 * Returns DL_OK, DL_EINVAL or DL_ENOMEM.
 */
#define DL_RULE_AKSVD 0
#define DL_RULE_SGK 1
#define DL_RULE_NSGK 2
int dl_set_update_rule(dl_ctx* ctx, int rule);

/*
 * dl_gram -- G = D^T D (n x n, row-major, device), the Gram matrix Batch-OMP
 * works from (the OMP-Box tool of Section 4).  D and G are device pointers.
 * Asynchronous.  Returns DL_OK, DL_EINVAL or DL_ECUDA.
 */
int dl_gram(dl_ctx* ctx, const float* D, float* G);

/*
 * dl_correlate -- A = Y^T D: A[i*n + j] = d_j^T y_i (m x n, row-major,
 * device), the correlations alpha0 = D^T y_i OMP starts from (Algorithm 1,
 * step 1).  Y, D, A are device pointers; m <= m_max.  Asynchronous.
 * Returns DL_OK, DL_EINVAL or DL_ECUDA.
 */
int dl_correlate(dl_ctx* ctx, const float* Y, int64_t m, const float* D, float* A);

/*
 * dl_correlate_noalloc -- the correlations of dl_correlate, A = Y^T D
 * (A[i*n + j] = d_j^T y_i, m x n row-major), computed without allocating any
 * device memory and without a context.  The paper has no counterpart: this is
 * an interface for callers that cannot call cudaMalloc -- code whose device
 * memory is entirely reserved by another allocator (a framework's caching pool
 * or a fixed arena) and code on a latency-critical path that cannot accept an
 * allocation's implicit synchronisation.
 *   Y, D, A  device pointers owned by the caller (inputs Y, D; output A).
 *   p, n     1 <= p <= DL_NOALLOC_MAX_P, 1 <= n <= DL_NOALLOC_MAX_N; larger
 *            sizes return DL_EINVAL.
 *   stream   cudaStream_t the work is enqueued on (asynchronous).
 * Scratch: the TF32 head/tail split of D lives in a fixed file-scope device
 * array of 2 * DL_NOALLOC_MAX_N * DL_NOALLOC_MAX_P floats (256 KB) plus an
 * error word, held on every GPU that loads the library until the process
 * exits.  The first call on each device looks up that array's device address
 * (cudaGetSymbolAddress, no allocation); make that first call before any
 * stream capture.  Every call on a device shares the array and it keeps the
 * previous call's contents (the error word is cleared by each call), so calls
 * whose executions overlap on the GPU (different streams) race: order them.
 * Calls no cudaMalloc, cudaFree or allocating library routine.
 * Returns DL_OK, DL_EINVAL or DL_ECUDA at enqueue time.  A bounded wait of the
 * tensor-core kernel that gives up (the product is then incomplete) is
 * recorded in the scratch array's error word and reported by
 * dl_correlate_noalloc_status, not by this call.
 */
#define DL_NOALLOC_MAX_N 512
#define DL_NOALLOC_MAX_P 64
int dl_correlate_noalloc(const float* Y, int64_t m, const float* D, int p, int n, float* A,
                         void* stream);

/*
 * dl_correlate_noalloc_status -- the device-side status of the allocation-free
 * correlations enqueued so far on the current device.  The paper has no
 * counterpart.  Synchronises `stream` (the stream the calls were enqueued on),
 * copies the error word of the shared scratch array into a host int, clears
 * it, and returns DL_ETIMEOUT if a bounded wait of the tensor-core kernel gave
 * up (its output A is then incomplete), DL_ENUMERIC if a non-finite value was
 * flagged, DL_OK otherwise, or DL_ECUDA if the copy or the synchronisation
 * failed.  Allocates nothing.  The word is shared by every call on the device
 * and each dl_correlate_noalloc call clears it when it starts, so ask for the
 * status after each call whose output matters, before the next call.
 */
int dl_correlate_noalloc_status(void* stream);

/*
 * dl_last_resolved -- synchronise and return how many signals of the most
 * recent sparse-coding pass were redone in FP64 because an FP32 Cholesky pivot
 * fell below 1e-6 (the FP64 pass uses the pivot threshold 1e-12 and the
 * residual threshold 1e-14 ||y||^2), or a negative status.
 */
int64_t dl_last_resolved(dl_ctx* ctx);

/*
 * dl_uses_tensor_cores -- 1 if this context's shape (p % 4 == 0, p <= 64,
 * n <= 1024) takes the split-TF32 tcgen05 path for D^T Y and D^T D, 0 if it
 * takes the FP32 CUDA-core path.  The environment variable
 * DL_FORCE_SIMT_GEMM forces the CUDA-core path.
 */
int dl_uses_tensor_cores(dl_ctx* ctx);

/*
 * dl_autotune -- pick this context's launch shapes for the problem (Y, m, D, s):
 * tensor-core or CUDA-core correlations, OMP warps per CTA (4/2/1), CTAs of the
 * error-accumulation pass (1x/2x), CTAs per SM of the row update (4/2/8), by a
 * coordinate search timing one DL iteration per candidate (best of 3, CUDA
 * events) from a scratch copy of D.  Y and D are device pointers and are not
 * modified.  Allocates and frees temporary device buffers and synchronises.
 * Later calls on the context use the chosen shapes.  Returns DL_OK, DL_EINVAL,
 * DL_ENOMEM or DL_ECUDA.
 */
int dl_autotune(dl_ctx* ctx, const float* Y, int64_t m, const float* D, int s);

/* dl_get_config -- the four launch-shape choices above, in that order. */
int dl_get_config(dl_ctx* ctx, int* cfg4);

/*
 * dl_last_omp_kernel -- which sparse-coding kernel the context's last coding
 * pass (omp_code, dl_iterate) ran (Algorithm 1 step 1), one of
 *   0  Batch-OMP, one warp per signal, from stored correlations alpha0
 *   1  the same with the progressive-Cholesky vectors in TMEM
 *   2  residual-form OMP, the correlations D^T r of every step on the tensor
 *      cores (FP16 hi/lo parts, or BF16 operands in the DL_BF16 form; FP32
 *      accumulation), no stored alpha0; taken for FP32 and BF16 calls without
 *      a proposer with 256 < n <= 512, p <= 64, p % 4 == 0, s <= 8
 *      and at least 3/4 of (SM count x 256) signals; the environment variable
 *      DL_OMP_RES, read by dl_init, turns it off (0) or takes it for every
 *      supported call (2)
 *   3  OMP restricted to proposed candidates (a proposer is attached)
 *  -1  no coding pass yet
 * written to *kind.  Returns DL_OK, or DL_EINVAL for a NULL argument.
 */
int dl_last_omp_kernel(dl_ctx* ctx, int* kind);

/*
 * Batches of independent DL problems of uneven shapes (p, n, m, s each their
 * own), run together: each problem gets its own context (workspace) and CUDA
 * stream; all problems' iterations are captured once into one CUDA graph with
 * one branch per problem, so one graph launch runs every problem's `iters`
 * iterations concurrently (Algorithm 1 per problem, group size n).
 */
typedef struct dl_problem {
  int p, n, s;          /* signal length, atoms, sparsity (limits as dl_init) */
  int64_t m;            /* signals */
  const float* Y;       /* device, p x m column-major */
  float* D;             /* device, p x n column-major, updated in place */
  int64_t* colptr;      /* device CSC output of X: m + 1 */
  int32_t* rowidx;      /* device, capacity s * m */
  float* val;           /* device, capacity s * m */
} dl_problem;

typedef struct dl_batch dl_batch;

/*
 * dl_batch_create -- contexts for `count` problems (pointers are kept: the
 * arrays must stay valid while the batch lives), precision as in dl_init,
 * optional autotuning of every problem (dl_autotune), and one eager iteration
 * of each problem on scratch D (sets kernel attributes before any capture).
 * `stream` must be a non-default cudaStream_t (graph capture).  Returns DL_OK,
 * DL_EINVAL, DL_ENOMEM or DL_ECUDA.
 */
int dl_batch_create(dl_batch** out, const dl_problem* problems, int count, int precision,
                    int autotune, void* stream);

/*
 * dl_batch_iterate -- run `iters` DL iterations of every problem as one CUDA
 * graph launch on the batch stream (the graph is captured on the first call
 * with a given `iters`).  rmse: NULL, or host double[count * 2 * iters] with,
 * for problem k, the pairs of dl_iterate at rmse[k * 2 * iters]; the call then
 * synchronises.  Returns DL_OK, DL_EINVAL, DL_ECUDA or DL_ENUMERIC.
 */
int dl_batch_iterate(dl_batch* batch, int iters, double* rmse);

/*
 * dl_batch_set_update_rule / dl_batch_set_group_size -- dl_set_update_rule and
 * dl_set_group_size applied to every problem of the batch (e.g. the P-NSGK and
 * P-SGK rows of the dictionary-recovery experiment, Section 4.1, as one batch).
 * The next dl_batch_iterate captures its graph again.  The P-NSGK previous
 * representations of each problem persist across dl_batch_iterate calls and
 * are dropped by the next dl_batch_set_update_rule.  dl_batch_iterate returns
 * DL_ENOTIMPL when a group size below n or P-NSGK is set for a problem without
 * the float4 data path (p % 4 == 0, Y and D 16-byte aligned).  Return as the
 * single-context calls (DL_EINVAL for a group size above some problem's n).
 */
int dl_batch_set_update_rule(dl_batch* batch, int rule);
int dl_batch_set_group_size(dl_batch* batch, int ntilde);

/* dl_batch_destroy -- free the batch's contexts, streams and graph. */
int dl_batch_destroy(dl_batch* batch);

/* dl_batch_kernel_launches -- kernels enqueued by all problems of the batch. */
int64_t dl_batch_kernel_launches(dl_batch* batch);

/* dl_batch_config -- launch shapes chosen for problem k (see dl_get_config). */
int dl_batch_config(dl_batch* batch, int k, int* cfg4);

/*
 * Learned support proposer.  A small MLP p -> hidden -> hidden -> n (GELU
 * activations, sigmoid outputs; BF16 weights with FP32 master copies) trained
 * with binary cross-entropy on the multi-hot OMP supports the method itself
 * produces, on the tensor cores with the library's own forward and backward
 * kernels and Adam.  At sparse coding it proposes the K atoms with the largest
 * logits per signal; OMP then runs over those candidates only, and a signal
 * whose residual norm exceeds (1 + tol) times the residual of its last full
 * OMP is coded again by full OMP (the fallback, which also judges the error).
 * This is the learned form of Algorithm 1 step 1; the atom update is unchanged.
 */
typedef struct dl_proposer dl_proposer;

/*
 * dl_proposer_create -- p <= DL_MAX_P, n and hidden multiples of 64, batch (rows
 * per training step and per inference chunk) a multiple of 64.  Weights start
 * at zero: set them with dl_proposer_set_weights.  Returns DL_OK, DL_EINVAL or
 * DL_ENOMEM.
 */
int dl_proposer_create(dl_proposer** out, int p, int n, int hidden, int64_t batch, void* stream);
int dl_proposer_destroy(dl_proposer* prop);

/* Host FP32 weights: W1 hidden x p, b1 hidden, W2 hidden x hidden, b2 hidden,
 * W3 n x hidden, b3 n (row-major, out x in).  Resets the Adam state. */
int dl_proposer_set_weights(dl_proposer* prop, const float* W1, const float* b1, const float* W2,
                            const float* b2, const float* W3, const float* b3);

/* which = 0: current weights; 1: gradients of the last training step.  Host
 * outputs, same shapes as dl_proposer_set_weights.  Synchronises. */
int dl_proposer_get(dl_proposer* prop, int which, float* W1, float* b1, float* W2, float* b2,
                    float* W3, float* b3);

/*
 * dl_proposer_train -- one pass over m training signals in batches of `batch`
 * rows (the last partial batch is skipped): Y device m x p, sup device m x s
 * support slots (-1 = empty), perm device int64 row order or NULL (in order),
 * Adam step lr (lr = 0 computes gradients only).  mean_loss: host, mean BCE of
 * the batches, or NULL.  Synchronises when mean_loss is given.
 */
int dl_proposer_train(dl_proposer* prop, const float* Y, int64_t m, const int32_t* sup, int s,
                      const int64_t* perm, int64_t batch, float lr, double* mean_loss);

/* dl_proposer_forward -- logits (device m x n FP32) and/or the K largest-logit
 * atoms (device m x K int32, ascending) of m signals.  Synchronises. */
int dl_proposer_forward(dl_proposer* prop, const float* Y, int64_t m, float* logits, int32_t* cand,
                        int K);

/*
 * dl_attach_proposer -- sparse coding of dl_iterate on ctx uses the proposer:
 * K candidates (s_max <= K <= 32) per signal; every full_every-th iteration
 * (starting with the first after attaching) runs full OMP for all signals and
 * records their residuals; tol is the fallback margin (0.01 = 1%).  prop NULL
 * detaches.  Returns DL_OK, DL_EINVAL or DL_ENOMEM.
 */
int dl_attach_proposer(dl_ctx* ctx, dl_proposer* prop, int K, int full_every, double tol);

/*
 * dl_attach_correlation_proposer -- the same sparse-coding scheme as
 * dl_attach_proposer (K candidates per signal, OMP restricted to them, full
 * OMP every full_every-th iteration and for the signals whose residual exceeds
 * their last full OMP's by the margin tol), with the candidates taken without
 * a network: the K atoms of largest |d_j^T y| (Algorithm 1 step 1's first
 * correlations).  It is the baseline that shows what the trained network
 * gains.  Replaces an attached learned proposer; dl_attach_proposer(ctx, NULL,
 * ...) detaches either.  Returns DL_OK, DL_EINVAL or DL_ENOMEM.
 */
int dl_attach_correlation_proposer(dl_ctx* ctx, int K, int full_every, double tol);

/* dl_last_fallbacks -- signals sent to full OMP by the most recent learned
 * iteration (synchronises). */
int64_t dl_last_fallbacks(dl_ctx* ctx);

/*
 * dl_sync -- wait for the context's stream and report a pending device-side
 * error (DL_ENUMERIC for non-finite inputs met by a kernel) or DL_OK.
 */
int dl_sync(dl_ctx* ctx);

/*
 * dl_kernel_launches -- number of kernels the library enqueued on this
 * context since it was created (graph replays count each kernel they hold).
 */
int64_t dl_kernel_launches(dl_ctx* ctx);

/*
 * dl_set_profiling -- when on != 0, dl_iterate records CUDA events on the
 * context's stream around each phase of every iteration (also inside the
 * replayed CUDA graph) and synchronises after each iteration to accumulate the
 * per-phase durations.  Turning it on or off resets the accumulated times.
 * Returns DL_OK or DL_EINVAL / DL_ECUDA.
 */
int dl_set_profiling(dl_ctx* ctx, int on);

/*
 * dl_phase_times -- average duration in milliseconds, per profiled iteration,
 * of the phases 0 Gram D^T D, 1 correlations D^T Y, 2 OMP, 3 colptr scan,
 * 4 error accumulation U = E X^T (+ fixed-order reduction), 5 atom update,
 * 6 row update + RMSE partials + CSC write, 7 RMSE finalisation + D copy.
 * Writes min(max_phases, 8) values to ms (host) and returns 8, the number of
 * phases, or DL_EINVAL.
 */
int dl_phase_times(dl_ctx* ctx, double* ms, int max_phases);

#ifdef __cplusplus
}
#endif

#endif /* DL_GB300_H */
