/*
 * dpp.h — C ABI of the GB300 (sm_103a) factorization-based DPP sampler.
 *
 * Method: J. Poulson, "High-performance sampling of generic Determinantal
 * Point Processes" (arXiv:1905.00165).
 *   - A DPP with marginal kernel K (n x n, complex or real) is defined by
 *     P[Y subset of the sample] = det(K_Y) (Section 2, Definition).
 *   - Sampling is an unpivoted right-looking LU factorization of K in which
 *     the j-th pivot d_j (the conditional inclusion probability of index j)
 *     drives a Bernoulli draw: keep j, or subtract 1 from the pivot and reject
 *     j; then the column is scaled and the Schur complement updated
 *     (Algorithm 1, Theorem 1, Props. 3-5). For Hermitian K the same process
 *     is an unpivoted LDL^H factorization with half the work (Theorem 1).
 *   - The blocked form factors a diagonal block with the sequential decisions,
 *     solves the two panels against it and applies a rank-nb Schur update
 *     (Algorithms 3 and 4, Section 4).
 *   - log P(Y) = sum_j log|d_j| over the final pivots, and on return the
 *     factored matrix holds the LU (LDL^H) factors of K - 1_{Y^c}
 *     (Algorithm 1's caption; Theorem 1).
 *
 * Conventions shared by every entry point
 *   - Matrices are column-major: entry (i, j) is at ptr[i + j * ld], ld >= n.
 *     Hermitian entry points read (and write) only the lower triangle.
 *   - Every pointer argument named "device" must point to device memory of the
 *     current CUDA device. The caller owns every buffer; the library allocates
 *     nothing per call and never writes the input K (unless factor_out == K).
 *   - All work is enqueued on `stream` (a cudaStream_t passed as void*, NULL =
 *     legacy default stream) and is asynchronous: results are valid once the
 *     stream has been synchronised. Calls are capture-safe (no synchronisation
 *     and no allocation inside).
 *   - Uniforms: unless an explicit `uniforms` array is given, u_j is drawn from
 *     Philox4x32-10 (Salmon et al., SC'11) with key = (seed & 0xffffffff,
 *     seed >> 32), counter = (j, instance & 0xffffffff, instance >> 32, 0),
 *     and u_j = ((x0 << 21 | x1 >> 11) + 0.5) * 2^-53, which lies in (0, 1).
 *   - Decision: index j is kept iff u_j < Re(d_j); otherwise d_j -= 1.
 *     Hermitian pivots are real (the imaginary part is dropped).
 *   - Host-detectable errors are returned as dpp_status (and described by
 *     dpp_last_error()); nothing is enqueued when a call returns an error.
 *     Errors detected on the device are OR-ed into dpp_result.status.
 */
#ifndef DPP_H_
#define DPP_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DPP_ABI_VERSION 1

typedef enum {
  DPP_OK = 0,
  DPP_ERR_INVALID_ARG = 1, /* bad size, pointer, alignment or enum       */
  DPP_ERR_CUDA = 2,        /* a CUDA runtime call failed                 */
  DPP_ERR_WORKSPACE = 3,   /* workspace too small or misaligned (256 B) */
  DPP_ERR_UNSUPPORTED = 4  /* combination not implemented (see below)   */
} dpp_status;

/* Element type of K, of factor_out and of dK. */
typedef enum {
  DPP_R64 = 0,  /* double                                    */
  DPP_C128 = 1  /* double complex, interleaved (re, im) pairs */
} dpp_dtype;

/* Arithmetic of the trailing Schur-complement update (step a3).
 *   DPP_PREC_FP64   : everything in FP64.
 *   DPP_PREC_3XTF32 : FP32 working copy; trailing update as three TF32
 *                     tensor-core products (hi*hi + hi*lo + lo*hi) with FP32
 *                     accumulation; pivots, decisions and log P in FP64; any
 *                     pivot whose uniform lies within the propagated error
 *                     bound of its threshold is recomputed in FP64 from the
 *                     original K before its decision.
 *   DPP_PREC_BF16X6 : as 3XTF32, but the trailing update splits each FP32
 *                     operand into three BF16 pieces (which represent it
 *                     exactly) and issues the six products of combined order
 *                     <= 2 on the BF16 tensor path: the same tensor time as
 *                     3XTF32 with FP32-level accuracy.                      */
typedef enum {
  DPP_PREC_FP64 = 0,
  DPP_PREC_3XTF32 = 1,
  DPP_PREC_BF16X6 = 2,
  DPP_PREC_FP32 = 3  /* FP32 SIMT updates, FP64 pivots and recomputes (batched) */
} dpp_precision;

/* Bits of dpp_result.status (device-side outcome of one draw). */
#define DPP_RES_OK 0
#define DPP_RES_NONFINITE 1     /* a pivot was NaN or Inf                     */
#define DPP_RES_TIMEOUT 2       /* a bounded device wait expired             */
#define DPP_RES_INADMISSIBLE 4  /* warning: a pivot left [-tol, 1 + tol]     */
#define DPP_RES_RECOMPUTE 8     /* warning: an FP64 recompute did not reach
                                   its target accuracy; the decision used the
                                   best available value                       */

/* Device-resident outcome of one draw (one per instance for batched calls). */
typedef struct {
  int32_t status;         /* DPP_RES_* bits                                  */
  int32_t n_kept;         /* |Y|                                             */
  int32_t n_borderline;   /* pivots recomputed in FP64 (mixed precision)     */
  int32_t n_out_of_range; /* pivots outside [-tol, 1 + tol] before decision  */
  double logp;            /* log P(Y) = sum_j log|d_j|                       */
  double max_err_ratio;   /* mixed precision: max over recomputed pivots of
                             |d_mixed - d_fp64| / tau_j (tau = error bound)  */
} dpp_result;

/* Operation selector for dpp_workspace_size. */
typedef enum {
  DPP_OP_SAMPLE_HERMITIAN = 0,
  DPP_OP_SAMPLE_LU = 1,
  DPP_OP_LOGPROB_BACKWARD = 2,
  DPP_OP_GREEDY_HERMITIAN = 3,
  DPP_OP_GREEDY_LU = 4,
  DPP_OP_SAMPLE_BATCHED = 5  /* tuning-table key of dpp_sample_batched only */
} dpp_op;

/* Bytes of device workspace needed by one call of `op` at order n.
 * Returns 0 for an unsupported combination. The workspace pointer passed to
 * the call must be 256-byte aligned and at least this large. */
size_t dpp_workspace_size(int32_t op, int64_t n, int32_t dtype,
                          int32_t precision, int32_t hermitian);

/* Sample DPP(K) for Hermitian K (LDL^H form of Algorithms 1 and 4).
 *   K          device, n x n column-major (ld >= n), lower triangle read.
 *   dtype      DPP_R64 or DPP_C128.
 *   precision  DPP_PREC_FP64, DPP_PREC_3XTF32 or DPP_PREC_BF16X6 (R64 and
 *              C128; a complex mixed draw keeps planar FP32 copies of K and
 *              runs each trailing update as two real tensor-core contractions).
 *   seed, instance  Philox stream (ignored if uniforms != NULL).
 *   uniforms   device, n doubles, or NULL for Philox.
 *   keep       device, n bytes: keep[j] = 1 iff j is in the sample.
 *   factor_out device n x ld of dtype, or NULL. Receives L (strictly lower,
 *              unit diagonal implied) and D (diagonal) of K - 1_{Y^c}. May
 *              equal K for an in-place factorization. With a mixed precision
 *              it receives the FP32 factor (pivots are the FP64 ones).
 *   pivots     device, n doubles, or NULL: final pivots d_j (after -1).
 *   result     device, one dpp_result.
 *   workspace  device, >= dpp_workspace_size(DPP_OP_SAMPLE_HERMITIAN, ...).
 * Returns DPP_OK once the work is enqueued. */
dpp_status dpp_sample_hermitian(const void* K, int64_t n, int64_t ld,
                                int32_t dtype, int32_t precision,
                                uint64_t seed, uint64_t instance,
                                const double* uniforms, uint8_t* keep,
                                void* factor_out, double* pivots,
                                dpp_result* result, void* workspace,
                                size_t workspace_bytes, void* stream);

/* Bytes of the device array that holds the scratch of
 * dpp_sample_hermitian_static, and the largest orders that fit in it. */
#define DPP_STATIC_SCRATCH_BYTES (4u << 20)
#define DPP_STATIC_MAX_N_R64 15418
#define DPP_STATIC_MAX_N_C128 7942

/* dpp_sample_hermitian at DPP_PREC_FP64 without any device allocation and
 * without a workspace argument. The paper has no counterpart: this entry point
 * serves callers that cannot allocate device memory when they sample (a
 * serving loop whose memory is planned once at start-up, where cudaMalloc
 * would synchronise the device or fail under memory pressure; a plain C caller
 * that owns only K and the outputs). Its scratch (the n x 32 panel of
 * D-scaled rows, 2n pivot doubles and a flag word: about 272 n bytes for
 * DPP_R64, 528 n for DPP_C128) lives in one file-scope device array of
 * DPP_STATIC_SCRATCH_BYTES bytes inside the library.
 *   K, n, ld, dtype, seed, instance, uniforms, keep, pivots, result, stream
 *              as in dpp_sample_hermitian.
 *   factor_out REQUIRED (n > 0): device n x ld of dtype, owned by the caller,
 *              receives L and D of K - 1_{Y^c}; may equal K (in place).
 * Keep, pivots and log P are those of dpp_sample_hermitian with
 * DPP_PREC_FP64 on the same arguments.
 * Errors: DPP_ERR_INVALID_ARG for bad sizes, NULL or misaligned pointers;
 * DPP_ERR_WORKSPACE (with the limit in dpp_last_error) when n is above
 * DPP_STATIC_MAX_N_R64 / DPP_STATIC_MAX_N_C128; DPP_ERR_CUDA if the set-up or
 * a launch fails. Nothing is enqueued on an error found on the host.
 * Set-up: the first call on each device, made with that device current, looks
 * up the array's device address (cudaGetSymbolAddress, which may load the
 * library's module onto the device); make that first call before any stream
 * capture begins. Every later call whose stream is not capturing looks the
 * address up again (so a device reset, after which the array may move, is
 * picked up); a call inside a capture uses the device's last address. Nothing in the array needs to start at zero: the call clears
 * its flag word on `stream` before the first kernel.
 * Concurrency: all calls on one device share the one array, so two calls in
 * flight at once on a device (different streams, or host threads without
 * ordering between their streams) race on it; issue them in order, e.g. on
 * one stream. */
dpp_status dpp_sample_hermitian_static(const void* K, int64_t n, int64_t ld,
                                       int32_t dtype, uint64_t seed,
                                       uint64_t instance,
                                       const double* uniforms, uint8_t* keep,
                                       void* factor_out, double* pivots,
                                       dpp_result* result, void* stream);

/* Sample DPP(K) for a general (non-Hermitian) K (Algorithm 1, blocked as in
 * Algorithm 4). Same arguments as dpp_sample_hermitian, except that the whole
 * of K is read, factor_out receives L (strictly lower, unit diagonal) and U
 * (upper, with the pivots on the diagonal), and `pivots`, when not NULL,
 * receives n doubles for DPP_R64 and 2n doubles (re, im) for DPP_C128.
 * Precision: DPP_PREC_FP64, DPP_PREC_3XTF32 or DPP_PREC_BF16X6 (R64 and
 * C128). The mixed precisions keep an FP32 copy of K (planar real and
 * imaginary copies for C128), make every decision on an FP64 pivot
 * (recomputed from K when it lies within the borderline band of its uniform;
 * for C128 the decision compares u_j with Re d_j) and apply the trailing
 * updates on the tensor cores (two real contractions of depth 2 kb per
 * complex update, outer blocks of at most 128 columns); factor_out then
 * receives the FP32 factor (FP64 pivots) and may not equal K. */
dpp_status dpp_sample_lu(const void* K, int64_t n, int64_t ld, int32_t dtype,
                         int32_t precision, uint64_t seed, uint64_t instance,
                         const double* uniforms, uint8_t* keep,
                         void* factor_out, double* pivots, dpp_result* result,
                         void* workspace, size_t workspace_bytes,
                         void* stream);

/* Greedy maximum-likelihood variant (Section 2, the remark after Prop. 1):
 * every Bernoulli draw of Algorithm 1 is replaced by its more likely outcome,
 * so index j is kept iff Re(d_j) > 1/2 (a tie, Re d_j = 1/2, rejects), with
 * d_j the conditional inclusion probability given the decisions on [0, j).
 * The result is deterministic: no seed. It equals the sampler's decision rule
 * "keep iff u_j < Re d_j" with every u_j = 1/2, and runs the same kernels:
 * on the mixed precisions a pivot within the borderline band of 1/2 is
 * recomputed in FP64 from K before its decision, so every decision is that
 * of the exact FP64 chain.
 *   Arguments as dpp_sample_hermitian / dpp_sample_lu without seed, instance
 *   and uniforms; workspace >= dpp_workspace_size(DPP_OP_GREEDY_HERMITIAN or
 *   DPP_OP_GREEDY_LU, n, dtype, precision, hermitian), whose first
 *   ceil(8 n / 256) * 256 bytes hold the thresholds.
 *   result->logp is log of the greedy set's probability, sum_j log|d_j|. */
dpp_status dpp_greedy_hermitian(const void* K, int64_t n, int64_t ld, int32_t dtype,
                                int32_t precision, uint8_t* keep, void* factor_out,
                                double* pivots, dpp_result* result, void* workspace,
                                size_t workspace_bytes, void* stream);
dpp_status dpp_greedy_lu(const void* K, int64_t n, int64_t ld, int32_t dtype, int32_t precision,
                         uint8_t* keep, void* factor_out, double* pivots, dpp_result* result,
                         void* workspace, size_t workspace_bytes, void* stream);

/* Elementary DPP sampler (Algorithm 2, Theorem 2): for a real symmetric
 * marginal kernel K that is an orthogonal projection of rank k, k steps of
 * left-looking, diagonally pivoted Cholesky factorization in which the pivot
 * of step j is drawn from the remaining diagonal d with probability
 * d_t / (k - j) give a sample of DPP(K); its size is k, and
 * P(Y) = prod_j A_jj^2 over the k pivots. FP64, O(n k^2), in ONE cooperative
 * launch (bounded grid barriers; DPP_RES_TIMEOUT if one runs out).
 * Step j uses one uniform u_j (Philox as above, counter j, or uniforms[j]):
 * with the positions in the order of the algorithm's symmetric swaps, the
 * position t is the first p >= j whose running sum of max(d_p, 0) exceeds
 * u_j S, S the sum over all p >= j (k - j in exact arithmetic); the last
 * position with d > 0 if rounding leaves none.
 *   K          device, n x ld column-major FP64 (read; K is symmetric).
 *   k          the rank (0 <= k <= n); exactly k steps are run.
 *   sample     device, k int64: the sampled indices in selection order.
 *   keep       device, n bytes, or NULL: keep[i] = 1 iff i is sampled.
 *   chol       device, k x k column-major (ld k), or NULL: the lower
 *              Cholesky factor of K_Y in selection order (pivots A_jj on the
 *              diagonal), as the listing of Algorithm 2 returns it.
 *   result     device; logp = 2 sum_j log A_jj, n_kept = k; a pivot that is
 *              not positive sets DPP_RES_INADMISSIBLE (K is not a projection
 *              of rank k) or DPP_RES_NONFINITE.
 *   workspace  >= dpp_elementary_workspace_size(n, k) bytes (8 n k bytes for
 *              the factor columns plus O(n)).
 * Limit: n <= 2048 x (number of SMs) (each CTA owns at most 2048 positions);
 * a larger n returns DPP_ERR_CUDA. */
size_t dpp_elementary_workspace_size(int64_t n, int64_t k);
dpp_status dpp_sample_elementary(const double* K, int64_t n, int64_t ld, int64_t k, uint64_t seed,
                                 uint64_t instance, const double* uniforms, int64_t* sample,
                                 uint8_t* keep, double* chol, dpp_result* result, void* workspace,
                                 size_t workspace_bytes, void* stream);

/* Many independent draws, one per Hermitian (real symmetric) kernel of its own
 * order, in ONE persistent launch (no host synchronisation). Each CTA takes
 * the next instance from a device work queue (largest n first) and draws it
 * alone: left-looking 32-wide panels, FP32 SIMT updates, FP64 pivots,
 * decisions and log P, FP64 recompute of any pivot inside the borderline band
 * (the band of dpp_sample_hermitian). Arguments (all arrays device memory):
 *   batch      number of instances (>= 0).
 *   n, ld      per-instance order and leading dimension (ld >= n).
 *   K          per-instance device pointer to the column-major FP64 kernel
 *              (lower triangle read).
 *   n_max      host bound on every n (instances with n > n_max are skipped
 *              and flagged DPP_RES_NONFINITE).
 *   precision  DPP_PREC_FP32.
 *   instance   per-instance Philox instance id, or NULL (id = index).
 *   keep       per-instance device pointer to n bytes (output).
 *   uniforms   per-instance device pointer to n doubles, or NULL (Philox).
 *   pivots     per-instance device pointer to n doubles, or NULL.
 *   results    batch dpp_result records.
 *   workspace  >= dpp_batched_workspace_size(batch, n_max, precision); the
 *              launch uses as many CTAs as fit (at most two per SM).
 * Calls that share a workspace must not overlap. */
size_t dpp_batched_workspace_size(int32_t batch, int64_t n_max, int32_t precision);

dpp_status dpp_sample_batched(int32_t batch, const int64_t* n,
                              const double* const* K, const int64_t* ld,
                              int64_t n_max, int32_t precision, uint64_t seed,
                              const uint64_t* instance, uint8_t* const* keep,
                              const double* const* uniforms,
                              double* const* pivots, dpp_result* results,
                              void* workspace, size_t workspace_bytes,
                              void* stream);

/* Adjoint of log P(Y) with the sample held fixed:
 *   dK = g * (K - 1_{Y^c})^{-H}          (g = *grad_logp, a device scalar)
 * which is the derivative of log|det(K - 1_{Y^c})| (Theorem 1's likelihood).
 * The factors are recomputed (no Bernoulli draws: the decisions are `keep`).
 *   hermitian  nonzero: K Hermitian, lower triangle read; dK is returned as a
 *              full (Hermitian) matrix, the gradient with respect to K taken
 *              as a general matrix (a symmetric perturbation E of K changes
 *              log P(Y) by Re tr(dK^H E)).
 *   dK         device, n x ld_dk of dtype (full matrix written).
 * Precision: DPP_PREC_FP64. */
dpp_status dpp_logprob_backward(const void* K, int64_t n, int64_t ld,
                                int32_t dtype, int32_t precision,
                                int32_t hermitian, const uint8_t* keep,
                                const double* grad_logp, void* dK,
                                int64_t ld_dk, void* workspace,
                                size_t workspace_bytes, void* stream);

/* Adjoint of log P(Y_i) for each instance of a batch of real symmetric
 * kernels (for instance the draws of dpp_sample_batched), Y_i fixed:
 * dK_i = g_i (K_i - 1_{Y_i^c})^{-T}, in FP64, exactly as dpp_logprob_backward
 * with hermitian = 1.
 *   batch      number of instances (>= 0).
 *   n, ld, ld_dk  HOST arrays of batch entries: order, leading dimension of
 *              K_i (>= max(1, n_i)) and of dK_i.
 *   K, keep, grad_logp, dK  HOST arrays of batch DEVICE pointers: K_i
 *              (column-major, lower triangle read), keep_i (n_i bytes),
 *              g_i (one double), dK_i (n_i x ld_dk_i doubles, written).
 *   workspace  device, dpp_logprob_backward_batched_workspace(batch, n_max)
 *              bytes (n_max = max_i n_i) for one CTA per SM; a smaller one runs
 *              on as many CTAs as it holds (at least one). All instances run in
 *              ONE persistent launch: each CTA takes the next instance, largest
 *              n first, and does its LDL^T, the triangular inverse and
 *              Z^T D^{-1} Z in FP64 in 32 x 32 tiles.
 * Errors: DPP_ERR_INVALID_ARG / DPP_ERR_WORKSPACE found on the host before
 * anything is enqueued; DPP_ERR_CUDA if a launch fails (earlier instances
 * may then already be enqueued). */
/* dpp_logprob_backward_batched in FP32 arithmetic: the LDL^T of K_i - 1_{Y^c},
 * the triangular inverse and Z^T D^{-1} Z run at the FP32 rate (GB300's FP64
 * rate is a small fraction of it); K, g and dK stay FP64 (dK carries FP32
 * rounding: about 1e-7 relative times the conditioning of K_i - 1_{Y^c}).
 * Same arguments, workspace and errors. */
dpp_status dpp_logprob_backward_batched_fp32(int32_t batch, const int64_t* n,
                                             const void* const* K, const int64_t* ld,
                                             const uint8_t* const* keep,
                                             const double* const* grad_logp,
                                             void* const* dK, const int64_t* ld_dk,
                                             void* workspace, size_t workspace_bytes,
                                             void* stream);

/* Workspace bytes for the one-launch form of dpp_logprob_backward_batched on
 * the current device (one CTA per SM, or DPP_TUNE_MAX_CTAS): a descriptor per
 * instance plus, per CTA, n_max^2 + 33 n_max + 32 n_max doubles (rounded up to
 * multiples of 32). Returns 0 for negative arguments. */
size_t dpp_logprob_backward_batched_workspace(int32_t batch, int64_t n_max);

dpp_status dpp_logprob_backward_batched(int32_t batch, const int64_t* n,
                                        const void* const* K, const int64_t* ld,
                                        const uint8_t* const* keep,
                                        const double* const* grad_logp,
                                        void* const* dK, const int64_t* ld_dk,
                                        void* workspace, size_t workspace_bytes,
                                        void* stream);

/* L-ensemble to marginal kernel (Section 5, stated there as future work):
 * for each real symmetric positive semi-definite L_i of a batch,
 *     K_i = L_i (L_i + I)^{-1} = I - (L_i + I)^{-1},
 * the marginal kernel of the L-ensemble DPP (P(Y) proportional to
 * det(L_Y)), ready for dpp_sample_batched. FP64, in ONE persistent launch:
 * each CTA takes the next instance (largest n first), factors L_i + I as
 * L D L^T (32 x 32 tiles), forms Z = L^{-1} and writes I - Z^T D^{-1} Z to both
 * triangles of K_i.
 *   batch      number of instances (>= 0).
 *   n, ld, ld_k  HOST arrays: order (0..4096), leading dimension of L_i and
 *              of K_i.
 *   L, K       HOST arrays of DEVICE pointers (L_i lower triangle read; K_i
 *              written in full; K_i may not alias L_i).
 *   workspace  device, dpp_logprob_backward_batched_workspace(batch, n_max)
 *              bytes for one CTA per SM (a smaller one runs on fewer CTAs).
 * Errors as dpp_logprob_backward_batched. */
dpp_status dpp_lensemble_to_marginal_batched(int32_t batch, const int64_t* n,
                                             const double* const* L, const int64_t* ld,
                                             double* const* K, const int64_t* ld_k,
                                             void* workspace, size_t workspace_bytes,
                                             void* stream);

/* Process-wide tuning knobs (read at each call; not for concurrent changes).
 *   DPP_TUNE_TAU_SAFETY   c in the mixed-precision borderline bound
 *                         tau_j = c * 2^-22 * sqrt(j + 1) * (K_jj + s_j),
 *                         s_j = sum_{k<j} |L_jk|^2 |d_k|            (default 8)
 *   DPP_TUNE_OUTER_BLOCK  outer block width of the mixed path: the trailing
 *                         update contracts this many columns at once (32..256,
 *                         multiple of 32; default 256)
 *   DPP_TUNE_UPDATE_KERNEL  mixed-path trailing update: 0 = tensor cores
 *                         (tcgen05), 1 = SIMT FP32 (default 0; real Hermitian
 *                         K only: the mixed LU and complex paths always use
 *                         the tensor cores)
 *   DPP_TUNE_MAX_CTAS     mixed path: CTAs per launch of the outer-block and
 *                         tensor-core kernels (0 = one per SM, the default;
 *                         else 8..4096, at most one per SM). With half the SMs,
 *                         two draws on two streams can overlap one draw's
 *                         latency-bound panels with the other's update.
 *   DPP_TUNE_PANEL_PIPELINE  mixed Hermitian path, panel kernel: 1 = single
 *                         helper (CTA 0 decides with one warp while its other
 *                         warps prepare the next block, CTA 1 streams the outer
 *                         block's rows), 2 = chunked (CTA 0 decides with all
 *                         its warps, helper CTAs own the outer block's 32-row
 *                         chunks, left-looking products are computed before
 *                         each panel is published; the LU path's kernel),
 *                         3 = split (also for the mixed LU path): the chunked
 *                         panel launch holds only CTA 0 and one helper CTA per
 *                         chunk of the outer block (8 CTAs), and the rows below
 *                         the outer block are brought through its panels
 *                         afterwards by a separate launch on the capped grid,
 *                         so the SMs of other draws in flight are not held
 *                         while the decisions run,
 *                         0 = automatic (the default): chunked when a launch
 *                         gets at least 96 CTAs, else single helper. The SIMT
 *                         trailing update always runs with pipeline 1.
 *   DPP_TUNE_WAIT_NS      limit, in nanoseconds, of every bounded wait between
 *                         the CTAs of the panel launches (FP64 panels, mixed
 *                         panel pipelines and their FP64 recomputes); a wait
 *                         that runs out ends its launch early and sets
 *                         DPP_RES_TIMEOUT (1e5..6e10, default 2e9)
 *   DPP_TUNE_FAULT_WITHHOLD  fault injection for tests of the bounded waits
 *                         (default 0). With 1, the CTA that makes the
 *                         decisions never releases a panel to the other CTAs
 *                         (the FP64 panel kernels and the chunked mixed
 *                         pipeline): their waits run out after DPP_TUNE_WAIT_NS,
 *                         every launch still ends, and the draw's status has
 *                         DPP_RES_TIMEOUT. Its outputs are then meaningless.
 *   DPP_TUNE_UPDATE_VARIANT  tensor-core trailing update (0..3, default 0):
 *                         bit 0 = accumulate 64 deep (3xTF32) / 32 deep
 *                         (BF16x6) in one tensor-memory accumulator before it
 *                         is drained into FP32 registers instead of 32 / 16;
 *                         bit 1 = 3xTF32 only: 16-deep operand stages, six of
 *                         them, instead of three 32-deep ones
 *   DPP_TUNE_PANEL_CTAS   split panel pipeline (DPP_TUNE_PANEL_PIPELINE 3):
 *                         CTAs of each outer block's cooperative decision
 *                         launch (0 = default: the launch cap DPP_TUNE_MAX_CTAS,
 *                         at least 8; else 8..4096). CTA 0 and seven helpers
 *                         decide and solve the block; the others only serve
 *                         FP64 recomputes, so a smaller grid leaves SMs to the
 *                         other draws in flight and a larger one recomputes
 *                         faster.
 *   DPP_TUNE_BATCHED_THREADS  dpp_sample_batched: threads per CTA, 128
 *                         (default: two CTAs, two instances, per SM) or 256
 *                         (one per SM, twice the threads per instance).
 *   DPP_TUNE_USE_CACHE    1 (default): when the autotuner's table (below) has
 *                         an entry for a call's key, that entry's outer block,
 *                         panel pipeline and CTA cap replace the three knobs
 *                         above for the call; 0: the knobs alone decide.
 * Returns DPP_ERR_INVALID_ARG for an unknown key or out-of-range value. */
typedef enum {
  DPP_TUNE_TAU_SAFETY = 0,
  DPP_TUNE_OUTER_BLOCK = 1,
  DPP_TUNE_UPDATE_KERNEL = 2,
  DPP_TUNE_MAX_CTAS = 3,
  DPP_TUNE_PANEL_PIPELINE = 4,
  DPP_TUNE_WAIT_NS = 5,
  DPP_TUNE_FAULT_WITHHOLD = 6,
  DPP_TUNE_USE_CACHE = 7,
  DPP_TUNE_UPDATE_VARIANT = 8,
  DPP_TUNE_PANEL_CTAS = 9,
  DPP_TUNE_BATCHED_THREADS = 10
} dpp_tune_key;

dpp_status dpp_set_tuning(int32_t key, double value);
double dpp_get_tuning(int32_t key);

/* Autotuner. The paper's only knobs are its tile and block sizes (Section 4,
 * chosen by hand per machine); here the launch configuration of a draw is
 * measured on the GPU at hand and kept in a table keyed by (GPU name, SM
 * count, op, dtype, precision, n bucket = floor(log2 n)).
 *
 * One entry: the configuration and the throughput it reached. `streams` is
 * the number of draws the caller should keep in flight (on that many
 * streams); `max_ctas` is the per-launch CTA cap that goes with it (0 = one
 * CTA per SM). The library applies outer_block, panel_pipeline and max_ctas
 * to every later call with the entry's key (unless DPP_TUNE_USE_CACHE is 0);
 * keeping `streams` draws in flight is the caller's part. */
typedef struct {
  int32_t op;              /* DPP_OP_SAMPLE_HERMITIAN, _LU or _BATCHED         */
  int32_t dtype;
  int32_t precision;
  int32_t n_bucket;        /* floor(log2 n) of the order it was tuned at       */
  int64_t n;               /* the order it was tuned at                        */
  int32_t outer_block;     /* as DPP_TUNE_OUTER_BLOCK                          */
  int32_t panel_pipeline;  /* as DPP_TUNE_PANEL_PIPELINE (0 = automatic)      */
  int32_t max_ctas;        /* as DPP_TUNE_MAX_CTAS                             */
  int32_t streams;         /* draws in flight                                  */
  double samples_per_s;    /* measured with this configuration                 */
  int32_t candidates;      /* configurations timed to choose it                */
  int32_t update_variant;  /* as DPP_TUNE_UPDATE_VARIANT                       */
  int32_t batched_threads; /* DPP_OP_SAMPLE_BATCHED entries: as
                              DPP_TUNE_BATCHED_THREADS (0 in the others)       */
} dpp_tune_entry;

/* Autotune dpp_sample_batched on the caller's batch (its arguments, with
 * precision DPP_PREC_FP32, no instance/uniform/pivot arrays): `draws` timed
 * draws (Philox seeds seed, seed + 1, ...; after one warm-up draw) with CTAs
 * of 128 and of 256 threads (DPP_TUNE_BATCHED_THREADS), CUDA events on
 * `stream`; the faster goes into the tuning table under (this GPU,
 * DPP_OP_SAMPLE_BATCHED, DPP_R64, DPP_PREC_FP32, floor(log2 n_max)), which
 * every later dpp_sample_batched call with that key uses. `best` (host,
 * nullable) receives the entry; samples_per_s counts instances per second.
 * The outputs (keep, results) hold the last timed draw. Blocks the host.
 * Errors: as dpp_sample_batched; DPP_ERR_INVALID_ARG if draws < 1. */
dpp_status dpp_autotune_batched(int32_t batch, const int64_t* n, const double* const* K,
                                const int64_t* ld, int64_t n_max, uint64_t seed,
                                uint8_t* const* keep, dpp_result* results, void* workspace,
                                size_t workspace_bytes, int32_t draws, dpp_tune_entry* best,
                                void* stream);

/* Device workspace for dpp_autotune: max_streams draws' workspaces, keep
 * masks and results (0 for an unsupported combination). */
size_t dpp_autotune_workspace_size(int32_t op, int64_t n, int32_t dtype, int32_t precision,
                                   int32_t max_streams);

/* Time every candidate configuration on the caller's kernel K (device,
 * column-major as for dpp_sample_hermitian / dpp_sample_lu; op selects which)
 * and keep the fastest in the table. Candidates: draws in flight 1, 2, 4 and
 * 8 (up to max_streams, 1..8), each launch then capped at SMs / streams CTAs;
 * outer block 128 and 256 (mixed precisions); panel pipelines 1, 2 and 3 for
 * real Hermitian mixed draws, 0 and 3 for real LU mixed draws; then, with the
 * winner's settings, the tensor-core update variants (DPP_TUNE_UPDATE_VARIANT;
 * 1..3 for 3xTF32, 1 for BF16x6). Each candidate runs one warm-up draw per stream and
 * then `draws` timed draws (Philox seeds 0, 1, ...) dealt round-robin to its
 * streams, timed with CUDA events between a start event on `stream` and the
 * last draw's end. Blocks the host until done; allocates only its own CUDA
 * streams and events (destroyed before returning). `best` (host, nullable)
 * receives the chosen entry.
 * Errors: DPP_ERR_INVALID_ARG / DPP_ERR_WORKSPACE / DPP_ERR_UNSUPPORTED on
 * the host before any work; DPP_ERR_CUDA if a draw or the timing fails. */
dpp_status dpp_autotune(int32_t op, const void* K, int64_t n, int64_t ld, int32_t dtype,
                        int32_t precision, int32_t max_streams, int32_t draws,
                        void* workspace, size_t workspace_bytes, dpp_tune_entry* best,
                        void* stream);

/* The table's entry for (op, n, dtype, precision) on the current device:
 * DPP_OK and *out filled, or DPP_ERR_UNSUPPORTED if there is none. */
dpp_status dpp_tune_lookup(int32_t op, int64_t n, int32_t dtype, int32_t precision,
                           dpp_tune_entry* out);

/* Write the whole table (entries of every GPU) to `path` as JSON, or merge
 * the entries of a JSON file written by dpp_tune_save into it (an entry with
 * the same key is replaced). The library loads the file named by the
 * environment variable DPP_TUNE_CACHE, if set, when it is loaded.
 * dpp_tune_clear empties the table. */
dpp_status dpp_tune_save(const char* path);
dpp_status dpp_tune_load(const char* path);
void dpp_tune_clear(void);

/* Fill `out` (device, n doubles) with the Philox uniforms u_0..u_{n-1} that
 * the samplers use for (seed, instance). */
dpp_status dpp_uniforms(uint64_t seed, uint64_t instance, int64_t n,
                        double* out, void* stream);

/* Per-kernel timing. While profiling is on (between dpp_profile_start and
 * dpp_profile_stop), every kernel launch of the library is bracketed by CUDA
 * events recorded on the stream it is launched on. dpp_profile_stop waits for
 * those events, writes one entry per kernel category that ran (at most
 * max_entries) and returns the number written. `flops` and `bytes` are the
 * ALGORITHMIC work of the recorded launches (e.g. m^2 b real flops for a
 * rank-b lower-triangular Schur update of order m), not executed instructions.
 * Profiling is process-wide and not meant for concurrent callers. */
typedef struct {
  char name[32];
  int64_t launches;
  double total_ms;
  double flops;
  double bytes;
} dpp_kernel_stat;

void dpp_profile_start(void);
int32_t dpp_profile_stop(dpp_kernel_stat* out, int32_t max_entries);

/* Number of kernels this library has enqueued since it was loaded. */
uint64_t dpp_launch_count(void);

/* Thread-local description of the last host-side error ("" if none). */
const char* dpp_last_error(void);

/* DPP_ABI_VERSION of the loaded library. */
int32_t dpp_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DPP_H_ */
