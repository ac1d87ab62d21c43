/*
 * compar.h — C ABI of a variant-selecting dense matrix multiply for one
 * B300 GPU (sm_103a).
 *
 * The idea follows COMPAR (Sec. 2): one component — here the matrix-multiply
 * interface "mmul" of Sec. 2.1 / Table 2 — is exposed through several
 * interchangeable implementation variants, and a runtime picks one variant per
 * call from the call's context (Sec. 2.2, "Runtime System": a task is mapped to
 * one of its codelets when it runs).  The lifecycle calls keep the names the
 * paper's pre-compiler generates (compar_init / compar_terminate, Sec. 2.1).
 *
 * The component computes
 *
 *     C = alpha * op_scale * (A x B) + beta * C
 *
 * with A (M x K), B (K x N), C (M x N), all ROW-MAJOR.  In compar_gemm the
 * matrices are contiguous (lda = K, ldb = N, ldc = N); compar_gemm_batched
 * takes explicit leading dimensions.  C is always float32.  op_scale is 1
 * except for FP8 inputs, where it is scale_a * scale_b (per-tensor
 * dequantisation factors: the real matrix is scale * decoded codes).
 *
 * Ownership: A, B, C are DEVICE pointers owned by the caller (for example
 * PyTorch tensors) unless a function says otherwise.  Everything else
 * (workspace, tensor maps, CUDA graphs, cost models, timing records) is owned
 * by the context and released by compar_terminate.
 *
 * Semantics: every compute call is asynchronous and stream-ordered on the
 * given cudaStream_t (passed as void*; NULL = legacy default stream).  Errors
 * found on the host are returned synchronously; kernel-side failures (a
 * bounded wait that ran out) are latched in a device error word and returned
 * by compar_check_device_error.  No call aborts the process.  Each call runs
 * on its context's device: the call makes that device current and restores
 * the caller's current device before returning, so one process may drive
 * several GPUs with one context each; the stream passed must belong to the
 * context's device.  A call clears a non-sticky CUDA error left pending on
 * the calling thread (cudaGetLastError) before it starts.  A context is not
 * thread-safe: use one context per host thread.  The calls on one context
 * share its device workspace (operand copies, partial sums, arrival
 * counters), so they must run in order on the GPU: issue them on one stream,
 * or order the streams yourself (events); calls that overlap on the GPU give
 * undefined results for those calls.
 *
 * beta == 0 means C is not read, and alpha == 0 that A and B are not read
 * (C = beta * C), as in BLAS.
 */
#ifndef COMPAR_H_
#define COMPAR_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define COMPAR_ABI_VERSION 1

typedef struct compar_ctx* compar_ctx_t;

/* Element type of A and B (the "type" clause of the parameter directive,
 * Sec. 2.1).  BF16 is passed as uint16 bit patterns, F8E4M3 as bytes (OCP
 * E4M3: bias 7, max finite 448, no infinities). */
typedef enum {
    COMPAR_F32 = 0,
    COMPAR_BF16 = 1,
    COMPAR_F8E4M3 = 2
} compar_dtype_t;

typedef enum {
    COMPAR_OK = 0,
    COMPAR_ERR_INVALID = -1,      /* bad argument, null/misaligned pointer   */
    COMPAR_ERR_UNSUPPORTED = -2,  /* variant cannot run this call           */
    COMPAR_ERR_CUDA = -3,         /* a CUDA runtime call failed             */
    COMPAR_ERR_TIMEOUT = -4,      /* a device-side bounded wait ran out     */
    COMPAR_ERR_IO = -5,           /* selector/record file error             */
    COMPAR_ERR_NO_VARIANT = -6    /* no eligible variant meets the tolerance */
} compar_status_t;

/* Stable implementation-variant ids (Table 2 lists the paper's mmul variants
 * BLAS/OMP/CUDA/CUBLAS; these are their B300 replacements). */
enum {
    COMPAR_V_NAIVE = 0,       /* one thread per C element, FP32 FMA         */
    COMPAR_V_SIMT = 1,        /* shared-memory tiled FP32 SIMT              */
    COMPAR_V_TC_TF32 = 2,     /* tcgen05 kind::tf32, TMEM FP32 accumulator  */
    COMPAR_V_TC_BF16 = 3,     /* tcgen05 kind::f16 (bf16 operands)          */
    COMPAR_V_TC_FP8 = 4,      /* tcgen05 kind::f8f6f4 (E4M3 operands)       */
    COMPAR_V_SPLIT3 = 5,      /* 3xBF16 split on tcgen05 (FP32 accuracy)    */
    COMPAR_V_GROUPED = 6,     /* persistent grouped kernel (batched only)   */
    COMPAR_V_SPLIT6 = 7,      /* 6-product 3-piece bf16 split on tcgen05
                                 (at or below the FP32 SIMT error level)    */
    COMPAR_V_SPLIT3_TF32 = 8, /* 3xTF32: 2-piece TF32 split, 3 kind::tf32
                                 products                                  */
    COMPAR_V_SPLIT3_FUSED = 9,/* 3xBF16 with the split done inside the GEMM
                                 kernel (float32 tiles split in shared
                                 memory, no pre-pass); float32 A and B with
                                 16-byte rows and 16-byte aligned bases    */
    COMPAR_V_COUNT = 10       /* ids 0 .. COUNT-1; ids never change once
                                 assigned, new variants take new ids        */
};

/* ---------------------------------------------------------------- lifecycle */

/* Create a context on CUDA device `device` (Sec. 2.1, `initialize` directive
 * -> compar_init()).  Reads COMPAR_* environment variables (COMPAR_FORCE_VARIANT,
 * COMPAR_SELECTOR = auto|history|mlp, COMPAR_SELECTOR_FILE, COMPAR_LOG,
 * COMPAR_WAIT_BUDGET_NS).  *out receives the context.  Returns COMPAR_OK,
 * COMPAR_ERR_INVALID (out == NULL), COMPAR_ERR_UNSUPPORTED (device is not
 * sm_103) or COMPAR_ERR_CUDA. */
int compar_init(compar_ctx_t* out, int device);

/* Create a HOST-ONLY context: no CUDA call is made and no device is needed.
 * Selection (compar_select), cost-model files, records and the error model
 * work; every compute call returns COMPAR_ERR_UNSUPPORTED.  `num_sms` is the
 * SM count the roofline prior assumes (<= 0: 148, one B300).  For offline
 * tooling and for testing the runtime's host logic. */
int compar_init_host(compar_ctx_t* out, int num_sms);

/* Release the context and everything it owns (Sec. 2.1, `terminate`
 * directive -> compar_terminate()).  Synchronises the device first.
 * NULL is accepted and ignored. */
int compar_terminate(compar_ctx_t ctx);

/* Human-readable name of a status code (static string, never NULL). */
const char* compar_status_string(int status);

/* Text of the last host-side error seen by this thread (CUDA call that
 * failed, injected failure, ...); empty string when none.  Never NULL. */
const char* compar_last_error(void);

/* ---------------------------------------------------------------- compute */

/* One GEMM call: the interface call of Sec. 2.1 ("mmul") submitted as a task
 * that the runtime maps to one variant (Sec. 2.2).
 *   m, n, k   : sizes, each >= 0 (m == 0 or n == 0: nothing to do;
 *               k == 0: C = beta * C).
 *   dtype     : element type of A and B.
 *   tol       : relative Frobenius error asked for, measured against the
 *               exact product of the inputs as given; tol <= 0 means 1e-5
 *               for every dtype.  A variant is eligible when its error
 *               model (relative Frobenius error on data that does not
 *               cancel) times the margin is at most tol; every input gets
 *               the variant's element-wise worst-case bound relative to
 *               |alpha| |A||B| + |beta| |C|, so a short dot product that
 *               cancels may exceed tol relatively.
 *   A, B      : device pointers, row-major contiguous (lda = k, ldb = n).
 *   C         : device float32, row-major contiguous (ldc = n); C must not
 *               overlap A or B (COMPAR_ERR_INVALID).
 *   stream    : cudaStream_t.
 * Variant choice: compar_force_variant > decision cache > learned MLP cost
 * model (when confident) > history-table model.  Returns COMPAR_OK,
 * COMPAR_ERR_INVALID, COMPAR_ERR_NO_VARIANT (nothing meets tol) or
 * COMPAR_ERR_CUDA.  alpha/beta and FP8 scales come from compar_set_scalars /
 * compar_set_fp8_scales (the listed signature has no slot for them).
 * Stream capture: a call may be captured into a CUDA graph and replayed
 * once a call of the same shape has run on the context outside the capture
 * (the decision is cached and the workspace has its size); a call that
 * would grow the workspace while `stream` is captured returns
 * COMPAR_ERR_UNSUPPORTED.  Such a refusal, or device memory that runs out
 * while the workspace grows (COMPAR_ERR_CUDA), is the caller's to handle:
 * it changes no later selection.  A variant whose own launch fails is
 * quarantined for the context and the call re-dispatched. */
int compar_gemm(compar_ctx_t ctx, int64_t m, int64_t n, int64_t k,
                compar_dtype_t dtype, double tol, const void* A,
                const void* B, float* C, void* stream);

/* The same GEMM on HOST matrices (no counterpart in the paper, whose tasks
 * received host data through StarPU's data management, Sec. 2.2): A (m x k),
 * B (k x n) and C (m x n, float32) are host pointers, row-major contiguous;
 * page-locked memory makes the transfers asynchronous.  The library uploads
 * B, then A (and C when beta != 0) in row panels on its own copy streams,
 * runs one selected-variant GEMM per panel on `stream` and downloads each
 * panel of C as soon as it is done, so transfers overlap the products; two
 * sets of context-owned device buffers let consecutive calls overlap too.
 * Ordering: A and B are read from the moment of the call (they must be
 * ready in host memory then, not merely by the time `stream` gets there);
 * C is in host memory once `stream` reaches the end of the call.  Errors
 * as compar_gemm; on a stream being captured into a CUDA graph it returns
 * COMPAR_ERR_UNSUPPORTED (its copy streams are its own). */
int compar_gemm_host(compar_ctx_t ctx, int64_t m, int64_t n, int64_t k, compar_dtype_t dtype,
                     double tol, const void* A, const void* B, float* C, void* stream);

/* One problem of a batched call.  Leading dimensions are in elements and must
 * be >= the row length (lda >= k, ldb >= n, ldc >= n). */
typedef struct {
    int64_t m, n, k;
    int64_t lda, ldb, ldc;
    compar_dtype_t dtype;
    const void* A;
    const void* B;
    float* C;
    float alpha, beta;
    float scale_a, scale_b;   /* FP8 dequantisation factors, else ignored */
} compar_problem_t;

/* Many independent GEMMs of uneven sizes in one call.  The paper has no
 * counterpart of this call: its runtime schedules each mmul task on its own
 * (Sec. 2.2); batching uneven products into one launch is this library's
 * addition for many small products on one GPU.  `probs` is a HOST
 * array of `count` problems and is copied before return.  F32 problems run at
 * FP32 accuracy when tol <= 1e-5 (3xBF16 mode), else on TF32; BF16 problems
 * on bf16 tensor cores.  The selector picks between one persistent grouped
 * launch captured in a CUDA graph (cached per batch signature) and one launch
 * per problem.  Returns as compar_gemm.  The call runs a graph of its own and
 * waits on its staging buffers, so it cannot itself be captured: on a stream
 * being captured it returns COMPAR_ERR_UNSUPPORTED and enqueues nothing.
 * The problems run concurrently: a problem's C may not share an element
 * with any problem's A, B or C (not checked; disjoint column blocks of one
 * matrix are fine). */
int compar_gemm_batched(compar_ctx_t ctx, int count,
                        const compar_problem_t* probs, double tol,
                        void* stream);

/* FP32 SIMT GEMM that allocates nothing, for callers that cannot allocate
 * device memory where they need the product: a host application or framework
 * that owns all device memory through its own pool, a latency-critical path
 * that cannot risk the synchronisation an allocation may cause, or a plug-in
 * given no allocator.  The paper has no counterpart of this call.
 *   C = alpha * A x B + beta * C, A (m x k), B (k x n), C (m x n), all float32,
 *   row-major contiguous DEVICE pointers owned by the caller, on the CURRENT
 *   device, asynchronous on `stream`.
 * It needs no context and calls no cudaMalloc / cudaFree or any allocating
 * routine.  Its only scratch, the split-K partial sums of the SIMT kernel,
 * is a fixed 16 MiB device array inside the library, which every GPU that
 * loads the library holds until the process exits.  A shape whose split-K
 * plan needs more than 16 MiB is refused with COMPAR_ERR_INVALID (the text is
 * in compar_last_error); nothing needs to start zeroed.  The first call on a
 * device does a one-time set-up (the device check and the SM count; it may
 * also load the library's device code), so make that first call before any
 * stream capture.  Every call looks up the array's device address again, so
 * the call keeps working after the device's context is reset.  All
 * calls share the one array: calls that may overlap on the GPU (different
 * streams or host threads without ordering) race on it; calls on one stream
 * are ordered and safe.  Returns COMPAR_OK, COMPAR_ERR_INVALID,
 * COMPAR_ERR_UNSUPPORTED (not an sm_103 device) or COMPAR_ERR_CUDA. */
int compar_gemm_simt_noalloc(int64_t m, int64_t n, int64_t k, float alpha,
                             const float* A, const float* B, float beta,
                             float* C, void* stream);

/* Time the implementations of a batched call on this batch and remember the
 * fastest for its signature (shapes, dtypes, tolerance class): 0 = one launch
 * per problem, 1 = grouped kernel with 128-column tiles, 2 = 256-column tiles,
 * 3 / 4 = as 1 / 2 with the largest problems first.  Each configuration runs
 * once untimed and three times timed (CUDA events on `stream`), so C is
 * written several times: with beta != 0 the final contents are not the
 * product.  times_ms (nullable, 5 floats) receives the medians, *best
 * (nullable) the choice.  Synchronises `stream`, so a stream being captured
 * into a CUDA graph is refused (COMPAR_ERR_UNSUPPORTED). */
int compar_autotune_batched(compar_ctx_t ctx, int count,
                            const compar_problem_t* probs, double tol,
                            void* stream, float* times_ms, int* best);

/* Run every following batched call in configuration `config` (0..4, as
 * numbered for compar_autotune_batched), or clear with -1 (autotuned choice
 * for known batch signatures, else configuration 1).  A forced variant
 * other than COMPAR_V_GROUPED still runs the per-GEMM loop.
 * COMPAR_ERR_INVALID for other values. */
int compar_set_batched_config(compar_ctx_t ctx, int config);

/* ---------------------------------------------------------------- control */

/* Force every following call onto `variant_id` (one of COMPAR_V_*), or clear
 * with -1 (the paper's STARPU_NCUDA / STARPU_NCPU switches, Sec. 3.2, pinned
 * whole architectures; this pins one variant).  A forced variant that cannot
 * run a call makes that call return COMPAR_ERR_UNSUPPORTED.  Forcing
 * COMPAR_V_GROUPED affects batched calls only (they then always use the
 * grouped kernel); forcing a single-call variant makes batched calls run one
 * launch per problem on that variant. */
int compar_force_variant(compar_ctx_t ctx, int variant_id);

/* alpha and beta used by compar_gemm (defaults 1 and 0). */
int compar_set_scalars(compar_ctx_t ctx, float alpha, float beta);

/* FP8 dequantisation factors used by compar_gemm for F8E4M3 inputs (default
 * 1, 1).  Must be finite and > 0. */
int compar_set_fp8_scales(compar_ctx_t ctx, float scale_a, float scale_b);

/* Selection policy: 0 = auto (the MLP when confident, else the history
 * table; a variant timed in the call's own history bucket is then ranked by
 * that measurement), 1 = history table only, 2 = MLP only. */
int compar_set_selector_mode(compar_ctx_t ctx, int mode);

/* Variant chosen by the most recent compar_gemm call (-1 before any). */
int compar_last_variant(compar_ctx_t ctx);

/* Number of variant ids (COMPAR_V_COUNT; id 6, the grouped kernel, runs
 * batched calls only) and their names (static strings; NULL if out of range). */
int compar_variant_count(void);
const char* compar_variant_name(int variant_id);

/* Whether variant `variant_id` can run (m, n, k, dtype) at all on
 * contiguous row-major operands with 16-byte aligned bases (dtype, row
 * alignment and shape rules; the tolerance is not considered).  1 / 0, or a
 * negative status. */
int compar_variant_supported(compar_ctx_t ctx, int variant_id, int64_t m,
                             int64_t n, int64_t k, compar_dtype_t dtype);

/* Drop every cached selection decision. */
int compar_clear_decisions(compar_ctx_t ctx);

/* The variant compar_gemm would run for this context, without running it
 * (forced variant, decision cache, MLP, history table, roofline prior, in that
 * order; caches the decision like compar_gemm).  `batch` is the batch-count
 * feature (1 for single calls).  Returns a variant id or a negative status
 * (COMPAR_ERR_NO_VARIANT when nothing meets tol). */
int compar_select(compar_ctx_t ctx, int64_t m, int64_t n, int64_t k,
                  compar_dtype_t dtype, double tol, int batch);

/* Error model used for eligibility: predicted relative Frobenius error of
 * `variant` on `dtype` inputs with inner dimension k is
 *     c0 + c1 * sqrt(k) * 2^-24 + c2 * k * 2^-24,
 * and a variant is eligible when prediction * margin <= tol.  c0 = +inf
 * marks (variant, dtype) pairs that can never meet any tolerance. */
int compar_error_model_set(compar_ctx_t ctx, int variant, compar_dtype_t dtype,
                           double c0, double c1, double c2);
int compar_error_model_get(compar_ctx_t ctx, int variant, compar_dtype_t dtype,
                           double* c0, double* c1, double* c2);
int compar_error_model_set_margin(compar_ctx_t ctx, double margin);
/* Predicted relative error of `variant` for (dtype, k); < 0 on bad input. */
double compar_error_model_predict(compar_ctx_t ctx, int variant,
                                  compar_dtype_t dtype, int64_t k);

/* ---------------------------------------------------------------- models */

/* Load a selector file: the performance models the selection rests on.
 * In the paper the runtime picks a variant from performance models trained
 * on earlier runs, their training decides how often it mis-selects (Sec. 3.2,
 * the matrix-multiply results) and better training is named as future work
 * (Sec. 5).  The file holds the history table, error model, MLP weights,
 * feature normaliser, grouped tile choice, stencil history, and a rehearsal
 * sample of up to 16384 of the timing records the MLP was trained on.  On any error
 * (missing file, bad magic, version, size or checksum) the models already
 * loaded are kept and COMPAR_ERR_IO is returned. */
int compar_selector_load(compar_ctx_t ctx, const char* path);

/* Write the current selector state to `path` (binary, versioned,
 * checksummed); the rehearsal sample is drawn uniformly from the loaded
 * sample and the records held. */
int compar_selector_save(compar_ctx_t ctx, const char* path);

/* ---------------------------------------------------------------- learned cost model */

/* The learned cost model is a 3-layer perceptron (8 -> 64 -> 64 -> 18, ReLU)
 * per ensemble member (4 members).  Inputs (features of a call):
 * log2 M, log2 N, log2 K, one-hot dtype (f32, bf16, f8), log10 tol,
 * log2 batch.  Outputs: for variant v (0..COMPAR_V_COUNT-1) output v is log2 of the run
 * time in ms and output COMPAR_V_COUNT+v log10 of the relative error (the
 * outputs of id 6, the batched-only grouped kernel, are never trained).  The paper's runtime
 * chooses variants with performance models it calls machine-learning models
 * and expects better-trained models to choose better (Sec. 3.2, Sec. 5).
 * Parameters of one member, float32, in this order: W1[64][8] b1[64]
 * W2[64][64] b2[64] W3[18][64] b3[18] (weights stored out x in). */
int compar_mlp_param_count(void);

/* Forward pass on the GPU for `members` parameter sets (host array
 * members x param_count) over `rows` raw (already standardised) feature rows
 * (host, rows x 8); Y (host) receives members x rows x 18.  Synchronous. */
int compar_mlp_forward(compar_ctx_t ctx, const float* params, int members,
                       const float* X, int rows, float* Y);

/* Training steps on the GPU (one CTA per member runs the whole loop):
 * loss = sum mask*(y-T)^2 / max(1, sum mask) over each mini-batch, gradients
 * by backpropagation, Adam (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected,
 * step counter starting at step0 >= 1).  All arrays are HOST arrays:
 * params/adam_m/adam_v (members x param_count, updated in place), X (rows x
 * 8), T and mask (rows x 18), batch_idx (members x steps x batch row indices,
 * batch <= 128).  When `grads` is non-NULL, steps must be 1: the gradients of
 * the first mini-batch are written to grads (members x param_count) and
 * params are left unchanged.  loss (nullable) receives members x steps batch
 * losses.  Synchronous. */
int compar_mlp_train_steps(compar_ctx_t ctx, float* params, float* adam_m,
                           float* adam_v, int members, const float* X,
                           const float* T, const float* mask, int rows,
                           const int32_t* batch_idx, int steps, int batch,
                           float lr, int step0, float* grads, float* loss);

/* Train the context's cost model from its timing records (compar_measure /
 * compar_record_add): standardises features and targets, holds out 1 row in
 * 10, trains the 4-member ensemble for `steps` Adam steps of `batch` rows
 * (bootstrap mini-batches from `seed`), then marks the model trained (used by
 * selection when confident) and clears the decision cache.  *val_loss
 * (nullable) receives the held-out standardised loss.  Synchronous. */
int compar_selector_train(compar_ctx_t ctx, int steps, int batch, float lr,
                          uint64_t seed, float* val_loss);

/* Continue training the current model from its weights and standardisation
 * on all records held plus the loaded rehearsal sample, so that new records
 * add to what the model knows instead of replacing it (fine-tuning; a fresh
 * training on the records held when no model exists yet).  The fine-tuned
 * weights are kept only if they lower the held-out loss below that of the
 * weights they started from; otherwise the model is left as it was (still
 * COMPAR_OK; *val_loss then holds the unchanged model's loss, and the
 * context's count of discarded fine-tunes, compar_online_stats, grows).
 * Arguments as compar_selector_train. */
int compar_selector_finetune(compar_ctx_t ctx, int steps, int batch, float lr,
                             uint64_t seed, float* val_loss);

/* Online selection (the paper expects better-trained models to choose
 * better, Sec. 3.2 and Sec. 5).  With probability `epsilon` a call (its
 * decision cached or not) runs another eligible variant instead of the
 * pick, drawn uniformly among those predicted within 4x of the pick's time
 * (among all others when none is): exploration, not cached, aimed at the
 * close calls the models must learn to rank.  Every
 * call is recorded, and once `retrain_every` (> 0) new records have
 * accumulated the MLP is fine-tuned for `finetune_steps` (0: 500) steps
 * inside the call that crosses the threshold (synchronous).  epsilon = 0 and
 * retrain_every = 0 turn it off; recording stays as it was set. */
int compar_set_online(compar_ctx_t ctx, double epsilon, int64_t retrain_every,
                      int finetune_steps);
/* Exploratory picks, fine-tunes run (online or by compar_selector_finetune)
 * and, of those, fine-tunes discarded because they did not lower the
 * held-out loss.  `rejected` may be NULL. */
int compar_online_stats(compar_ctx_t ctx, int64_t* explored, int64_t* retrains,
                        int64_t* rejected);

/* The trained model's prediction for one call: per variant (arrays of
 * COMPAR_V_COUNT floats, indexed by variant id) the ensemble-mean run time in
 * ms, relative error, and the ensemble std of log2 time (spread, nullable).
 * COMPAR_ERR_UNSUPPORTED when untrained. */
int compar_predict(compar_ctx_t ctx, int64_t m, int64_t n, int64_t k,
                   compar_dtype_t dtype, double tol, int batch,
                   float* time_ms, float* rel_err, float* spread);

/* Relative Frobenius error of C against alpha * op_scale * A x B computed in
 * FP64 on the GPU over `nrows` rows drawn from `seed` (all rows when nrows >=
 * m); op_scale is the context's fp8 scales for F8E4M3 inputs, else 1.  A, B,
 * C are device pointers, row-major contiguous; C was computed with beta = 0.
 * Labels the accuracy of recorded runs.  Synchronises `stream` (refused,
 * COMPAR_ERR_UNSUPPORTED, while `stream` is being captured into a graph). */
int compar_residual_check(compar_ctx_t ctx, int64_t m, int64_t n, int64_t k,
                          compar_dtype_t dtype, const void* A, const void* B,
                          const float* C, float alpha, int nrows, uint64_t seed,
                          double* rel_err, void* stream);

/* ---------------------------------------------------------------- timing */

/* Time variant `variant_id` on one call with CUDA events on `stream`:
 * `warmup` untimed runs, then `reps` timed runs; *median_ms receives the
 * median.  Adds one timing record per timed run when recording is on, and one
 * observation to the history table.  Synchronises the stream (refused,
 * COMPAR_ERR_UNSUPPORTED, while it is being captured into a graph). */
int compar_measure(compar_ctx_t ctx, int variant_id, int64_t m, int64_t n,
                   int64_t k, compar_dtype_t dtype, double tol, const void* A,
                   const void* B, float* C, int warmup, int reps,
                   void* stream, float* median_ms);

/* One timing record: the call's context and the measured time (and, when a
 * residual check ran, the relative error; -1 otherwise). */
typedef struct {
    int64_t m, n, k;
    int32_t dtype;
    int32_t variant;
    int32_t batch;
    float tol;
    float time_ms;
    float rel_err;
} compar_record_t;

/* Recording of timing records (off by default). */
int compar_record_enable(compar_ctx_t ctx, int on);
/* Number of records held (ring buffer of 1<<20 records). */
int64_t compar_record_count(compar_ctx_t ctx);
/* Copy up to `max` records, oldest first, into host array `out`;
 * returns the number copied or a negative status. */
int64_t compar_record_get(compar_ctx_t ctx, compar_record_t* out, int64_t max);
/* Append externally measured records (host array). */
int compar_record_add(compar_ctx_t ctx, const compar_record_t* recs,
                      int64_t count);
int compar_record_clear(compar_ctx_t ctx);

/* ---------------------------------------------------------------- stencil */

/* The second component behind the same runtime: a thermal 2-D stencil (the
 * paper evaluates Rodinia's Hotspot, Table 2, with CUDA and OpenMP variants;
 * the computation is read here as the explicit step of the 2-D heat
 * equation).  One step updates every cell of a rows x cols grid:
 *   T'[i][j] = T[i][j] + c * ( P[i][j]
 *                + (T[i-1][j] + T[i+1][j] - 2 T[i][j]) * gy
 *                + (T[i][j-1] + T[i][j+1] - 2 T[i][j]) * gx
 *                + (amb - T[i][j]) * gz )
 * with a neighbour outside the grid replaced by the cell itself (insulated
 * edge).  Stable for c * (2 gx + 2 gy + gz) <= 1. */
typedef struct {
    float c;              /* time step / heat capacity                     */
    float gx, gy, gz;     /* conductance to column / row neighbours, ambient */
    float amb;            /* ambient temperature                           */
} compar_stencil_params_t;

/* Stencil variant ids (their own id space). */
enum {
    COMPAR_S_NAIVE = 0,   /* one thread per cell, one launch per step       */
    COMPAR_S_TILED = 1,   /* shared-memory temporal blocking, 8 steps/launch */
    COMPAR_S_TMA = 2,     /* the same with TMA region loads                 */
    COMPAR_S_COUNT = 3
};

/* `iters` steps from T_in into T_out (device float32 grids, row-major
 * contiguous, rows x cols; P the power grid).  T_in and P are not written;
 * T_out must not overlap T_in or P.  iters == 0 copies T_in.  The variant is
 * the forced one, else the decision cache, else the fastest by the stencil
 * history table (compar_stencil_measure feeds it; selector files carry it),
 * else by a roofline prior.  Every variant computes bit-identical grids.
 * Returns COMPAR_OK, COMPAR_ERR_INVALID (bad sizes, parameters, pointers or
 * overlap), COMPAR_ERR_UNSUPPORTED (forced variant cannot run this grid) or
 * COMPAR_ERR_CUDA; a TMA wait that runs out is reported through
 * compar_check_device_error.  Scratch (one grid) comes from the context's
 * workspace. */
int compar_stencil(compar_ctx_t ctx, int64_t rows, int64_t cols, int iters,
                   const compar_stencil_params_t* params, const float* T_in,
                   const float* P, float* T_out, void* stream);

/* Force stencil variant `v` (COMPAR_S_*), or clear with -1. */
int compar_stencil_force_variant(compar_ctx_t ctx, int v);
/* Variant used by the most recent compar_stencil call (-1 before any). */
int compar_stencil_last_variant(compar_ctx_t ctx);
/* Static name of stencil variant v, NULL if out of range. */
const char* compar_stencil_variant_name(int v);
/* Whether variant v can run a rows x cols grid (16-byte aligned grids
 * assumed): 1 / 0, or COMPAR_ERR_INVALID. */
int compar_stencil_supported(compar_ctx_t ctx, int v, int64_t rows, int64_t cols);
/* The variant compar_stencil would choose (works on host-only contexts). */
int compar_stencil_select(compar_ctx_t ctx, int64_t rows, int64_t cols, int iters);
/* Median time (ms, CUDA events on `stream`) of `reps` runs of variant v
 * after `warmup` runs; the result also feeds the stencil history table.
 * Synchronises `stream` (refused, COMPAR_ERR_UNSUPPORTED, while it is being
 * captured into a graph). */
int compar_stencil_measure(compar_ctx_t ctx, int v, int64_t rows, int64_t cols, int iters,
                           const compar_stencil_params_t* params, const float* T_in,
                           const float* P, float* T_out, int warmup, int reps,
                           void* stream, float* median_ms);

/* ---------------------------------------------------------------- profiling */

/* Kernel timing: when on, the main GEMM kernel of every call (not its
 * operand pre-passes) is bracketed by CUDA events on the call's stream and
 * its duration added to a per-variant total; for a stencil call, all its
 * launches together.  Off by default.  Slots: 0..COMPAR_V_COUNT-1
 * the GEMM variant ids, COMPAR_V_COUNT + s the stencil variant s. */
int compar_profile_enable(compar_ctx_t ctx, int on);
/* Total kernel milliseconds and number of timed launches of `variant` since
 * the last reset (synchronises on the pending events). */
int compar_profile_read(compar_ctx_t ctx, int variant, double* kernel_ms,
                        int64_t* launches);
int compar_profile_reset(compar_ctx_t ctx);

/* Number of CUDA kernels this library has launched in this process (every
 * variant kernel and every pre-pass kernel). */
int64_t compar_launch_count(void);

/* Measured FP32 FMA-pipe throughput of this GPU (TFLOP/s, 2 flops per FMA):
 * register-resident independent FMA chains at full occupancy, median of 5
 * timed launches on `stream`.  The roofline denominator of the naive and SIMT
 * variants.  Synchronises `stream`. */
int compar_peak_ffma(compar_ctx_t ctx, float* tflops, void* stream);

/* ---------------------------------------------------------------- errors */

/* Read and clear the device error word after synchronising `stream`.
 * Returns COMPAR_OK, COMPAR_ERR_TIMEOUT (a bounded wait in a kernel ran out;
 * the kernel returned early and C is undefined) or COMPAR_ERR_CUDA. */
int compar_check_device_error(compar_ctx_t ctx, void* stream);

/* Budget of every device-side bounded wait, in nanoseconds of %globaltimer
 * (default 2e9).  Values below 1000 are raised to 1000. */
int compar_set_wait_budget(compar_ctx_t ctx, uint64_t ns);

/* Launch one small kernel whose wait on an mbarrier can never complete, so
 * the bounded wait runs out after the wait budget; the kernel records
 * COMPAR_ERR_TIMEOUT in the device error word and returns.  Used to test the
 * timeout path without faulting or hanging the GPU.  Asynchronous. */
int compar_selftest_timeout(compar_ctx_t ctx, void* stream);

/* Launch plan of tensor-core variant `variant_id` (COMPAR_V_TC_TF32 ..
 * COMPAR_V_SPLIT3_FUSED, not GROUPED) for an m x n x k call on a GPU with
 * `num_sms` SMs, without a device: out[0] K blocks, [1] 128 x 256 output
 * tiles, [2] K splits (> 1: split-K with a reduce), [3] K blocks per split,
 * [4] first stream-K tile (tiles before it are dealt whole, round-robin),
 * [5] stream-K chunks per tile, [6] stream-K chunks in all (0: no stream-K
 * tail), [7] CTAs sharing the tail, [8] K blocks per stream-K chunk.
 * COMPAR_ERR_INVALID for other variants or sizes < 1. */
int compar_tc_plan(int variant_id, int64_t m, int64_t n, int64_t k, int num_sms,
                   int64_t* out);

/* The same plan for the CTA-pair kernels (no counterpart in the paper; a
 * B300 kernel design): a pair of CTAs on one TPC computes a 256 x 256 tile
 * with tcgen05 pair MMAs (cta_group::2), each CTA holding half of A's rows
 * and half of B's columns in its shared memory.  `num_pairs` pairs run at
 * once; out[] as compar_tc_plan, with tiles of 256 x 256, "CTAs" counting
 * pairs, and K never split (out[2] = 1).  Variants TF32, BF16, FP8 and
 * SPLIT3; COMPAR_ERR_INVALID for the others or sizes < 1. */
int compar_tc_pair_plan(int variant_id, int64_t m, int64_t n, int64_t k, int num_pairs,
                        int64_t* out);

/* When the tensor-core variants TF32, BF16, FP8 and SPLIT3 run on CTA
 * pairs: mode -1 (default) when the single-CTA plan has a full wave of
 * 128 x 256 tiles or more, 0 never, 1 always.  Results agree with the
 * single-CTA kernels within the variant's tolerance (the tile and stream-K
 * decomposition, and with it the rounding, differ).  Returns COMPAR_OK or
 * COMPAR_ERR_INVALID. */
int compar_set_tc_pairs(compar_ctx_t ctx, int mode);

/* Launch plan of the SIMT variant (COMPAR_V_SIMT) for an m x n x k call
 * with inputs of `dtype`, B's row stride `ldb` (elements) and a 16-byte
 * aligned B, on a GPU with `num_sms` SMs, without a device: out[0] 1 for the
 * skinny-M kernel (a few rows of A against a wide, deep B: K chunks summed
 * in thread-block clusters), 0 for the tiled kernel; [1] rows and [2]
 * columns of C per CTA; [3] partial sums added by the reduce pass (1: none);
 * [4] K per chunk or split (the longest FMA chain); [5] CTAs per cluster
 * (1 for the tiled kernel).  COMPAR_ERR_INVALID for sizes < 1, ldb < n or
 * an unknown dtype. */
int compar_simt_plan(int64_t m, int64_t n, int64_t k, compar_dtype_t dtype, int64_t ldb,
                     int num_sms, int64_t* out);

#ifdef __cplusplus
}
#endif
#endif /* COMPAR_H_ */
