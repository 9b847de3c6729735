/*
 * qiht.h -- C ABI of the QIHT library (GB300, sm_103a).
 *
 * QIHT is normalized iterative hard thresholding run on stochastically
 * quantized data: Gurel et al., "Compressive Sensing Using Iterative Hard
 * Thresholding with Low Precision Data Representation", IEEE TSP 2020.
 *   problem      y = Phi x + e, minimise ||y - Phi x||^2 s.t. ||x||_0 <= s     (Section I-A)
 *   quantizer    Q(v, b): 2^b levels on [-1, 1], stochastic rounding            (Section III-A)
 *                or 2^(b-1) + 1 levels, 0 among them                          (Appendix, remark on FPGAs)
 *   iteration    x <- H_s(x + mu Q1^T (Q(y) - Q2 x)), adaptive mu, backtracking (Algorithm 2)
 *
 * Conventions (every entry point):
 *   - Pointers marked [device] are CUDA device addresses; [host] are host
 *     addresses. The caller owns every buffer, including workspaces. The
 *     library never allocates device memory on these paths.
 *   - Calls are asynchronous on `stream` unless stated otherwise; results are
 *     valid after the stream is synchronised. NULL stream = legacy default stream.
 *   - Argument errors are detected on the host before any launch and returned
 *     as a status; nothing is launched then. Errors found on the device (non-
 *     finite scales, a backtracking cap) are written to the device report.
 *   - No exception crosses this boundary.
 *
 * Code matrix layout ("column-packed"): a quantized rows x cols matrix is
 * stored as cols columns of ld_words 32-bit words each, column j starting at
 * word j * ld_words (16-byte aligned). With G = 32 / bits codes per word, word
 * q of a column holds rows q*G .. q*G+G-1; the code of row q*G + 4k + p
 * (k = 0 .. G/4-1, p = 0..3) sits at bit 8p + bits*k. Rows past `rows` hold
 * code 0 and never contribute. A vector is a matrix with one column.
 * Grids: L = 2^bits levels (Section III-A; the default), or the odd grid of
 * L = 2^(bits-1) + 1 levels with spacing 1/2^(bits-2) on [-1, 1] (the
 * Appendix's remark on fixed-point hardware; 0 is a level), stored in the same
 * bits (codes 0 .. L-1). The value of code c is scale * (2c - (L - 1)) / (L - 1).
 *
 * Random numbers of the quantizer: Philox4x32-10 (Salmon et al., SC'11) with
 * key (seed low 32 bits, seed high 32 bits) and counter (e>>2 low, e>>2 high,
 * stream_id, 0), where e = j * rows + i is the column-major index of element
 * (i, j); element e uses output word e & 3 and u = (word >> 8) * 2^-24.
 * The rounding decision is taken in binary32: t = (v / c + 1) * (L - 1) / 2,
 * clamped to [0, L - 1], code = floor(t) + (u < t - floor(t)) (at most L - 1),
 * each operation correctly rounded. (The kernels divide by c with a reciprocal and
 * two FMAs; where |v / c| < 2^-25 their quotient may differ in its last bits, but
 * 1 + v / c rounds to 1 either way, so t and the code are the same.)
 */
#ifndef QIHT_H
#define QIHT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QIHT_ABI_VERSION 4

/* Same type as cudaStream_t. */
typedef struct CUstream_st* qiht_stream_t;

typedef enum {
    QIHT_OK = 0,
    QIHT_ERR_ARG = 1,            /* null pointer, size out of range, s > m or s > n, ... */
    QIHT_ERR_BITS = 2,           /* bits not in {2, 4, 8} */
    QIHT_ERR_NONFINITE = 3,      /* NaN or Inf in the input (its scale is not finite) */
    QIHT_ERR_TIMEOUT = 4,        /* a device-side wait ran out of its budget */
    QIHT_ERR_BACKTRACK_CAP = 5,  /* the step size was shrunk max_backtrack times in one iteration */
    QIHT_ERR_CUDA = 6,           /* a CUDA runtime call failed */
    QIHT_ERR_WORKSPACE = 7       /* workspace missing, too small or not 256-byte aligned */
} qiht_status;

/* Human-readable name of a status (static string). */
const char* qiht_status_string(int32_t status);

/* Version of this ABI (QIHT_ABI_VERSION of the built library). */
int32_t qiht_abi_version(void);

/* Description of the last CUDA runtime failure seen by this thread inside the
 * library (the call and the CUDA error string), or "" if there was none. */
const char* qiht_last_error(void);

/* A quantized matrix or vector in the column-packed layout (see above). */
typedef struct {
    const uint32_t* words;   /* [device] cols * ld_words words */
    const float* scale;      /* [device] one float: c = max |v| used by the quantizer */
    int32_t rows;            /* rows of the logical matrix (length of a vector) */
    int32_t cols;            /* columns (1 for a vector) */
    int32_t bits;            /* 2, 4 or 8 */
    int32_t ld_words;        /* words per column; must equal qiht_ld_words(rows, bits) */
    int32_t levels;          /* grid the codes were made on: 0 or 2^bits (the default grid),
                                or 2^(bits-1) + 1 (the odd grid, QIHT_ODD_LEVELS); any other
                                value is QIHT_ERR_ARG */
    int32_t reserved;        /* 0 */
} qiht_codes;

/* Words per column of the column-packed layout: ceil(rows / (32/bits)) rounded
 * up to a multiple of 4. Returns -1 for bits not in {2, 4, 8} or rows < 1. */
int32_t qiht_ld_words(int32_t rows, int32_t bits);

/* ---------------------------------------------------------------------- */
/* Quantization (Section III-A; scale c_v = max |v| from the Appendix's    */
/* quantization-error lemma)                                                */
/* ---------------------------------------------------------------------- */

#define QIHT_SCALE_GIVEN   1  /* use *scale as it is (do not compute max |v|) */
#define QIHT_CHECK_FINITE  2  /* synchronise `stream` and return QIHT_ERR_NONFINITE if the scale is not finite */
#define QIHT_ODD_LEVELS    4  /* quantize on the odd grid of 2^(bits-1) + 1 levels; the codes are then
                                 described by a qiht_codes with levels = 2^(bits-1) + 1 */

/* Quantize a rows x cols float32 matrix `in` [device], row-major with row
 * stride ld_in >= cols (floats), to `bits`-bit codes in the column-packed
 * layout at `words` [device, cols * ld_words words, 16-byte aligned]. *scale
 * [device] receives c = max |in| (or is read, with QIHT_SCALE_GIVEN). A
 * non-finite input makes *scale non-finite. seed and stream_id select the
 * random numbers (the solver uses 0 for Q1, 1 for Q2, 2 for y by convention).
 * Launches two kernels (max |v|, then quantize + pack) unless the scale is given. */
qiht_status qiht_quantize(const float* in, int32_t rows, int32_t cols, int64_t ld_in, int32_t bits,
                          uint64_t seed, uint32_t stream_id, int32_t flags,
                          uint32_t* words, int32_t ld_words, float* scale, qiht_stream_t stream);

/* Two independent quantizations of the same matrix in one pass over `in` (the double
 * sampling of Algorithm 2: Q1 and Q2 of Phi, sharing the scale c). Element by element
 * the result is bit-identical to two qiht_quantize calls with stream_a -> words_a and
 * stream_b -> words_b (same seed and scale); the rounding decision, which does not
 * depend on the random number, is computed once. Arguments as for qiht_quantize;
 * words_a and words_b are distinct buffers of cols * ld_words words each. */
qiht_status qiht_quantize_pair(const float* in, int32_t rows, int32_t cols, int64_t ld_in, int32_t bits,
                               uint64_t seed, uint32_t stream_a, uint32_t stream_b, int32_t flags,
                               uint32_t* words_a, uint32_t* words_b, int32_t ld_words, float* scale,
                               qiht_stream_t stream);

/* ---------------------------------------------------------------------- */
/* Building blocks of one iteration (exposed for tests and measurement)     */
/* ---------------------------------------------------------------------- */

/* g = Q^T r: the gradient product of Algorithm 2 (g = Q1^T r), one pass over
 * all codes of Q. r [device, Q->rows floats], g [device, Q->cols floats].
 * Inner sums are exact: r is converted to 24-bit block fixed point (scale =
 * a power of two set by max |r|) and codes times fixed-point r are summed in
 * integers; the result is scaled once per column. Requires Q->rows <= 16384.
 * Workspace: qiht_gemv_t_workspace_size() bytes, 256-byte aligned. */
size_t qiht_gemv_t_workspace_size(void);
qiht_status qiht_gemv_t(const qiht_codes* Q, const float* r, float* g,
                        void* workspace, size_t workspace_bytes, qiht_stream_t stream);

/* The same product when max |r| is already known: rmax [device, one float]
 * must hold max |r| exactly (as the solver keeps it). Launches one kernel,
 * the one the solver runs every iteration, with the same launch plan. */
qiht_status qiht_gemv_t_prescaled(const qiht_codes* Q, const float* r, const float* rmax, float* g,
                                  qiht_stream_t stream);

/* z = Q[:, cols] coef: product with a column subset, the products of Algorithm 2 with
 * the second quantization: Q2 x on the support (the residual), Q2_G g_G of the step size
 * (the Eq. for mu) and Q2 (x' - x) of the backtracking test (Section II-A).
 * cols [device, count int32 in [0, Q->cols)], coef [device, count floats],
 * z [device, Q->rows floats]. FP32 sums in a fixed order (deterministic).
 * The indices are read on the device only: an entry outside [0, Q->cols) is never
 * used to address the codes; it makes every entry of z NaN instead.
 * Workspace: qiht_gemv_cols_workspace_size(Q->rows, count) bytes. */
size_t qiht_gemv_cols_workspace_size(int32_t rows, int32_t count);
qiht_status qiht_gemv_cols(const qiht_codes* Q, const int32_t* cols, const float* coef, int32_t count,
                           float* z, void* workspace, size_t workspace_bytes, qiht_stream_t stream);


/* Allocation-free variant of qiht_gemv_cols. The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory when they
 * need the product (code running while its stream is captured into a CUDA graph,
 * real-time loops that forbid allocation once running, plug-ins whose host owns
 * every device allocation). Same arguments and results as qiht_gemv_cols, but
 * the scratch is a fixed array of QIHT_STATIC_SCRATCH_BYTES inside this library,
 * held on every GPU that loads the library until the process exits; the call
 * allocates nothing. Limit: qiht_gemv_cols_workspace_size(Q->rows, count) must not
 * exceed QIHT_STATIC_SCRATCH_BYTES, else QIHT_ERR_WORKSPACE is returned and nothing
 * is launched. The first call in a CUDA context (the runtime's primary context of a
 * device, or a context made current through the driver API) looks up the array's
 * device address in that context (cudaGetSymbolAddress, with the context current);
 * make that first call before any stream capture. All calls share the one array:
 * calls whose kernels overlap on the GPU (other streams, other threads) race and
 * give wrong results. Indices outside [0, Q->cols) give a NaN z, as for
 * qiht_gemv_cols. */
#define QIHT_STATIC_SCRATCH_BYTES (2u << 20)
qiht_status qiht_gemv_cols_static(const qiht_codes* Q, const int32_t* cols, const float* coef, int32_t count,
                                  float* z, qiht_stream_t stream);

/* G = Q^T R for nrhs residual vectors at once: the gradient products of Algorithm 2 for
 * many right-hand sides sharing one quantized matrix (many observations y_k of the same
 * Phi), a dense contraction run on the tensor cores. R [device] nrhs x ldr floats (row k
 * = residual k, Q->rows entries used, ldr >= Q->rows), G [device] nrhs x ldg floats
 * (row k = Q^T r_k, Q->cols entries written, ldg >= Q->cols). Arithmetic: the centred
 * codes 2c - (L-1) are exact in f16; each residual is scaled by a power of two and split
 * into two f16 parts (hi + lo, about 22 significant bits); the products are exact and
 * summed in FP32, then scaled once. Requires Q->rows <= 16384. status [device, one
 * int32, may be NULL] is set to QIHT_ERR_TIMEOUT if a device-side wait ran out (and
 * left as it was otherwise). Launches two kernels, or three when the product's last wave
 * of 256 x 256 tiles would hold at most half the SMs: those tiles are then summed in two
 * halves of the rows, added (in either order, with the same result) into their part of
 * G, which a third kernel zeroes first.
 * Workspace: qiht_gemv_t_multi_workspace_size(Q->rows, nrhs) bytes, 256-byte aligned. */
size_t qiht_gemv_t_multi_workspace_size(int32_t rows, int32_t nrhs);
qiht_status qiht_gemv_t_multi(const qiht_codes* Q, const float* R, int64_t ldr, int32_t nrhs, float* G,
                              int64_t ldg, int32_t* status, void* workspace, size_t workspace_bytes,
                              qiht_stream_t stream);

/* The same product with FP8 operands, for codes of 2 or 4 bits (else QIHT_ERR_BITS): the centred
 * codes 2c - (L-1) are exact in e4m3 (|2c - (L-1)| <= 15), the residual is scaled by a power of
 * two (max |r| 2^-e in [2^7, 2^8)) and split into three e4m3 terms, r' ~ t1 + t2 + t3 with
 * |r' - t1 - t2 - t3| <= 2^-12 |r'| + 2^-10, and tcgen05.mma kind::f8f6f4 sums the products in
 * FP32 (K = 32 rows per MMA instead of 16, three terms instead of two parts: 3/4 of the MMA work
 * of the f16 split, at about 12 significant bits instead of 22). This is the paper's observation
 * that codes of b <= 4 bits are exact in an 8-bit floating-point format (Section III-A, the
 * quantizer's levels), carried to the tensor cores. Arguments, workspace and errors as for
 * qiht_gemv_t_multi. */
qiht_status qiht_gemv_t_multi_fp8(const qiht_codes* Q, const float* R, int64_t ldr, int32_t nrhs, float* G,
                                  int64_t ldg, int32_t* status, void* workspace, size_t workspace_bytes,
                                  qiht_stream_t stream);

/* Hard threshold H_s (Eq. NIHT): the s entries of a [device, n floats] of
 * largest magnitude, ties broken by the lower index; exactly s are kept.
 * idx [device, s int32] receives their indices in ascending order, val
 * [device, s floats, may be NULL] their values, kth [device, 2 floats, may be
 * NULL] the s-th and (s+1)-th largest magnitudes (0 if s == n).
 * Requires 1 <= s <= n <= 2^24. Up to 49152 entries one CTA selects (no workspace); above,
 * a multi-CTA radix select with the same result needs qiht_top_s_workspace_size(n) bytes
 * of workspace (256-byte aligned, else QIHT_ERR_WORKSPACE). */
size_t qiht_top_s_workspace_size(int32_t n);
qiht_status qiht_top_s(const float* a, int32_t n, int32_t s, int32_t* idx, float* val, float* kth,
                       void* workspace, size_t workspace_bytes, qiht_stream_t stream);

/* ---------------------------------------------------------------------- */
/* The solver (Algorithm 2)                                                 */
/* ---------------------------------------------------------------------- */

#define QIHT_SOLVE_EAGER 1  /* launch the kernels one by one from the host (no graph; synchronises the
                              stream every iteration). Same kernels and results as the graph;
                              meant for debugging and per-kernel profiling. */

#define QIHT_SOLVE_TEST_TIMEOUT 2  /* test hook, not part of the method: the iteration kernel's CTA 0
                                     withholds its first step-size decision, so every other CTA's
                                     bounded wait on it runs out (about 0.2 s) and the solve stops
                                     with QIHT_ERR_TIMEOUT in the report; the CUDA context stays
                                     usable. Honoured by the kernel used for s <= 1024. */

#define QIHT_SOLVE_FP8 4   /* qiht_niht_solve_multi only, codes of 2 or 4 bits: the gradient products run
                              as qiht_gemv_t_multi_fp8 (e4m3 operands, about 12 significant bits of the
                              residual) instead of the two-part f16 split (about 22 bits) */

/* Denominator of the step size mu = ||g_G||^2 / den on the current support G (Eq. for mu). */
#define QIHT_MU_FORWARD_SQ 0  /* den = ||Q2_G g_G||^2 (positive; the default) */
#define QIHT_MU_CROSS      1  /* den = (Q1_G g_G)^T (Q2_G g_G), the product of the two quantizations that
                                 Algorithm 2 prints (with fresh realizations: Phi-hat_{2n-1} and
                                 Phi-hat_{2n}); when it is not positive, the forward square is used */

typedef struct {
    double k;               /* shrinkage of the step size, k > 1/(1-c) (Section II-A); default 2 */
    double c;               /* small constant of the descent test, 0 < c < 1; default 0.01 */
    int32_t max_backtrack;  /* shrinks allowed per iteration before QIHT_ERR_BACKTRACK_CAP; default 32 */
    int32_t flags;          /* 0 or QIHT_SOLVE_EAGER, QIHT_SOLVE_TEST_TIMEOUT */
    double tol;             /* 0: off. > 0: stop after the first iteration whose ||Q(y) - Q2 x||^2 (FP64) is
                               at most tol. The paper stops after a fixed number of iterations,
                               n* = ceil(log2(||x^s|| / eps_s)) (Section III-B, after Theorem 4); tol states
                               the same criterion on the residual, for when eps_s is not known. Must be
                               finite and >= 0. */
    int32_t mu_mode;        /* QIHT_MU_FORWARD_SQ (default) or QIHT_MU_CROSS; Q1 and Q2 must then be on
                               the same grid */
    int32_t reserved;       /* 0 */
} qiht_params;

typedef struct {            /* written on the device after every iteration */
    int32_t iters_run;      /* iterations completed (an iteration that stopped early is not counted) */
    int32_t backtracks;     /* total step-size shrinks */
    int32_t support_changes;/* iterations whose accepted support differs from the previous one */
    int32_t status;         /* qiht_status of the run: OK, NONFINITE, BACKTRACK_CAP or TIMEOUT */
    double resid_norm2;     /* ||Q(y) - Q2 x||^2 of the returned x (FP64 sum of FP32 residuals) */
    double mu;              /* last accepted step size */
    int32_t full_selects;   /* selections that ranked all n entries (the rest used the candidate list) */
    int32_t reserved;
    float phase_us[8];      /* diagnostics: device-clock durations of the last iteration's phases
                               (step size, filter, select, backtracking tests, residual, commit) */
} qiht_report;

typedef struct {            /* optional per-iteration record [device]; any field may be NULL */
    int32_t* support;       /* (iters+1) x s: row 0 = initial support, row t = support after iteration t */
    float* kth;             /* (iters+1) x 2: s-th and (s+1)-th |x + mu g| of the accepted selection */
    double* mu;             /* (iters+1): accepted step size (row 0 = 0) */
    int32_t* bt;            /* (iters+1): shrinks in that iteration */
    double* resid2;         /* (iters+1): ||Q(y) - Q2 x||^2 after that iteration */
} qiht_trace;

/* Workspace bytes for qiht_niht_solve with these sizes (256-byte aligned buffer). */
size_t qiht_solve_workspace_size(int32_t m, int32_t n, int32_t s);

/* Run `iters` iterations of QIHT (Algorithm 2) with fixed quantizations:
 * g = Q1^T (Q(y) - Q2 x) with Q1, Q2 two independent quantizations of Phi
 * (m x n) and y (m, one column); mu = ||g_G||^2 / ||Q2_G g_G||^2 on the
 * current support G; x' = H_s(x + mu g); when the support changes, the step is
 * shrunk by k(1-c) while mu > (1-c) ||x'-x||^2 / ||Q2 (x'-x)||^2.
 * Initial state: x = 0, G = supp H_s(Q1^T Q(y)). The run stops early when
 * ||g_G||^2 or ||Q2_G g_G||^2 is zero (converged) or on a device error.
 * Outputs: x [device, n floats, dense, s-sparse], support [device, s int32,
 * ascending], report [device, one qiht_report]. trace may be NULL.
 * The whole run is one CUDA-graph launch (built on the first call with a given
 * set of arguments and cached); control never returns to the host between
 * iterations. Requires 1 <= s <= min(m, n), m <= 16384, n <= 49152.
 * params may be NULL (the defaults). With params->tol > 0 the run stops after the
 * first iteration whose residual is at most tol; the report's iters_run says which. */
qiht_status qiht_niht_solve(const qiht_codes* Q1, const qiht_codes* Q2, const qiht_codes* y,
                            int32_t s, int32_t iters, const qiht_params* params,
                            float* x, int32_t* support, qiht_report* report, const qiht_trace* trace,
                            void* workspace, size_t workspace_bytes, qiht_stream_t stream);

/* Drop every cached solver graph (e.g. before freeing buffers they reference). */
void qiht_clear_graph_cache(void);

/* ---------------------------------------------------------------------- */
/* Fresh realizations per iteration (Algorithm 2 as written: 2 n* matrix    */
/* realizations and n* observation realizations)                           */
/* ---------------------------------------------------------------------- */

/* Workspace bytes for qiht_niht_solve_fresh (0 if a size is out of range). */
size_t qiht_solve_fresh_workspace_size(int32_t m, int32_t n, int32_t s, int32_t bits_phi, int32_t bits_y);

/* Algorithm 2 with a new quantization of Phi and y in every iteration: iteration t
 * (1..iters) forms g = Phi-hat_{2t-1}^T (y-hat_t - Phi-hat_{2t} x), the step size and the
 * backtracking test with Phi-hat_{2t}, and records ||y-hat_t - Phi-hat_{2t} x||^2; the initial
 * support comes from Phi-hat_1^T y-hat_1. Realization k of Q(Phi) uses random-number stream
 * (k <= 2 ? k - 1 : 0x1000 + k), realization t of Q(y) stream (t == 1 ? 2 : 0x2000 + t), all with
 * `seed` and the scales max |Phi|, max |y| (so iteration 1 equals qiht_niht_solve's on the
 * quantizations with streams 0, 1, 2). phi [device] m x n row-major (row stride ld_phi
 * >= n floats), y [device] m floats; quant_flags 0 or QIHT_ODD_LEVELS. Outputs and
 * params as for qiht_niht_solve (params->flags must be 0; with QIHT_MU_CROSS the step size
 * takes the product of the iteration's two realizations, as Algorithm 2 prints it). Every
 * iteration re-quantizes
 * Phi twice (one pass over the FP32 matrix) and y, then runs the iteration as separate
 * kernels; the host reads the solver state after every iteration and backtracking test,
 * so the call returns when the solve is done (the stream is synchronised). Requires
 * m <= 16384, n <= 49152. */
qiht_status qiht_niht_solve_fresh(const float* phi, int64_t ld_phi, const float* y, int32_t m, int32_t n,
                                  int32_t bits_phi, int32_t bits_y, uint64_t seed, int32_t quant_flags, int32_t s,
                                  int32_t iters, const qiht_params* params, float* x, int32_t* support,
                                  qiht_report* report, const qiht_trace* trace, void* workspace,
                                  size_t workspace_bytes, qiht_stream_t stream);

/* ---------------------------------------------------------------------- */
/* Many independent problems in one launch (the batched workload of the    */
/* solver: Algorithm 2 applied to each problem separately)                  */
/* ---------------------------------------------------------------------- */

#define QIHT_BATCH_MAX_ROWS 2048   /* m of every problem of a batch */
#define QIHT_BATCH_MAX_COLS 8192   /* n */
#define QIHT_BATCH_MAX_S 256       /* s */

typedef struct {
    qiht_codes Q1, Q2, y;   /* as for qiht_niht_solve; Q1 and Q2 of every problem of a batch have the same bits */
    int32_t s;              /* sparsity, 1 <= s <= min(m, n, QIHT_BATCH_MAX_S) */
    int32_t reserved;       /* 0 */
    float* x;               /* [device] n: the returned x (dense) */
    int32_t* support;       /* [device] s: its support, ascending */
    qiht_report* report;    /* [device] the problem's report (phase_us zero) */
} qiht_problem;

/* Bytes of workspace for a batch of nprob problems (0 if nprob < 1). */
size_t qiht_solve_batched_workspace_size(int32_t nprob);

/* qiht_niht_solve for each of nprob independent problems (`problems`: a HOST array,
 * read during the call; all buffers it points to are device memory), `iters` iterations
 * each, in one persistent launch: every CTA solves whole problems, largest first,
 * entirely in its shared memory (the limits above keep a problem's vectors there).
 * Results per problem are those of the same algorithm and arithmetic as
 * qiht_niht_solve (exact-integer gradient, FP32 products, FP64 step size; the order of
 * some FP32 sums differs). params->tol must be 0 and params->mu_mode QIHT_MU_FORWARD_SQ.
 * Errors: QIHT_ERR_ARG (a problem out of the limits, mixed bits,
 * bad pointers), QIHT_ERR_BITS, QIHT_ERR_WORKSPACE, QIHT_ERR_CUDA; per-problem numeric
 * failures are in the problem's report. Asynchronous on `stream` after the descriptor
 * copy. */
qiht_status qiht_niht_solve_batched(const qiht_problem* problems, int32_t nprob, int32_t iters,
                                    const qiht_params* params, void* workspace, size_t workspace_bytes,
                                    qiht_stream_t stream);

/* ---------------------------------------------------------------------- */
/* Many right-hand sides sharing one quantized matrix (Algorithm 2 run for  */
/* many observations y_k of the same Phi)                                   */
/* ---------------------------------------------------------------------- */

#define QIHT_MULTI_MAX_ROWS 16384  /* m */
#define QIHT_MULTI_MAX_COLS 32768  /* n */
#define QIHT_MULTI_MAX_S 256       /* s */

/* Bytes of workspace for qiht_niht_solve_multi (0 if a size is out of range). */
size_t qiht_solve_multi_workspace_size(int32_t m, int32_t n, int32_t s, int32_t nrhs);

/* qiht_niht_solve for nrhs observations y[k] (a HOST array of nrhs vector descriptors,
 * each of Q1->rows entries, read during the call) sharing Q1 and Q2, `iters` iterations
 * each. One iteration computes the gradients of all right-hand sides as one tensor-core
 * product (qiht_gemv_t_multi), then the step size, H_s with backtracking and the
 * residual of every right-hand side (one CTA each). Results: X [device] nrhs x n (row k
 * = x of y[k], dense), support [device] nrhs x s (ascending), reports [device] nrhs.
 * Arithmetic: that of qiht_niht_solve except the gradient (f16 products of the exact
 * codes with a two-part f16 split of the residual, FP32 sums; see qiht_gemv_t_multi).
 * Requires m <= QIHT_MULTI_MAX_ROWS, n <= QIHT_MULTI_MAX_COLS, 1 <= s <= min(m, n,
 * QIHT_MULTI_MAX_S); params->flags 0 or QIHT_SOLVE_FP8 (2- and 4-bit codes: the FP8 gradient
 * product), params->tol 0 and params->mu_mode QIHT_MU_FORWARD_SQ. Errors as for qiht_niht_solve; numeric
 * failures of a right-hand side are in its report, a device-side timeout of the
 * gradient product (QIHT_ERR_TIMEOUT) in every report. Asynchronous on `stream` after
 * the descriptor copy. */
qiht_status qiht_niht_solve_multi(const qiht_codes* Q1, const qiht_codes* Q2, const qiht_codes* y, int32_t nrhs,
                                  int32_t s, int32_t iters, const qiht_params* params, float* X,
                                  int32_t* support, qiht_report* reports, void* workspace, size_t workspace_bytes,
                                  qiht_stream_t stream);

/* ---------------------------------------------------------------------- */
/* K unrolled iterations and their adjoint (calibration of a per-row gain)   */
/* ---------------------------------------------------------------------- */

/* Bytes of workspace for qiht_unrolled_forward / _backward (0 if a size is out of range). */
size_t qiht_unrolled_workspace_size(int32_t nprob, int32_t m, int32_t n, int32_t s, int32_t K);

/* K iterations of Algorithm 2 without the backtracking test, for nprob problems sharing m,
 * n and bits: Q1[p], Q2[p] (HOST arrays of descriptors, read during the call) are the two
 * quantizations of problem p's Phi; the operator is the stacked real system
 * A_i = [diag(a); diag(b)] Q_i (2m x n) of the per-row complex gain g = a + i b
 * (gain_re = a, gain_im = b: [device] nprob x m floats); y [device] nprob x 2m floats (not
 * quantized). With x_0 = 0: r_t = y - A2 x_t, h_t = A1^T r_t, G_t = supp H_s(h_0) for t = 0
 * and the support of x_t after, mu_t = ||h_t on G_t||^2 / ||A2 (h_t on G_t)||^2,
 * x_{t+1} = H_s(x_t + mu_t h_t). X [device] nprob x n receives x_K. The workspace keeps the
 * state every ceil(sqrt(K)) steps for qiht_unrolled_backward. Requires m <= 16384,
 * n <= 32768, 1 <= s <= min(m, n, 256), K >= 0 (K = 0 gives X = 0).
 * Definition: the iteration of Algorithm 2 with the adaptive step size (Eq. for mu) and H_s,
 * on the stacked real form of a complex measurement (Section IV-B); the backtracking test is
 * left out so that the map is differentiable with the supports held fixed.
 * Ownership: the caller owns every buffer; the workspace (qiht_unrolled_workspace_size bytes,
 * 256-byte aligned, device) holds the checkpoints and must be passed unchanged to the
 * matching qiht_unrolled_backward. Errors: QIHT_ERR_ARG (null pointers, problems of different
 * m, n or bits, sizes out of range), QIHT_ERR_BITS (bits not 2, 4 or 8), QIHT_ERR_WORKSPACE
 * (too small or misaligned), QIHT_ERR_CUDA (a failed launch or copy; qiht_last_error says
 * which). Nothing is launched when an argument check fails. Asynchronous on `stream` after
 * the descriptor copies. */
qiht_status qiht_unrolled_forward(const qiht_codes* Q1, const qiht_codes* Q2, int32_t nprob, const float* y,
                                  const float* gain_re, const float* gain_im, int32_t s, int32_t K, float* X,
                                  void* workspace, size_t workspace_bytes, qiht_stream_t stream);

/* The adjoint of qiht_unrolled_forward with the supports held fixed: from Xbar = dL/dx_K
 * [device, nprob x n] it writes ybar = dL/dy (nprob x 2m), gain_re_bar = dL/da and
 * gain_im_bar = dL/db (nprob x m each). Call it after qiht_unrolled_forward with the same
 * arguments and workspace: each segment between checkpoints is recomputed, recording what
 * the reverse steps need. The adjoint is that of the map defined for qiht_unrolled_forward
 * (masks fixed): through x_{t+1} = P_{t+1}(x_t + mu_t h_t), mu_t = N_t / D_t, h_t = A1^T r_t
 * and r_t = y - A2 x_t, with the gains entering A1 and A2 by rows. FP32 products, FP64
 * scalars. Xbar may alias nothing that the call writes. Errors as for qiht_unrolled_forward.
 * Asynchronous on `stream`. */
qiht_status qiht_unrolled_backward(const qiht_codes* Q1, const qiht_codes* Q2, int32_t nprob, const float* y,
                                   const float* gain_re, const float* gain_im, int32_t s, int32_t K, const float* Xbar,
                                   float* ybar, float* gain_re_bar, float* gain_im_bar, void* workspace,
                                   size_t workspace_bytes, qiht_stream_t stream);

/* ---------------------------------------------------------------------- */
/* Phi computed on the fly (Section IV-C: the entries of Phi generated      */
/* inside the device instead of read from memory), for the gridded         */
/* radio-interferometry matrix of Section IV-B                              */
/* ---------------------------------------------------------------------- */

#define QIHT_FLY_MAX_GRID 256

/* The interferometry measurement matrix (Section IV-B: Phi_kp = exp(-2 pi i (u_k l_p + v_k m_p)),
 * stacked real) with gridded visibilities: baseline k lies on the uv grid of a g x g sky image at
 * integer coordinates (u_k, v_k), and pixel p = ix * g + iy (direction cosines proportional to
 * ix - g/2 and iy - g/2, spacing the inverse of the grid's extent). The phase of entry (k, p) is
 * then 2 pi t_kp / g with the integer index
 *   t_kp = (u_k (ix - g/2) + v_k (iy - g/2)) mod g,
 * and the stacked real matrix (m = 2K rows, n = g^2 columns) is
 *   Phi[k][p]     = table[t_kp]        (k < K, the real part)
 *   Phi[K + k][p] = table[g + t_kp]    (the imaginary part)
 * where table [device, 2g floats] holds cos(2 pi t / g) for t < g, then -sin(2 pi t / g)
 * (the values are the caller's; any 2g floats define a matrix the same way). An entry costs one
 * integer index and one table read; nothing of size m x n is stored. The scale of this
 * operator's quantizations is c = max |table|, which is max |Phi| whenever the table's largest
 * magnitude is reached (table[0] = cos 0 = 1 is, by the centre pixel, for every baseline). */
typedef struct {
    const int32_t* uv;      /* [device] 2K ints: u_0, v_0, u_1, v_1, ... (any integers; taken mod g) */
    const float* table;     /* [device] 2g floats */
    int32_t baselines;      /* K: a multiple of 4, 4 <= K <= 8192 (m = 2K <= 16384 rows) */
    int32_t grid;           /* g: a power of two, 2 <= g <= QIHT_FLY_MAX_GRID */
} qiht_fly_op;

/* Codes of the operator's Phi in the column-packed layout: bit-identical to qiht_quantize (and,
 * with words_b, qiht_quantize_pair) of the materialized m x n matrix with the same bits, seed,
 * streams, flags (0 or QIHT_ODD_LEVELS) and scale. *scale [device] receives max |table|.
 * words_a, words_b [device, n * ld_words words each; words_b NULL for one quantization],
 * ld_words = qiht_ld_words(2K, bits). One kernel launch (after one for the scale);
 * asynchronous on `stream`. Errors: QIHT_ERR_BITS, QIHT_ERR_ARG (operator out of its limits,
 * bad pointers or ld_words). */
qiht_status qiht_fly_quantize(const qiht_fly_op* op, int32_t bits, uint64_t seed, uint32_t stream_a,
                              uint32_t stream_b, int32_t flags, uint32_t* words_a, uint32_t* words_b,
                              int32_t ld_words, float* scale, qiht_stream_t stream);

/* g = Q^T r where Q is the quantization (bits, seed, stream_id, flags) of the operator's Phi,
 * generated, quantized and multiplied inside one kernel and never stored. The result is
 * bit-identical to qiht_gemv_t on the codes qiht_fly_quantize makes (the same exact integer sums
 * and final scaling). r [device, 2K floats], g [device, g^2 floats], scale [device, one float,
 * receives max |table|]. Asynchronous on `stream`. Errors as for qiht_fly_quantize. */
qiht_status qiht_gemv_t_fly(const qiht_fly_op* op, int32_t bits, uint64_t seed, uint32_t stream_id, int32_t flags,
                            const float* r, float* g, float* scale, qiht_stream_t stream);

/* qiht_niht_solve_fresh with Phi given by the operator: each iteration's two realizations of
 * Q(Phi) are drawn from the operator (as qiht_fly_quantize does) instead of from a stored FP32
 * matrix, so the solve holds no copy of Phi; results are identical to qiht_niht_solve_fresh on
 * the materialized matrix. y [device, 2K floats]; the workspace is
 * qiht_solve_fresh_workspace_size(2K, g^2, s, bits_phi, bits_y) bytes; g^2 <= 49152. Other
 * arguments, errors and synchronisation as for qiht_niht_solve_fresh. */
qiht_status qiht_niht_solve_fresh_fly(const qiht_fly_op* op, const float* y, int32_t bits_phi, int32_t bits_y,
                                      uint64_t seed, int32_t quant_flags, int32_t s, int32_t iters,
                                      const qiht_params* params, float* x, int32_t* support, qiht_report* report,
                                      const qiht_trace* trace, void* workspace, size_t workspace_bytes,
                                      qiht_stream_t stream);

/* ---------------------------------------------------------------------- */
/* Separable operator with quantized transform factors (Section IV-B, MRI: */
/* Phi formed by the Fourier and inverse wavelet transforms and the        */
/* sampling operator, the transformation matrices themselves quantized)    */
/* ---------------------------------------------------------------------- */

#define QIHT_SEP_MAX_N 512     /* n = N^2 <= 262144 (above 49152 the threshold is the multi-CTA select) */

/* Phi = S (A (x) A), stacked real: A is the N x N complex 1D transform of the separable 2D
 * transform (for MRI, the orthonormal DFT times the Haar synthesis, A = F_1 H^T), x the N x N
 * coefficient image in row-major order (index j1 N + j2), S the M sampled positions
 * (k1 N + k2). Row k of the complex operator is kron(A[k1], A[k2]); the stacked real matrix has
 * m = 2M rows (real parts, then imaginary parts) and n = N^2 columns. The factor is given as its
 * real and imaginary parts stacked into one 2N x N row-major float matrix [Re A; Im A], which
 * is what is quantized: one scale c = max |[Re A; Im A]|, element (i, j) of the stacked matrix
 * numbered j * 2N + i for the quantizer's random numbers. */
typedef struct {
    const float* factor;    /* [device] 2N x N floats: Re A (rows 0..N-1), then Im A */
    const int32_t* mask;    /* [device] M ints: sampled positions k1 * N + k2, distinct (one off the grid samples 0) */
    int32_t N;              /* 2 <= N <= QIHT_SEP_MAX_N */
    int32_t M;              /* 1 <= M <= N^2 */
} qiht_sep_op;

/* Workspace bytes for qiht_niht_solve_separable (0 if out of range). */
size_t qiht_solve_separable_workspace_size(int32_t N, int32_t M, int32_t s);

/* Algorithm 2 on the separable operator with its factor quantized: Q1 and Q2 are two
 * quantizations of the stacked factor to bits_factor bits (2..16; 2^bits levels, or
 * 2^(bits-1) + 1 with QIHT_ODD_LEVELS in quant_flags), random-number streams 0 and 1 with
 * `seed`; Phi-hat_k = S (A-hat_k (x) A-hat_k). y [device, 2M floats: real parts, then imaginary]
 * is quantized to bits_y bits (2..16) with stream 2. Then, as qiht_niht_solve:
 * g = Phi-hat_1^T (y-hat - Phi-hat_2 x), mu = ||g_G||^2 / ||Phi-hat_2 g_G||^2,
 * x' = H_s(x + mu g), shrink mu by k(1 - c) while mu > (1 - c) ||x'-x||^2 / ||Phi-hat_2 (x'-x)||^2.
 * The operator is applied as dense transforms of the N x N image (FP32 products of the
 * dequantized factors, the sampling as a gather and its adjoint as a scatter), never as an
 * m x n matrix. The host drives the iteration and reads scalars after every product, so the
 * call returns when the solve is done. params: as for qiht_niht_solve (flags must be 0;
 * mu_mode QIHT_MU_FORWARD_SQ only). s <= M, s <= N^2. Outputs and trace as for qiht_niht_solve. */
qiht_status qiht_niht_solve_separable(const qiht_sep_op* op, const float* y, int32_t bits_factor, int32_t bits_y,
                                      uint64_t seed, int32_t quant_flags, int32_t s, int32_t iters,
                                      const qiht_params* params, float* x, int32_t* support, qiht_report* report,
                                      const qiht_trace* trace, void* workspace, size_t workspace_bytes,
                                      qiht_stream_t stream);

/* The building blocks, for tests: the quantized factor (codes [device, 2N x N uint16, may be
 * NULL] and dequantized values [device, 2N x N floats]: scale/(L-1) (2c - (L-1)), rounded once)
 * of one realization, and the products of its operator: forward out = Phi-hat x
 * (x [device, N^2 floats] -> out [device, 2M floats]) and adjoint out = Phi-hat^T r
 * (r [device, 2M] -> out [device, N^2]). Workspace: qiht_solve_separable_workspace_size(N, M, 1).
 * Asynchronous on `stream`. */
qiht_status qiht_sep_quantize_factor(const qiht_sep_op* op, int32_t bits, uint64_t seed, uint32_t stream_id,
                                     int32_t quant_flags, uint16_t* codes, float* factor_hat, float* scale,
                                     qiht_stream_t stream);
qiht_status qiht_sep_apply(const qiht_sep_op* op, const float* factor_hat, int32_t adjoint, const float* in,
                           float* out, void* workspace, size_t workspace_bytes, qiht_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* QIHT_H */
