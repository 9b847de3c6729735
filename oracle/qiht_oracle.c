/*
 * qiht_oracle.c -- slow, plain reference implementation of QIHT.
 *
 * TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline leg of bench.py may load this library. The CUDA library of the
 * package shares no code, header, table or constant generator with it, and
 * neither side calls the other.
 *
 * Method: Gurel et al., "Compressive Sensing Using Iterative Hard Thresholding
 * with Low Precision Data Representation" (IEEE TSP 2020):
 *   - stochastic quantizer Q(v, b)                       Section III-A
 *   - max-abs normalisation c_v before quantizing        Appendix, Lemma (quantization error)
 *   - normalized IHT with adaptive step and backtracking Section II-A, Algorithm 1, Eq. (step_size)
 *   - QIHT: NIHT on two independent quantizations        Section III-A, Algorithm 2
 *
 * Arithmetic: FP64 everywhere except the quantisation decision, which is
 * taken in binary32 because the paper defines Q on single-precision inputs
 * (Section III-A) and the decision must be identical on both sides.
 * Build with -O2 -ffp-contract=off: no fused multiply-add anywhere.
 * With -fopenmp the dense products and the quantiser split their OUTPUTS over
 * threads (columns of A^T r, rows of A[:, list] v, elements of Q(v)); every
 * output is still one sum in the serial order, so results do not depend on the
 * number of threads.
 *
 * Readings of the paper (where it is silent or garbled):
 *   - 2^b equally spaced levels on [-1, 1], spacing 2/(2^b - 1)   (Section III-A)
 *   - the Appendix's remark on fixed-point hardware gives a second grid of
 *     2^(b-1) + 1 levels, spacing 1/2^(b-2), on which 0 is a level; the
 *     quantizer takes the number of levels as an argument and treats both
 *     grids (and any other level count) with the same rule
 *   - scale c = max |v| over the whole matrix / vector; c = 0 -> the
 *     normalised value is taken as 0 (the dequantised value is 0 anyway)
 *   - random numbers: Philox4x32-10 (Salmon et al., SC'11), one stream per
 *     quantisation (the paper used XORShift on CPU; the generator is free)
 *   - Algorithm 2's "x^{[n]}" inside g is x^{[n-1]}; the branches that set
 *     x^{[n]} = x^{[n-1]} are read as "accept the proposal" (Section II-A text)
 *   - the mu denominator, by default, uses the second quantisation only:
 *     ||Q2[:, G] g_G||^2 (a positive number), and omega uses Q2 as well;
 *     mu_mode = 1 takes the denominator Algorithm 2 prints, the cross product
 *     (Q1[:, G] g_G)^T (Q2[:, G] g_G) of the two quantisations, and falls back
 *     to the forward square when that product is not positive
 *   - tol > 0 stops the run after the first iteration whose residual
 *     ||y - Q2 x||^2 is at most tol (the paper stops after a fixed number of
 *     iterations n*, Theorem 4's n* = ceil(log2(||x^s|| / eps_s)); tol is the
 *     same criterion stated on the residual, for when eps_s is not known)
 *   - H_s keeps exactly s indices: order by |a| descending, then index ascending
 *   - if ||g_G||^2 == 0 or ||Q2 g_G||^2 == 0 the solve stops (converged)
 *   - grad_e4m3 = 1 forms the gradient from the residual held as three e4m3 terms
 *     (the 8-bit floating-point gradient for codes of at most 4 bits, which e4m3
 *     holds exactly, Section III-A): r -> 2^e (t1 + t2 + t3), e such that max |r| 2^-e
 *     lies in [2^7, 2^8), each term the e4m3 value nearest to what the earlier terms
 *     leave; A1^T is applied to that vector in FP64. The same holds for y in the
 *     initial gradient A1^T y.
 *
 * QO_MUTANT (default 0) plants one deliberate mistake; it is set only by the
 * mutation tests, which build such variants to show that the pins catch them.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads of the OpenMP split (1 when built without OpenMP). */
void qo_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int qo_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

#define QO_OK 0
#define QO_ERR_ARG 1
#define QO_ERR_BITS 2
#define QO_ERR_NONFINITE 3
#define QO_ERR_BACKTRACK_CAP 5

#ifndef QO_MUTANT
#define QO_MUTANT 0
#endif

/* ------------------------------------------------------------------ */
/* Philox4x32-10: Salmon, Moraes, Dror, Shaw, "Parallel Random Numbers: As   */
/* Easy as 1, 2, 3", SC'11. Multipliers and Weyl key increments as published. */
/* ------------------------------------------------------------------ */
void qo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0 && QO_MUTANT != 7) {  /* key schedule: add the Weyl constants */
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Uniform in [0, 1) for logical element e of one quantisation.
 * Counter (e>>2 low word, e>>2 high word, stream, 0), key (seed low, seed high);
 * element e uses output word e & 3; u = (word >> 8) * 2^-24. */
float qo_uniform(uint64_t seed, uint32_t stream, uint64_t e)
{
    uint64_t q = e >> 2;
    uint32_t ctr[4] = {(uint32_t)q, (uint32_t)(q >> 32), stream, 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t w[4];
    qo_philox4x32_10(ctr, key, w);
    return (float)(w[e & 3u] >> 8) * 0x1p-24f;
}

/* c_v = max_i |v_i| (Appendix, quantization-error lemma). Counts non-finite entries. */
float qo_absmax(const float* v, int64_t count, int64_t* nonfinite)
{
    float c = 0.0f;
    int64_t bad = 0;
    for (int64_t i = 0; i < count; ++i) {
        float a = fabsf(v[i]);
        if (!isfinite(a)) { ++bad; continue; }
        if (a > c) c = a;
    }
    if (nonfinite) *nonfinite = bad;
    return c;
}

/* One quantisation decision, Section III-A.
 * Levels q_k = -1 + 2k/(L-1), k = 0..L-1, for a grid of L levels (L = 2^b in
 * the main text; L = 2^(b-1) + 1 for the odd grid of the Appendix's remark).
 * With t = (v/c + 1)(L-1)/2, v lies between q_i and q_{i+1} for i = floor(t);
 * it is rounded up to q_{i+1} with probability f = t - i (so E[Q(v)] = v) and
 * down to q_i otherwise. */
static int qo_code(float v, float c, int L, float u)
{
    const float half = (QO_MUTANT == 2) ? (float)L * 0.5f : (float)(L - 1) * 0.5f;  /* exact */
    float vt = (c > 0.0f) ? v / c : 0.0f;               /* binary32, round to nearest */
    float t = (vt + 1.0f) * half;
    if (t < 0.0f) t = 0.0f;
    if (t > (float)(L - 1)) t = (float)(L - 1);
    float fi = floorf(t);
    float f = t - fi;                                    /* exact */
    int code = (int)fi + ((QO_MUTANT == 1) ? (u > f ? 1 : 0) : (u < f ? 1 : 0));
    if (code > L - 1) code = L - 1;
    return code;
}

/* Quantise a block of a matrix on a grid of `levels` levels (2 <= levels <=
 * 65536). The block is rows x cols, row-major with row stride ld, and sits at
 * (row0, col0) of a matrix with rows_total rows. The random number of element
 * (i, j) is the one of logical index e = j*rows_total + i (column-major
 * numbering), so the codes depend only on (i, j, seed, stream).
 * codes: rows x cols, row-major. A vector is a matrix with one column. */
int qo_quantize(const float* v, int64_t rows, int64_t cols, int64_t ld,
                int64_t row0, int64_t col0, int64_t rows_total,
                int levels, uint64_t seed, uint32_t stream, float scale, uint16_t* codes)
{
    if (levels < 2 || levels > 65536) return QO_ERR_BITS;
    if (!(scale >= 0.0f) || !isfinite(scale)) return QO_ERR_NONFINITE;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < rows; ++i) {
        for (int64_t j = 0; j < cols; ++j) {
            uint64_t e = (uint64_t)(col0 + j) * (uint64_t)rows_total + (uint64_t)(row0 + i);
            float u = qo_uniform(seed, stream, e);
            codes[i * cols + j] = (uint16_t)qo_code(v[i * ld + j], scale, levels, u);
        }
    }
    return QO_OK;
}

/* Dequantised value c * q_code = (c / (L-1)) * (2 code - (L-1)), in FP64. */
void qo_dequantize(const uint16_t* codes, int64_t count, int levels, float scale, double* out)
{
    const double lm1 = (double)(levels - 1);
    const double alpha = (double)scale / lm1;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < count; ++i)
        out[i] = alpha * (2.0 * (double)codes[i] - ((QO_MUTANT == 9) ? lm1 + 1.0 : lm1));
}

/* ------------------------------------------------------------------ */
/* Dense products (A row-major m x n, FP64). Each output is one sum in     */
/* ascending index order; loops are arranged so A is read row by row.     */
/* ------------------------------------------------------------------ */

/* g = A^T r. Each thread owns a range of columns and walks all rows, so g[j] is summed
 * over i in ascending order whatever the number of threads. */
void qo_gemv_t(const double* A, const double* r, int64_t m, int64_t n, double* g)
{
#pragma omp parallel
    {
        int64_t j0 = 0, j1 = n;
#ifdef _OPENMP
        const int64_t nt = omp_get_num_threads(), id = omp_get_thread_num();
        j0 = n * id / nt;
        j1 = n * (id + 1) / nt;
#endif
        for (int64_t j = j0; j < j1; ++j) g[j] = 0.0;
        for (int64_t i = 0; i < m; ++i) {
            const double* row = A + i * n;
            const double ri = r[i];
            for (int64_t j = j0; j < j1; ++j) g[j] += row[j] * ri;
        }
    }
}

/* z = A[:, idx] v over a list of columns (in list order) */
void qo_gemv_cols(const double* A, int64_t m, int64_t n, const int32_t* idx, const double* v,
                  int64_t k, double* z)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        const double* row = A + i * n;
        double acc = 0.0;
        for (int64_t t = 0; t < k; ++t) acc += row[idx[t]] * v[t];
        z[i] = acc;
    }
}

/* ------------------------------------------------------------------ */
/* Hard threshold H_s (Eq. NIHT): keep the s entries of largest magnitude.  */
/* Order: |a| descending, ties by index ascending; exactly s are kept.      */
/* ------------------------------------------------------------------ */
typedef struct { double key; int32_t idx; } qo_kv;

static int qo_kv_cmp(const void* pa, const void* pb)
{
    const qo_kv* a = (const qo_kv*)pa;
    const qo_kv* b = (const qo_kv*)pb;
    if (QO_MUTANT == 5) { if (a->key < b->key) return -1; if (a->key > b->key) return 1; }
    else { if (a->key > b->key) return -1; if (a->key < b->key) return 1; }
    return (a->idx < b->idx) ? -1 : (a->idx > b->idx);
}

static int qo_int_cmp(const void* pa, const void* pb)
{
    int32_t a = *(const int32_t*)pa, b = *(const int32_t*)pb;
    return (a > b) - (a < b);
}

/* sel: s indices sorted ascending; kth[0] = s-th largest |a|, kth[1] = (s+1)-th (0 if s == n).
 * work: n entries of scratch. */
void qo_hard_threshold(const double* a, int32_t n, int32_t s, int32_t* sel, double kth[2], qo_kv* work)
{
    for (int32_t j = 0; j < n; ++j) { work[j].key = fabs(a[j]); work[j].idx = j; }
    qsort(work, (size_t)n, sizeof(qo_kv), qo_kv_cmp);
    for (int32_t t = 0; t < s; ++t) sel[t] = work[t].idx;
    qsort(sel, (size_t)s, sizeof(int32_t), qo_int_cmp);
    kth[0] = (s > 0) ? work[s - 1].key : 0.0;
    kth[1] = (s < n) ? work[s].key : 0.0;
}

/* exported for tests: H_s on a vector */
void qo_top_s(const double* a, int32_t n, int32_t s, int32_t* sel, double* kth)
{
    qo_kv* work = (qo_kv*)malloc(sizeof(qo_kv) * (size_t)(n > 0 ? n : 1));
    qo_hard_threshold(a, n, s, sel, kth, work);
    free(work);
}

/* ------------------------------------------------------------------ */
/* QIHT / NIHT (Algorithm 2; Algorithm 1 when A1 = A2 = Phi).               */
/* ------------------------------------------------------------------ */
typedef struct {
    double k;              /* shrinkage, k > 1/(1-c) (Section II-A) */
    double c;              /* small constant in (0, 1) */
    int32_t max_backtrack; /* cap on mu shrinks per iteration */
    int32_t mu_mode;       /* 0: ||A2_G g_G||^2; 1: Algorithm 2's cross product, forward square if <= 0 */
    double tol;            /* > 0: stop after the first iteration with ||y - A2 x||^2 <= tol */
    int32_t grad_e4m3;     /* 1: the gradient's residual as three e4m3 terms (qo_e4m3_terms) */
    int32_t reserved;
} qo_params;

/* Nearest value of the 8-bit floating-point format E4M3 (OCP 8-bit floating point
 * specification: sign, 4 exponent bits with bias 7, 3 fraction bits, subnormals with
 * spacing 2^-9, largest finite value 448), ties to the even fraction, magnitudes past 448
 * saturated to 448. The quantum of a value with leading bit 2^E (E >= -6) is 2^(E-3). */
double qo_e4m3(double v)
{
    if (v == 0.0 || v != v) return v;
    const double a = fabs(v);
    int e;
    frexp(a, &e);                    /* a = f 2^e, f in [0.5, 1): leading bit 2^(e-1) */
    int E = e - 1;
    if (E < -6) E = -6;              /* subnormal range: one quantum 2^-9 */
    const double q = ldexp(1.0, E - 3);
    double rnd = nearbyint(a / q) * q; /* a / q is exact; nearbyint rounds ties to even */
    if (rnd > 448.0) rnd = 448.0;
    return copysign(rnd, v);
}

/* r (m values) -> out = 2^e (t_1 + ... + t_terms): e puts max |r| 2^-e in [2^7, 2^8)
 * (0 when r is all zero or not finite), t_k = qo_e4m3 of r 2^-e - (t_1 + ... + t_{k-1}). */
void qo_e4m3_terms(const double* r, int64_t m, int terms, double* out)
{
    double mx = 0.0;
    for (int64_t i = 0; i < m; ++i) if (fabs(r[i]) > mx) mx = fabs(r[i]);
    int e = 0;
    if (mx > 0.0 && isfinite(mx)) {
        int ex;
        frexp(mx, &ex);
        e = ex - ((QO_MUTANT == 13) ? 7 : 8);
    }
    const int nt = (QO_MUTANT == 12) ? terms - 1 : terms;
    for (int64_t i = 0; i < m; ++i) {
        double v = ldexp(r[i], -e), acc = 0.0;
        for (int k = 0; k < nt; ++k) {
            const double t = qo_e4m3(v);
            acc += t;
            v -= t;
        }
        out[i] = ldexp(acc, e);
    }
}

/* Step size on support G (Eq. step_size; Algorithm 2): num = ||g_G||^2 and
 *   mu_mode 0: den = ||A2[:, G] g_G||^2
 *   mu_mode 1: den = (A1[:, G] g_G)^T (A2[:, G] g_G), the product of the two realizations
 *              Algorithm 2 prints; when it is not positive, den = ||A2[:, G] g_G||^2.
 * out[0] = num, out[1] = den used, out[2] = the cross product (mode 1; else 0),
 * out[3] = 1 when mode 1 fell back to the forward square. z1, z2: m doubles of scratch;
 * coef: s doubles of scratch. */
void qo_step_size(const double* A1, const double* A2, int32_t m, int32_t n, const int32_t* sup,
                  const double* g, int32_t s, int32_t mu_mode, double* out, double* coef, double* z1, double* z2)
{
    double num = 0.0;
    for (int32_t q = 0; q < s; ++q) {
        const double gq = g[sup[q]];
        num += (QO_MUTANT == 4) ? fabs(gq) : gq * gq;
        coef[q] = gq;
    }
    qo_gemv_cols(A2, m, n, sup, coef, s, z2);
    double fwd = 0.0;
    for (int32_t i = 0; i < m; ++i) fwd += z2[i] * z2[i];
    double cross = 0.0, den = fwd, fell = 0.0;
    if (mu_mode == 1) {
        qo_gemv_cols((QO_MUTANT == 10) ? A2 : A1, m, n, sup, coef, s, z1);
        for (int32_t i = 0; i < m; ++i) cross += z1[i] * z2[i];
        if (cross > 0.0) den = cross;
        else fell = 1.0;
    }
    out[0] = num;
    out[1] = den;
    out[2] = cross;
    out[3] = fell;
}

typedef struct {           /* all optional (NULL); arrays have iters + 1 rows */
    int32_t* support;      /* (iters+1) x s: row 0 = initial support, row t = after iteration t */
    double* kth;           /* (iters+1) x 2: s-th and (s+1)-th |a| of the accepted selection */
    double* min_gap;       /* (iters+1): min relative gap (kth0-kth1)/kth0 over this iteration's selections */
    double* mu;            /* (iters+1): accepted step size (row 0: 0) */
    int32_t* bt;           /* (iters+1): number of shrinks */
    double* min_margin;    /* (iters+1): min |mu - (1-c) omega| / mu over omega tests (INFINITY if none) */
    double* resid2;        /* (iters+1): ||y - A2 x||^2 after the iteration */
    double* x;             /* (iters+1) x n: iterate after each iteration (row 0 = 0) */
    int32_t* mu_fallback;  /* (iters+1): 1 when mu_mode 1 fell back to the forward square */
    double* num;           /* (iters+1): ||g_G||^2 of the iteration's step size (row 0: 0) */
    double* xnorm2;        /* (iters+1): ||x||^2 after the iteration */
} qo_trace;

typedef struct {
    int32_t iters_run;
    int32_t backtracks;
    int32_t support_changes;
    int32_t status;
    double resid_norm2;
    double mu;
} qo_report;

static double qo_rel_gap(const double kth[2])
{
    return kth[0] > 0.0 ? (kth[0] - kth[1]) / kth[0] : 0.0;
}

static int qo_same_set(const int32_t* a, const int32_t* b, int32_t s)
{
    for (int32_t t = 0; t < s; ++t) if (a[t] != b[t]) return 0;
    return 1;
}

static double qo_resid2(const double* A2, const double* y, int32_t m, int32_t n,
                        const int32_t* sup, const double* x, int32_t s, double* xs, double* z)
{
    for (int32_t t = 0; t < s; ++t) xs[t] = x[sup[t]];
    qo_gemv_cols(A2, m, n, sup, xs, s, z);
    double acc = 0.0;
    for (int32_t i = 0; i < m; ++i) { double r = y[i] - z[i]; acc += r * r; }
    return acc;
}

/* Algorithm 2 with one realization of the matrices and observation per iteration:
 * A1s[t], A2s[t], ys[t] (t = 1..iters) are the matrices of iteration t (Phi-hat_{2t-1} for the
 * gradient, Phi-hat_{2t} for A2 x, the step size and the backtracking test) and its
 * observation y-hat_t; A1s[0], ys[0] give the initial support. Each A is m x n row-major.
 * x: n (output, s-sparse). support: s (output, ascending). The residual recorded after
 * iteration t is ||ys[t] - A2s[t] x||^2. Returns a status code; rep is filled in any case. */
int qo_niht_seq(const double* const* A1s, const double* const* A2s, const double* const* ys, int32_t m,
                int32_t n, int32_t s, int32_t iters, const qo_params* p, double* x, int32_t* support,
                qo_trace* tr, qo_report* rep)
{
    const double* A1 = A1s[0];
    const double* A2 = A2s[0];
    const double* y = ys[0];
    memset(rep, 0, sizeof(*rep));
    if (m <= 0 || n <= 0 || s <= 0 || s > n || s > m || iters < 0) {
        rep->status = QO_ERR_ARG;
        return QO_ERR_ARG;
    }
    const double shrink = p->k * (1.0 - p->c);
    double* g = (double*)malloc(sizeof(double) * (size_t)n);
    double* a = (double*)malloc(sizeof(double) * (size_t)n);
    double* r = (double*)malloc(sizeof(double) * (size_t)m);
    double* z = (double*)malloc(sizeof(double) * (size_t)m);
    double* z1 = (double*)malloc(sizeof(double) * (size_t)m);
    double* xn = (double*)malloc(sizeof(double) * (size_t)n);
    double* coef = (double*)malloc(sizeof(double) * (size_t)(2 * s));
    int32_t* uni = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * s));
    int32_t* sel = (int32_t*)malloc(sizeof(int32_t) * (size_t)s);
    qo_kv* work = (qo_kv*)malloc(sizeof(qo_kv) * (size_t)n);
    int status = QO_OK;

    /* Initialisation (Algorithm 2): x = 0, support of H_s(A1^T y). */
    for (int32_t j = 0; j < n; ++j) x[j] = 0.0;
    if (p->grad_e4m3) {
        qo_e4m3_terms(y, m, 3, r);
        qo_gemv_t(A1, r, m, n, g);
    } else {
        qo_gemv_t(A1, y, m, n, g);
    }
    double kth[2];
    qo_hard_threshold(g, n, s, support, kth, work);
    if (tr) {
        if (tr->support) memcpy(tr->support, support, sizeof(int32_t) * (size_t)s);
        if (tr->kth) { tr->kth[0] = kth[0]; tr->kth[1] = kth[1]; }
        if (tr->min_gap) tr->min_gap[0] = qo_rel_gap(kth);
        if (tr->mu) tr->mu[0] = 0.0;
        if (tr->bt) tr->bt[0] = 0;
        if (tr->min_margin) tr->min_margin[0] = INFINITY;
        if (tr->resid2) { double acc = 0.0; for (int32_t i = 0; i < m; ++i) acc += y[i] * y[i]; tr->resid2[0] = acc; }
        if (tr->x) memcpy(tr->x, x, sizeof(double) * (size_t)n);
        if (tr->mu_fallback) tr->mu_fallback[0] = 0;
        if (tr->num) tr->num[0] = 0.0;
        if (tr->xnorm2) tr->xnorm2[0] = 0.0;
    }

    int32_t t;
    int tol_stop = 0;
    for (t = 1; t <= iters; ++t) {
        A1 = A1s[t];
        A2 = A2s[t];
        y = ys[t];
        /* g = A1^T (y - A2 x) */
        for (int32_t q = 0; q < s; ++q) coef[q] = x[support[q]];
        qo_gemv_cols(A2, m, n, support, coef, s, z);
        for (int32_t i = 0; i < m; ++i) r[i] = (QO_MUTANT == 8) ? z[i] - y[i] : y[i] - z[i];
        if (p->grad_e4m3) {
            qo_e4m3_terms(r, m, 3, z1);
            memcpy(r, z1, sizeof(double) * (size_t)m);
        }
        qo_gemv_t((QO_MUTANT == 3) ? A2 : A1, r, m, n, g);

        /* step size (Eq. step_size on the current support) */
        double ss[4];
        qo_step_size(A1, A2, m, n, support, g, s, p->mu_mode, ss, coef, z1, z);
        const double num = ss[0], den = ss[1];
        if (num == 0.0 || den == 0.0) break;               /* converged: x unchanged */
        double mu = num / den;

        /* proposal x' = H_s(x + mu g) */
#pragma omp parallel for schedule(static)
        for (int32_t j = 0; j < n; ++j) a[j] = x[j] + mu * g[j];
        qo_hard_threshold(a, n, s, sel, kth, work);
        double min_gap = qo_rel_gap(kth);
        double min_margin = INFINITY;
        int32_t nbt = 0;
        int changed = !qo_same_set(sel, support, s);

        if (changed) {
            for (;;) {
                /* x' on its support; Delta = x' - x over the union of supports */
                for (int32_t j = 0; j < n; ++j) xn[j] = 0.0;
                for (int32_t q = 0; q < s; ++q) xn[sel[q]] = a[sel[q]];
                int32_t nu = 0;
                for (int32_t q = 0; q < s; ++q) uni[nu++] = sel[q];
                for (int32_t q = 0; q < s; ++q) {
                    int32_t j = support[q];
                    int in_new = 0;
                    for (int32_t w = 0; w < s; ++w) if (sel[w] == j) { in_new = 1; break; }
                    if (!in_new) uni[nu++] = j;
                }
                double dn = 0.0;
                for (int32_t q = 0; q < nu; ++q) { coef[q] = xn[uni[q]] - x[uni[q]]; dn += coef[q] * coef[q]; }
                if (dn == 0.0) break;                        /* nothing moves: accept */
                qo_gemv_cols(A2, m, n, uni, coef, nu, z);
                double dd = 0.0;
                for (int32_t i = 0; i < m; ++i) dd += z[i] * z[i];
                double omega = (dd > 0.0) ? dn / dd : INFINITY;
                double bound = (1.0 - p->c) * omega;
                double margin = fabs(mu - bound) / mu;
                if (margin < min_margin) min_margin = margin;
                if ((QO_MUTANT == 6) ? (mu > bound) : (mu <= bound)) break;  /* sufficient decrease holds */
                if (nbt >= p->max_backtrack) { status = QO_ERR_BACKTRACK_CAP; break; }
                mu = mu / shrink;
                ++nbt;
                for (int32_t j = 0; j < n; ++j) a[j] = x[j] + mu * g[j];
                qo_hard_threshold(a, n, s, sel, kth, work);
                double gp = qo_rel_gap(kth);
                if (gp < min_gap) min_gap = gp;
                if (qo_same_set(sel, support, s)) break;
            }
        }
        if (status != QO_OK) break;

        /* accept x' */
        if (!qo_same_set(sel, support, s)) rep->support_changes++;
        for (int32_t q = 0; q < s; ++q) x[support[q]] = 0.0;
        for (int32_t q = 0; q < s; ++q) x[sel[q]] = a[sel[q]];
        memcpy(support, sel, sizeof(int32_t) * (size_t)s);
        rep->backtracks += nbt;
        rep->mu = mu;
        if (tr) {
            if (tr->support) memcpy(tr->support + (size_t)t * s, support, sizeof(int32_t) * (size_t)s);
            if (tr->kth) { tr->kth[2 * t] = kth[0]; tr->kth[2 * t + 1] = kth[1]; }
            if (tr->min_gap) tr->min_gap[t] = min_gap;
            if (tr->mu) tr->mu[t] = mu;
            if (tr->bt) tr->bt[t] = nbt;
            if (tr->min_margin) tr->min_margin[t] = min_margin;
            if (tr->resid2) tr->resid2[t] = qo_resid2(A2, y, m, n, support, x, s, coef, z);
            if (tr->x) memcpy(tr->x + (size_t)t * n, x, sizeof(double) * (size_t)n);
            if (tr->mu_fallback) tr->mu_fallback[t] = (int32_t)ss[3];
            if (tr->num) tr->num[t] = num;
            if (tr->xnorm2) {
                double acc = 0.0;
                for (int32_t q = 0; q < s; ++q) acc += x[support[q]] * x[support[q]];
                tr->xnorm2[t] = acc;
            }
        }
        if (p->tol > 0.0 && ((QO_MUTANT == 11) ? qo_resid2(A2, y, m, n, support, x, s, coef, z) >= p->tol
                                               : qo_resid2(A2, y, m, n, support, x, s, coef, z) <= p->tol)) {
            tol_stop = 1;                                  /* residual reached tol: stop */
            break;
        }
    }
    rep->iters_run = tol_stop ? t : ((t > iters) ? iters : t - 1);
    rep->status = status;
    rep->resid_norm2 = qo_resid2(A2, y, m, n, support, x, s, coef, z);

    free(g); free(a); free(r); free(z); free(z1); free(xn); free(coef); free(uni); free(sel); free(work);
    return status;
}

/* A1, A2: m x n row-major (the two dequantised matrices, or Phi twice), the same in every
 * iteration; y: m. Arguments and results as for qo_niht_seq. */
int qo_niht(const double* A1, const double* A2, const double* y, int32_t m, int32_t n, int32_t s,
            int32_t iters, const qo_params* p, double* x, int32_t* support, qo_trace* tr,
            qo_report* rep)
{
    const int32_t cnt = (iters > 0 ? iters : 0) + 1;
    const double** a1 = (const double**)malloc(sizeof(double*) * (size_t)cnt);
    const double** a2 = (const double**)malloc(sizeof(double*) * (size_t)cnt);
    const double** yy = (const double**)malloc(sizeof(double*) * (size_t)cnt);
    for (int32_t t = 0; t < cnt; ++t) { a1[t] = A1; a2[t] = A2; yy[t] = y; }
    const int st = qo_niht_seq(a1, a2, yy, m, n, s, iters, p, x, support, tr, rep);
    free(a1); free(a2); free(yy);
    return st;
}
