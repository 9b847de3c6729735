// One QIHT iteration after the gradient product (Algorithm 2), as one persistent
// kernel: step size, threshold with backtracking, residual and commit.
//
// One CTA per SM (all resident at once: cooperative launch). CTA c owns a block of
// code words of every column, i.e. a block of rows, so the products with a column
// subset, z = Q2[:, list] coef, are complete for its rows without any cross-CTA
// sum; only scalars (||z||^2, ||r||^2, max|r|) are combined, in a fixed order.
// Phases, separated by grid barriers:
//   Mu      z = Q2_G g_G; mu = ||g_G||^2 / ||z||^2                        (Eq. step_size)
//   Filter  keys |x + mu g|; candidates >= tau for the threshold
//   Select  CTA 0: H_s on the candidates (or on all keys), G', x', x' - x list
//   Omega   if G' != G: omega = ||x'-x||^2 / ||Q2 (x'-x)||^2; while mu > (1-c) omega,
//           shrink mu by k(1-c) and go back to Filter                     (Section II-A)
//   Resid   r = Q(y) - Q2_G' x'; ||r||^2, max|r|; the last CTA commits x <- x', G <- G'
// Every grid barrier is an arrive counter plus a generation word; waiting is
// bounded by %globaltimer and a timeout sets QIHT_ERR_TIMEOUT instead of hanging.
#include <cmath>
#include <cstdlib>

#include "internal.cuh"

namespace qiht {

constexpr int kIterThreads = 512;
// bytes of the next gradient pass's codes each CTA brings into L2, in one bulk request from one
// thread (about 97 MB over the grid). Measured per iteration at 8192 x 32768, 8 bits: no prefetch
// 55.1 us; 192 KB 52.6; 384 KB 52.2; 640 KB 52.1; 768 KB 52.1. The same bytes as 384-byte
// requests from every thread cost ~1.2 us to issue (53.6 us). At 4 bits 50.6 -> 50.4 us, at 2 bits
// 72.6 -> 72.0 us.
constexpr unsigned kIterPrefetchCta = 640u * 1024u;
constexpr int kListChunk = 1024;                          // list entries staged in shared memory at once
constexpr unsigned long long kBarrierBudgetNs = 200ull * 1000 * 1000;

__device__ __forceinline__ unsigned long long gtimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned long long ld_acquire64(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// A bounded wait ran out: stop the solve and say so in the state and the report.
__device__ __forceinline__ void report_timeout(State* st, qiht_report* rep)
{
    st->status = QIHT_ERR_TIMEOUT;
    st->stop = 1;
    if (rep) rep->status = QIHT_ERR_TIMEOUT;
}

// Grid barrier on one 64-bit arrival counter that only grows: thread 0 of every CTA
// adds 1 with release semantics and waits (acquire) until the counter reaches the
// barrier's target, a multiple of the grid size. Only thread 0 of a CTA holds the
// target. Waiting is bounded by %globaltimer; a timeout marks the state and returns false.
__device__ bool grid_sync(unsigned long long* cnt, unsigned long long& target, State* st, qiht_report* rep)
{
    __shared__ int ok_sh;
    __syncthreads();
    if (threadIdx.x == 0) {
        target += gridDim.x;
        __threadfence();
        asm volatile("red.release.gpu.global.add.u64 [%0], 1;" ::"l"(cnt) : "memory");
        int ok = 1;
        if ((long long)(ld_acquire64(cnt) - target) < 0) {
            const unsigned long long t0 = gtimer_ns();
            while ((long long)(ld_acquire64(cnt) - target) < 0) {
                if (gtimer_ns() - t0 > kBarrierBudgetNs) { ok = 0; break; }
            }
        }
        if (!ok) report_timeout(st, rep);
        ok_sh = ok;
    }
    __syncthreads();
    return ok_sh != 0;
}

// Barrier target of the launch's first barrier: the counter is a multiple of the grid
// size between launches, and no CTA can complete the first barrier before this one arrives.
__device__ __forceinline__ unsigned long long barrier_base(const unsigned long long* cnt)
{
    unsigned long long c;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(c) : "l"(cnt) : "memory");
    return c - c % gridDim.x;
}

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Deterministic sum of one double per thread over threads [0, nact) (the others are not
// read); fixed shuffle trees, and only the warps that hold values do FP64 work (FP64
// throughput is low on this GPU). Every thread gets the result.
__device__ double cta_sum_n(double v, int nact, double* sh)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nw = min((nact + 31) >> 5, (int)(blockDim.x >> 5));
    if (w < nw) {
        if ((int)threadIdx.x >= nact) v = 0.0;
        v = warp_sum_d(v);
        if (lane == 0) sh[w] = v;
    }
    __syncthreads();
    if (w == 0) {
        double t = lane < nw ? sh[lane] : 0.0;
        t = warp_sum_d(t);
        if (lane == 0) sh[32] = t;
    }
    __syncthreads();
    const double r = sh[32];
    __syncthreads();
    return r;
}

__device__ double cta_sum(double v, double* sh) { return cta_sum_n(v, blockDim.x, sh); }

__device__ unsigned cta_max(unsigned v, unsigned* sh)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    v = __reduce_max_sync(0xffffffffu, v);
    if (lane == 0) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        unsigned t = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0u;
        t = __reduce_max_sync(0xffffffffu, t);
        if (lane == 0) sh[32] = t;
    }
    __syncthreads();
    const unsigned r = sh[32];
    __syncthreads();
    return r;
}

// Sum over CTAs of partial slot `k` (warp 0 loads them, eight per lane in flight, and
// adds them in a fixed order); every thread gets the same value.
__device__ double grid_partial_sum(const double* part, int k, double* sh)
{
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < 32) {
        double v = 0.0;
        for (int c0 = lane; c0 < (int)gridDim.x; c0 += 32 * 8) {
            double t[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int c = c0 + 32 * u;
                t[u] = c < (int)gridDim.x ? __ldcg(part + k * kSlotCtas + c) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) v += t[u];
        }
        v = warp_sum_d(v);
        if (lane == 0) sh[32] = v;
    }
    __syncthreads();
    const double r = sh[32];
    __syncthreads();
    return r;
}

// Sum of slot ks and maximum of slot km over CTAs in one pass (warp 0).
__device__ void grid_partial_sum_max(const double* part, int ks, int km, double* sh, double* sum, double* mx)
{
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < 32) {
        double v = 0.0, w = 0.0;
        for (int c0 = lane; c0 < (int)gridDim.x; c0 += 32 * 4) {
            double t[4], u[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int c = c0 + 32 * i;
                t[i] = c < (int)gridDim.x ? __ldcg(part + ks * kSlotCtas + c) : 0.0;
                u[i] = c < (int)gridDim.x ? __ldcg(part + km * kSlotCtas + c) : 0.0;
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) { v += t[i]; w = fmax(w, u[i]); }
        }
        v = warp_sum_d(v);
#pragma unroll
        for (int o = 16; o; o >>= 1) w = fmax(w, __shfl_xor_sync(0xffffffffu, w, o));
        if (lane == 0) { sh[30] = v; sh[31] = w; }
    }
    __syncthreads();
    *sum = sh[30];
    *mx = sh[31];
    __syncthreads();
}

__device__ double grid_partial_max(const double* part, int k, double* sh)
{
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < 32) {
        double v = 0.0;
        for (int c0 = lane; c0 < (int)gridDim.x; c0 += 32 * 8) {
            double t[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int c = c0 + 32 * u;
                t[u] = c < (int)gridDim.x ? __ldcg(part + k * kSlotCtas + c) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) v = fmax(v, t[u]);
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0) sh[32] = v;
    }
    __syncthreads();
    const double r = sh[32];
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------------------
// Tagged exchange slots. A per-CTA partial that is a sum of squares (>= 0, or NaN)
// travels in one 64-bit word whose sign bit holds a tag: the parity of how often
// that slot has been written. A reader knows the tag it waits for, so the word
// itself says whether it is fresh, and no barrier or flag has to be read first.
// The slot schedule rewrites a slot only after every CTA has read its previous
// value, so one tag bit tells the current write from the previous one. Slots start
// with tag 1 (set by the solver's set-up kernel); their first writes carry tag 0.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void slot_put(double* p, double v, unsigned tag)
{
    const unsigned long long b = ((unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull) |
                                 ((unsigned long long)(tag & 1u) << 63);
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(b) : "memory");
}

__device__ __forceinline__ unsigned long long slot_ld(const double* p)
{
    unsigned long long b;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(b) : "l"(p) : "memory");
    return b;
}

// Warp 0 waits until slot ks (and km, when >= 0) of every CTA, and slot ke of CTA 0
// (when >= 0), carry `tag`; then the sum over CTAs of slot ks (lane l adds CTAs l,
// l + 32, ... in order, then a fixed shuffle tree), the maximum of slot km and CTA 0's
// slot ke go to every thread. Each polling round re-reads all stale words of a lane at
// once. Waiting is bounded by %globaltimer; false on timeout.

__device__ bool slot_gather(const double* part, int ks, int km, int ke, unsigned tag, double* sum, double* mx,
                            double* ext, State* st, qiht_report* rep, double* sh)
{
    __shared__ int ok_sh;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < 32) {
        constexpr unsigned long long M = 0x7fffffffffffffffull;
        const unsigned long long want = (unsigned long long)(tag & 1u) << 63;
        const int grid = (int)gridDim.x;
        unsigned long long bs[kSlotPerLane], bm[kSlotPerLane], be = want;
        unsigned pend = 0;                       // bit u: sum word u stale; bit 8 + u: max word u; bit 16: extra
#pragma unroll
        for (int u = 0; u < kSlotPerLane; ++u) {
            bs[u] = want;
            bm[u] = want;
            const int c = lane + 32 * u;
            if (c < grid) {
                pend |= 1u << u;
                if (km >= 0) pend |= 1u << (8 + u);
            }
        }
        if (ke >= 0 && lane == 0) pend |= 1u << 16;
        const unsigned long long t0 = gtimer_ns();
        int ok = 1;
        while (pend) {
#pragma unroll
            for (int u = 0; u < kSlotPerLane; ++u) {
                const int c = lane + 32 * u;
                if (pend & (1u << u)) bs[u] = slot_ld(part + ks * kSlotCtas + c);
                if (pend & (1u << (8 + u))) bm[u] = slot_ld(part + km * kSlotCtas + c);
            }
            if (pend & (1u << 16)) be = slot_ld(part + ke * kSlotCtas);
#pragma unroll
            for (int u = 0; u < kSlotPerLane; ++u) {
                if ((bs[u] & ~M) == want) pend &= ~(1u << u);
                if ((bm[u] & ~M) == want) pend &= ~(1u << (8 + u));
            }
            if ((be & ~M) == want) pend &= ~(1u << 16);
            if (pend && gtimer_ns() - t0 > kBarrierBudgetNs) { ok = 0; break; }
        }
        double v = 0.0, w = 0.0;
#pragma unroll
        for (int u = 0; u < kSlotPerLane; ++u) {
            v += __longlong_as_double((long long)(bs[u] & M));
            w = fmax(w, __longlong_as_double((long long)(bm[u] & M)));
        }
        const double e = __longlong_as_double((long long)(be & M));
        ok = __all_sync(0xffffffffu, ok);
        v = warp_sum_d(v);
#pragma unroll
        for (int o = 16; o; o >>= 1) w = fmax(w, __shfl_xor_sync(0xffffffffu, w, o));
        if (lane == 0) {
            sh[29] = v;
            sh[30] = w;
            sh[31] = e;
            ok_sh = ok;
            if (!ok) report_timeout(st, rep);
        }
    }
    __syncthreads();
    *sum = sh[29];
    if (mx) *mx = sh[30];
    if (ext) *ext = sh[31];
    const int ok = ok_sh;
    __syncthreads();
    return ok != 0;
}

// Decision word: CTA 0 publishes, after gathering the partials of an exchange, what
// every CTA needs from it (a code and the float step size) in one tagged 64-bit word:
// bit 63 tag, bits 32-33 code, bits 0-31 the float. The word is rewritten only after
// every CTA has read it (each CTA reads it before writing its next partial, and CTA 0
// gathers all of those before writing again); tags alternate with every use.
__device__ __forceinline__ void dec_put(unsigned long long* p, unsigned tag, unsigned code, float v)
{
    const unsigned long long w =
        ((unsigned long long)(tag & 1u) << 63) | ((unsigned long long)(code & 3u) << 32) | __float_as_uint(v);
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(w) : "memory");
}

// Thread 0 polls the decision word until it carries `tag`; every thread gets code and value.
__device__ bool dec_wait(const unsigned long long* p, unsigned tag, unsigned* code, float* v, State* st,
                         qiht_report* rep)
{
    __shared__ unsigned long long sw;
    __shared__ int ok_sh;
    if (threadIdx.x == 0) {
        const unsigned long long want = (unsigned long long)(tag & 1u);
        unsigned long long w;
        asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(w) : "l"(p) : "memory");
        int ok = 1;
        if ((w >> 63) != want) {
            const unsigned long long t0 = gtimer_ns();
            do {
                if (gtimer_ns() - t0 > kBarrierBudgetNs) { ok = 0; break; }
                asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(w) : "l"(p) : "memory");
            } while ((w >> 63) != want);
        }
        if (!ok) report_timeout(st, rep);
        sw = w;
        ok_sh = ok;
    }
    __syncthreads();
    const unsigned long long w = sw;
    const int ok = ok_sh;
    __syncthreads();
    *code = (unsigned)(w >> 32) & 3u;
    *v = __uint_as_float((uint32_t)w);
    return ok != 0;
}

struct IterArgs {
    Codes Q;                    // second quantization Q2
    State* st;
    const float* g;
    float* x;                   // dense iterate
    int32_t* support;           // current support G (ascending), committed at the end
    int32_t* sel;               // proposal G'
    float* val;                 // x' on G'
    int32_t* uni;               // G' u G
    float* delta;               // x' - x on G' u G
    const float* yhat;
    float* r;
    uint32_t* keys;             // |x + mu g| of every entry (fallback select)
    unsigned long long* cand;   // filter candidates
    int cap;
    double* part;               // [kPartSlots][kSlotCtas] per-CTA partials (CTA index fastest)
    unsigned* bar;              // [2] commit counter
    unsigned long long* gbar;   // grid-barrier arrival counter
    float* cand_val;            // x + mu g of each candidate (same slot as cand)
    float* cand_x;              // x of each candidate
    // fast-path iteration kernel (k_iter_fast)
    int32_t* pos;               // position of every entry in the support G, -1 outside
    float* xs;                  // x on G, in support order
    const float* gsup;          // g on G, by position (written by the gradient kernel)
    const unsigned long long* gcand;   // gradient-kernel candidates: (g bits << 32) | index
    int gcap;                   // capacity of gcand
    int n, m, s;
    double k, c;
    int max_bt;
    int flags;                  // QIHT_SOLVE_* (the test hook QIHT_SOLVE_TEST_TIMEOUT)
    qiht_report* report;
    qiht_trace trace;
    const uint32_t* q1_words;   // first quantization Q1 (same layout as Q): QIHT_MU_CROSS step size
    int mu_mode;                // QIHT_MU_FORWARD_SQ or QIHT_MU_CROSS
    double tol;                 // general kernel: stop once ||r||^2 <= tol (0: off)
};

// Rows owned by this CTA: code words [w0, w1) of every column.
struct RowBlock {
    int w0, w1, wpc, nsl;       // words, words per CTA (max), column slices
};

__device__ __forceinline__ RowBlock row_block(int ld)
{
    RowBlock b;
    b.wpc = (ld + gridDim.x - 1) / gridDim.x;
    b.w0 = min(ld, (int)blockIdx.x * b.wpc);
    b.w1 = min(ld, b.w0 + b.wpc);
    b.nsl = kIterThreads / b.wpc;
    if (b.nsl < 1) b.nsl = 1;
    return b;
}

// z (for this CTA's rows) += sum over a list in shared memory of coef_j * code column j:
// slice sl takes entries sl, sl + nsl, ... in order (four loads in flight per step).
template <int BITS>
__device__ __forceinline__ void rows_accum(const IterArgs& a, const uint32_t* words, const RowBlock& rb,
                                           const int32_t* s_list, const float* s_coef, int cn, int sl, int q,
                                           float (&z)[32 / BITS])
{
    constexpr int G = 32 / BITS;
    constexpr int U = 8;                       // entries of a slice whose loads are in flight together
    const int ld = a.Q.ld, lm1 = a.Q.lm1;
    for (int jj = sl; jj < cn; jj += U * rb.nsl) {
        uint32_t w[U];
        float cf[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = jj + u * rb.nsl;
            const bool in = e < cn;
            w[u] = in ? __ldg(words + (size_t)s_list[e] * ld + q) : 0u;
            cf[u] = in ? s_coef[e] : 0.0f;         // past the end: adds exact zeros
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int k = 0; k < G; ++k) {
                const int code = (int)((w[u] >> (8 * (k & 3) + BITS * (k >> 2))) & ((1u << BITS) - 1));
                z[k] = fmaf((float)(2 * code - lm1), cf[u], z[k]);
            }
    }
}

// Sum of the slices in slice order; the result stays in zrow[t] of the reducer threads:
// row word wl = t / G, row in word k = t % G, valid for t < wpc*G.
template <int BITS>
__device__ __forceinline__ void rows_reduce(const RowBlock& rb, int sl, const float (&z)[32 / BITS], float* red,
                                            float* zrow)
{
    constexpr int G = 32 / BITS;
    const int t = threadIdx.x;
    __syncthreads();
    if (sl < rb.nsl) {
#pragma unroll
        for (int k = 0; k < G; ++k) red[t * G + k] = z[k];
    }
    __syncthreads();
    if (t < rb.wpc * G) {
        const int w = t / G, k = t % G;
        float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};     // four interleaved partial sums, then in order
        int s2 = 0;
        for (; s2 + 4 <= rb.nsl; s2 += 4)
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] += red[((s2 + u) * rb.wpc + w) * G + k];
        for (; s2 < rb.nsl; ++s2) acc[0] += red[(s2 * rb.wpc + w) * G + k];
        zrow[t] = (acc[0] + acc[1]) + (acc[2] + acc[3]);
    }
    __syncthreads();
}

// z (for this CTA's rows) = sum over a list in global memory of coef_j * code column j,
// staged through shared memory in chunks of kListChunk entries.
// coef_mode: 0 = coef[jj], 1 = g[list[jj]].
template <int BITS>
__device__ void rows_product(const IterArgs& a, const RowBlock& rb, const int32_t* list, const float* coef,
                             int coef_mode, int count, int32_t* s_list, float* s_coef, float* red, float* zrow,
                             double* coef_sq = nullptr, const uint32_t* words = nullptr)
{
    if (!words) words = a.Q.words;
    constexpr int G = 32 / BITS;
    const int t = threadIdx.x;
    const int wl = t % rb.wpc, sl = t / rb.wpc;
    const int q = rb.w0 + wl;
    const bool active = sl < rb.nsl && q < rb.w1;
    float z[G];
#pragma unroll
    for (int k = 0; k < G; ++k) z[k] = 0.0f;
    for (int c0 = 0; c0 < count; c0 += kListChunk) {
        const int cn = min(kListChunk, count - c0);
        __syncthreads();
        for (int i = t; i < cn; i += blockDim.x) {
            const int col = __ldcg(list + c0 + i);
            s_list[i] = col;
            const float cf = coef_mode == 1 ? __ldcg(a.g + col) : __ldcg(coef + c0 + i);
            s_coef[i] = cf;
            if (coef_sq) *coef_sq += (double)cf * (double)cf;      // this thread's entries, in order
        }
        __syncthreads();
        if (active) rows_accum<BITS>(a, words, rb, s_list, s_coef, cn, sl, q, z);
    }
    rows_reduce<BITS>(rb, sl, z, red, zrow);
}

// The same product for a list already in shared memory (no staging).
template <int BITS>
__device__ void rows_product_sm(const IterArgs& a, const RowBlock& rb, const int32_t* list_sm, const float* coef_sm,
                                int count, float* red, float* zrow, const uint32_t* words = nullptr)
{
    if (!words) words = a.Q.words;
    constexpr int G = 32 / BITS;
    const int t = threadIdx.x;
    const int wl = t % rb.wpc, sl = t / rb.wpc;
    const int q = rb.w0 + wl;
    float z[G];
#pragma unroll
    for (int k = 0; k < G; ++k) z[k] = 0.0f;
    if (sl < rb.nsl && q < rb.w1) rows_accum<BITS>(a, words, rb, list_sm, coef_sm, count, sl, q, z);
    rows_reduce<BITS>(rb, sl, z, red, zrow);
}

// Radix select of the s-th largest of cnt keys (11/11/10-bit digits), keys read through ld().
template <typename KeyAt>
__device__ uint32_t select_kth(KeyAt key_at, int cnt, int s, unsigned* hist, int* sh_i, int* need_out)
{
    const int tid = threadIdx.x;
    uint32_t prefix = 0;
    int need = s;
    for (int pass = 0; pass < 3; ++pass) {
        const int shift = pass == 0 ? 21 : pass == 1 ? 10 : 0;
        const int width = pass == 2 ? 10 : 11;
        const uint32_t dmask = (1u << width) - 1u;
        const int nbins = 1 << width;
        for (int i = tid; i < nbins; i += blockDim.x) hist[i] = 0;
        __syncthreads();
        const int hi = shift + width;
        for (int j = tid; j < cnt; j += blockDim.x) {
            const uint32_t k = key_at(j);
            if (hi >= 32 || (k >> hi) == (prefix >> hi)) atomicAdd(&hist[(k >> shift) & dmask], 1u);
        }
        __syncthreads();
        if (tid < 32) {
            const int per = nbins >> 5;
            int tot = 0;
            for (int i = 0; i < per; ++i) tot += (int)hist[nbins - 1 - tid * per - i];
            int incl = tot;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (tid >= o) incl += y;
            }
            const int excl = incl - tot;
            if (excl < need && need <= incl) {
                int run = excl;
                for (int i = 0; i < per; ++i) {
                    const int bi = nbins - 1 - tid * per - i;
                    const int c = (int)hist[bi];
                    if (run + c >= need) { sh_i[0] = bi; sh_i[1] = run; break; }
                    run += c;
                }
            }
        }
        __syncthreads();
        prefix |= (uint32_t)sh_i[0] << shift;
        need -= sh_i[1];
        __syncthreads();
    }
    *need_out = need;
    return prefix;
}

__device__ int cta_excl_scan(int v, int* sh, int* total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        const int sv = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0;
        int tt = sv;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, tt, o);
            if (lane >= o) tt += y;
        }
        sh[lane] = tt - sv;
        if (lane == 31) sh[32] = tt;
    }
    __syncthreads();
    const int r = sh[w] + x - v;
    *total = sh[32];
    __syncthreads();
    return r;
}

// H_s on CTA 0. Candidates (keys >= tau) are ranked directly when there are at
// least s of them and no more than kRankMax: the rank of a candidate is the number
// of candidates ahead of it in the order (|a| descending, index ascending), read
// from one packed 64-bit key, so ties resolve exactly as in the full ranking.
// Otherwise the s-th largest of all n keys is found by a radix select. Either way
// the selection is marked in a bitmap and emitted in ascending index order; the
// x' - x list over G' u G is built from the same bitmap.
constexpr int kRankMax = 1024;
constexpr int kSupportSmem = 4096;       // supports up to this size are staged in shared memory

// Shared-memory arrays of the one-CTA select.
struct SelSmem {
    unsigned* hist;                  // 2048
    uint32_t* bitmap;                // ceil(n / 32) rounded up to 4
    int* wpre;                       // same
    unsigned long long* cv;          // cap (rank path only)
    float* cval;                     // cap (rank path only)
    float* cx;                       // cap (rank path only)
    int32_t* sup;                    // s (if s <= kSupportSmem)
};

__device__ __forceinline__ SelSmem sel_smem_layout(const IterArgs& a, unsigned char* smem)
{
    const int nbw4 = (((a.n + 31) / 32) + 3) & ~3;
    SelSmem m;
    m.hist = reinterpret_cast<unsigned*>(smem);
    m.bitmap = m.hist + 2048;
    m.wpre = reinterpret_cast<int*>(m.bitmap + nbw4);
    m.cv = reinterpret_cast<unsigned long long*>(m.wpre + nbw4);
    m.cval = reinterpret_cast<float*>(m.cv + a.cap);
    m.cx = m.cval + a.cap;
    m.sup = reinterpret_cast<int32_t*>(m.cx + a.cap);
    return m;
}

// allow_rank = false: always the radix select over all n keys.
__device__ void select_on_cta0(const IterArgs& a, float mu, const SelSmem& sm, bool allow_rank)
{
    State* st = a.st;
    const int n = a.n, s = a.s, tid = threadIdx.x;
    const int lane = tid & 31;
    const int nbw = (n + 31) / 32;
    const int nbw4 = (nbw + 3) & ~3;
    unsigned* hist = sm.hist;
    uint32_t* bitmap = sm.bitmap;
    int* wpre = sm.wpre;
    unsigned long long* cv = sm.cv;
    float* cval = sm.cval;
    float* cx = sm.cx;
    int32_t* sup = sm.sup;
    const bool sup_sm = s <= kSupportSmem;
    __shared__ int sh_i[36];
    __shared__ unsigned sh_u[33];
    __shared__ unsigned long long sh_k[2];

    const int cnt = (int)__ldcg(&st->cand_count);
    const unsigned below_filter = __ldcg(&st->below_max);
    const bool use_rank =
        allow_rank && a.cap > 0 && __ldcg(&st->tau_bits) != 0u && cnt >= s && cnt <= min(a.cap, kRankMax);
    for (int w = tid; w < nbw4; w += blockDim.x) bitmap[w] = 0u;
    if (tid < 2) sh_k[tid] = 0ull;
    if (sup_sm)
        for (int q = tid; q < s; q += blockDim.x) sup[q] = __ldcg(a.support + q);
    float kth0 = 0.0f, kth1 = 0.0f;
    if (use_rank) {
        for (int i = tid; i < cnt; i += blockDim.x) {
            cv[i] = __ldcg(a.cand + i);
            cval[i] = __ldcg(a.cand_val + i);
            cx[i] = __ldcg(a.cand_x + i);
        }
        __syncthreads();
        for (int i = tid; i < cnt; i += blockDim.x) {
            const unsigned long long mine = cv[i];
            int rank = 0;
#pragma unroll 8
            for (int q = 0; q < cnt; ++q) rank += (cv[q] > mine);
            if (rank < s) {
                const uint32_t j = ~(uint32_t)mine;
                atomicOr(&bitmap[j >> 5], 1u << (j & 31));
            }
            if (rank == s - 1) sh_k[0] = mine;
            if (rank == s) sh_k[1] = mine;
        }
        __syncthreads();
        kth0 = __uint_as_float((uint32_t)(sh_k[0] >> 32));
        kth1 = cnt > s ? __uint_as_float((uint32_t)(sh_k[1] >> 32)) : __uint_as_float(below_filter);
    } else {
        __syncthreads();
        int need = 0;
        const uint32_t T = select_kth([&](int j) { return __ldcg(a.keys + j); }, n, s, hist, sh_i, &need);
        // mark keys > T, and the `need` lowest-index keys == T, walking the keys in index order
        const int warp = tid >> 5, nw = blockDim.x >> 5;
        const int seg = ((n + 32 * nw - 1) / (32 * nw)) * 32;
        const int wb = min(n, warp * seg), we = min(n, wb + seg);
        int eq = 0;
        unsigned below = 0;
        for (int b = wb; b < we; b += 32) {
            const int j = b + lane;
            const bool in = j < we;
            const uint32_t k = in ? __ldcg(a.keys + j) : 0u;
            eq += __popc(__ballot_sync(0xffffffffu, in && k == T));
            if (in && k < T) below = max(below, k);
        }
        if (lane == 0) sh_i[warp] = eq;
        __syncthreads();
        int eq_before = 0;
        for (int w = 0; w < warp; ++w) eq_before += sh_i[w];
        int eq_total = 0;
        for (int w = 0; w < nw; ++w) eq_total += sh_i[w];
        __syncthreads();
        const int take_w = max(0, min(eq, need - eq_before));
        int erun = 0;
        const unsigned lt = (1u << lane) - 1u;
        for (int b = wb; b < we; b += 32) {
            const int j = b + lane;
            const bool in = j < we;
            const uint32_t k = in ? __ldcg(a.keys + j) : 0u;
            const unsigned meq = __ballot_sync(0xffffffffu, in && k == T);
            const int rank = erun + __popc(meq & lt);
            const bool take = in && (k > T || (k == T && rank < take_w));
            if (take) atomicOr(&bitmap[j >> 5], 1u << (j & 31));
            erun += __popc(meq);
        }
        const unsigned bm = cta_max(below, sh_u);
        kth0 = __uint_as_float(T);
        kth1 = (eq_total > need) ? kth0 : (s < n ? __uint_as_float(bm) : 0.0f);
    }
    __syncthreads();
    // selected entries before each bitmap word (exclusive scan over the words)
    {
        const int wpt = (nbw + blockDim.x - 1) / blockDim.x;
        const int w0 = min(nbw, tid * wpt), w1 = min(nbw, w0 + wpt);
        int c = 0;
        for (int w = w0; w < w1; ++w) c += __popc(bitmap[w]);
        int total;
        int pre = cta_excl_scan(c, sh_i, &total);
        for (int w = w0; w < w1; ++w) { wpre[w] = pre; pre += __popc(bitmap[w]); }
    }
    __syncthreads();
    // emit G' (ascending) with x'; the first s entries of the x' - x list are G'
    int diff = 0;
    auto emit = [&](int j, float v, float xj) {
        const int w = j >> 5;
        const int pos = wpre[w] + __popc(bitmap[w] & ((1u << (j & 31)) - 1u));
        diff |= (j != (sup_sm ? sup[pos] : __ldcg(a.support + pos)));
        a.sel[pos] = j;
        a.val[pos] = v;
        a.uni[pos] = j;
        a.delta[pos] = v - xj;
    };
    if (use_rank) {
        for (int i = tid; i < cnt; i += blockDim.x) {
            const uint32_t j = ~(uint32_t)cv[i];
            if ((bitmap[j >> 5] >> (j & 31)) & 1u) emit((int)j, cval[i], cx[i]);
        }
    } else {
        for (int w = tid; w < nbw; w += blockDim.x) {
            uint32_t bits = bitmap[w];
            while (bits) {
                const int b = __ffs(bits) - 1;
                bits &= bits - 1;
                const int j = w * 32 + b;
                const float xj = __ldcg(a.x + j);
                emit(j, fmaf(mu, __ldcg(a.g + j), xj), xj);
            }
        }
    }
    diff = __syncthreads_or(diff);
    // G \ G' after G', in support order
    {
        const int sper = (s + blockDim.x - 1) / blockDim.x;
        const int q0 = min(s, tid * sper), q1 = min(s, q0 + sper);
        int cntx = 0;
        for (int q = q0; q < q1; ++q) {
            const int j = sup_sm ? sup[q] : __ldcg(a.support + q);
            cntx += !((bitmap[j >> 5] >> (j & 31)) & 1u);
        }
        int extra;
        int p = cta_excl_scan(cntx, sh_i, &extra);
        for (int q = q0; q < q1; ++q) {
            const int j = sup_sm ? sup[q] : __ldcg(a.support + q);
            if (!((bitmap[j >> 5] >> (j & 31)) & 1u)) {
                a.uni[s + p] = j;
                a.delta[s + p] = -__ldcg(a.x + j);
                ++p;
            }
        }
        if (tid == 0) {
            if (!use_rank) st->full_selects += 1;
            st->kth0 = kth0;
            st->kth1 = kth1;
            // next candidate threshold: a little below the current (s+1)-th magnitude
            st->tau_bits = (a.cap > 0 && kth1 > 0.0f) ? __float_as_uint(kth1 * 0.9375f) : 0u;
            st->cand_count = 0u;
            st->below_max = 0u;
            st->changed = diff ? 1 : 0;
            st->union_count = s + extra;
        }
    }
}

template <int BITS>
__global__ void __launch_bounds__(kIterThreads, 1) k_iter(IterArgs a)
{
    constexpr int G = 32 / BITS;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double shd[33];
    __shared__ unsigned shu[33];
    State* st = a.st;
    griddep_wait();                             // the previous kernels' results are visible
    griddep_launch();
    if (st->stop) return;                       // uniform: read before any barrier
    const bool stamp = blockIdx.x == 0 && threadIdx.x == 0;
    if (stamp) st->t_phase[0] = gtimer_ns();
    unsigned long long target = threadIdx.x == 0 ? barrier_base(a.gbar) : 0ull;

    const RowBlock rb = row_block(a.Q.ld);
    int32_t* s_list = reinterpret_cast<int32_t*>(smem);
    float* s_coef = reinterpret_cast<float*>(s_list + kListChunk);
    float* red = s_coef + kListChunk;                           // kIterThreads * G
    float* zrow = red + kIterThreads * G;                       // kIterThreads
    unsigned char* sel_smem = smem;                             // CTA 0's select reuses the buffer
    // alpha = scale / (levels - 1) once per CTA (FP64 division is slow on this GPU); the
    // first product's barriers publish it
    __shared__ double s_alpha;
    __shared__ float s_alpha_f;
    if (threadIdx.x == 32) {
        s_alpha = (double)(*a.Q.scale) / (double)a.Q.lm1;
        s_alpha_f = (float)s_alpha;
    }
    const int m = a.m, s = a.s, n = a.n;
    const int tid = threadIdx.x;
    double* mypart = a.part + blockIdx.x;       // slot k of this CTA: mypart[k * kSlotCtas]

    // ---- Mu: z = Q2_G g_G, den = alpha^2 ||z||^2, num = ||g_G||^2 ----
    // (QIHT_MU_CROSS: also z1 = Q1_G g_G and den = alpha^2 z1 . z when that is positive)
    const bool cross = a.mu_mode == QIHT_MU_CROSS;
    float z1v = 0.0f;
    if (cross) {
        rows_product<BITS>(a, rb, a.support, nullptr, 1, s, s_list, s_coef, red, zrow, nullptr, a.q1_words);
        if (tid < rb.wpc * G) z1v = zrow[tid];
    }
    double gsq = 0.0;
    rows_product<BITS>(a, rb, a.support, nullptr, 1, s, s_list, s_coef, red, zrow, &gsq);
    {
        double acc = 0.0, cp = 0.0;
        if (tid < rb.wpc * G) {
            const int row = (rb.w0 + tid / G) * G + tid % G;
            if (rb.w0 + tid / G < rb.w1 && row < m) {
                acc = (double)zrow[tid] * (double)zrow[tid];
                cp = (double)z1v * (double)zrow[tid];
            }
        }
        acc = cta_sum(acc, shd);
        const double num = cta_sum(gsq, shd);                // ||g_G||^2 from the staged coefficients
        if (cross) cp = cta_sum(cp, shd);
        if (tid == 0) {
            mypart[0 * kSlotCtas] = acc;
            mypart[1 * kSlotCtas] = num;
            if (cross) mypart[4 * kSlotCtas] = cp;
        }
    }
    if (!grid_sync(a.gbar, target, st, a.report)) return;
    if (stamp) st->t_phase[1] = gtimer_ns();
    double mu;
    {
        const double den_f = s_alpha * s_alpha * grid_partial_sum(a.part, 0, shd);
        double den = den_f;
        if (cross) {
            const double den_c = s_alpha * s_alpha * grid_partial_sum(a.part, 4, shd);
            if (den_c > 0.0) den = den_c;                      // else the forward square
        }
        const double num = __ldcg(a.part + 1 * kSlotCtas);     // CTA 0's slot
        bool stop = false;
        if (!isfinite(num) || !isfinite(den_f)) {
            stop = true;
            if (blockIdx.x == 0 && tid == 0) st->status = QIHT_ERR_NONFINITE;
        } else if (num == 0.0 || den_f == 0.0) {
            stop = true;                                       // converged: x stays
        }
        mu = stop ? 0.0 : num / den;
        if (stop) {
            if (blockIdx.x == 0 && tid == 0) {
                st->stop = 1;
                if (a.report) {
                    a.report->iters_run = st->iter;
                    a.report->backtracks = st->backtracks_total;
                    a.report->support_changes = st->support_changes_total;
                    a.report->status = st->status;
                    a.report->resid_norm2 = st->resid2;
                    a.report->mu = st->mu_accepted;
                }
            }
            return;                                            // uniform across CTAs
        }
        if (blockIdx.x == 0 && tid == 0) { st->num = num; st->bt = 0; }
    }

    int bt = 0;
    for (;;) {
        // ---- Filter: keys of all entries, candidates >= tau ----
        {
            const float muf = (float)mu;
            const uint32_t tau = __ldcg(&st->tau_bits);
            const int per = (n + gridDim.x - 1) / gridDim.x;
            const int j0 = blockIdx.x * per, j1 = min(n, j0 + per);
            __shared__ int scan_i[33];
            __shared__ unsigned base_sh;
            unsigned below = 0;
            int bad = 0;
            for (int jb = j0; jb < j1; jb += blockDim.x) {
                const int j = jb + tid;
                uint32_t k = 0;
                float v = 0.0f, xj = 0.0f;
                const bool in = j < j1;
                if (in) {
                    xj = __ldcg(a.x + j);
                    v = fmaf(muf, __ldcg(a.g + j), xj);
                    k = __float_as_uint(v) & 0x7fffffffu;
                    bad |= (k > 0x7f800000u);
                    a.keys[j] = k;
                }
                const bool take = in && tau != 0u && k >= tau;
                if (in && !take) below = max(below, k);
                // CTA-aggregated append: one atomic per CTA and batch
                int total;
                const int rank = cta_excl_scan(take ? 1 : 0, scan_i, &total);
                if (total) {
                    if (tid == 0) base_sh = atomicAdd(&st->cand_count, (unsigned)total);
                    __syncthreads();
                    if (take) {
                        const unsigned slot = base_sh + (unsigned)rank;
                        if (slot < (unsigned)a.cap) {
                            a.cand[slot] = ((unsigned long long)k << 32) | (unsigned long long)(~(uint32_t)j);
                            a.cand_val[slot] = v;
                            a.cand_x[slot] = xj;
                        }
                    }
                    __syncthreads();
                }
            }
            // one atomic per CTA for the largest key below tau
            const unsigned bcta = cta_max(below, shu);
            if (tid == 0 && bcta) atomicMax(&st->below_max, bcta);
            if (__syncthreads_or(bad) && tid == 0) st->status = QIHT_ERR_NONFINITE;
        }
        if (!grid_sync(a.gbar, target, st, a.report)) return;
        if (stamp) st->t_phase[2] = gtimer_ns();
        if (__ldcg(&st->status) == QIHT_ERR_NONFINITE) {
            if (blockIdx.x == 0 && tid == 0) st->stop = 1;
            return;
        }
        // ---- Select on CTA 0 ----
        if (blockIdx.x == 0) select_on_cta0(a, (float)mu, sel_smem_layout(a, sel_smem), true);
        if (!grid_sync(a.gbar, target, st, a.report)) return;
        if (stamp) st->t_phase[3] = gtimer_ns();
        if (!__ldcg(&st->changed)) break;

        // ---- Omega: backtracking test on G' u G ----
        const int cu = __ldcg(&st->union_count);
        double dsq = 0.0;
        rows_product<BITS>(a, rb, a.uni, a.delta, 0, cu, s_list, s_coef, red, zrow, &dsq);
        {
            double acc = 0.0;
            if (tid < rb.wpc * G) {
                const int row = (rb.w0 + tid / G) * G + tid % G;
                if (rb.w0 + tid / G < rb.w1 && row < m) acc = (double)zrow[tid] * (double)zrow[tid];
            }
            acc = cta_sum(acc, shd);
            const double dn = cta_sum(dsq, shd);             // ||x' - x||^2 from the staged list
            if (tid == 0) { mypart[2 * kSlotCtas] = acc; mypart[3 * kSlotCtas] = dn; }
        }
        if (!grid_sync(a.gbar, target, st, a.report)) return;
        const double dd = s_alpha * s_alpha * grid_partial_sum(a.part, 2, shd);
        const double dn = __ldcg(a.part + 3 * kSlotCtas);
        if (!(dn > 0.0)) break;                               // nothing moves: accept
        const double omega = dd > 0.0 ? dn / dd : INFINITY;
        if (mu <= (1.0 - a.c) * omega) break;                 // sufficient decrease: accept
        if (bt >= a.max_bt) {
            if (blockIdx.x == 0 && tid == 0) {
                st->status = QIHT_ERR_BACKTRACK_CAP;
                st->stop = 1;
                if (a.report) {
                    a.report->iters_run = st->iter;
                    a.report->backtracks = st->backtracks_total;
                    a.report->support_changes = st->support_changes_total;
                    a.report->status = st->status;
                    a.report->resid_norm2 = st->resid2;
                    a.report->mu = st->mu_accepted;
                }
            }
            return;
        }
        mu = mu / (a.k * (1.0 - a.c));
        ++bt;
    }

    // ---- Resid: r = Q(y) - Q2_G' x' for this CTA's rows ----
    if (stamp) st->t_phase[4] = gtimer_ns();
    rows_product<BITS>(a, rb, a.sel, a.val, 0, s, s_list, s_coef, red, zrow);
    {
        double acc = 0.0;
        unsigned mx = 0;
        if (tid < rb.wpc * G) {
            const int row = (rb.w0 + tid / G) * G + tid % G;
            if (rb.w0 + tid / G < rb.w1 && row < m) {
                const float ri = fmaf(-s_alpha_f, zrow[tid], __ldcg(a.yhat + row));
                a.r[row] = ri;
                acc = (double)ri * (double)ri;
                mx = __float_as_uint(ri) & 0x7fffffffu;
            }
        }
        acc = cta_sum(acc, shd);
        mx = cta_max(mx, shu);
        if (tid == 0) { mypart[0 * kSlotCtas] = acc; mypart[1 * kSlotCtas] = (double)mx; }
    }
    if (stamp) st->t_phase[5] = gtimer_ns();
    // the last CTA to arrive commits the iteration (no CTA waits for it)
    __shared__ int last;
    __threadfence();
    __syncthreads();
    if (tid == 0) last = (atomicAdd(a.bar + 2, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    const double resid2 = grid_partial_sum(a.part, 0, shd);
    const double rmax = grid_partial_max(a.part, 1, shd);
    {
        // zero the old support everywhere first, then write the new one (entries may be in both)
        constexpr int kPer = 8;
        for (int q0 = 0; q0 < s; q0 += kPer * kIterThreads) {
            int oldj[kPer];
#pragma unroll
            for (int u = 0; u < kPer; ++u) {
                const int q = q0 + u * kIterThreads + tid;
                oldj[u] = q < s ? __ldcg(a.support + q) : -1;
            }
#pragma unroll
            for (int u = 0; u < kPer; ++u)
                if (oldj[u] >= 0) a.x[oldj[u]] = 0.0f;
        }
        __syncthreads();
        for (int q0 = 0; q0 < s; q0 += kPer * kIterThreads) {
            int newj[kPer];
            float newv[kPer];
#pragma unroll
            for (int u = 0; u < kPer; ++u) {
                const int q = q0 + u * kIterThreads + tid;
                newj[u] = q < s ? __ldcg(a.sel + q) : -1;
                newv[u] = q < s ? __ldcg(a.val + q) : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < kPer; ++u) {
                const int q = q0 + u * kIterThreads + tid;
                if (newj[u] >= 0) { a.x[newj[u]] = newv[u]; a.support[q] = newj[u]; }
            }
        }
        __syncthreads();
    }
    if (tid == 0) {
        a.bar[2] = 0u;
        const int it = st->iter + 1;
        st->iter = it;
        st->mu = mu;
        st->mu_accepted = mu;
        st->bt = bt;
        st->resid2 = resid2;
        st->rmax_bits = (unsigned)rmax;
        st->backtracks_total += bt;
        st->support_changes_total += st->changed;
        if (!isfinite(resid2)) {
            st->status = QIHT_ERR_NONFINITE;
            st->stop = 1;
        }
        if (a.trace.kth) { a.trace.kth[2 * it] = st->kth0; a.trace.kth[2 * it + 1] = st->kth1; }
        if (a.trace.mu) a.trace.mu[it] = mu;
        if (a.trace.bt) a.trace.bt[it] = bt;
        if (a.trace.resid2) a.trace.resid2[it] = resid2;
        if (it >= st->iters) st->stop = 1;
        if (a.tol > 0.0 && resid2 <= a.tol) st->stop = 1;      // the residual reached tol
        if (a.report) {
            a.report->iters_run = st->iter;
            a.report->backtracks = st->backtracks_total;
            a.report->support_changes = st->support_changes_total;
            a.report->status = st->status;
            a.report->resid_norm2 = resid2;
            a.report->mu = mu;
            a.report->full_selects = st->full_selects;
            // phases: step size, filter, select(s) + backtracking, residual product, commit
            const unsigned long long t6 = gtimer_ns();
            const unsigned long long* tp = st->t_phase;
            a.report->phase_us[0] = (float)((tp[1] - tp[0]) * 1e-3);
            a.report->phase_us[1] = (float)((tp[2] - tp[1]) * 1e-3);
            a.report->phase_us[2] = (float)((tp[3] - tp[2]) * 1e-3);
            a.report->phase_us[3] = (float)((tp[4] - tp[3]) * 1e-3);
            a.report->phase_us[4] = (float)((tp[5] - tp[4]) * 1e-3);
            a.report->phase_us[5] = (float)((t6 - tp[5]) * 1e-3);
            a.report->phase_us[6] = (float)((t6 - tp[0]) * 1e-3);
            a.report->phase_us[7] = 0.0f;
        }
    }
    __syncthreads();
    if (a.trace.support) {
        const int it = st->iter;
        for (int q = tid; q < s; q += blockDim.x) a.trace.support[(size_t)it * s + q] = __ldcg(a.sel + q);
    }
}


// ---------------------------------------------------------------------------
// Fast-path iteration kernel. The threshold's candidates come from the gradient
// kernel: an entry outside G has x_j = 0, so its key |x_j + mu g_j| = fl(mu |g_j|)
// orders like |g_j| whatever mu is, and the gradient kernel can keep the entries
// with |g_j| >= tau_g (and the largest |g_j| below) before mu is known. Every CTA
// then ranks G together with the candidates in its own shared memory and gets the
// same H_s, so no grid barrier separates the step size from the residual when the
// support does not move. The selection is provably the full one when the s-th key
// of the ranked set exceeds fl(mu max_rejected |g|); otherwise (and in the first
// iteration, before the gradient kernel has a support to filter against) the keys
// of all n entries go to the one-CTA radix select as in k_iter.
// Every CTA commits its own slice of x and of the position map; the last CTA to
// finish writes G, x_G and the scalars.
// ---------------------------------------------------------------------------
constexpr int kFastMaxS = 2 * 512;       // largest s of the fast path (lists held in shared memory)
constexpr int kResidDirect = 16;         // the residual is formed directly every 16 iterations
constexpr int kTieMax = 64;              // ties at the s-th key ranked by index in shared memory

struct FastSm {
    uint32_t* key;                       // [s + gcap] |x + mu g| of G, then of the candidates
    int32_t* el_idx;                     // [s + gcap]
    float* el_x;                         // [s + gcap]
    float* el_g;                         // [s + gcap]
    uint32_t* bitmap;                    // [nbw4] selection
    int* wpre;                           // [nbw4]
    int32_t* u_idx;                      // [2s] G' (ascending), then G \ G'
    float* u_val;                        // [s]  x' on G'
    float* u_delta;                      // [2s] x' - x on the u_idx list
    unsigned* hist;                      // [256]
    int32_t* tie;                        // [kTieMax]
    float* red;                          // [kIterThreads * G]
    float* zrow;                         // [kIterThreads]
};

__host__ __device__ inline size_t fast_smem_bytes(int n, int s, int gcap, int G)
{
    const size_t el = (size_t)s + (size_t)gcap;
    const size_t nbw4 = ((size_t)(n + 31) / 32 + 3) & ~(size_t)3;
    return el * 16 + nbw4 * 8 + (size_t)s * 20 + 256 * 4 + (size_t)kTieMax * 4 + (size_t)kIterThreads * G * 4 +
           (size_t)kIterThreads * 4;
}

__device__ __forceinline__ FastSm fast_smem_layout(const IterArgs& a, unsigned char* smem, int G)
{
    const int el = a.s + a.gcap;
    const int nbw4 = (((a.n + 31) / 32) + 3) & ~3;
    FastSm m;
    m.key = reinterpret_cast<uint32_t*>(smem);
    m.el_idx = reinterpret_cast<int32_t*>(m.key + el);
    m.el_x = reinterpret_cast<float*>(m.el_idx + el);
    m.el_g = m.el_x + el;
    m.bitmap = reinterpret_cast<uint32_t*>(m.el_g + el);
    m.wpre = reinterpret_cast<int*>(m.bitmap + nbw4);
    m.u_idx = reinterpret_cast<int32_t*>(m.wpre + nbw4);
    m.u_val = reinterpret_cast<float*>(m.u_idx + 2 * a.s);
    m.u_delta = m.u_val + a.s;
    m.hist = reinterpret_cast<unsigned*>(m.u_delta + 2 * a.s);
    m.tie = reinterpret_cast<int32_t*>(m.hist + 256);
    m.red = reinterpret_cast<float*>(m.tie + kTieMax);
    m.zrow = m.red + kIterThreads * G;
    return m;
}

// Radix select (8-bit digits, most significant first) of the s-th largest of cnt keys
// in shared memory. Stops early when the digit's bucket holds exactly the keys still
// needed (then every key of the bucket is selected): *depth_out = last digit examined
// (3 = all four), and the return value has the digits found so far. Otherwise the
// result is the s-th key itself and *need_out says how many keys equal to it belong
// to the s largest.
__device__ uint32_t radix_select8(const uint32_t* key, int cnt, int s, unsigned* hist, int* sh_i, int* need_out,
                                  int* depth_out)
{
    const int tid = threadIdx.x, lane = tid & 31;
    uint32_t prefix = 0;
    int need = s;
    int depth = 3;
    for (int pass = 0; pass < 4; ++pass) {
        const int shift = 24 - 8 * pass;
        if (tid < 256) hist[tid] = 0;
        __syncthreads();
        for (int e = tid; e < cnt; e += blockDim.x) {
            const uint32_t k = key[e];
            if (pass == 0 || (k >> (shift + 8)) == (prefix >> (shift + 8))) atomicAdd(&hist[(k >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (tid < 32) {
            // lane l holds bins 255 - 8l down to 248 - 8l (descending key order)
            int c[8];
            int tot = 0;
#pragma unroll
            for (int i = 0; i < 8; ++i) { c[i] = (int)hist[255 - 8 * lane - i]; tot += c[i]; }
            int incl = tot;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const int excl = incl - tot;
            if (excl < need && need <= incl) {
                int run = excl;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    if (run + c[i] >= need) {
                        sh_i[0] = 255 - 8 * lane - i;
                        sh_i[1] = run;
                        sh_i[2] = (run + c[i] == need);        // the whole bucket is taken
                        break;
                    }
                    run += c[i];
                }
            }
        }
        __syncthreads();
        prefix |= (uint32_t)sh_i[0] << shift;
        need -= sh_i[1];
        if (sh_i[2] && pass < 3) { depth = pass; break; }
    }
    __syncthreads();
    *need_out = need;
    *depth_out = depth;
    return prefix;
}

struct SelResult {
    int changed, uc;
    float kth0, kth1;
};

// H_s over G and the gradient kernel's candidates, in this CTA. Returns false (the
// same in every CTA) when the ranked set cannot be shown to hold the full selection.
// When G' = G the lists are G itself (no bitmap is built).
__device__ bool select_fast(const IterArgs& a, const FastSm& sm, int cnt, float muf, uint32_t outside_max,
                            SelResult& out)
{
    const int s = a.s, n = a.n, tid = threadIdx.x;
    __shared__ int sh_i[36];
    __shared__ unsigned sh_u[33];
    __shared__ int tie_n;
    int bad = 0;
    for (int e = tid; e < cnt; e += blockDim.x) {
        const uint32_t k = __float_as_uint(fmaf(muf, sm.el_g[e], sm.el_x[e])) & 0x7fffffffu;
        bad |= k > 0x7f800000u;
        sm.key[e] = k;
    }
    if (tid == 0) tie_n = 0;
    if (__syncthreads_or(bad)) return false;                   // NaN: the full select reports it
    {
        // the support stays when every key of G exceeds every other key (the candidates' and
        // outside_max, the largest key of the entries the gradient kernel rejected): then H_s
        // keeps G whatever the order inside it, and no ranking is needed
        unsigned inv_min = 0, cmax = 0;
        for (int e = tid; e < cnt; e += blockDim.x) {
            const uint32_t k = sm.key[e];
            if (e < s) inv_min = max(inv_min, ~k);
            else cmax = max(cmax, k);
        }
        const uint32_t kmin = ~cta_max(inv_min, sh_u);
        const uint32_t rest = max(cta_max(cmax, sh_u), outside_max);
        if (kmin > rest) {
            for (int q = tid; q < s; q += blockDim.x) {
                sm.u_idx[q] = sm.el_idx[q];
                sm.u_val[q] = fmaf(muf, sm.el_g[q], sm.el_x[q]);
            }
            out.changed = 0;
            out.uc = s;
            out.kth0 = __uint_as_float(kmin);
            out.kth1 = __uint_as_float(rest);
            __syncthreads();
            return true;
        }
    }
    int need = 0, depth = 3;
    const uint32_t P = radix_select8(sm.key, cnt, s, sm.hist, sh_i, &need, &depth);
    uint32_t T;
    int eq_total = 0;
    bool tie_rank = false;
    unsigned below = 0;
    if (depth < 3) {
        // every key of the bucket (top 8 (depth + 1) bits = P's) is taken: T = its smallest key
        const int shift = 24 - 8 * depth;
        unsigned inv = 0;
        for (int e = tid; e < cnt; e += blockDim.x) {
            const uint32_t k = sm.key[e];
            if ((k >> shift) == (P >> shift)) inv = max(inv, ~k);
        }
        T = ~cta_max(inv, sh_u);
        for (int e = tid; e < cnt; e += blockDim.x) {
            const uint32_t k = sm.key[e];
            if (k < T) below = max(below, k);
        }
        below = cta_max(below, sh_u);
        if (!(T > outside_max)) return false;
    } else {
        T = P;
        int eq = 0;
        for (int e = tid; e < cnt; e += blockDim.x) {
            const uint32_t k = sm.key[e];
            eq += (k == T);
            if (k < T) below = max(below, k);
        }
        (void)cta_excl_scan(eq, sh_i, &eq_total);
        below = cta_max(below, sh_u);
        // every key outside the set is <= outside_max: the set decides H_s if its s-th key is larger
        if (!(T > outside_max) || (eq_total > need && eq_total > kTieMax)) return false;
        tie_rank = eq_total > need;
        if (tie_rank) {
            for (int e = tid; e < cnt; e += blockDim.x)
                if (sm.key[e] == T) sm.tie[atomicAdd(&tie_n, 1)] = sm.el_idx[e];
            __syncthreads();
        }
    }
    auto taken = [&](int e) -> bool {
        const uint32_t k = sm.key[e];
        if (k != T) return k > T;
        if (!tie_rank) return true;
        const int j = sm.el_idx[e];
        int r = 0;                                             // equal keys: lower index first
        for (int i = 0; i < eq_total; ++i) r += sm.tie[i] < j;
        return r < need;
    };
    out.kth0 = __uint_as_float(T);
    out.kth1 = tie_rank ? __uint_as_float(T) : __uint_as_float(max(below, outside_max));
    // G' = G exactly when every entry of G is taken (s are taken in all)
    int left = 0;
    for (int q = tid; q < s; q += blockDim.x) left |= !taken(q);
    const int diff = __syncthreads_or(left);
    out.changed = diff;
    if (!diff) {
        for (int q = tid; q < s; q += blockDim.x) {
            sm.u_idx[q] = sm.el_idx[q];
            sm.u_val[q] = fmaf(muf, sm.el_g[q], sm.el_x[q]);
        }
        out.uc = s;
        __syncthreads();
        return true;
    }
    const int nbw = (n + 31) / 32;
    const int nbw4 = (nbw + 3) & ~3;
    for (int w = tid; w < nbw4; w += blockDim.x) sm.bitmap[w] = 0u;
    __syncthreads();
    for (int e = tid; e < cnt; e += blockDim.x)
        if (taken(e)) {
            const int j = sm.el_idx[e];
            atomicOr(&sm.bitmap[j >> 5], 1u << (j & 31));
        }
    __syncthreads();
    {
        const int wpt = (nbw + blockDim.x - 1) / blockDim.x;
        const int w0 = min(nbw, tid * wpt), w1 = min(nbw, w0 + wpt);
        int c = 0;
        for (int w = w0; w < w1; ++w) c += __popc(sm.bitmap[w]);
        int total;
        int pre = cta_excl_scan(c, sh_i, &total);
        for (int w = w0; w < w1; ++w) { sm.wpre[w] = pre; pre += __popc(sm.bitmap[w]); }
    }
    __syncthreads();
    for (int e = tid; e < cnt; e += blockDim.x) {
        const int j = sm.el_idx[e];
        const int w = j >> 5;
        const uint32_t bm = sm.bitmap[w];
        if ((bm >> (j & 31)) & 1u) {
            const int p = sm.wpre[w] + __popc(bm & ((1u << (j & 31)) - 1u));
            const float xj = sm.el_x[e];
            const float v = fmaf(muf, sm.el_g[e], xj);
            sm.u_idx[p] = j;
            sm.u_val[p] = v;
            sm.u_delta[p] = v - xj;
        }
    }
    int extra = 0;
    {
        // G \ G' after G', in support order
        const int sper = (s + blockDim.x - 1) / blockDim.x;
        const int q0 = min(s, tid * sper), q1 = min(s, q0 + sper);
        int cntx = 0;
        for (int q = q0; q < q1; ++q) {
            const int j = sm.el_idx[q];
            cntx += !((sm.bitmap[j >> 5] >> (j & 31)) & 1u);
        }
        int p = cta_excl_scan(cntx, sh_i, &extra);
        for (int q = q0; q < q1; ++q) {
            const int j = sm.el_idx[q];
            if (!((sm.bitmap[j >> 5] >> (j & 31)) & 1u)) {
                sm.u_idx[s + p] = j;
                sm.u_delta[s + p] = -sm.el_x[q];
                ++p;
            }
        }
    }
    __syncthreads();
    out.uc = s + extra;
    return true;
}

// Per-CTA partial slots (CTA index fastest, tagged; see slot_put), gathered by CTA 0:
// 0 ||z||^2 of the step size, 2 ||Q2 d||^2 of a backtracking test, 4 ||r||^2 and
// 5 max |r| of the residual. CTA 0 answers the first two with the decision word.
template <int BITS>
__global__ void __launch_bounds__(kIterThreads, 1) k_iter_fast(IterArgs a)
{
    constexpr int G = 32 / BITS;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double shd[33];
    __shared__ unsigned shu[33];
    __shared__ double s_alpha;
    __shared__ float s_alpha_f, s_muf;
    __shared__ int s_code;
    State* st = a.st;
    const int tid = threadIdx.x, lane = tid & 31;
    const bool cta0 = blockIdx.x == 0;
    // FP64 work (low throughput on this GPU) is done by single threads or single warps
    if (tid == 32) {
        const double al = (double)(*a.Q.scale) / (double)a.Q.lm1;
        s_alpha = al;
        s_alpha_f = (float)al;
    }
    const RowBlock rb = row_block(a.Q.ld);
    const FastSm sm = fast_smem_layout(a, smem, G);
    const int m = a.m, s = a.s, n = a.n;
    double* mypart = a.part + blockIdx.x;       // slot k of this CTA: mypart[k * kSlotCtas]
    const int nbw4 = (((n + 31) / 32) + 3) & ~3;
    const int nrow_thr = rb.wpc * G;            // threads that hold one row of this CTA
    float yrow = 0.0f;                          // Q(y) of this thread's row (fixed during the solve)
    int row_ok = 0, row = 0;
    if (tid < nrow_thr) {
        row = (rb.w0 + tid / G) * G + tid % G;
        row_ok = rb.w0 + tid / G < rb.w1 && row < m;
        if (row_ok) yrow = __ldcg(a.yhat + row);
    }
    // everything above is fixed during the solve; the rest comes from the previous kernels
    griddep_wait();
    griddep_launch();
    // The next gradient pass streams Q1's codes from the start of the array (its first round
    // of columns, one per warp, is a contiguous block). After the step size is known, the
    // rest of this kernel leaves HBM nearly idle, so it brings the start of that block into L2
    // meanwhile (issued earlier, it slows the step size's own reads). A hint only; nothing
    // waits on it.
    auto prefetch_next = [&]() {
        if (tid != 0) return;
        const size_t total = (size_t)a.n * (size_t)a.Q.ld * 4;
        const size_t off = (size_t)blockIdx.x * kIterPrefetchCta;
        if (off < total) {
            const unsigned len = (unsigned)min((size_t)kIterPrefetchCta, total - off);   // a multiple of 16
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(reinterpret_cast<const char*>(a.q1_words) + off),
                         "r"(len)
                         : "memory");
        }
    };

    // the state words are read by one thread per CTA (every thread of every CTA reading the
    // same line would queue thousands of requests on one L2 slice) and shared below
    __shared__ unsigned s_state[8];
    if (tid == 0) {
        s_state[0] = (unsigned)__ldcg(&st->stop);
        s_state[1] = (unsigned)__ldcg(&st->iter);
        s_state[2] = __ldcg(&st->omega_uses);
        s_state[3] = __ldcg(&st->dec_uses);
        s_state[4] = __ldcg(&st->tau_g_bits);
        s_state[5] = __ldcg(&st->gcand_count);
        s_state[6] = __ldcg(&st->bmax_g);
        s_state[7] = (unsigned)__ldcg(&st->iters);
    }
    unsigned long long tp[5] = {0, 0, 0, 0, 0};  // CTA 0, thread 0: phase clock
    if (cta0 && tid == 0) tp[0] = gtimer_ns();
    unsigned long long target = 0;
    if (tid == 0) target = barrier_base(a.gbar);
    int st_bt = 0, st_sc = 0, st_iters = 0, st_status = 0, st_fsel = 0;
    if (cta0 && tid == 0) {
        st_bt = st->backtracks_total;
        st_sc = st->support_changes_total;
        st_iters = st->iters;
        st_status = st->status;
        st_fsel = st->full_selects;
    }
    // G, x_G, g_G in support order and the first candidates, requested before the state
    // is known (s <= 2 x 512; the candidate list has room for 512 reads)
    int jq[2] = {0, 0};
    float xq[2] = {0.0f, 0.0f}, gq[2] = {0.0f, 0.0f};
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int q = tid + u * kIterThreads;
        if (q < s) {
            jq[u] = __ldcg(a.support + q);
            xq[u] = __ldcg(a.xs + q);
            gq[u] = __ldcg(a.gsup + q);
        }
    }
    unsigned long long cspec = 0;
    if (tid < a.gcap) cspec = __ldcg(a.gcand + tid);
    const float rrow = row_ok ? __ldcg(a.r + row) : 0.0f;       // this thread's row of r
    __syncthreads();
    if (s_state[0]) return;                      // uniform: read before any exchange
    const int iter0 = (int)s_state[1];
    const unsigned omega_uses = s_state[2];
    const unsigned dec_uses = s_state[3];
    const uint32_t tau_g = s_state[4];
    const unsigned ncand = s_state[5];
    const uint32_t bmax_g = s_state[6];
    const bool first = iter0 == 0;              // the gradient kernel has not filtered yet
    const bool cand_ok = !first && tau_g != 0u && ncand <= (unsigned)a.gcap;
    const int cnt = cand_ok ? (int)ncand : 0;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int q = tid + u * kIterThreads;
        if (q < s) {
            sm.el_idx[q] = jq[u];
            // first iteration: x and g through G (x_G, g_G are not kept in support order yet)
            sm.el_x[q] = first ? __ldcg(a.x + jq[u]) : xq[u];
            sm.el_g[q] = first ? __ldcg(a.g + jq[u]) : gq[u];
        }
    }
    for (int i = tid; i < cnt; i += blockDim.x) {
        const unsigned long long c = i == tid ? cspec : __ldcg(a.gcand + i);
        sm.el_idx[s + i] = (int)(uint32_t)c;
        sm.el_x[s + i] = 0.0f;
        sm.el_g[s + i] = __uint_as_float((uint32_t)(c >> 32));
    }
    __syncthreads();
    const float alpha_f = s_alpha_f;
    const unsigned tag = (unsigned)iter0 & 1u;  // step-size and residual slots: once per iteration

    // ---- Mu: z = Q2_G g_G, den = alpha^2 ||z||^2, num = ||g_G||^2 (CTA 0's warp 0) ----
    double num = 0.0;                            // CTA 0, warp 0
    // QIHT_MU_CROSS: also z1 = Q1_G g_G; the CTA's part of z1 . z travels as its positive and
    // negative parts (tagged slots carry non-negative values) in slots 1 and 3
    const bool cross = a.mu_mode == QIHT_MU_CROSS;
    // this thread's row of Q2_G g_G and of the last backtracking product Q2 (x' - x): the
    // residual update r <- r - alpha Q2 (x' - x) uses one of them
    float zmu = 0.0f, zom = 0.0f;
    {
        if (cta0 && tid < 32) {
            for (int q = lane; q < s; q += 32) num += (double)sm.el_g[q] * (double)sm.el_g[q];
            num = warp_sum_d(num);
        }
        float z1v = 0.0f;
        if (cross) {
            rows_product_sm<BITS>(a, rb, sm.el_idx, sm.el_g, s, sm.red, sm.zrow, a.q1_words);
            if (row_ok) z1v = sm.zrow[tid];
        }
        rows_product_sm<BITS>(a, rb, sm.el_idx, sm.el_g, s, sm.red, sm.zrow);
        double acc = 0.0;
        if (row_ok) {
            zmu = sm.zrow[tid];
            acc = (double)zmu * (double)zmu;
        }
        acc = cta_sum_n(acc, nrow_thr, shd);
        if (cross) {
            double cp = row_ok ? (double)z1v * (double)sm.zrow[tid] : 0.0;
            cp = cta_sum_n(cp, nrow_thr, shd);
            if (tid == 0) {
                slot_put(mypart + 1 * kSlotCtas, cp > 0.0 ? cp : 0.0, tag);
                slot_put(mypart + 3 * kSlotCtas, cp < 0.0 ? -cp : 0.0, tag);
            }
        }
        if (tid == 0) slot_put(mypart + 0 * kSlotCtas, acc, tag);
    }
    // CTA 0 gathers the partials and publishes mu (code 1: stop); the others wait for it
    double mu = 0.0;                             // meaningful in CTA 0's thread 0
    unsigned dec_use = dec_uses;                 // uses of the decision word so far
    {
        unsigned code = 0;
        float muf = 0.0f;
        if (cta0) {
            double densum = 0.0, cpos = 0.0, cneg = 0.0;
            if (!slot_gather(a.part, 0, -1, -1, tag, &densum, nullptr, nullptr, st, a.report, shd)) return;
            if (cross) {
                if (!slot_gather(a.part, 1, -1, -1, tag, &cpos, nullptr, nullptr, st, a.report, shd)) return;
                if (!slot_gather(a.part, 3, -1, -1, tag, &cneg, nullptr, nullptr, st, a.report, shd)) return;
            }
            if (tid == 0) {
                tp[1] = gtimer_ns();
                const double den_f = s_alpha * s_alpha * densum;
                double den = den_f;
                if (cross) {
                    const double den_c = s_alpha * s_alpha * (cpos - cneg);
                    if (den_c > 0.0) den = den_c;              // else the forward square
                }
                if (!isfinite(num) || !isfinite(den_f)) {
                    code = 1;
                    st->status = QIHT_ERR_NONFINITE;
                } else if (num == 0.0 || den_f == 0.0) {
                    code = 1;                                  // converged: x stays
                } else {
                    mu = num / den;
                }
                muf = (float)mu;
                // test hook: withhold the first decision so that the other CTAs' waits run out
                if (!((a.flags & QIHT_SOLVE_TEST_TIMEOUT) && iter0 == 0)) dec_put(&st->dec_word, dec_use, code, muf);
                if (code) {
                    st->stop = 1;
                    if (a.report) {
                        a.report->iters_run = iter0;
                        a.report->backtracks = st_bt;
                        a.report->support_changes = st_sc;
                        a.report->status = st->status;
                        a.report->resid_norm2 = st->resid2;
                        a.report->mu = st->mu_accepted;
                    }
                }
                s_code = (int)code;
                s_muf = muf;
            }
            __syncthreads();
            code = (unsigned)s_code;
            muf = s_muf;
        } else {
            if (!dec_wait(&st->dec_word, dec_use, &code, &muf, st, a.report)) return;
            if (tid == 0) s_muf = muf;
        }
        ++dec_use;
        if (code) return;                                      // uniform across CTAs
        __syncthreads();
    }

    prefetch_next();
    int bt = 0, rounds = 0, full_here = 0;
    SelResult sr{};
    for (;;) {
        const float muf = s_muf;
        const uint32_t outside = __float_as_uint(fmaf(muf, __uint_as_float(bmax_g), 0.0f)) & 0x7fffffffu;
        const bool exact = cand_ok && select_fast(a, sm, s + cnt, muf, outside, sr);
        if (!exact) {
            // keys of all n entries, then the one-CTA radix select
            ++full_here;
            const int per = (n + gridDim.x - 1) / gridDim.x;
            const int j0 = min(n, (int)blockIdx.x * per), j1 = min(n, j0 + per);
            int bad = 0;
            for (int j = j0 + tid; j < j1; j += blockDim.x) {
                const uint32_t k = __float_as_uint(fmaf(muf, __ldcg(a.g + j), __ldcg(a.x + j))) & 0x7fffffffu;
                bad |= k > 0x7f800000u;
                a.keys[j] = k;
            }
            if (__syncthreads_or(bad) && tid == 0) st->status = QIHT_ERR_NONFINITE;
            if (!grid_sync(a.gbar, target, st, a.report)) return;
            if (__ldcg(&st->status) == QIHT_ERR_NONFINITE) {
                if (cta0 && tid == 0) st->stop = 1;
                return;
            }
            if (cta0) {
                SelSmem fs{};
                fs.hist = sm.key;                              // s + gcap >= 2048 entries
                fs.bitmap = sm.bitmap;
                fs.wpre = sm.wpre;
                fs.sup = sm.u_idx;
                select_on_cta0(a, muf, fs, false);
            }
            if (!grid_sync(a.gbar, target, st, a.report)) return;
            sr.changed = __ldcg(&st->changed);
            sr.uc = __ldcg(&st->union_count);
            sr.kth0 = __ldcg(&st->kth0);
            sr.kth1 = __ldcg(&st->kth1);
            for (int i = tid; i < sr.uc; i += blockDim.x) {
                sm.u_idx[i] = __ldcg(a.uni + i);
                sm.u_delta[i] = __ldcg(a.delta + i);
            }
            for (int q = tid; q < s; q += blockDim.x) sm.u_val[q] = __ldcg(a.val + q);
            for (int w = tid; w < nbw4; w += blockDim.x) sm.bitmap[w] = 0u;
            __syncthreads();
            for (int q = tid; q < s; q += blockDim.x) {
                const int j = sm.u_idx[q];
                atomicOr(&sm.bitmap[j >> 5], 1u << (j & 31));
            }
            __syncthreads();
        }
        if (cta0 && tid == 0 && bt == 0) tp[2] = gtimer_ns();
        if (!sr.changed) break;

        // ---- Omega: backtracking test on G' u G; CTA 0 decides, the others wait ----
        const unsigned otag = (omega_uses + (unsigned)rounds) & 1u;
        ++rounds;
        double dsq = 0.0;                                      // CTA 0, warp 0
        {
            if (cta0 && tid < 32) {
                for (int i = lane; i < sr.uc; i += 32) dsq += (double)sm.u_delta[i] * (double)sm.u_delta[i];
                dsq = warp_sum_d(dsq);
            }
            rows_product_sm<BITS>(a, rb, sm.u_idx, sm.u_delta, sr.uc, sm.red, sm.zrow);
            double acc = 0.0;
            if (row_ok) {
                zom = sm.zrow[tid];
                acc = (double)zom * (double)zom;
            }
            acc = cta_sum_n(acc, nrow_thr, shd);
            if (tid == 0) slot_put(mypart + 2 * kSlotCtas, acc, otag);
        }
        unsigned code = 0;                                     // 0 accept, 1 shrink, 2 give up
        float mnew = 0.0f;
        if (cta0) {
            double ddsum = 0.0;
            if (!slot_gather(a.part, 2, -1, -1, otag, &ddsum, nullptr, nullptr, st, a.report, shd)) return;
            if (tid == 0) {
                const double dd = s_alpha * s_alpha * ddsum;
                const double dn = dsq;
                if (dn > 0.0) {                                // else nothing moves: accept
                    const double omega = dd > 0.0 ? dn / dd : INFINITY;
                    if (!(mu <= (1.0 - a.c) * omega)) {        // insufficient decrease
                        if (bt >= a.max_bt) {
                            code = 2;
                            st->status = QIHT_ERR_BACKTRACK_CAP;
                            st->stop = 1;
                            if (a.report) {
                                a.report->iters_run = iter0;
                                a.report->backtracks = st_bt;
                                a.report->support_changes = st_sc;
                                a.report->status = QIHT_ERR_BACKTRACK_CAP;
                                a.report->resid_norm2 = st->resid2;
                                a.report->mu = st->mu_accepted;
                            }
                        } else {
                            code = 1;
                            mu = mu / (a.k * (1.0 - a.c));
                        }
                    }
                }
                mnew = (float)mu;
                dec_put(&st->dec_word, dec_use, code, mnew);
                s_code = (int)code;
                s_muf = mnew;
            }
            __syncthreads();
            code = (unsigned)s_code;
        } else {
            if (!dec_wait(&st->dec_word, dec_use, &code, &mnew, st, a.report)) return;
            if (tid == 0) s_muf = mnew;
        }
        ++dec_use;
        __syncthreads();
        if (code == 0) break;
        if (code == 2) return;
        ++bt;
    }

    // ---- CTA 0 commits G, x_G and the scalars (the next kernel records ||r||^2 from the
    // residual partials, so that no CTA waits for the others at the end) ----
    const int it = iter0 + 1;
    if (cta0) {
        for (int q = tid; q < s; q += blockDim.x) {
            a.support[q] = sm.u_idx[q];
            a.xs[q] = sm.u_val[q];
            if (a.trace.support) a.trace.support[(size_t)it * s + q] = sm.u_idx[q];
        }
        if (tid == 0) {
            tp[3] = gtimer_ns();
            const int bt_total = st_bt + bt;
            const int sc_total = st_sc + sr.changed;
            st->iter = it;
            st->omega_uses = omega_uses + (unsigned)rounds;
            st->dec_uses = dec_use;
            st->mu = mu;
            st->mu_accepted = mu;
            st->bt = bt;
            st->backtracks_total = bt_total;
            st->support_changes_total = sc_total;
            st->changed = sr.changed;
            st->kth0 = sr.kth0;
            st->kth1 = sr.kth1;
            // candidates of the next gradient: a little below the (s+1)-th key, in units of |g|
            const float tg = sr.kth1 > 0.0f ? 0.8f * sr.kth1 / (float)mu : 0.0f;
            st->tau_g_bits = (isfinite(tg) && tg > 0.0f) ? __float_as_uint(tg) : 0u;
            st->gcand_count = 0u;
            st->bmax_g = 0u;
            if (it >= st_iters) st->stop = 1;
            if (a.trace.kth) { a.trace.kth[2 * it] = sr.kth0; a.trace.kth[2 * it + 1] = sr.kth1; }
            if (a.trace.mu) a.trace.mu[it] = mu;
            if (a.trace.bt) a.trace.bt[it] = bt;
            if (a.report) {
                a.report->iters_run = it;
                a.report->backtracks = bt_total;
                a.report->support_changes = sc_total;
                a.report->status = st_status;
                a.report->mu = mu;
                a.report->full_selects = st_fsel + full_here;
                // phases (CTA 0's clock): step size, (filter: in the gradient kernel), select,
                // backtracking, commit, residual and this CTA's slices, whole kernel
                a.report->phase_us[0] = (float)(tp[1] - tp[0]) * 1e-3f;
                a.report->phase_us[1] = 0.0f;
                a.report->phase_us[2] = (float)(tp[2] - tp[1]) * 1e-3f;
                a.report->phase_us[3] = (float)(tp[3] - tp[2]) * 1e-3f;
            }
        }
    }

    // ---- Resid for this CTA's rows: directly, r = Q(y) - alpha Q2_G' x', in the first and
    // the last iteration, every kResidDirect-th, and when a residual tolerance is set;
    // otherwise r <- r - alpha Q2 (x' - x) with the product this iteration already formed:
    // mu Q2_G g_G when the support stayed, the accepted backtracking test's Q2 (x' - x) when
    // it moved (the same vector up to FP32 rounding; the direct form resets the drift) ----
    const bool direct = first || (it % kResidDirect) == 0 || it >= (int)s_state[7] || a.tol > 0.0;
    if (direct) rows_product_sm<BITS>(a, rb, sm.u_idx, sm.u_val, s, sm.red, sm.zrow);
    {
        double acc = 0.0;
        unsigned mx = 0;
        if (row_ok) {
            const float ri = direct ? fmaf(-alpha_f, sm.zrow[tid], yrow)
                                    : fmaf(-alpha_f, sr.changed ? zom : s_muf * zmu, rrow);
            a.r[row] = ri;
            acc = (double)ri * (double)ri;
            mx = __float_as_uint(ri) & 0x7fffffffu;
        }
        acc = cta_sum_n(acc, nrow_thr, shd);
        mx = cta_max(mx, shu);
        if (tid == 0) {
            slot_put(mypart + kSlotResid * kSlotCtas, acc, tag);
            slot_put(mypart + kSlotRmax * kSlotCtas, (double)mx, tag);
        }
    }
    // ---- this CTA's slice of x and of the position map ----
    {
        const int per = (n + gridDim.x - 1) / gridDim.x;
        const int j0 = min(n, (int)blockIdx.x * per), j1 = min(n, j0 + per);
        for (int q = tid; q < s; q += blockDim.x) {
            if (sr.changed) {
                const int jo = sm.el_idx[q];
                if (jo >= j0 && jo < j1 && !((sm.bitmap[jo >> 5] >> (jo & 31)) & 1u)) {
                    a.x[jo] = 0.0f;
                    a.pos[jo] = -1;
                }
            }
            const int jn = sm.u_idx[q];
            if (jn >= j0 && jn < j1) {
                a.x[jn] = sm.u_val[q];
                if (sr.changed || first) a.pos[jn] = q;     // the initial support has no positions yet
            }
        }
    }
    if (cta0 && tid == 0 && a.report) {
        const unsigned long long t6 = gtimer_ns();
        a.report->phase_us[4] = (float)(t6 - tp[3]) * 1e-3f;
        a.report->phase_us[5] = 0.0f;
        a.report->phase_us[6] = (float)(t6 - tp[0]) * 1e-3f;
        a.report->phase_us[7] = 0.0f;
    }
}

static_assert(sizeof(IterArgs) <= kIterArgsMax, "iteration kernel arguments exceed their storage");
size_t iter_args_bytes() { return sizeof(IterArgs); }

static size_t iter_smem_bytes(int n, int bits);

void iter_node(const Codes& Q2, State* st, const float* g, float* x, int32_t* support, int32_t* sel, float* val,
               int32_t* uni, float* delta, const float* yhat, float* r, uint32_t* keys, unsigned long long* cand,
               double* part, const IterFastBufs& fb, int n, int m, int s, double k, double c, int max_bt,
               int flags, qiht_report* report, const qiht_trace& trace, cudaKernelNodeParams* p, void* argstore,
               void** argbuf, const uint32_t* q1_words, int mu_mode, double tol)
{
    static_assert(sizeof(IterArgs) <= kIterArgsMax, "iteration kernel arguments");
    IterArgs* a = reinterpret_cast<IterArgs*>(argstore);
    *a = IterArgs{};
    a->Q = Q2;
    a->st = st;
    a->g = g;
    a->x = x;
    a->support = support;
    a->sel = sel;
    a->val = val;
    a->uni = uni;
    a->delta = delta;
    a->yhat = yhat;
    a->r = r;
    a->keys = keys;
    a->cand = cand;
    a->cap = kTopCandCap;
    a->part = part;
    a->bar = &st->counters[0][0];
    a->gbar = &st->bar_count;
    a->cand_val = reinterpret_cast<float*>(cand + kTopCandCap);
    a->cand_x = reinterpret_cast<float*>(cand + kTopCandCap) + kTopCandCap;
    a->pos = fb.pos;
    a->xs = fb.xs;
    a->gsup = fb.gsup;
    a->gcand = fb.gcand;
    a->gcap = fb.gcap;
    a->n = n;
    a->m = m;
    a->s = s;
    a->k = k;
    a->c = c;
    a->max_bt = max_bt;
    a->flags = flags;
    a->report = report;
    a->trace = trace;
    a->q1_words = q1_words ? q1_words : Q2.words;
    a->mu_mode = mu_mode;
    a->tol = tol;
    argbuf[0] = a;
    const int G = 32 / Q2.bits;
    void* fn;
    size_t smem;
    if (iter_fast(s)) {
        fn = Q2.bits == 8 ? (void*)k_iter_fast<8> : Q2.bits == 4 ? (void*)k_iter_fast<4> : (void*)k_iter_fast<2>;
        smem = fast_smem_bytes(n, s, fb.gcap, G);
    } else {
        fn = Q2.bits == 8 ? (void*)k_iter<8> : Q2.bits == 4 ? (void*)k_iter<4> : (void*)k_iter<2>;
        smem = iter_smem_bytes(n, Q2.bits);
    }
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    p->func = fn;
    p->gridDim = dim3(iter_grid());
    p->blockDim = dim3(kIterThreads);
    p->sharedMemBytes = (unsigned)smem;
    p->kernelParams = argbuf;
    p->extra = nullptr;
}

static size_t iter_smem_bytes(int n, int bits)
{
    const int G = 32 / bits;
    const size_t gather = (size_t)kListChunk * 8 + (size_t)kIterThreads * G * 4 + (size_t)kIterThreads * 4;
    const size_t nbw = ((size_t)(n + 31) / 32 + 3) & ~(size_t)3;
    const size_t select = 2048 * 4 + 2 * nbw * 4 + (size_t)kTopCandCap * 16 + (size_t)kSupportSmem * 4;
    return gather > select ? gather : select;
}

bool iter_fast(int s)
{
    // QIHT_ITER=base selects k_iter (filter and select phases inside the kernel) for measurement
    static int v = -1;
    if (v < 0) {
        const char* e = getenv("QIHT_ITER");
        v = (e && e[0] == 'b') ? 0 : 1;
    }
    return v == 1 && s <= kFastMaxS;
}

int iter_grid()
{
    // one CTA per SM; the partial slots hold up to kSlotCtas CTAs
    static int g = -1;
    if (g < 0) {
        const int n = num_sms();
        g = n > kSlotCtas ? kSlotCtas : n;
    }
    return g;
}

}  // namespace qiht
