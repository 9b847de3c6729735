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
constexpr int kListChunk = 1024;                          // list entries staged in shared memory at once
constexpr unsigned long long kBarrierBudgetNs = 200ull * 1000 * 1000;

__device__ __forceinline__ unsigned long long gtimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void st_release(unsigned* p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid barrier without contended atomics: CTA c release-stores the barrier's epoch in
// its own flag; CTA 0 acquires every flag (in parallel) and then releases the epoch in
// the generation word, which every CTA acquires. Epochs only grow (wrap-safe
// comparisons), so flags never need resetting. Waiting is bounded by %globaltimer;
// a timeout marks the state and returns false.
__device__ bool grid_sync(unsigned* flags, unsigned* gen, unsigned& epoch, State* st)
{
    __shared__ int ok_sh;
    ++epoch;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        st_release(flags + blockIdx.x, epoch);
        ok_sh = 1;
    }
    __syncthreads();
    if (blockIdx.x == 0) {
        int ok = 1;
        for (int c = threadIdx.x; c < (int)gridDim.x; c += blockDim.x) {
            if ((int)(ld_acquire(flags + c) - epoch) < 0) {
                const unsigned long long t0 = gtimer_ns();
                while ((int)(ld_acquire(flags + c) - epoch) < 0) {
                    if (gtimer_ns() - t0 > kBarrierBudgetNs) { ok = 0; break; }
                }
            }
        }
        ok = __syncthreads_and(ok);
        if (threadIdx.x == 0) {
            if (ok) {
                __threadfence();
                st_release(gen, epoch);
            } else {
                st->status = QIHT_ERR_TIMEOUT;
                st->stop = 1;
                ok_sh = 0;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && ok_sh) {
        if ((int)(ld_acquire(gen) - epoch) < 0) {
            const unsigned long long t0 = gtimer_ns();
            while ((int)(ld_acquire(gen) - epoch) < 0) {
                if (gtimer_ns() - t0 > kBarrierBudgetNs) {
                    ok_sh = 0;
                    st->status = QIHT_ERR_TIMEOUT;
                    st->stop = 1;
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok_sh != 0;
}

// Deterministic sum of one double per thread (fixed shuffle tree, warps in order).
__device__ double cta_sum(double v, double* sh)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sh[i];
        sh[32] = t;
    }
    __syncthreads();
    const double r = sh[32];
    __syncthreads();
    return r;
}

__device__ unsigned cta_max(unsigned v, unsigned* sh)
{
    v = __reduce_max_sync(0xffffffffu, v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t = max(t, sh[i]);
        sh[32] = t;
    }
    __syncthreads();
    const unsigned r = sh[32];
    __syncthreads();
    return r;
}

// Sum over CTAs of partial slot `k` of the per-CTA partials (every CTA gets the same value).
__device__ double grid_partial_sum(const double* part, int k, double* sh)
{
    double v = 0.0;
    for (int c = threadIdx.x; c < (int)gridDim.x; c += blockDim.x) v += __ldcg(part + 4 * c + k);
    return cta_sum(v, sh);
}

__device__ double grid_partial_max(const double* part, int k, double* sh)
{
    double v = 0.0;
    for (int c = threadIdx.x; c < (int)gridDim.x; c += blockDim.x) v = fmax(v, __ldcg(part + 4 * c + k));
#pragma unroll
    for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t = fmax(t, sh[i]);
        sh[32] = t;
    }
    __syncthreads();
    const double r = sh[32];
    __syncthreads();
    return r;
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
    double* part;               // [grid][4] per-CTA partials
    unsigned* bar;              // [0] generation of the grid barrier, [2] commit counter
    unsigned* flags;            // [grid] barrier epoch of every CTA
    float* cand_val;            // x + mu g of each candidate (same slot as cand)
    float* cand_x;              // x of each candidate
    int n, m, s;
    double k, c;
    int max_bt;
    qiht_report* report;
    qiht_trace trace;
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

// z (for this CTA's rows) = sum over the list of coef_j * code column j, in list order
// per slice and slices in order; the result stays in red[t*G + k] of the reducer threads:
// row word wl = t / G, row in word k = t % G, valid for t < wpc*G.
// coef_mode: 0 = coef[jj], 1 = g[list[jj]].
template <int BITS>
__device__ void rows_product(const IterArgs& a, const RowBlock& rb, const int32_t* list, const float* coef,
                             int coef_mode, int count, int32_t* s_list, float* s_coef, float* red, float* zrow,
                             double* coef_sq = nullptr)
{
    constexpr int G = 32 / BITS;
    constexpr int L = 1 << BITS;
    const int t = threadIdx.x;
    const int wl = t % rb.wpc, sl = t / rb.wpc;
    const int q = rb.w0 + wl;
    const bool active = sl < rb.nsl && q < rb.w1;
    const int ld = a.Q.ld;
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
        if (active) {
            int jj = sl;
            for (; jj + 3 * rb.nsl < cn; jj += 4 * rb.nsl) {
                uint32_t w[4];
                float cf[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    w[u] = __ldg(a.Q.words + (size_t)s_list[jj + u * rb.nsl] * ld + q);
                    cf[u] = s_coef[jj + u * rb.nsl];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int k = 0; k < G; ++k) {
                        const int code = (int)((w[u] >> (8 * (k & 3) + BITS * (k >> 2))) & (uint32_t)(L - 1));
                        z[k] = fmaf((float)(2 * code - (L - 1)), cf[u], z[k]);
                    }
            }
            for (; jj < cn; jj += rb.nsl) {
                const uint32_t w = __ldg(a.Q.words + (size_t)s_list[jj] * ld + q);
                const float cf = s_coef[jj];
#pragma unroll
                for (int k = 0; k < G; ++k) {
                    const int code = (int)((w >> (8 * (k & 3) + BITS * (k >> 2))) & (uint32_t)(L - 1));
                    z[k] = fmaf((float)(2 * code - (L - 1)), cf, z[k]);
                }
            }
        }
    }
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

__device__ void select_on_cta0(const IterArgs& a, float mu, unsigned char* smem)
{
    State* st = a.st;
    const int n = a.n, s = a.s, tid = threadIdx.x;
    const int lane = tid & 31;
    const int nbw = (n + 31) / 32;
    const int nbw4 = (nbw + 3) & ~3;
    unsigned* hist = reinterpret_cast<unsigned*>(smem);                       // 2048
    uint32_t* bitmap = hist + 2048;                                           // nbw4
    int* wpre = reinterpret_cast<int*>(bitmap + nbw4);                        // nbw4: selected before word w
    unsigned long long* cv = reinterpret_cast<unsigned long long*>(wpre + nbw4);   // cap
    float* cval = reinterpret_cast<float*>(cv + a.cap);                       // cap
    float* cx = cval + a.cap;                                                 // cap
    int32_t* sup = reinterpret_cast<int32_t*>(cx + a.cap);                    // s (if it fits)
    const bool sup_sm = s <= kSupportSmem;
    __shared__ int sh_i[36];
    __shared__ unsigned sh_u[33];
    __shared__ unsigned long long sh_k[2];

    const int cnt = (int)__ldcg(&st->cand_count);
    const unsigned below_filter = __ldcg(&st->below_max);
    const bool use_rank = a.cap > 0 && __ldcg(&st->tau_bits) != 0u && cnt >= s && cnt <= min(a.cap, kRankMax);
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
    constexpr int L = 1 << BITS;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double shd[33];
    __shared__ unsigned shu[33];
    State* st = a.st;
    if (st->stop) return;                       // uniform: read before any barrier
    const bool stamp = blockIdx.x == 0 && threadIdx.x == 0;
    if (stamp) st->t_phase[0] = gtimer_ns();
    // barrier epochs continue from the generation left by the previous launch; no CTA can
    // move it on before every CTA has arrived at the first barrier, so all read the same value
    unsigned epoch = ld_acquire(a.bar);

    const RowBlock rb = row_block(a.Q.ld);
    int32_t* s_list = reinterpret_cast<int32_t*>(smem);
    float* s_coef = reinterpret_cast<float*>(s_list + kListChunk);
    float* red = s_coef + kListChunk;                           // kIterThreads * G
    float* zrow = red + kIterThreads * G;                       // kIterThreads
    unsigned char* sel_smem = smem;                             // CTA 0's select reuses the buffer
    const double alpha = (double)(*a.Q.scale) / (double)(L - 1);
    const float alpha_f = (float)alpha;
    const int m = a.m, s = a.s, n = a.n;
    const int tid = threadIdx.x;
    double* mypart = a.part + 4 * blockIdx.x;

    // ---- Mu: z = Q2_G g_G, den = alpha^2 ||z||^2, num = ||g_G||^2 ----
    double gsq = 0.0;
    rows_product<BITS>(a, rb, a.support, nullptr, 1, s, s_list, s_coef, red, zrow, &gsq);
    {
        double acc = 0.0;
        if (tid < rb.wpc * G) {
            const int row = (rb.w0 + tid / G) * G + tid % G;
            if (rb.w0 + tid / G < rb.w1 && row < m) acc = (double)zrow[tid] * (double)zrow[tid];
        }
        acc = cta_sum(acc, shd);
        const double num = cta_sum(gsq, shd);                // ||g_G||^2 from the staged coefficients
        if (tid == 0) { mypart[0] = acc; mypart[1] = num; }
    }
    if (!grid_sync(a.flags, a.bar, epoch, st)) return;
    if (stamp) st->t_phase[1] = gtimer_ns();
    double mu;
    {
        const double den = alpha * alpha * grid_partial_sum(a.part, 0, shd);
        const double num = __ldcg(a.part + 1);                 // CTA 0's slot
        bool stop = false;
        if (!isfinite(num) || !isfinite(den)) {
            stop = true;
            if (blockIdx.x == 0 && tid == 0) st->status = QIHT_ERR_NONFINITE;
        } else if (num == 0.0 || den == 0.0) {
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
        if (!grid_sync(a.flags, a.bar, epoch, st)) return;
        if (stamp) st->t_phase[2] = gtimer_ns();
        if (__ldcg(&st->status) == QIHT_ERR_NONFINITE) {
            if (blockIdx.x == 0 && tid == 0) st->stop = 1;
            return;
        }
        // ---- Select on CTA 0 ----
        if (blockIdx.x == 0) select_on_cta0(a, (float)mu, sel_smem);
        if (!grid_sync(a.flags, a.bar, epoch, st)) return;
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
            if (tid == 0) { mypart[2] = acc; mypart[3] = dn; }
        }
        if (!grid_sync(a.flags, a.bar, epoch, st)) return;
        const double dd = alpha * alpha * grid_partial_sum(a.part, 2, shd);
        const double dn = __ldcg(a.part + 3);
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
                const float ri = fmaf(-alpha_f, zrow[tid], __ldcg(a.yhat + row));
                a.r[row] = ri;
                acc = (double)ri * (double)ri;
                mx = __float_as_uint(ri) & 0x7fffffffu;
            }
        }
        acc = cta_sum(acc, shd);
        mx = cta_max(mx, shu);
        if (tid == 0) { mypart[0] = acc; mypart[1] = (double)mx; }
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

static_assert(sizeof(IterArgs) <= kIterArgsMax, "iteration kernel arguments exceed their storage");
size_t iter_args_bytes() { return sizeof(IterArgs); }

void iter_node(const Codes& Q2, State* st, const float* g, float* x, int32_t* support, int32_t* sel, float* val,
               int32_t* uni, float* delta, const float* yhat, float* r, uint32_t* keys, unsigned long long* cand,
               double* part, int n, int m, int s, double k, double c, int max_bt, qiht_report* report,
               const qiht_trace& trace, cudaKernelNodeParams* p, void* argstore, void** argbuf)
{
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
    a->flags = &st->counters[1][0];
    a->cand_val = reinterpret_cast<float*>(cand + kTopCandCap);
    a->cand_x = reinterpret_cast<float*>(cand + kTopCandCap) + kTopCandCap;
    a->n = n;
    a->m = m;
    a->s = s;
    a->k = k;
    a->c = c;
    a->max_bt = max_bt;
    a->report = report;
    a->trace = trace;
    argbuf[0] = a;
    void* fn = Q2.bits == 8 ? (void*)k_iter<8> : Q2.bits == 4 ? (void*)k_iter<4> : (void*)k_iter<2>;
    const size_t smem = iter_smem_bytes(n, Q2.bits);
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    p->func = fn;
    p->gridDim = dim3(iter_grid());
    p->blockDim = dim3(kIterThreads);
    p->sharedMemBytes = (unsigned)smem;
    p->kernelParams = argbuf;
    p->extra = nullptr;
}

size_t iter_smem_bytes(int n, int bits)
{
    const int G = 32 / bits;
    const size_t gather = (size_t)kListChunk * 8 + (size_t)kIterThreads * G * 4 + (size_t)kIterThreads * 4;
    const size_t nbw = ((size_t)(n + 31) / 32 + 3) & ~(size_t)3;
    const size_t select = 2048 * 4 + 2 * nbw * 4 + (size_t)kTopCandCap * 16 + (size_t)kSupportSmem * 4;
    return gather > select ? gather : select;
}

int iter_grid()
{
    // QIHT_ITER_GRID overrides the number of CTAs (for measurement); default one per SM
    static int g = -1;
    if (g < 0) {
        int n = num_sms();
        const char* e = getenv("QIHT_ITER_GRID");
        if (e && atoi(e) > 0 && atoi(e) < n) n = atoi(e);
        g = n > 1024 ? 1024 : n;
    }
    return g;
}

}  // namespace qiht
