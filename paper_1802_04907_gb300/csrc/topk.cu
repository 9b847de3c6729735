// Hard threshold H_s (Eq. NIHT): keep the s entries of a = x + mu g of largest
// magnitude, ties broken by the lower index, exactly s entries.
//
// One CTA of 1024 threads. Keys are the float bits of |a| (monotone for
// non-negative floats) held in shared memory. A 3-pass MSB-first radix select
// (11/11/10-bit digits, warp-aggregated shared histograms) finds the s-th largest key T; an
// ordered compaction (two block scans) then emits every key > T plus the
// lowest-index keys == T, in ascending index order. In the solver the same CTA
// compares the new support G' with the current one and builds the list of
// x' - x over G' u G for the backtracking test (Section II-A).
#include "internal.cuh"

namespace qiht {

constexpr int kTopThreads = 1024;

__device__ __forceinline__ bool tid0() { return threadIdx.x == 0; }

// Exclusive block scan of one int per thread (thread order); returns the total in *total.
__device__ int block_excl_scan(int v, int* sh, int* total)
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
        int s = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0;
        int t = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        sh[lane] = t - s;            // exclusive prefix of warp totals
        if (lane == 31) sh[32] = t;  // grand total
    }
    __syncthreads();
    const int r = sh[w] + x - v;
    *total = sh[32];
    __syncthreads();
    return r;
}

// Candidate filter (many CTAs): keys |x + mu g| >= tau go to a short list. When
// the list holds at least s keys it contains every key >= the s-th largest, so the
// selection over the list is exact; otherwise the select falls back to all keys.
__global__ void __launch_bounds__(256) k_top_filter(TopArgs a)
{
    State* st = a.st;
    if (st->stop || st->tau_bits == 0u) return;
    const uint32_t tau = st->tau_bits;
    const float mu = (float)(*a.mu);
    const int lane = threadIdx.x & 31;
    unsigned below = 0;
    const int stride = gridDim.x * blockDim.x;
    for (int j0 = blockIdx.x * blockDim.x; j0 < a.n; j0 += stride) {
        const int j = j0 + threadIdx.x;
        uint32_t k = 0;
        if (j < a.n) {
            const float v = fmaf(mu, __ldcg(a.g + j), __ldcg(a.x + j));
            k = __float_as_uint(v) & 0x7fffffffu;
            if (k > 0x7f800000u) { st->status = QIHT_ERR_NONFINITE; st->stop = 1; }
        }
        const bool take = j < a.n && k >= tau;
        if (j < a.n && !take) below = max(below, k);
        const unsigned mask = __ballot_sync(0xffffffffu, take);
        if (mask) {
            unsigned base = 0;
            if (lane == __ffs(mask) - 1) base = atomicAdd(&st->cand_count, (unsigned)__popc(mask));
            base = __shfl_sync(0xffffffffu, base, __ffs(mask) - 1);
            if (take) {
                const unsigned slot = base + __popc(mask & ((1u << lane) - 1u));
                if (slot < (unsigned)a.cap) a.cand[slot] = ((unsigned long long)k << 32) | (unsigned long long)(~(uint32_t)j);
            }
        }
    }
    below = __reduce_max_sync(0xffffffffu, below);
    if (lane == 0 && below) atomicMax(&st->below_max, below);
}

// Radix select of the s-th largest of `cnt` keys in shared memory: digits of 11, 11
// and 10 bits, MSB first. Returns T; *need_out = how many keys equal to T belong
// to the top s (the others above T all do). Keys are strided over the threads.
__device__ uint32_t radix_select(const uint32_t* keys, int cnt, int s, unsigned* hist, int* sel_digit,
                                 int* sel_above, int* need_out)
{
    const int tid = threadIdx.x;
    uint32_t prefix = 0;
    int need = s;
    for (int pass = 0; pass < 3; ++pass) {
        const int shift = pass == 0 ? 21 : pass == 1 ? 10 : 0;
        const int width = pass == 2 ? 10 : 11;
        const uint32_t dmask = (1u << width) - 1u;
        const int nbins = 1 << width;
        for (int i = tid; i < nbins; i += kTopThreads) hist[i] = 0;
        __syncthreads();
        const int hi = shift + width;
#pragma unroll 4
        for (int j = tid; j < cnt; j += kTopThreads) {
            const uint32_t k = keys[j];
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
                    if (run + c >= need) { *sel_digit = bi; *sel_above = run; break; }
                    run += c;
                }
            }
        }
        __syncthreads();
        prefix |= (uint32_t)(*sel_digit) << shift;
        need -= *sel_above;
        __syncthreads();
    }
    *need_out = need;
    return prefix;
}

__global__ void __launch_bounds__(kTopThreads) k_top(TopArgs a)
{
    extern __shared__ uint32_t keys[];            // full path: n keys; fast path: cap keys + cap indices
    __shared__ unsigned hist[2048];
    __shared__ int scan_sh[33];
    __shared__ int sel_digit, sel_above;
    __shared__ unsigned red_u[32];
    __shared__ int s_flag;
    State* st = a.st;
    const int tid = threadIdx.x;
    if (a.h_bt && tid == 0) cudaGraphSetConditional((cudaGraphConditionalHandle)a.h_bt, 0u);
    if (st && st->stop) return;

    const int n = a.n, s = a.s;
    const float mu = a.mu ? (float)(*a.mu) : 1.0f;
    const int lane = tid & 31, warp = tid >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    uint32_t* bitmap = keys + ((n > 2 * a.cap) ? n : 2 * a.cap);   // n bits
    const int nbw = (n + 31) / 32;

    uint32_t T = 0;
    int need = 0, eq_total = 0;
    unsigned below = 0;
    bool fast = false;

    // ---- fast path: select among the filter's candidates ----
    if (st && a.cap > 0 && st->tau_bits != 0u) {
        const int cnt = (int)st->cand_count;
        if (cnt >= s && cnt <= a.cap) {
            uint32_t* ckey = keys;
            uint32_t* cidx = keys + a.cap;
            for (int i = tid; i < cnt; i += kTopThreads) {
                const unsigned long long v = __ldcg(a.cand + i);
                ckey[i] = (uint32_t)(v >> 32);
                cidx[i] = ~(uint32_t)v;
            }
            __syncthreads();
            T = radix_select(ckey, cnt, s, hist, &sel_digit, &sel_above, &need);
            int eq = 0;
            for (int i = tid; i < cnt; i += kTopThreads) {
                const uint32_t k = ckey[i];
                eq += (k == T);
                if (k < T) below = max(below, k);
            }
            {
                int v = eq;
#pragma unroll
                for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0) scan_sh[warp] = v;
                __syncthreads();
                if (tid == 0) {
                    int t = 0;
                    for (int w = 0; w < kTopThreads / 32; ++w) t += scan_sh[w];
                    s_flag = t;
                }
                __syncthreads();
                eq_total = s_flag;
                __syncthreads();
            }
            if (eq_total == need) {
                // every key > T and every key == T is selected: mark them, then emit in index order
                fast = true;
                for (int w = tid; w < nbw; w += kTopThreads) bitmap[w] = 0u;
                __syncthreads();
                for (int i = tid; i < cnt; i += kTopThreads) {
                    if (ckey[i] >= T) {
                        const uint32_t j = cidx[i];
                        atomicOr(&bitmap[j >> 5], 1u << (j & 31));
                    }
                }
                below = max(below, st->below_max);
            }
            __syncthreads();
        }
    }

    if (fast) {
        const int wpt = (nbw + kTopThreads - 1) / kTopThreads;
        const int w0 = min(nbw, tid * wpt), w1 = min(nbw, w0 + wpt);
        int c = 0;
        for (int w = w0; w < w1; ++w) c += __popc(bitmap[w]);
        int total;
        int pos = block_excl_scan(c, scan_sh, &total);
        for (int w = w0; w < w1; ++w) {
            uint32_t bits = bitmap[w];
            while (bits) {
                const int b = __ffs(bits) - 1;
                bits &= bits - 1;
                const int j = w * 32 + b;
                a.sel[pos] = j;
                if (a.val) {
                    const float x = a.x ? __ldcg(a.x + j) : 0.0f;
                    a.val[pos] = fmaf(mu, __ldcg(a.g + j), x);
                }
                ++pos;
            }
        }
    } else {
        // ---- full path: keys of all n entries ----
        int bad = 0;
#pragma unroll 8
        for (int j = tid; j < n; j += kTopThreads) {
            const float x = a.x ? __ldcg(a.x + j) : 0.0f;
            const float v = fmaf(mu, __ldcg(a.g + j), x);
            const uint32_t k = __float_as_uint(v) & 0x7fffffffu;
            bad |= (k > 0x7f800000u);
            keys[j] = k;
        }
        bad = __syncthreads_or(bad);
        if (bad && st) {
            if (tid == 0) { st->status = QIHT_ERR_NONFINITE; st->stop = 1; }
            return;
        }
        T = radix_select(keys, n, s, hist, &sel_digit, &sel_above, &need);

        // ordered compaction: warp w owns the contiguous segment [w*seg, (w+1)*seg) and walks it
        // 32 keys at a time (lane = key), so shared reads are conflict-free and order is kept
        const int seg = ((n + 32 * 32 - 1) / (32 * 32)) * 32;
        const int wb = min(n, warp * seg), we = min(n, wb + seg);
        int gt = 0, eq = 0;
        for (int b = wb; b < we; b += 32) {
            const int j = b + lane;
            const uint32_t k = (j < we) ? keys[j] : 0u;
            const bool in = j < we;
            gt += __popc(__ballot_sync(0xffffffffu, in && k > T));
            eq += __popc(__ballot_sync(0xffffffffu, in && k == T));
            if (in && k < T) below = max(below, k);
        }
        int eq_before_w = 0, pos_w = 0;
        {
            if (lane == 0) scan_sh[warp] = eq;
            __syncthreads();
            if (warp == 0) {
                const int v = scan_sh[lane];
                int incl = v;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                scan_sh[lane] = incl - v;
                if (lane == 31) scan_sh[32] = incl;
            }
            __syncthreads();
            eq_before_w = scan_sh[warp];
            eq_total = scan_sh[32];
            __syncthreads();
        }
        const int take_eq_w = max(0, min(eq, need - eq_before_w));
        {
            if (lane == 0) scan_sh[warp] = gt + take_eq_w;
            __syncthreads();
            if (warp == 0) {
                const int v = scan_sh[lane];
                int incl = v;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                scan_sh[lane] = incl - v;
            }
            __syncthreads();
            pos_w = scan_sh[warp];
            __syncthreads();
        }
        int pos = pos_w, erun = 0;
        for (int b = wb; b < we; b += 32) {
            const int j = b + lane;
            const bool in = j < we;
            const uint32_t k = in ? keys[j] : 0u;
            const unsigned meq = __ballot_sync(0xffffffffu, in && k == T);
            const int rank = erun + __popc(meq & lt_mask);
            const bool take = in && (k > T || (k == T && rank < take_eq_w));
            const unsigned mt = __ballot_sync(0xffffffffu, take);
            if (take) {
                const int p = pos + __popc(mt & lt_mask);
                a.sel[p] = j;
                if (a.val) {
                    const float x = a.x ? __ldcg(a.x + j) : 0.0f;
                    a.val[p] = fmaf(mu, __ldcg(a.g + j), x);
                }
            }
            pos += __popc(mt);
            erun += __popc(meq);
        }
    }

    // (s+1)-th largest key: T again if more keys equal T than were taken, else the largest key below T
    below = __reduce_max_sync(0xffffffffu, below);
    if (lane == 0) red_u[warp] = below;
    __syncthreads();
    float kth0 = __uint_as_float(T), kth1 = 0.0f;
    if (tid == 0) {
        unsigned bm = 0;
        for (int w = 0; w < kTopThreads / 32; ++w) bm = max(bm, red_u[w]);
        kth1 = (eq_total > need) ? __uint_as_float(T) : (s < n ? __uint_as_float(bm) : 0.0f);
        if (a.kth) { a.kth[0] = kth0; a.kth[1] = kth1; }
        if (st) {
            if (!fast) st->full_selects += 1;
            st->kth0 = kth0;
            st->kth1 = kth1;
            // next candidate threshold: a little below the current (s+1)-th magnitude
            st->tau_bits = (a.cap > 0 && kth1 > 0.0f) ? __float_as_uint(kth1 * 0.9375f) : 0u;
            st->cand_count = 0u;
            st->below_max = 0u;
        }
    }
    __syncthreads();   // a.sel / a.val visible to the whole CTA

    if (a.init) {
        // initial support (Algorithm 2 initialisation): G = supp H_s(Q1^T Q(y))
        for (int q = tid; q < s; q += kTopThreads) {
            const int j = a.sel[q];
            a.support_init[q] = j;
            if (a.trace.support) a.trace.support[q] = j;
        }
        if (tid == 0 && a.trace.kth) { a.trace.kth[0] = kth0; a.trace.kth[1] = kth1; }
        return;
    }
    if (!st) return;

    // compare G' with G (both ascending) and build the x' - x list over G' u G
    for (int w = tid; w < nbw; w += kTopThreads) bitmap[w] = 0u;
    __syncthreads();
    int diff = 0;
    for (int q = tid; q < s; q += kTopThreads) {
        const int j = a.sel[q];
        diff |= (j != __ldcg(a.support + q));
        atomicOr(&bitmap[j >> 5], 1u << (j & 31));
        a.uni[q] = j;
        a.delta[q] = a.val[q] - __ldcg(a.x + j);
    }
    diff = __syncthreads_or(diff);
    // old support entries not in G', in support order
    const int sper = (s + kTopThreads - 1) / kTopThreads;
    const int q0 = min(s, tid * sper), q1 = min(s, q0 + sper);
    int cntx = 0;
    for (int q = q0; q < q1; ++q) {
        const int j = __ldcg(a.support + q);
        cntx += !((bitmap[j >> 5] >> (j & 31)) & 1u);
    }
    int extra;
    int p = block_excl_scan(cntx, scan_sh, &extra);
    for (int q = q0; q < q1; ++q) {
        const int j = __ldcg(a.support + q);
        if (!((bitmap[j >> 5] >> (j & 31)) & 1u)) {
            a.uni[s + p] = j;
            a.delta[s + p] = -__ldcg(a.x + j);
            ++p;
        }
    }
    if (tid == 0) {
        st->changed = diff ? 1 : 0;
        st->union_count = s + extra;
    }
}

size_t top_smem_bytes(int n)
{
    const size_t base = (size_t)n > 2 * (size_t)kTopCandCap ? (size_t)n : 2 * (size_t)kTopCandCap;
    return base * 4 + (size_t)((n + 31) / 32) * 4;
}

static bool g_top_attr_set = false;

static void ensure_top_attr()
{
    if (!g_top_attr_set) {
        cudaFuncSetAttribute((const void*)k_top, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)top_smem_bytes(kMaxTopN));
        g_top_attr_set = true;
    }
}

void top_filter_node(const TopArgs& a, cudaKernelNodeParams* p, void** argbuf)
{
    int blocks = (a.n + 255) / 256;
    const int cap = num_sms() * 4;
    if (blocks > cap) blocks = cap;
    p->func = (void*)k_top_filter;
    p->gridDim = dim3(blocks < 1 ? 1 : blocks);
    p->blockDim = dim3(256);
    p->sharedMemBytes = 0;
    p->kernelParams = argbuf;
    p->extra = nullptr;
}

void top_node(const TopArgs& a, cudaKernelNodeParams* p, void** argbuf)
{
    ensure_top_attr();
    p->func = (void*)k_top;
    p->gridDim = dim3(1);
    p->blockDim = dim3(kTopThreads);
    p->sharedMemBytes = (unsigned)top_smem_bytes(a.n);
    p->kernelParams = argbuf;
    p->extra = nullptr;
}

cudaError_t launch_top(const TopArgs& a, cudaStream_t s)
{
    cudaKernelNodeParams p{};
    TopArgs copy = a;
    void* args[1] = {&copy};
    top_node(a, &p, args);
    return cudaLaunchKernel(p.func, p.gridDim, p.blockDim, args, p.sharedMemBytes, s);
}

}  // namespace qiht
