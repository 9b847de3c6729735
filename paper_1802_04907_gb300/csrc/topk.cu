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

__global__ void __launch_bounds__(kTopThreads) k_top(TopArgs a)
{
    extern __shared__ uint32_t keys[];            // n keys, then n/32 bitmap words
    __shared__ unsigned hist[2048];
    __shared__ int scan_sh[33];
    __shared__ int sel_digit, sel_above;
    __shared__ unsigned red_u[32];
    State* st = a.st;
    if (a.h_bt && tid0()) cudaGraphSetConditional((cudaGraphConditionalHandle)a.h_bt, 0u);
    if (st && st->stop) return;

    const int n = a.n, s = a.s;
    const int tid = threadIdx.x;
    const float mu = a.mu ? (float)(*a.mu) : 1.0f;

    // keys of |x + mu g| (strided: coalesced global reads, conflict-free shared writes)
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

    // radix select of the s-th largest key: digits of 11, 11 and 10 bits (MSB first).
    // Keys of similar magnitude share their top bits, so histogram updates are
    // aggregated per warp (__match_any_sync): one shared atomic per distinct bin.
    uint32_t prefix = 0;
    int need = s;
    for (int pass = 0; pass < 3; ++pass) {
        const int shift = pass == 0 ? 21 : pass == 1 ? 10 : 0;
        const int width = pass == 2 ? 10 : 11;
        const uint32_t dmask = (1u << width) - 1u;
        const int nbins = 1 << width;
        for (int i = tid; i < nbins; i += kTopThreads) hist[i] = 0;
        __syncthreads();
        const int hi = shift + width;             // bits above this digit must equal the prefix
#pragma unroll 4
        for (int j0 = 0; j0 < n; j0 += kTopThreads) {
            const int j = j0 + tid;
            int bin = -1;
            if (j < n) {
                const uint32_t k = keys[j];
                if (hi >= 32 || (k >> hi) == (prefix >> hi)) bin = (int)((k >> shift) & dmask);
            }
            const unsigned peers = __match_any_sync(0xffffffffu, bin);
            if (bin >= 0 && (__ffs(peers) - 1) == (tid & 31)) atomicAdd(&hist[bin], (unsigned)__popc(peers));
        }
        __syncthreads();
        if (tid < 32) {
            // lane l holds bins nbins-1-l*per .. (descending), per = nbins / 32
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
                    if (run + c >= need) { sel_digit = bi; sel_above = run; break; }
                    run += c;
                }
            }
        }
        __syncthreads();
        prefix |= (uint32_t)sel_digit << shift;
        need -= sel_above;
        __syncthreads();
    }
    const uint32_t T = prefix;    // s-th largest key; take `need` of the keys equal to T

    // ordered compaction: warp w owns the contiguous segment [w*seg, (w+1)*seg) and walks it
    // 32 keys at a time (lane = key), so shared reads are conflict-free and order is kept
    const int lane = tid & 31, warp = tid >> 5;
    const int seg = ((n + 32 * 32 - 1) / (32 * 32)) * 32;
    const int wb = min(n, warp * seg), we = min(n, wb + seg);
    const unsigned lt_mask = (1u << lane) - 1u;
    int gt = 0, eq = 0;
    unsigned below = 0;
    for (int b = wb; b < we; b += 32) {
        const int j = b + lane;
        const uint32_t k = (j < we) ? keys[j] : 0u;
        const bool in = j < we;
        gt += __popc(__ballot_sync(0xffffffffu, in && k > T));
        eq += __popc(__ballot_sync(0xffffffffu, in && k == T));
        if (in && k < T) below = max(below, k);
    }
    int eq_before_w = 0, eq_total = 0, pos_w = 0;
    {
        // scans over the 32 warp totals (warp order = index order)
        if (lane == 0) { scan_sh[warp] = eq; }
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
            if (lane == 31) scan_sh[32] = incl;
        }
        __syncthreads();
        pos_w = scan_sh[warp];
        __syncthreads();
    }
    {
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
        if (st) { st->kth0 = kth0; st->kth1 = kth1; }
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
    uint32_t* bitmap = keys + n;                  // n/32 words (keys no longer needed)
    const int nbw = (n + 31) / 32;
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
    int cnt = 0;
    for (int q = q0; q < q1; ++q) {
        const int j = __ldcg(a.support + q);
        cnt += !((bitmap[j >> 5] >> (j & 31)) & 1u);
    }
    int extra;
    int p = block_excl_scan(cnt, scan_sh, &extra);
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

size_t top_smem_bytes(int n) { return (size_t)n * 4 + (size_t)((n + 31) / 32) * 4; }

static bool g_top_attr_set = false;

static void ensure_top_attr()
{
    if (!g_top_attr_set) {
        cudaFuncSetAttribute((const void*)k_top, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)top_smem_bytes(kMaxTopN));
        g_top_attr_set = true;
    }
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
