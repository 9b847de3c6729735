// H_s (Eq. NIHT) over more keys than one CTA's shared memory holds: a multi-CTA radix select.
//
// The keys are the binary32 magnitudes |fmaf(mu, g_j, x_j)| as unsigned integers (monotone
// for finite values). The threshold key T (the s-th largest) is found one digit at a time,
// most significant first (digits of 11, 11 and 10 bits): a grid-wide histogram of the digit
// among the keys that share the digits chosen so far, then one CTA picks the digit where the
// count from the top reaches the number still wanted. The selection is then every key above T
// and, among the keys equal to T, the ones of lowest index, as many as are still wanted
// (ties to the lower index, exactly s kept): chunks of the index range count their keys above
// and equal to T, one CTA scans the counts, and every chunk writes its selected indices in
// ascending order at its offset. kth = (T, the largest key below T, or T when the keys equal to
// T are not all taken).
#include "internal.cuh"

namespace qiht {
namespace {

constexpr int kBsThreads = 256;
constexpr int kBsChunk = kBsThreads * 16;          // indices per chunk of the final passes
constexpr int kBsBins = 2048;

struct BsInfo {
    unsigned prefix;     // digits chosen so far
    unsigned need;       // keys still wanted among those sharing the prefix
    unsigned above;      // keys above the prefix's range (all selected)
    unsigned eq_total;   // keys equal to T (after the last level)
    unsigned below_max;  // largest key below T
};

__device__ __forceinline__ uint32_t bs_key(const float* g, const float* x, float muf, int j)
{
    const float v = x ? fmaf(muf, __ldg(g + j), __ldg(x + j)) : __ldg(g + j);
    return __float_as_uint(v) & 0x7fffffffu;
}

// level 0 writes the keys; every level histograms its digit among the keys matching the prefix
__global__ void __launch_bounds__(kBsThreads) k_bs_hist(const float* __restrict__ g, const float* __restrict__ x,
                                                        const double* __restrict__ mu, int n, uint32_t* __restrict__ keys,
                                                        const BsInfo* __restrict__ info, int level,
                                                        unsigned* __restrict__ hist)
{
    __shared__ unsigned h[kBsBins];
    for (int b = threadIdx.x; b < kBsBins; b += kBsThreads) h[b] = 0u;
    __syncthreads();
    const float muf = mu ? (float)*mu : 1.0f;
    const int shift = level == 0 ? 21 : level == 1 ? 10 : 0;
    const unsigned mask = level == 2 ? 1023u : 2047u;
    const unsigned prefix = level == 0 ? 0u : info->prefix;
    const int pshift = shift + (level == 2 ? 10 : 11);              // bits above this digit
    for (int j = blockIdx.x * kBsThreads + threadIdx.x; j < n; j += gridDim.x * kBsThreads) {
        uint32_t k;
        if (level == 0) {
            k = bs_key(g, x, muf, j);
            keys[j] = k;
        } else {
            k = keys[j];
            if ((k >> pshift) != prefix) continue;
        }
        atomicAdd(&h[(k >> shift) & mask], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kBsBins; b += kBsThreads)
        if (h[b]) atomicAdd(&hist[b], h[b]);
}

// one CTA: the digit where the count from the top reaches `need`; clears the histogram
__global__ void __launch_bounds__(1024) k_bs_pick(unsigned* __restrict__ hist, BsInfo* __restrict__ info, int level,
                                                  int s)
{
    __shared__ unsigned suf[kBsBins + 1];
    const int nb = level == 2 ? 1024 : 2048;
    const unsigned need = level == 0 ? (unsigned)s : info->need;
    // suffix sums from the top digit down (sequential per thread over two bins, then a scan)
    for (int b = threadIdx.x; b < nb; b += 1024) suf[b] = hist[b];
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned acc = 0;
        suf[nb] = 0;
        for (int b = nb - 1; b >= 0; --b) {
            acc += suf[b];
            suf[b] = acc;                                            // keys with digit >= b
        }
        int d = 0;
        for (int b = nb - 1; b >= 0; --b)
            if (suf[b] >= need) { d = b; break; }
        const unsigned higher = suf[d + 1 <= nb - 1 ? d + 1 : nb];   // keys with digit > d
        BsInfo v = level == 0 ? BsInfo{0u, (unsigned)s, 0u, 0u, 0u} : *info;
        v.prefix = (v.prefix << (level == 2 ? 10 : 11)) | (unsigned)d;
        v.above += higher;
        v.need = need - higher;
        if (level == 2) v.eq_total = suf[d] - higher;
        *info = v;
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kBsBins; b += 1024) hist[b] = 0u;
}

// per chunk of the index range: keys above T and equal to T; the largest key below T
__global__ void __launch_bounds__(kBsThreads) k_bs_count(const uint32_t* __restrict__ keys, int n,
                                                         BsInfo* __restrict__ info, unsigned* __restrict__ cnt)
{
    const uint32_t T = info->prefix;
    const int nch = (n + kBsChunk - 1) / kBsChunk;
    __shared__ unsigned s_gt[kBsThreads / 32], s_eq[kBsThreads / 32], s_mx[kBsThreads / 32];
    for (int c = blockIdx.x; c < nch; c += gridDim.x) {
        unsigned gt = 0, eq = 0, mx = 0;
        const int j0 = c * kBsChunk, j1 = min(n, j0 + kBsChunk);
        for (int j = j0 + threadIdx.x; j < j1; j += kBsThreads) {
            const uint32_t k = keys[j];
            gt += k > T;
            eq += k == T;
            if (k < T) mx = max(mx, k);
        }
        gt = __reduce_add_sync(0xffffffffu, gt);
        eq = __reduce_add_sync(0xffffffffu, eq);
        mx = __reduce_max_sync(0xffffffffu, mx);
        if ((threadIdx.x & 31) == 0) {
            s_gt[threadIdx.x >> 5] = gt;
            s_eq[threadIdx.x >> 5] = eq;
            s_mx[threadIdx.x >> 5] = mx;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned a = 0, b = 0, m = 0;
            for (int w = 0; w < kBsThreads / 32; ++w) { a += s_gt[w]; b += s_eq[w]; m = max(m, s_mx[w]); }
            cnt[2 * c] = a;
            cnt[2 * c + 1] = b;
            if (m) atomicMax(&info->below_max, m);
        }
        __syncthreads();
    }
}

// one CTA: exclusive prefix counts over the chunks (in place)
__global__ void __launch_bounds__(1024) k_bs_scan(unsigned* __restrict__ cnt, int nch)
{
    if (threadIdx.x == 0) {
        unsigned a = 0, b = 0;
        for (int c = 0; c < nch; ++c) {
            const unsigned ga = cnt[2 * c], gb = cnt[2 * c + 1];
            cnt[2 * c] = a;
            cnt[2 * c + 1] = b;
            a += ga;
            b += gb;
        }
    }
}

// every chunk writes its selected indices (ascending) and the values fmaf(mu, g, x) at its offset
__global__ void __launch_bounds__(kBsThreads) k_bs_write(const uint32_t* __restrict__ keys, const float* __restrict__ g,
                                                         const float* __restrict__ x, const double* __restrict__ mu,
                                                         int n, const BsInfo* __restrict__ info,
                                                         const unsigned* __restrict__ cnt, int32_t* __restrict__ sel,
                                                         float* __restrict__ val, float* __restrict__ kth)
{
    const uint32_t T = info->prefix;
    const unsigned need = info->need;
    const float muf = mu ? (float)*mu : 1.0f;
    const int nch = (n + kBsChunk - 1) / kBsChunk;
    __shared__ unsigned s_w[kBsThreads / 32][2];
    __shared__ unsigned s_base[2];
    if (blockIdx.x == 0 && threadIdx.x == 0 && kth) {
        kth[0] = __uint_as_float(T);
        kth[1] = info->eq_total > need ? __uint_as_float(T) : __uint_as_float(info->below_max);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int c = blockIdx.x; c < nch; c += gridDim.x) {
        unsigned base_gt = cnt[2 * c], base_eq = cnt[2 * c + 1];
        const int j0 = c * kBsChunk, j1 = min(n, j0 + kBsChunk);
        // the chunk in rounds of kBsThreads consecutive indices, in index order
        for (int r0 = j0; r0 < j1; r0 += kBsThreads) {
            const int j = r0 + threadIdx.x;
            const uint32_t k = j < j1 ? keys[j] : 0u;
            const bool gt = j < j1 && k > T, eq = j < j1 && k == T;
            const unsigned bgt = __ballot_sync(0xffffffffu, gt), beq = __ballot_sync(0xffffffffu, eq);
            if (lane == 0) {
                s_w[warp][0] = __popc(bgt);
                s_w[warp][1] = __popc(beq);
            }
            __syncthreads();
            unsigned pgt = 0, peq = 0, tgt = 0, teq = 0;
            for (int w = 0; w < kBsThreads / 32; ++w) {
                if (w < warp) { pgt += s_w[w][0]; peq += s_w[w][1]; }
                tgt += s_w[w][0];
                teq += s_w[w][1];
            }
            const unsigned lt = (1u << lane) - 1u;
            const unsigned rgt = base_gt + pgt + __popc(bgt & lt);         // keys above T before j
            const unsigned req = base_eq + peq + __popc(beq & lt);         // keys equal to T before j
            const bool take = gt || (eq && req < need);
            if (take) {
                const unsigned pos = rgt + min(req, need);
                sel[pos] = j;
                if (val) val[pos] = x ? fmaf(muf, __ldg(g + j), __ldg(x + j)) : __ldg(g + j);
            }
            base_gt += tgt;
            base_eq += teq;
            __syncthreads();
        }
    }
}

}  // namespace

size_t big_top_workspace(int n)
{
    const size_t nch = ((size_t)n + kBsChunk - 1) / kBsChunk;
    return ((size_t)n * 4 + 255) / 256 * 256 + (size_t)kBsBins * 4 + 256 + (nch * 8 + 255) / 256 * 256;
}

cudaError_t launch_big_top(const float* g, const float* x, const double* mu, int n, int s, int32_t* sel, float* val,
                           float* kth, void* ws, cudaStream_t st)
{
    char* w = reinterpret_cast<char*>(ws);
    uint32_t* keys = reinterpret_cast<uint32_t*>(w);
    w += ((size_t)n * 4 + 255) / 256 * 256;
    unsigned* hist = reinterpret_cast<unsigned*>(w);
    w += (size_t)kBsBins * 4;
    BsInfo* info = reinterpret_cast<BsInfo*>(w);
    w += 256;
    unsigned* cnt = reinterpret_cast<unsigned*>(w);
    const int nch = (n + kBsChunk - 1) / kBsChunk;
    cudaError_t e = cudaMemsetAsync(hist, 0, (size_t)kBsBins * 4 + sizeof(BsInfo), st);
    if (e != cudaSuccess) return e;
    int grid = (n + kBsThreads * 8 - 1) / (kBsThreads * 8);
    const int cap = num_sms() * 4;
    if (grid > cap) grid = cap;
    if (grid < 1) grid = 1;
    for (int level = 0; level < 3; ++level) {
        k_bs_hist<<<grid, kBsThreads, 0, st>>>(g, x, mu, n, keys, info, level, hist);
        k_bs_pick<<<1, 1024, 0, st>>>(hist, info, level, s);
    }
    const int cgrid = nch < num_sms() * 4 ? nch : num_sms() * 4;
    k_bs_count<<<cgrid, kBsThreads, 0, st>>>(keys, n, info, cnt);
    k_bs_scan<<<1, 1024, 0, st>>>(cnt, nch);
    k_bs_write<<<cgrid, kBsThreads, 0, st>>>(keys, g, x, mu, n, info, cnt, sel, val, kth);
    return cudaGetLastError();
}

}  // namespace qiht
