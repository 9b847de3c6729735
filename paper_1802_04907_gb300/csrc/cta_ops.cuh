// Building blocks of one-CTA-per-problem kernels (1024 threads): deterministic CTA
// reductions, products with column subsets of a code matrix, and the hard threshold H_s
// over the keys of all n entries held in shared memory. Included by the translation units
// whose kernels solve one right-hand side or one problem per CTA.
#pragma once

#include "internal.cuh"

namespace qiht {
namespace cta {
namespace {                               // internal linkage in every including unit

constexpr int kST = 1024;                 // threads per CTA
// ssum, smax and sscan combine one partial per warp in warp 0 (lane w reads warp w's slot):
// every kernel that calls them runs kST threads, 32 warps
static_assert(kST == 1024, "the CTA reductions take one partial from each of 32 warps");
constexpr int kSW = kST / 32;

struct SSh {
    double d[34];
    int i[36];
    double mu, alpha1, alpha2, alpha_y;
    float muf, alpha2f;
    int code;
};

// Shared memory of one right-hand side.
struct MSm {
    uint32_t* keys;      // max(n, 16384): selection keys; scratch of the column products
    uint32_t* bitmap;    // n / 32: selected set
    uint32_t* gbit;      // n / 32: current support
    int* wpre;           // n / 32
    float* z;            // mk: column-subset product, then the residual
    int* sup;            // s: G (ascending)
    float* xs;           // s: x on G
    int* sel;            // s: G'
    float* val;          // s: x' on G'
    int* uni;            // 2s: G' then G \ G'
    float* dlt;          // 2s: x' - x on uni
    unsigned* hist;      // 256
};

__host__ __device__ inline size_t mrhs_keys_words(int n) { return (size_t)(n > 16384 ? n : 16384); }

__host__ __device__ inline size_t mrhs_step_smem_bytes(int n, int mk, int s)
{
    const size_t nb = (size_t)(n + 31) / 32;
    return mrhs_keys_words(n) * 4 + 3 * nb * 4 + (size_t)mk * 4 + (size_t)s * 4 * 4 + (size_t)s * 2 * 4 * 2 +
           256 * 4 + 64;
}

__host__ __device__ inline size_t msm_bytes(int n, int mk, int s) { return mrhs_step_smem_bytes(n, mk, s); }

__device__ MSm msm_layout(unsigned char* p, int n, int mk, int s)
{
    const size_t nb = (size_t)(n + 31) / 32;
    MSm m;
    m.keys = reinterpret_cast<uint32_t*>(p);
    m.bitmap = m.keys + mrhs_keys_words(n);
    m.gbit = m.bitmap + nb;
    m.wpre = reinterpret_cast<int*>(m.gbit + nb);
    m.z = reinterpret_cast<float*>(m.wpre + nb);
    m.sup = reinterpret_cast<int*>(m.z + mk);
    m.xs = reinterpret_cast<float*>(m.sup + s);
    m.sel = reinterpret_cast<int*>(m.xs + s);
    m.val = reinterpret_cast<float*>(m.sel + s);
    m.uni = reinterpret_cast<int*>(m.val + s);
    m.dlt = reinterpret_cast<float*>(m.uni + 2 * s);
    m.hist = reinterpret_cast<unsigned*>(m.dlt + 2 * s);
    return m;
}

// ---- deterministic CTA reductions ----
__device__ double ssum(double v, double* sh)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        double t = sh[lane];
#pragma unroll
        for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) sh[32] = t;
    }
    __syncthreads();
    const double r = sh[32];
    __syncthreads();
    return r;
}

__device__ unsigned smax(unsigned v, int* sh)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    v = __reduce_max_sync(0xffffffffu, v);
    if (lane == 0) sh[w] = (int)v;
    __syncthreads();
    if (w == 0) {
        unsigned t = (unsigned)sh[lane];
        t = __reduce_max_sync(0xffffffffu, t);
        if (lane == 0) sh[32] = (int)t;
    }
    __syncthreads();
    const unsigned r = (unsigned)sh[32];
    __syncthreads();
    return r;
}

__device__ int sscan(int v, int* sh, int* total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        const int sv = sh[lane];
        int t = sv;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        sh[lane] = t - sv;
        if (lane == 31) sh[32] = t;
    }
    __syncthreads();
    const int r = sh[w] + x - v;
    *total = sh[32];
    __syncthreads();
    return r;
}

// z[0..m) = sum over the list (in list order) of coef_e * (2 c_{i, list_e} - (L-1)).
// Thread t takes 16-row group t % ngr of every column and the list entries of slice
// t / ngr; several slices are summed in slice order.
template <int BITS>
__device__ void mcols(const Codes& Q, const int* list, const float* coef, int count, float* z, float* part)
{
    constexpr int G = 32 / BITS;
    constexpr int WG = 16 / G;                // words per 16-row group
    constexpr uint32_t MASK = (1u << BITS) - 1;
    constexpr int kSU = BITS == 8 ? 4 : 8;    // list entries of a thread in flight (64 registers per thread)
    const int ld = Q.ld, m = Q.rows, lm1 = Q.lm1;
    const int ngr = ld / WG;                  // <= kST under the row limit
    const int nsl = kST / ngr;
    const int tid = threadIdx.x, gi = tid % ngr, sl = tid / ngr;
    float acc[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) acc[r] = 0.0f;
    if (sl < nsl) {
        const uint32_t* base = Q.words + (size_t)gi * WG;
        for (int e0 = sl; e0 < count; e0 += kSU * nsl) {
            uint32_t w[kSU][WG];
            float cf[kSU];
#pragma unroll
            for (int u = 0; u < kSU; ++u) {
                const int e = e0 + u * nsl;
                const bool in = e < count;
                const uint32_t* src = base + (size_t)(in ? list[e] : 0) * ld;
                if (WG == 4) {
                    const uint4 v = in ? __ldg(reinterpret_cast<const uint4*>(src)) : make_uint4(0, 0, 0, 0);
                    w[u][0] = v.x; w[u][WG > 1 ? 1 : 0] = v.y; w[u][WG > 2 ? 2 : 0] = v.z; w[u][WG > 3 ? 3 : 0] = v.w;
                } else if (WG == 2) {
                    const uint2 v = in ? __ldg(reinterpret_cast<const uint2*>(src)) : make_uint2(0, 0);
                    w[u][0] = v.x; w[u][WG > 1 ? 1 : 0] = v.y;
                } else {
                    w[u][0] = in ? __ldg(src) : 0u;
                }
                cf[u] = in ? coef[e] : 0.0f;          // past the end: exact zeros
            }
#pragma unroll
            for (int u = 0; u < kSU; ++u)
#pragma unroll
                for (int q = 0; q < WG; ++q)
#pragma unroll
                    for (int k = 0; k < G; ++k) {
                        const int code = (int)((w[u][q] >> (8 * (k & 3) + BITS * (k >> 2))) & MASK);
                        acc[q * G + k] = fmaf((float)(2 * code - lm1), cf[u], acc[q * G + k]);
                    }
        }
    }
    if (nsl == 1) {
        if (sl == 0)
#pragma unroll
            for (int r = 0; r < 16; ++r)
                if (gi * 16 + r < m) z[gi * 16 + r] = acc[r];
        __syncthreads();
        return;
    }
    if (sl < nsl)
#pragma unroll
        for (int r = 0; r < 16; ++r) part[(sl * ngr + gi) * 16 + r] = acc[r];
    __syncthreads();
    for (int i = tid; i < m; i += kST) {
        const int g2 = i / 16, r = i % 16;
        float a = 0.0f;
        for (int t = 0; t < nsl; ++t) a += part[(t * ngr + g2) * 16 + r];
        z[i] = a;
    }
    __syncthreads();
}

// ---- exact-integer column-subset products (8- and 4-bit codes) ----
__device__ __forceinline__ uint32_t cdp4a_uu(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("dp4a.u32.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}
__device__ __forceinline__ int32_t cdp4a_us(uint32_t a, uint32_t b, int32_t c)
{
    int32_t d;
    asm("dp4a.u32.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}
// 4 x 4 byte transpose: out[p] byte u = byte p of in[u]
__device__ __forceinline__ void transpose4(const uint32_t (&in)[4], uint32_t (&out)[4])
{
    const uint32_t t0 = __byte_perm(in[0], in[1], 0x5140), t1 = __byte_perm(in[0], in[1], 0x7362);
    const uint32_t t2 = __byte_perm(in[2], in[3], 0x5140), t3 = __byte_perm(in[2], in[3], 0x7362);
    out[0] = __byte_perm(t0, t2, 0x5410);
    out[1] = __byte_perm(t0, t2, 0x7632);
    out[2] = __byte_perm(t1, t3, 0x5410);
    out[3] = __byte_perm(t1, t3, 0x7632);
}

// z[0..m) = sum over the list of coef_e (2 c_{i, list_e} - (L-1)), as exact integer sums: the
// coefficients in 24-bit block fixed point, kappa_e = rn(coef_e 2^sh) with |kappa_e| <= 2^22 and
// sh from max |coef|; four list entries' codes of a row (a byte transpose of their code words)
// times the three byte planes of their kappa by dp4a; z_i = 2^-sh (2 sum_e kappa_e c_ie - (L-1)
// sum_e kappa_e), rounded once to FP32. planes: scratch of 3 ceil(count / 4) words. A coefficient
// that is not finite makes every z_i NaN.
template <int BITS>
__device__ void mcols_fx(const Codes& Q, const int* list, const float* coef, int count, float* z, uint32_t* planes,
                         SSh& sh)
{
    static_assert(BITS == 8 || BITS == 4, "8- and 4-bit codes");
    constexpr int WPT = BITS == 8 ? 2 : 1;      // code words of a column per thread
    constexpr int R = 4 * WPT * (BITS == 4 ? 2 : 1);   // rows per thread
    const int tid = threadIdx.x;
    const int ld = Q.ld, m = Q.rows;
    const int ng = (count + 3) / 4;
    unsigned mx = 0;
    for (int e = tid; e < count; e += kST) mx = max(mx, __float_as_uint(coef[e]) & 0x7fffffffu);
    mx = smax(mx, sh.i);
    const bool finite = mx < 0x7f800000u;
    int fsh = 0;
    if (finite && mx) {
        int ex;
        frexpf(__uint_as_float(mx), &ex);       // max |coef| < 2^ex
        fsh = 22 - ex;
    }
    double ksum = 0.0;
    for (int gq = tid; gq < ng; gq += kST) {
        uint32_t p0 = 0, p1 = 0, p2 = 0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int e = 4 * gq + u;
            const int kv = (e < count && finite) ? __float2int_rn(ldexpf(coef[e], fsh)) : 0;
            ksum += (double)kv;
            p0 |= (uint32_t)(kv & 255) << (8 * u);
            p1 |= (uint32_t)((kv >> 8) & 255) << (8 * u);
            p2 |= (uint32_t)((kv >> 16) & 255) << (8 * u);
        }
        planes[3 * gq] = p0;
        planes[3 * gq + 1] = p1;
        planes[3 * gq + 2] = p2;
    }
    const long long K = (long long)ssum(ksum, sh.d);   // exact (|K| < 2^31); its barriers publish the planes
    const long long lk = (long long)Q.lm1 * K;
    for (int rw = tid * WPT; rw < ld; rw += kST * WPT) {
        uint32_t a0[R], a1[R];
        int32_t a2[R];
#pragma unroll
        for (int r = 0; r < R; ++r) { a0[r] = 0u; a1[r] = 0u; a2[r] = 0; }
#pragma unroll 2
        for (int gq = 0; gq < ng; ++gq) {
            uint32_t w[WPT][4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = 4 * gq + u;
                const uint32_t* src = Q.words + (size_t)(e < count ? list[e] : 0) * ld + rw;
                if (WPT == 2) {
                    const uint2 v = e < count ? __ldg(reinterpret_cast<const uint2*>(src)) : make_uint2(0u, 0u);
                    w[0][u] = v.x;
                    w[WPT - 1][u] = v.y;
                } else {
                    w[0][u] = e < count ? __ldg(src) : 0u;
                }
            }
            const uint32_t P0 = planes[3 * gq], P1 = planes[3 * gq + 1], P2 = planes[3 * gq + 2];
#pragma unroll
            for (int h = 0; h < WPT * (BITS == 4 ? 2 : 1); ++h) {
                uint32_t in[4], T[4];
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    in[u] = BITS == 8 ? w[h][u] : (h == 0 ? (w[0][u] & 0x0F0F0F0Fu) : ((w[0][u] >> 4) & 0x0F0F0F0Fu));
                transpose4(in, T);
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    a0[4 * h + p] = cdp4a_uu(T[p], P0, a0[4 * h + p]);
                    a1[4 * h + p] = cdp4a_uu(T[p], P1, a1[4 * h + p]);
                    a2[4 * h + p] = cdp4a_us(T[p], P2, a2[4 * h + p]);
                }
            }
        }
        // rows: 8 bits: 4 rw + r; 4 bits: 8 rw + r (low nibbles rows 0-3, high 4-7)
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int i = (BITS == 8 ? 4 : 8) * rw + r;
            if (i < m) {
                const long long S = (long long)a0[r] + ((long long)a1[r] << 8) + ((long long)a2[r] << 16);
                z[i] = finite ? ldexpf(__ll2float_rn(2 * S - lk), -fsh) : __int_as_float(0x7fc00000);
            }
        }
    }
    __syncthreads();
}

// x_j of the current iterate (0 off the support): binary search of the ascending support
__device__ __forceinline__ float x_at(const MSm& sm, int s, int j)
{
    if (!((sm.gbit[j >> 5] >> (j & 31)) & 1u)) return 0.0f;
    int lo = 0, hi = s - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (sm.sup[mid] < j) lo = mid + 1;
        else hi = mid;
    }
    return sm.xs[lo];
}

// keys |fmaf(mu, g_j, x_j)| for all j (x is 0 off the support); returns 1 if one is not finite
// Keys |fmaf(mu, g_j, x_j)| of all n entries (x is 0 off the support G). With sh != nullptr
// also the smallest key on G (*kmin) and the largest key off G (*rest): when kmin > rest,
// H_s keeps G whatever the order inside it. Returns nonzero if a key is not finite.
__device__ int mkeys(int n, int s, float muf, const float* g, const MSm& sm, int* sh = nullptr,
                     uint32_t* kmin = nullptr, uint32_t* rest = nullptr)
{
    const int tid = threadIdx.x;
    int bad = 0;
    unsigned cmax = 0, inv_min = 0;
    constexpr int KU = 8;                       // a thread's loads of g issued KU at a time
    for (int j0 = tid; j0 < n; j0 += KU * kST) {
        float gv[KU];
#pragma unroll
        for (int u = 0; u < KU; ++u) {
            const int j = j0 + u * kST;
            gv[u] = j < n ? __ldg(g + j) : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < KU; ++u) {
            const int j = j0 + u * kST;
            if (j < n) {
                const uint32_t k = __float_as_uint(fmaf(muf, gv[u], 0.0f)) & 0x7fffffffu;
                sm.keys[j] = k;
                bad |= k > 0x7f800000u;
                if (sh && !((sm.gbit[j >> 5] >> (j & 31)) & 1u)) cmax = max(cmax, k);
            }
        }
    }
    __syncthreads();
    for (int q = tid; q < s; q += kST) {
        const int j = sm.sup[q];
        const uint32_t k = __float_as_uint(fmaf(muf, __ldg(g + j), sm.xs[q])) & 0x7fffffffu;
        sm.keys[j] = k;
        bad |= k > 0x7f800000u;
        inv_min = max(inv_min, ~k);
    }
    if (sh) {
        *rest = smax(cmax, sh);
        *kmin = ~smax(inv_min, sh);
    }
    return __syncthreads_or(bad);
}

// mkeys for a step from the support G, which also lists the candidates of H_s: the s-th
// largest key is at least the smallest key on G (*kmin; the smallest of any s keys bounds it),
// so H_s over all n keys is H_s over G and the entries off G whose key reaches *kmin. The list
// gets G's s indices, then those entries (list[0 .. s + *ncand)), at most cap in all; *ncand is
// -1 when they do not fit. *rest = the largest key off G. Returns nonzero if a key is not finite.
__device__ int mkeys_cand(int n, int s, float muf, const float* g, const MSm& sm, int* sh, uint32_t* kmin,
                          uint32_t* rest, int* list, int cap, int* ncand)
{
    const int tid = threadIdx.x, lane = tid & 31;
    int bad = 0;
    unsigned inv_min = 0, cmax = 0;
    for (int q = tid; q < s; q += kST) {
        const int j = sm.sup[q];
        const uint32_t k = __float_as_uint(fmaf(muf, __ldg(g + j), sm.xs[q])) & 0x7fffffffu;
        sm.keys[j] = k;
        list[q] = j;
        bad |= k > 0x7f800000u;
        inv_min = max(inv_min, ~k);
    }
    const uint32_t km = ~smax(inv_min, sh);
    if (tid == 0) sh[35] = 0;                   // candidate count
    __syncthreads();
    // the entries of a thread in groups of KU, their loads of g issued together (one after the
    // other, the pass is a chain of global-load latencies)
    constexpr int KU = 8;
    for (int j0 = tid; j0 - lane < n; j0 += KU * kST) {   // warp-uniform trip count (the ballots below)
        float gv[KU];
#pragma unroll
        for (int u = 0; u < KU; ++u) {
            const int j = j0 + u * kST;
            gv[u] = j < n ? __ldg(g + j) : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < KU; ++u) {
            const int j = j0 + u * kST;
            bool cand = false;
            if (j < n && !((sm.gbit[j >> 5] >> (j & 31)) & 1u)) {
                const uint32_t k = __float_as_uint(fmaf(muf, gv[u], 0.0f)) & 0x7fffffffu;
                sm.keys[j] = k;
                bad |= k > 0x7f800000u;
                cmax = max(cmax, k);
                cand = k >= km;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, cand);
            if (bal) {
                int base = 0;
                if (lane == 0) base = atomicAdd(&sh[35], __popc(bal));
                base = __shfl_sync(0xffffffffu, base, 0);
                const int pos = s + base + __popc(bal & ((1u << lane) - 1u));
                if (cand && pos < cap) list[pos] = j;
            }
        }
    }
    *rest = smax(cmax, sh);                     // its barriers make the count final
    *kmin = km;
    const int c = sh[35];
    *ncand = s + c <= cap ? c : -1;
    return __syncthreads_or(bad);
}

// H_s over the keys: the s largest, ties to the lower index. G' ascending in sel / val
// (val = x'), the list x' - x over G' u G in uni / dlt (G \ G' after G', in support
// order; only with with_old). Returns 1 if G' != G, else 0; *uc = entries of the list.
// bin of the next radix digit from the histogram in sm.hist (warp 0): the digit whose bucket
// holds the need-th largest key; sh.i[0] = digit, sh.i[1] = keys in higher buckets,
// sh.i[2] = keys in the digit's bucket
__device__ void radix_pick(const MSm& sm, SSh& sh, int need)
{
    const int lane = threadIdx.x & 31;
    if ((threadIdx.x >> 5) == 0) {
        int c[8];
        int tot = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) { c[i] = (int)sm.hist[255 - 8 * lane - i]; tot += c[i]; }
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
                if (run + c[i] >= need) { sh.i[0] = 255 - 8 * lane - i; sh.i[1] = run; sh.i[2] = c[i]; break; }
                run += c[i];
            }
        }
    }
    __syncthreads();
}

// H_s over the keys: the s largest, ties to the lower index. G' ascending in sel / val
// (val = x'), the list x' - x over G' u G in uni / dlt (G \ G' after G', in support
// order; only with with_old). Returns 1 if G' != G, else 0; *uc = entries of the list.
// list (capacity listcap ints, free shared memory) holds the candidates of the top digit's
// bucket: the three later radix passes run over them only. With given >= 0 the list already
// holds every entry H_s can take (given of them, from mkeys_cand): all four passes run over it.
__device__ int mselect(int n, int s, float muf, const float* g, const MSm& sm, SSh& sh, int* uc, bool with_old,
                       int* list, int listcap, int given = -1)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t prefix = 0;
    int need = s, cnt = 0, pass0 = 1;
    bool compact = true;
    if (given >= 0) {
        cnt = given;
        pass0 = 0;
    } else {
    // first digit (top 8 bits) over all keys
    if (tid < 256) sm.hist[tid] = 0;
    __syncthreads();
    for (int b = warp * 32; b < n; b += kST) {
        const int j = b + lane;
        const bool in = j < n;
        const uint32_t k = in ? sm.keys[j] : 0u;
        const unsigned bin = k >> 24;
        // lanes with the same bin add once (keys crowd into few bins)
        const unsigned peers = __match_any_sync(0xffffffffu, in ? bin : 0x100u);
        if (in && lane == __ffs(peers) - 1) atomicAdd(&sm.hist[bin], (unsigned)__popc(peers));
    }
    __syncthreads();
    radix_pick(sm, sh, s);
    prefix = (uint32_t)sh.i[0] << 24;
    need = s - sh.i[1];
    const int c0 = sh.i[2];
    compact = c0 <= listcap;
    __syncthreads();
    if (compact) {
        // the bucket's keys into the list (order does not matter for the histograms)
        if (tid == 0) sh.i[3] = 0;
        __syncthreads();
        const uint32_t top = prefix >> 24;
        for (int b = warp * 32; b < n; b += kST) {
            const int j = b + lane;
            const bool hit = j < n && (sm.keys[j] >> 24) == top;
            const unsigned bal = __ballot_sync(0xffffffffu, hit);
            if (!bal) continue;
            int base = 0;
            if (lane == 0) base = atomicAdd(&sh.i[3], __popc(bal));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (hit) list[base + __popc(bal & ((1u << lane) - 1u))] = j;
        }
        __syncthreads();
        cnt = sh.i[3];
        __syncthreads();
    }
    }
    for (int pass = pass0; pass < 4; ++pass) {
        const int shift = 24 - 8 * pass;
        if (tid < 256) sm.hist[tid] = 0;
        __syncthreads();
        if (compact) {
            for (int e = tid; e < cnt; e += kST) {
                const uint32_t k = sm.keys[list[e]];
                if (pass == 0 || (k >> (shift + 8)) == (prefix >> (shift + 8)))
                    atomicAdd(&sm.hist[(k >> shift) & 255u], 1u);
            }
        } else {
            for (int b = warp * 32; b < n; b += kST) {
                const int j = b + lane;
                const bool in = j < n;
                const uint32_t k = in ? sm.keys[j] : 0u;
                const bool take = in && (k >> (shift + 8)) == (prefix >> (shift + 8));
                if (!__any_sync(0xffffffffu, take)) continue;
                const unsigned bin = (k >> shift) & 255u;
                const unsigned peers = __match_any_sync(0xffffffffu, take ? bin : 0x100u);
                if (take && lane == __ffs(peers) - 1) atomicAdd(&sm.hist[bin], (unsigned)__popc(peers));
            }
        }
        __syncthreads();
        radix_pick(sm, sh, need);
        prefix |= (uint32_t)sh.i[0] << shift;
        need -= sh.i[1];
        __syncthreads();
    }
    const uint32_t T = prefix;
    const int nbw = (n + 31) / 32;
    // every key equal to T taken (the usual case, T's bucket at the last digit holds exactly
    // `need` keys): the selection is every key >= T, marked in one pass
    const bool all_ties = sh.i[2] == need;
    __syncthreads();
    if (all_ties && given >= 0) {
        // the keys >= T are all in the list (the others are below *kmin <= T)
        for (int w = tid; w < nbw; w += kST) sm.bitmap[w] = 0u;
        __syncthreads();
        for (int e = tid; e < cnt; e += kST) {
            const int j = list[e];
            if (sm.keys[j] >= T) atomicOr(&sm.bitmap[j >> 5], 1u << (j & 31));
        }
        __syncthreads();
    } else if (all_ties) {
        for (int b = warp * 32; b < n; b += kST) {
            const int j = b + lane;
            const unsigned bal = __ballot_sync(0xffffffffu, j < n && sm.keys[j] >= T);
            if (lane == 0 && b < n) sm.bitmap[b >> 5] = bal;
        }
        __syncthreads();
    } else {
    for (int w = tid; w < nbw; w += kST) sm.bitmap[w] = 0u;
    const int seg = ((n + 32 * kSW - 1) / (32 * kSW)) * 32;
    const int wb = min(n, warp * seg), we = min(n, wb + seg);
    int eq = 0;
    for (int b = wb; b < we; b += 32) {
        const int j = b + lane;
        eq += __popc(__ballot_sync(0xffffffffu, j < we && sm.keys[j] == T));
    }
    if (lane == 0) sh.i[warp] = eq;
    __syncthreads();
    int eq_before = 0;
    for (int w = 0; w < warp; ++w) eq_before += sh.i[w];
    const int take_w = max(0, min(eq, need - eq_before));
    int erun = 0;
    for (int b = wb; b < we; b += 32) {
        const int j = b + lane;
        const bool in = j < we;
        const uint32_t k = in ? sm.keys[j] : 0u;
        const unsigned meq = __ballot_sync(0xffffffffu, in && k == T);
        const int rank = erun + __popc(meq & ((1u << lane) - 1u));
        if (in && (k > T || (k == T && rank < take_w))) atomicOr(&sm.bitmap[j >> 5], 1u << (j & 31));
        erun += __popc(meq);
    }
    __syncthreads();
    }
    {
        const int wpt = (nbw + kST - 1) / kST;
        const int w0 = min(nbw, tid * wpt), w1 = min(nbw, w0 + wpt);
        int c = 0;
        for (int w = w0; w < w1; ++w) c += __popc(sm.bitmap[w]);
        int total;
        int pre = sscan(c, sh.i, &total);
        for (int w = w0; w < w1; ++w) { sm.wpre[w] = pre; pre += __popc(sm.bitmap[w]); }
    }
    __syncthreads();
    for (int w = tid; w < nbw; w += kST) {
        uint32_t bits = sm.bitmap[w];
        int p = sm.wpre[w];
        while (bits) {
            const int b = __ffs(bits) - 1;
            bits &= bits - 1;
            const int j = w * 32 + b;
            const float xj = x_at(sm, s, j);
            const float v = fmaf(muf, __ldg(g + j), xj);
            sm.sel[p] = j;
            sm.val[p] = v;
            sm.uni[p] = j;
            sm.dlt[p] = v - xj;
            ++p;
        }
    }
    __syncthreads();
    int diff = 0;
    *uc = s;
    if (with_old) {
        const int sper = (s + kST - 1) / kST;
        const int q0 = min(s, tid * sper), q1 = min(s, q0 + sper);
        int cntx = 0;
        for (int q = q0; q < q1; ++q) {
            const int j = sm.sup[q];
            cntx += !((sm.bitmap[j >> 5] >> (j & 31)) & 1u);
        }
        int extra;
        int p = sscan(cntx, sh.i, &extra);
        for (int q = q0; q < q1; ++q) {
            const int j = sm.sup[q];
            if (!((sm.bitmap[j >> 5] >> (j & 31)) & 1u)) {
                sm.uni[s + p] = j;
                sm.dlt[s + p] = -sm.xs[q];
                ++p;
            }
        }
        diff = extra > 0;
        *uc = s + extra;
    }
    __syncthreads();
    return diff;
}


}  // namespace
}  // namespace cta
}  // namespace qiht
