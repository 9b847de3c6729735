// Algorithm 2 for many right-hand sides sharing one quantized matrix: everything of an
// iteration except the gradient product, one CTA per right-hand side.
//
// The gradients of all right-hand sides come from one tensor-core GEMM (mrhs_gemm.cu);
// the rest of an iteration is per right-hand side and runs here with the single-solve
// arithmetic: the step size mu = ||g_G||^2 / ||Q2_G g_G||^2 (FP64 sums of FP32 products
// with column subsets of Q2, summed in list order), H_s as a radix select over the
// binary32 keys |fmaf(mu, g, x)| with ties to the lower index, the backtracking test
// omega = ||x' - x||^2 / ||Q2 (x' - x)||^2, and the residual r = Q(y) - Q2_G' x', updated
// from the product the step already formed (Q2 (x' - x) of the backtracking test, or
// mu Q2_G g_G when the support is unchanged), and directly as Q(y) - Q2_G' x' every few
// iterations and on the last. The CTA then splits r into the scaled f16 parts the next
// GEMM reads.
// The iterate of a right-hand side is kept sparse (its support and the values on it).
#include <cuda_fp16.h>

#include <cmath>

#include "internal.cuh"

namespace qiht {
namespace {

constexpr int kST = 1024;                 // threads per CTA
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
__device__ int mkeys(int n, int s, float muf, const float* g, const MSm& sm)
{
    const int tid = threadIdx.x;
    int bad = 0;
    for (int j = tid; j < n; j += kST) {
        const uint32_t k = __float_as_uint(fmaf(muf, __ldg(g + j), 0.0f)) & 0x7fffffffu;
        sm.keys[j] = k;
        bad |= k > 0x7f800000u;
    }
    __syncthreads();
    for (int q = tid; q < s; q += kST) {
        const int j = sm.sup[q];
        const uint32_t k = __float_as_uint(fmaf(muf, __ldg(g + j), sm.xs[q])) & 0x7fffffffu;
        sm.keys[j] = k;
        bad |= k > 0x7f800000u;
    }
    return __syncthreads_or(bad);
}

// H_s over the keys: the s largest, ties to the lower index. G' ascending in sel / val
// (val = x'), the list x' - x over G' u G in uni / dlt (G \ G' after G', in support
// order; only with with_old). Returns 1 if G' != G, else 0; *uc = entries of the list.
__device__ int mselect(int n, int s, float muf, const float* g, const MSm& sm, SSh& sh, int* uc, bool with_old)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t prefix = 0;
    int need = s;
    for (int pass = 0; pass < 4; ++pass) {
        const int shift = 24 - 8 * pass;
        if (tid < 256) sm.hist[tid] = 0;
        __syncthreads();
        for (int b = warp * 32; b < n; b += kST) {
            const int j = b + lane;
            const bool in = j < n;
            const uint32_t k = in ? sm.keys[j] : 0u;
            const bool take = in && (pass == 0 || (k >> (shift + 8)) == (prefix >> (shift + 8)));
            if (!__any_sync(0xffffffffu, take)) continue;   // later passes: most steps have no candidate
            const unsigned bin = (k >> shift) & 255u;
            // lanes with the same bin add once (keys crowd into few bins); the other lanes share
            // one value so that the match stays cheap
            const unsigned peers = __match_any_sync(0xffffffffu, take ? bin : 0x100u);
            if (take && lane == __ffs(peers) - 1) atomicAdd(&sm.hist[bin], (unsigned)__popc(peers));
        }
        __syncthreads();
        if (warp == 0) {
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
                    if (run + c[i] >= need) { sh.i[0] = 255 - 8 * lane - i; sh.i[1] = run; break; }
                    run += c[i];
                }
            }
        }
        __syncthreads();
        prefix |= (uint32_t)sh.i[0] << shift;
        need -= sh.i[1];
        __syncthreads();
    }
    const uint32_t T = prefix;
    const int nbw = (n + 31) / 32;
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

// dequantized observation value of row i (FP64 product, rounded once)
__device__ __forceinline__ float yhat_at(const qiht_codes& Y, int lm1y, double alpha_y, int i)
{
    const int Gy = 32 / Y.bits;
    const uint32_t w = __ldg(Y.words + i / Gy);
    const int k = i % Gy;
    const int code = (int)((w >> (8 * (k & 3) + Y.bits * (k >> 2))) & ((1u << Y.bits) - 1));
    return (float)(alpha_y * (double)(2 * code - lm1y));
}

// r (in z[0..m)) -> the scaled f16 parts of the next gradient product
__device__ void split_residual(const float* r, int m, int mk, __half* hi, __half* lo, float* sc_k, double alpha1,
                               SSh& sh)
{
    unsigned mx = 0;
    for (int i = threadIdx.x; i < m; i += kST) mx = max(mx, __float_as_uint(r[i]) & 0x7fffffffu);
    mx = smax(mx, sh.i);
    int e = 0;
    const float M = __uint_as_float(mx);
    if (M > 0.0f && isfinite(M)) {
        int ex;
        frexpf(M, &ex);
        e = ex - 15;
    }
    for (int i = threadIdx.x; i < mk; i += kST) {
        const float v = i < m ? ldexpf(r[i], -e) : 0.0f;
        const __half h = __float2half_rn(v);
        hi[i] = h;
        lo[i] = __float2half_rn(v - __half2float(h));
    }
    if (threadIdx.x == 0) *sc_k = (float)ldexp(alpha1, e);
}

template <int BITS>
__global__ void __launch_bounds__(kST, 1) k_mrhs_step(MrhsStepArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ SSh sh;
    const int k = blockIdx.x, tid = threadIdx.x;
    MrhsState* st = a.st + k;
    if (st->stop) return;
    const int n = a.n, m = a.m, s = a.s;
    const MSm sm = msm_layout(smem, n, a.mk, s);
    const float* g = a.G + (size_t)k * n;
    int32_t* gsup = a.sup + (size_t)k * s;
    float* gxs = a.xs + (size_t)k * s;
    if (tid == 0) {
        sh.alpha1 = (double)(*a.scale1) / (double)a.lm1_1;
        sh.alpha2 = (double)(*a.Q2.scale) / (double)a.Q2.lm1;
        sh.alpha2f = (float)sh.alpha2;
    }
    const int nbw = (n + 31) / 32;
    for (int w = tid; w < nbw; w += kST) sm.gbit[w] = 0u;
    __syncthreads();
    int status = QIHT_OK;
    int uc = 0;
    if (a.mode == 0) {
        // initial support H_s(g) (x = 0, keys |g|)
        for (int q = tid; q < s; q += kST) { sm.sup[q] = 0; sm.xs[q] = 0.0f; }
        __syncthreads();
        if (mkeys(n, 0, 1.0f, g, sm)) {
            status = QIHT_ERR_NONFINITE;
        } else {
            mselect(n, s, 1.0f, g, sm, sh, &uc, false);
            for (int q = tid; q < s; q += kST) { gsup[q] = sm.sel[q]; gxs[q] = 0.0f; }
        }
        if (tid == 0 && status != QIHT_OK) { st->status = status; st->stop = 2; }
        return;
    }
    for (int q = tid; q < s; q += kST) {
        const int j = gsup[q];
        sm.sup[q] = j;
        sm.xs[q] = gxs[q];
        atomicOr(&sm.gbit[j >> 5], 1u << (j & 31));
    }
    __syncthreads();
    // step size mu = ||g_G||^2 / (alpha2^2 ||Q2_G g_G||^2)
    for (int q = tid; q < s; q += kST) sm.val[q] = __ldg(g + sm.sup[q]);
    __syncthreads();
    double num = 0.0;
    if (tid < 32) {
        for (int q = tid; q < s; q += 32) num += (double)sm.val[q] * (double)sm.val[q];
#pragma unroll
        for (int o = 16; o; o >>= 1) num += __shfl_xor_sync(0xffffffffu, num, o);
    }
    mcols<BITS>(a.Q2, sm.sup, sm.val, s, sm.z, reinterpret_cast<float*>(sm.keys));
    double zz = 0.0;
    float* zmu = a.zmu + (size_t)k * m;             // kept for the residual update
    for (int i = tid; i < m; i += kST) {
        zz += (double)sm.z[i] * (double)sm.z[i];
        zmu[i] = sm.z[i];
    }
    zz = ssum(zz, sh.d);
    if (tid == 0) {
        const double den = sh.alpha2 * sh.alpha2 * zz;
        int code = 0;
        if (!isfinite(num) || !isfinite(den)) code = 2;
        else if (num == 0.0 || den == 0.0) code = 1;      // converged: x stays
        sh.mu = code ? 0.0 : num / den;
        sh.muf = (float)sh.mu;
        sh.code = code;
    }
    __syncthreads();
    if (sh.code != 0) {
        if (tid == 0) {
            if (sh.code == 2) st->status = QIHT_ERR_NONFINITE;
            st->stop = sh.code;
        }
        return;
    }
    int bt = 0, changed = 0;
    for (;;) {
        if (mkeys(n, s, sh.muf, g, sm)) { changed = -1; break; }
        changed = mselect(n, s, sh.muf, g, sm, sh, &uc, true);
        if (!changed) break;
        // backtracking test on G' u G
        double dn = 0.0;
        if (tid < 32) {
            for (int q = tid; q < uc; q += 32) dn += (double)sm.dlt[q] * (double)sm.dlt[q];
#pragma unroll
            for (int o = 16; o; o >>= 1) dn += __shfl_xor_sync(0xffffffffu, dn, o);
        }
        mcols<BITS>(a.Q2, sm.uni, sm.dlt, uc, sm.z, reinterpret_cast<float*>(sm.keys));
        double dz = 0.0;
        for (int i = tid; i < m; i += kST) dz += (double)sm.z[i] * (double)sm.z[i];
        dz = ssum(dz, sh.d);
        if (tid == 0) {
            const double dd = sh.alpha2 * sh.alpha2 * dz;
            int code = 0;                                   // 0 accept, 1 shrink, 2 give up
            if (dn > 0.0) {
                const double omega = dd > 0.0 ? dn / dd : INFINITY;
                if (!(sh.mu <= (1.0 - a.cc) * omega)) {
                    if (bt >= a.max_bt) code = 2;
                    else {
                        code = 1;
                        sh.mu = sh.mu / (a.kk * (1.0 - a.cc));
                        sh.muf = (float)sh.mu;
                    }
                }
            }
            sh.code = code;
        }
        __syncthreads();
        if (sh.code == 0) break;
        if (sh.code == 2) { changed = -2; break; }
        ++bt;
    }
    if (changed < 0) {
        if (tid == 0) {
            st->status = changed == -1 ? QIHT_ERR_NONFINITE : QIHT_ERR_BACKTRACK_CAP;
            st->stop = 2;
        }
        return;
    }
    // commit G' and x'
    for (int q = tid; q < s; q += kST) {
        gsup[q] = sm.sel[q];
        gxs[q] = sm.val[q];
    }
    // residual: r - alpha2 Q2 (x' - x) with the product already formed for this step (the
    // backtracking test's Q2 (x' - x) if G' != G, else mu Q2_G g_G of the step size), or
    // directly r = Q(y) - alpha2 Q2_G' x' on refresh iterations (periodically and on the last)
    double rr = 0.0;
    float* rk = a.resid + (size_t)k * m;
    if (a.refresh) {
        mcols<BITS>(a.Q2, sm.sel, sm.val, s, sm.z, reinterpret_cast<float*>(sm.keys));
        const float* yk = a.yhat + (size_t)k * m;
        for (int i = tid; i < m; i += kST) {
            const float ri = fmaf(-sh.alpha2f, sm.z[i], __ldg(yk + i));
            sm.z[i] = ri;
            rk[i] = ri;
            rr += (double)ri * (double)ri;
        }
    } else if (changed) {
        for (int i = tid; i < m; i += kST) {
            const float ri = fmaf(-sh.alpha2f, sm.z[i], rk[i]);
            sm.z[i] = ri;
            rk[i] = ri;
            rr += (double)ri * (double)ri;
        }
    } else {
        const float cz = sh.alpha2f * sh.muf;
        for (int i = tid; i < m; i += kST) {
            const float ri = fmaf(-cz, zmu[i], rk[i]);
            sm.z[i] = ri;
            rk[i] = ri;
            rr += (double)ri * (double)ri;
        }
    }
    rr = ssum(rr, sh.d);
    if (tid == 0) {
        st->iters_run += 1;
        st->backtracks += bt;
        st->changes += changed;
        st->mu = sh.mu;
        st->resid2 = rr;
        if (!isfinite(rr)) { st->status = QIHT_ERR_NONFINITE; st->stop = 2; }
    }
    if (!a.last && isfinite(rr))
        split_residual(sm.z, m, a.mk, a.R16 + (size_t)k * a.mk, a.R16 + (size_t)(a.rhi + k) * a.mk, a.sc + k,
                       sh.alpha1, sh);
}

// Q(y_k) -> r = Q(y_k), its f16 parts, ||Q(y_k)||^2; the state of every right-hand side reset.
// Rows of the padded tensor past nrhs become zeros.
__global__ void __launch_bounds__(kST) k_mrhs_init(MrhsStepArgs a)
{
    __shared__ SSh sh;
    extern __shared__ __align__(16) unsigned char smem[];
    float* r = reinterpret_cast<float*>(smem);
    const int k = blockIdx.x, tid = threadIdx.x, m = a.m;
    __half* hi = a.R16 + (size_t)k * a.mk;
    __half* lo = a.R16 + (size_t)(a.rhi + k) * a.mk;
    if (k >= a.nrhs) {
        for (int i = tid; i < a.mk; i += kST) { hi[i] = __float2half_rn(0.0f); lo[i] = __float2half_rn(0.0f); }
        if (tid == 0) a.sc[k] = 0.0f;
        return;
    }
    const qiht_codes Y = a.ydesc[k];
    const int lm1y = grid_levels(Y.bits, Y.levels) - 1;
    if (tid == 0) {
        const float c1 = *a.scale1, c2 = *a.Q2.scale, cy = *Y.scale;
        sh.code = (isfinite(c1) && isfinite(c2) && isfinite(cy)) ? 0 : 1;
        sh.alpha1 = (double)c1 / (double)a.lm1_1;
        sh.alpha_y = (double)cy / (double)lm1y;
    }
    __syncthreads();
    double acc = 0.0;
    for (int i = tid; i < m; i += kST) {
        const float v = yhat_at(Y, lm1y, sh.alpha_y, i);
        r[i] = v;
        a.yhat[(size_t)k * m + i] = v;
        a.resid[(size_t)k * m + i] = v;
        acc += (double)v * (double)v;
    }
    acc = ssum(acc, sh.d);
    MrhsState* st = a.st + k;
    // a valid support until the first selection (a right-hand side stopped here keeps x = 0)
    for (int q = tid; q < a.s; q += kST) {
        a.sup[(size_t)k * a.s + q] = q;
        a.xs[(size_t)k * a.s + q] = 0.0f;
    }
    if (tid == 0) {
        st->mu = 0.0;
        st->resid2 = acc;
        st->stop = sh.code ? 2 : 0;
        st->status = sh.code ? QIHT_ERR_NONFINITE : QIHT_OK;
        st->iters_run = 0;
        st->backtracks = 0;
        st->changes = 0;
    }
    split_residual(r, m, a.mk, hi, lo, a.sc + k, sh.alpha1, sh);
}

// dense x, the support and the report of every right-hand side
__global__ void __launch_bounds__(256) k_mrhs_final(MrhsStepArgs a, float* X, qiht_report* reports,
                                                    const int* gemm_status)
{
    const int k = blockIdx.x;
    const MrhsState* st = a.st + k;
    float* x = X + (size_t)k * a.n;
    for (int j = threadIdx.x; j < a.n; j += 256) x[j] = 0.0f;
    __syncthreads();
    for (int q = threadIdx.x; q < a.s; q += 256) x[a.sup[(size_t)k * a.s + q]] = a.xs[(size_t)k * a.s + q];
    if (threadIdx.x == 0) {
        qiht_report* rp = reports + k;
        rp->iters_run = st->iters_run;
        rp->backtracks = st->backtracks;
        rp->support_changes = st->changes;
        rp->status = *gemm_status ? *gemm_status : st->status;
        rp->resid_norm2 = st->resid2;
        rp->mu = st->mu;
        rp->full_selects = st->iters_run + 1;
        rp->reserved = 0;
        for (int i = 0; i < 8; ++i) rp->phase_us[i] = 0.0f;
    }
}

}  // namespace

size_t mrhs_step_smem(int n, int mk, int s) { return mrhs_step_smem_bytes(n, mk, s); }

cudaError_t launch_mrhs_init(const MrhsStepArgs& a, cudaStream_t s)
{
    const size_t smem = (size_t)a.mk * 4;
    cudaError_t e = cudaFuncSetAttribute(k_mrhs_init, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_mrhs_init<<<a.rhi, kST, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_mrhs_step(const MrhsStepArgs& a, int bits, cudaStream_t s)
{
    const size_t smem = mrhs_step_smem_bytes(a.n, a.mk, a.s);
    void* fn = bits == 8 ? (void*)k_mrhs_step<8> : bits == 4 ? (void*)k_mrhs_step<4> : (void*)k_mrhs_step<2>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    MrhsStepArgs b = a;
    void* args[] = {(void*)&b};
    return cudaLaunchKernel(fn, dim3((unsigned)a.nrhs), dim3(kST), args, smem, s);
}

cudaError_t launch_mrhs_final(const MrhsStepArgs& a, float* X, qiht_report* reports, const int* gemm_status,
                              cudaStream_t s)
{
    k_mrhs_final<<<a.nrhs, 256, 0, s>>>(a, X, reports, gemm_status);
    return cudaGetLastError();
}

}  // namespace qiht
