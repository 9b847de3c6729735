// Many independent QIHT problems (Algorithm 2) in one persistent launch.
//
// One CTA (1024 threads) per SM takes whole problems from a work counter, largest
// first, and runs every step of the solve for a problem inside the CTA: all vectors of
// a problem (Q(y), r, the fixed-point residual planes, g, x, the support lists) live in
// shared memory, so no step needs a grid-wide exchange or any wait on another CTA. The
// arithmetic is the single-solve path's: the gradient g = Q1^T r in exact integer sums
// (24-bit fixed-point residual, dp4a), products with column subsets of Q2 in FP32 in
// list order, sums of squares and the step size in FP64, H_s as a radix select over the
// binary32 keys |fmaf(mu, g, x)| with ties by the lower index.
#include <cmath>

#include "internal.cuh"

namespace qiht {
namespace {

constexpr int kBT = 1024;                 // threads per CTA
constexpr int kBWarps = kBT / 32;
// bmax, bsum_ll and bexcl_scan combine one partial per warp in warp 0, lane w reading warp w's
// slot: they need exactly 32 warps (with fewer, the upper lanes would read stale slots)
static_assert(kBWarps == 32, "the CTA reductions take one partial from each of 32 warps");
constexpr int kBItems = 4;                // loads of a lane in flight (64 registers per thread)

__device__ __forceinline__ uint32_t bdp4a_uu(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("dp4a.u32.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

__device__ __forceinline__ int32_t bdp4a_us(uint32_t a, uint32_t b, int32_t c)
{
    int32_t d;
    asm("dp4a.u32.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

// 24-bit fixed-point shift of the residual: |r| * 2^sh < 2^22
__device__ __forceinline__ int bfixed_shift(unsigned rmax_bits)
{
    const float M = __uint_as_float(rmax_bits);
    if (!(M > 0.0f) || !isfinite(M)) return 0;
    int ex;
    frexpf(M, &ex);
    return 22 - ex;
}

// ---- deterministic CTA reductions (fixed shuffle trees; FP64 only in warps with data) ----
__device__ double bsum_n(double v, int nact, double* sh)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nw = min((nact + 31) >> 5, kBWarps);
    if (w < nw) {
        if ((int)threadIdx.x >= nact) v = 0.0;
#pragma unroll
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sh[w] = v;
    }
    __syncthreads();
    if (w == 0) {
        double t = lane < nw ? sh[lane] : 0.0;
#pragma unroll
        for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) sh[32] = t;
    }
    __syncthreads();
    const double r = sh[32];
    __syncthreads();
    return r;
}

__device__ unsigned bmax(unsigned v, unsigned* sh)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    v = __reduce_max_sync(0xffffffffu, v);
    if (lane == 0) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        unsigned t = sh[lane];
        t = __reduce_max_sync(0xffffffffu, t);
        if (lane == 0) sh[32] = t;
    }
    __syncthreads();
    const unsigned r = sh[32];
    __syncthreads();
    return r;
}

__device__ long long bsum_ll(long long v, long long* sh)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        long long t = sh[lane];
#pragma unroll
        for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) sh[32] = t;
    }
    __syncthreads();
    const long long r = sh[32];
    __syncthreads();
    return r;
}

// exclusive prefix sum of one int per thread, in thread order
__device__ int bexcl_scan(int v, int* sh, int* total)
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

// Shared memory of one problem (sizes for the batch limits).
struct BSm {
    float* yhat;       // m
    float* r;          // m
    float* z;          // m: column-subset product
    uint32_t* limb;    // 3 planes x m bytes: the residual's fixed-point bytes [3][E][P][4]
    float* g;          // n
    float* x;          // n (dense iterate)
    uint32_t* bitmap;  // n / 32 (selection)
    int* wpre;         // n / 32
    int* sup;          // s: G (ascending)
    int* sel;          // s: G'
    float* val;        // s: x' on G'
    int* uni;          // 2s: G' then G \ G'
    float* dlt;        // 2s: x' - x on uni
    float* red;        // kBT * 16: slice partials of the column-subset product
    unsigned* hist;    // 256
};

constexpr int kBMaxBitmap = QIHT_BATCH_MAX_COLS / 32;

__host__ __device__ inline size_t batched_smem_bytes()
{
    return (size_t)3 * QIHT_BATCH_MAX_ROWS * 4 + (size_t)3 * QIHT_BATCH_MAX_ROWS + (size_t)2 * QIHT_BATCH_MAX_COLS * 4 +
           (size_t)2 * kBMaxBitmap * 4 + (size_t)QIHT_BATCH_MAX_S * 4 * 7 + (size_t)kBT * 16 * 4 + 256 * 4 + 64;
}

__device__ BSm bsm_layout(unsigned char* p)
{
    BSm m;
    m.yhat = reinterpret_cast<float*>(p);
    m.r = m.yhat + QIHT_BATCH_MAX_ROWS;
    m.z = m.r + QIHT_BATCH_MAX_ROWS;
    m.limb = reinterpret_cast<uint32_t*>(m.z + QIHT_BATCH_MAX_ROWS);
    m.g = reinterpret_cast<float*>(m.limb + 3 * QIHT_BATCH_MAX_ROWS / 4);
    m.x = m.g + QIHT_BATCH_MAX_COLS;
    m.bitmap = reinterpret_cast<uint32_t*>(m.x + QIHT_BATCH_MAX_COLS);
    m.wpre = reinterpret_cast<int*>(m.bitmap + kBMaxBitmap);
    m.sup = m.wpre + kBMaxBitmap;
    m.sel = m.sup + QIHT_BATCH_MAX_S;
    m.val = reinterpret_cast<float*>(m.sel + QIHT_BATCH_MAX_S);
    m.uni = reinterpret_cast<int*>(m.val + QIHT_BATCH_MAX_S);
    m.dlt = reinterpret_cast<float*>(m.uni + 2 * QIHT_BATCH_MAX_S);
    m.red = m.dlt + 2 * QIHT_BATCH_MAX_S;
    m.hist = reinterpret_cast<unsigned*>(m.red + kBT * 16);
    return m;
}

struct BShared {          // small scalars shared by the CTA
    double d[34];
    unsigned u[34];
    long long ll[34];
    int i[36];
    double alpha1, alpha2, mu;
    float alpha2f, muf;
    int code;
};

// g = Q1^T r for the whole problem, inside the CTA (the single-solve arithmetic): the
// residual becomes 24-bit fixed point in three byte planes in shared memory; each warp takes
// columns w, w + 32, ... in groups of 32 / LPC, one group of LPC lanes per column; a lane walks
// its 16-byte pieces (lane % LPC, + LPC, ...) of its columns kBItems at a time (that many loads
// in flight), multiplies the codes by dp4a, and each lane group reduces its finished column's
// integer sums. LPC (lanes per column) is the tile shape the batch's autotuner picks per
// problem size (one kernel per shape): short columns (few 16-byte pieces) keep more lanes
// busy with small groups.
template <int BITS, int LPC>
__device__ void bgemv_t(const qiht_codes& Q, const BSm& sm, BShared& sh)
{
    constexpr int G = 32 / BITS;
    constexpr int E = G / 4;
    constexpr int CPW = 32 / LPC;                      // columns a warp works on at once
    constexpr uint32_t MASK = 0x01010101u * (uint32_t)((1 << BITS) - 1);
    const int m = Q.rows, n = Q.cols, ld = Q.ld_words;
    const long long lm1 = grid_levels(BITS, Q.levels) - 1;   // levels - 1 of the grid
    const int P = ld / 4;                              // 16-byte pieces per column
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int sub = lane / LPC, sl = lane % LPC;

    unsigned mx = 0;
    for (int i = tid; i < m; i += kBT) mx = max(mx, __float_as_uint(sm.r[i]) & 0x7fffffffu);
    mx = bmax(mx, sh.u);
    const int shf = bfixed_shift(mx);
    long long rsum = 0;
    for (int lw = tid; lw < P * G; lw += kBT) {
        uint32_t b0 = 0, b1 = 0, b2 = 0;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const int i = 4 * lw + p;
            const int v = i < m ? __float2int_rn(ldexpf(sm.r[i], shf)) : 0;
            rsum += v;
            b0 |= (uint32_t)(v & 255) << (8 * p);
            b1 |= (uint32_t)((v >> 8) & 255) << (8 * p);
            b2 |= (uint32_t)((v >> 16) & 255) << (8 * p);
        }
        const int piece = lw / G, rem = lw - piece * G, q = rem >> 2, w = rem & 3;
        const int idx = (q * P + piece) * 4 + w;
        sm.limb[idx] = b0;
        sm.limb[E * P * 4 + idx] = b1;
        sm.limb[2 * E * P * 4 + idx] = b2;
    }
    const long long R = lm1 * bsum_ll(rsum, sh.ll);    // (L-1) sum_i r_i; also orders the limb stores
    const double outscale = ldexp(sh.alpha1, -shf);
    const uint4* L0 = reinterpret_cast<const uint4*>(sm.limb);
    const uint4* L1 = L0 + E * P;
    const uint4* L2 = L0 + 2 * E * P;

    // the warp's items: column group kg (columns warp + kBWarps (kg CPW + sub)) and piece
    // sl + LPC t of this lane's column
    const int ppl = (P + LPC - 1) / LPC;               // pieces per lane and column
    const int ncol_w = warp < n ? (n - warp + kBWarps - 1) / kBWarps : 0;
    const int ngrp = (ncol_w + CPW - 1) / CPW;
    const int nitem = ngrp * ppl;
    uint32_t s0[E], s1[E];
    int32_t s2[E];
#pragma unroll
    for (int k = 0; k < E; ++k) { s0[k] = 0; s1[k] = 0; s2[k] = 0; }
    for (int i0 = 0; i0 < nitem; i0 += kBItems) {
        uint4 cv[kBItems];
#pragma unroll
        for (int u = 0; u < kBItems; ++u) {
            const int it = i0 + u;
            const int kg = it / ppl, t = it - kg * ppl;
            const int piece = sl + LPC * t;
            const int kc = kg * CPW + sub;
            const int j = warp + kc * kBWarps;
            if (it < nitem && piece < P && kc < ncol_w)
                cv[u] = __ldg(reinterpret_cast<const uint4*>(Q.words + (size_t)j * ld) + piece);
            else
                cv[u] = make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int u = 0; u < kBItems; ++u) {
            const int it = i0 + u;
            if (it >= nitem) break;                    // uniform within the warp
            const int kg = it / ppl, t = it - kg * ppl;
            const int piece = min(sl + LPC * t, P - 1);    // lanes past P hold zero codes
            const uint32_t wv[4] = {cv[u].x, cv[u].y, cv[u].z, cv[u].w};
#pragma unroll
            for (int q = 0; q < E; ++q) {
                const uint4 A0 = L0[q * P + piece];
                const uint4 A1 = L1[q * P + piece];
                const uint4 A2 = L2[q * P + piece];
                const uint32_t y0[4] = {A0.x, A0.y, A0.z, A0.w};
                const uint32_t y1[4] = {A1.x, A1.y, A1.z, A1.w};
                const uint32_t y2[4] = {A2.x, A2.y, A2.z, A2.w};
#pragma unroll
                for (int tt = 0; tt < 4; ++tt) {
                    const int lw = q * 4 + tt, w = lw / E, k = lw - w * E;
                    const uint32_t x = wv[w] & (MASK << (BITS * k));
                    s0[k] = bdp4a_uu(x, y0[tt], s0[k]);
                    s1[k] = bdp4a_uu(x, y1[tt], s1[k]);
                    s2[k] = bdp4a_us(x, y2[tt], s2[k]);
                }
            }
            if (t == ppl - 1) {                        // the group's columns are complete
                long long S = 0;
#pragma unroll
                for (int k = 0; k < E; ++k) {
                    uint32_t t0 = s0[k], t1 = s1[k];
                    int32_t t2 = s2[k];
                    if (LPC == 32) {                   // the whole warp: one reduction instruction
                        t0 = __reduce_add_sync(0xffffffffu, t0);
                        t1 = __reduce_add_sync(0xffffffffu, t1);
                        t2 = __reduce_add_sync(0xffffffffu, t2);
                    } else {
#pragma unroll
                        for (int o = LPC / 2; o; o >>= 1) {   // exact: the sums stay below 2^32
                            t0 += __shfl_xor_sync(0xffffffffu, t0, o);
                            t1 += __shfl_xor_sync(0xffffffffu, t1, o);
                            t2 += __shfl_xor_sync(0xffffffffu, t2, o);
                        }
                    }
                    S += ((long long)t0 + ((long long)t1 << 8) + ((long long)t2 << 16)) >> (BITS * k);
                    s0[k] = 0; s1[k] = 0; s2[k] = 0;
                }
                const int kc = kg * CPW + sub;
                if (sl == 0 && kc < ncol_w) {
                    const long long T = 2 * S - R;
                    sm.g[warp + kc * kBWarps] = (float)((double)T * outscale);
                }
            }
        }
    }
    __syncthreads();
}

// z[0..m) = sum over the list (indices and coefficients in shared memory, in list order)
// of coef_j * (2 c_ij - (L-1)) for the problem's Q2 (L levels). Thread t owns code word t % ld of
// every column (G rows) and the list entries of slice t / ld; the slices are summed in
// order.
template <int BITS>
__device__ void bcols(const qiht_codes& Q, const int* list, const float* coef, int count, const BSm& sm)
{
    constexpr int G = 32 / BITS;
    constexpr uint32_t MASK = (1u << BITS) - 1;
    const int ld = Q.ld_words, m = Q.rows;
    const int lm1 = grid_levels(BITS, Q.levels) - 1;
    const int tid = threadIdx.x;
    const int nsl = kBT / ld;                          // ld <= 512 under the batch limits
    const int wr = tid % ld, sl = tid / ld;
    float zk[G];
#pragma unroll
    for (int k = 0; k < G; ++k) zk[k] = 0.0f;
    if (sl < nsl) {
        for (int j0 = sl; j0 < count; j0 += kBItems * nsl) {
            uint32_t w[kBItems];
            float cf[kBItems];
#pragma unroll
            for (int u = 0; u < kBItems; ++u) {
                const int e = j0 + u * nsl;
                const bool in = e < count;
                w[u] = in ? __ldg(Q.words + (size_t)list[e] * ld + wr) : 0u;
                cf[u] = in ? coef[e] : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < kBItems; ++u)
#pragma unroll
                for (int k = 0; k < G; ++k) {
                    const int code = (int)((w[u] >> (8 * (k & 3) + BITS * (k >> 2))) & MASK);
                    zk[k] = fmaf((float)(2 * code - lm1), cf[u], zk[k]);
                }
        }
#pragma unroll
        for (int k = 0; k < G; ++k) sm.red[(sl * ld + wr) * G + k] = zk[k];
    }
    __syncthreads();
    for (int i = tid; i < ld * G; i += kBT) {
        const int w = i / G, k = i % G;
        float acc = 0.0f;
        for (int s2 = 0; s2 < nsl; ++s2) acc += sm.red[(s2 * ld + w) * G + k];
        const int row = w * G + k;
        if (row < m) sm.z[row] = acc;
    }
    __syncthreads();
}

// H_s(x + mu g) over all n entries: radix select (8-bit digits) of the s-th largest key
// |fmaf(mu, g, x)| (binary32 bits), then the keys above it and the lowest-index keys equal
// to it; Gamma' ascending in sm.sel / sm.val, the x' - x list over Gamma' u Gamma in
// sm.uni / sm.dlt (with_old: Gamma is in sm.sup; without it only Gamma' is produced).
// Returns -1 if a key is not finite, else 1 if Gamma' != Gamma, 0 if equal; *uc = entries
// of the union list.
__device__ int bselect(int n, int s, float muf, const BSm& sm, BShared& sh, int* uc, bool with_old)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    auto key = [&](int j) { return __float_as_uint(fmaf(muf, sm.g[j], sm.x[j])) & 0x7fffffffu; };
    int bad = 0;
    for (int j = tid; j < n; j += kBT) bad |= key(j) > 0x7f800000u;
    if (__syncthreads_or(bad)) return -1;
    uint32_t prefix = 0;
    int need = s;
    for (int pass = 0; pass < 4; ++pass) {
        const int shift = 24 - 8 * pass;
        if (tid < 256) sm.hist[tid] = 0;
        __syncthreads();
        for (int j = tid; j < n; j += kBT) {
            const uint32_t k = key(j);
            if (pass == 0 || (k >> (shift + 8)) == (prefix >> (shift + 8))) atomicAdd(&sm.hist[(k >> shift) & 255u], 1u);
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
    // mark the keys > T and the `need` lowest-index keys == T: warp w walks indices
    // [w seg, (w + 1) seg) in order
    const int nbw = (n + 31) / 32;
    for (int w = tid; w < nbw; w += kBT) sm.bitmap[w] = 0u;
    const int seg = ((n + 32 * kBWarps - 1) / (32 * kBWarps)) * 32;
    const int wb = min(n, warp * seg), we = min(n, wb + seg);
    int eq = 0;
    for (int b = wb; b < we; b += 32) {
        const int j = b + lane;
        eq += __popc(__ballot_sync(0xffffffffu, j < we && key(j) == T));
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
        const uint32_t k = in ? key(j) : 0u;
        const unsigned meq = __ballot_sync(0xffffffffu, in && k == T);
        const int rank = erun + __popc(meq & ((1u << lane) - 1u));
        if (in && (k > T || (k == T && rank < take_w))) atomicOr(&sm.bitmap[j >> 5], 1u << (j & 31));
        erun += __popc(meq);
    }
    __syncthreads();
    // selected entries before each bitmap word (words in order, thread t takes words t*wpt..)
    {
        const int wpt = (nbw + kBT - 1) / kBT;
        const int w0 = min(nbw, tid * wpt), w1 = min(nbw, w0 + wpt);
        int c = 0;
        for (int w = w0; w < w1; ++w) c += __popc(sm.bitmap[w]);
        int total;
        int pre = bexcl_scan(c, sh.i, &total);
        for (int w = w0; w < w1; ++w) { sm.wpre[w] = pre; pre += __popc(sm.bitmap[w]); }
    }
    __syncthreads();
    for (int w = tid; w < nbw; w += kBT) {
        uint32_t bits = sm.bitmap[w];
        int p = sm.wpre[w];
        while (bits) {
            const int b = __ffs(bits) - 1;
            bits &= bits - 1;
            const int j = w * 32 + b;
            const float xj = sm.x[j];
            const float v = fmaf(muf, sm.g[j], xj);
            sm.sel[p] = j;
            sm.val[p] = v;
            sm.uni[p] = j;
            sm.dlt[p] = v - xj;
            ++p;
        }
    }
    __syncthreads();
    // G \ G' after G', in support order
    int diff = 0;
    *uc = s;
    if (with_old) {
        const int sper = (s + kBT - 1) / kBT;
        const int q0 = min(s, tid * sper), q1 = min(s, q0 + sper);
        int cntx = 0;
        for (int q = q0; q < q1; ++q) {
            const int j = sm.sup[q];
            cntx += !((sm.bitmap[j >> 5] >> (j & 31)) & 1u);
        }
        int extra;
        int p = bexcl_scan(cntx, sh.i, &extra);
        for (int q = q0; q < q1; ++q) {
            const int j = sm.sup[q];
            if (!((sm.bitmap[j >> 5] >> (j & 31)) & 1u)) {
                sm.uni[s + p] = j;
                sm.dlt[s + p] = -sm.x[j];
                ++p;
            }
        }
        diff = extra > 0;
        *uc = s + extra;
    }
    __syncthreads();
    return diff;
}

template <int BITS, int LPC>
__device__ void solve_one(const qiht_problem& P, int iters, double kk, double cc, int max_bt, const BSm& sm,
                          BShared& sh)
{
    const int tid = threadIdx.x;
    const int m = P.Q1.rows, n = P.Q1.cols, s = P.s;
    const uint32_t ymask = (1u << P.y.bits) - 1;
    const int lm1y = grid_levels(P.y.bits, P.y.levels) - 1, Gy = 32 / P.y.bits;
    if (tid == 0) {
        const float c1 = *P.Q1.scale, c2 = *P.Q2.scale, cy = *P.y.scale;
        sh.code = (isfinite(c1) && isfinite(c2) && isfinite(cy)) ? 0 : 1;
        sh.alpha1 = (double)c1 / (double)(grid_levels(BITS, P.Q1.levels) - 1);
        sh.alpha2 = (double)c2 / (double)(grid_levels(BITS, P.Q2.levels) - 1);
        sh.alpha2f = (float)sh.alpha2;
        sh.d[33] = (double)cy / (double)lm1y;          // alpha of y
    }
    __syncthreads();
    const double alpha_y = sh.d[33];
    const bool finite = sh.code == 0;
    // Q(y) dequantized, r = Q(y), x = 0
    double acc = 0.0;
    for (int i = tid; i < m; i += kBT) {
        const uint32_t w = __ldg(P.y.words + i / Gy);
        const int k = i % Gy;
        const int code = (int)((w >> (8 * (k & 3) + P.y.bits * (k >> 2))) & ymask);
        const float v = (float)(alpha_y * (double)(2 * code - lm1y));
        sm.yhat[i] = v;
        sm.r[i] = v;
        acc += (double)v * (double)v;
    }
    for (int j = tid; j < n; j += kBT) sm.x[j] = 0.0f;
    double resid2 = bsum_n(acc, min(m, kBT), sh.d);
    int status = finite ? QIHT_OK : QIHT_ERR_NONFINITE;
    int it = 0, bt_total = 0, changes = 0;
    double mu_acc = 0.0;
    int uc = 0;
    if (finite) {
        bgemv_t<BITS, LPC>(P.Q1, sm, sh);
        // initial support: H_s(g)
        const int sel0 = bselect(n, s, 1.0f, sm, sh, &uc, false);   // x = 0: the keys are |g|
        if (sel0 < 0) {
            status = QIHT_ERR_NONFINITE;
        } else {
            for (int q = tid; q < s; q += kBT) sm.sup[q] = sm.sel[q];
        }
        __syncthreads();
    }
    while (status == QIHT_OK && it < iters) {
        // step size: mu = ||g_G||^2 / (alpha2^2 ||Q2_G g_G||^2)
        for (int q = tid; q < s; q += kBT) sm.val[q] = sm.g[sm.sup[q]];
        __syncthreads();
        double num = 0.0;
        if (tid < 32) {
            for (int q = tid; q < s; q += 32) num += (double)sm.val[q] * (double)sm.val[q];
#pragma unroll
            for (int o = 16; o; o >>= 1) num += __shfl_xor_sync(0xffffffffu, num, o);
        }
        bcols<BITS>(P.Q2, sm.sup, sm.val, s, sm);
        // sums of squares: each thread's terms in FP32, the CTA sum of the partials in FP64
        float zzf = 0.0f;
        for (int i = tid; i < m; i += kBT) zzf = fmaf(sm.z[i], sm.z[i], zzf);
        const double zz = bsum_n((double)zzf, min(m, kBT), sh.d);
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
        if (sh.code == 2) { status = QIHT_ERR_NONFINITE; break; }
        if (sh.code == 1) break;
        int bt = 0;
        int changed = 0;
        for (;;) {
            changed = bselect(n, s, sh.muf, sm, sh, &uc, true);
            if (changed < 0) break;
            if (!changed) break;
            // backtracking test on G' u G
            double dn = 0.0;
            if (tid < 32) {
                for (int q = tid; q < uc; q += 32) dn += (double)sm.dlt[q] * (double)sm.dlt[q];
#pragma unroll
                for (int o = 16; o; o >>= 1) dn += __shfl_xor_sync(0xffffffffu, dn, o);
            }
            bcols<BITS>(P.Q2, sm.uni, sm.dlt, uc, sm);
            float dzf = 0.0f;
            for (int i = tid; i < m; i += kBT) dzf = fmaf(sm.z[i], sm.z[i], dzf);
            const double dz = bsum_n((double)dzf, min(m, kBT), sh.d);
            if (tid == 0) {
                const double dd = sh.alpha2 * sh.alpha2 * dz;
                int code = 0;                                   // 0 accept, 1 shrink, 2 give up
                if (dn > 0.0) {
                    const double omega = dd > 0.0 ? dn / dd : INFINITY;
                    if (!(sh.mu <= (1.0 - cc) * omega)) {
                        if (bt >= max_bt) code = 2;
                        else {
                            code = 1;
                            sh.mu = sh.mu / (kk * (1.0 - cc));
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
        if (changed == -1) { status = QIHT_ERR_NONFINITE; break; }
        if (changed == -2) { status = QIHT_ERR_BACKTRACK_CAP; break; }
        // commit x and G
        for (int q = tid; q < s; q += kBT) {
            const int j = sm.sup[q];
            if (!((sm.bitmap[j >> 5] >> (j & 31)) & 1u)) sm.x[j] = 0.0f;
        }
        __syncthreads();
        for (int q = tid; q < s; q += kBT) {
            sm.x[sm.sel[q]] = sm.val[q];
            sm.sup[q] = sm.sel[q];
        }
        __syncthreads();
        // residual r = Q(y) - alpha2 Q2_G' x'
        bcols<BITS>(P.Q2, sm.sel, sm.val, s, sm);
        float rrf = 0.0f;
        for (int i = tid; i < m; i += kBT) {
            const float ri = fmaf(-sh.alpha2f, sm.z[i], sm.yhat[i]);
            sm.r[i] = ri;
            rrf = fmaf(ri, ri, rrf);
        }
        resid2 = bsum_n((double)rrf, min(m, kBT), sh.d);
        ++it;
        bt_total += bt;
        changes += changed;
        mu_acc = sh.mu;
        if (!isfinite(resid2)) { status = QIHT_ERR_NONFINITE; break; }
        if (it < iters) bgemv_t<BITS, LPC>(P.Q1, sm, sh);
    }
    // outputs
    for (int j = tid; j < n; j += kBT) P.x[j] = sm.x[j];
    for (int q = tid; q < s; q += kBT) P.support[q] = sm.sup[q];
    if (tid == 0) {
        qiht_report* rp = P.report;
        rp->iters_run = it;
        rp->backtracks = bt_total;
        rp->support_changes = changes;
        rp->status = status;
        rp->resid_norm2 = resid2;
        rp->mu = mu_acc;
        rp->full_selects = it + 1;
        rp->reserved = 0;
        for (int i = 0; i < 8; ++i) rp->phase_us[i] = 0.0f;
    }
    __syncthreads();
}

template <int BITS, int LPC>
__global__ void __launch_bounds__(kBT, 1) k_batched(const qiht_problem* __restrict__ probs,
                                                    const int* __restrict__ order, int nprob, int iters, double kk,
                                                    double cc, int max_bt, unsigned* next)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ BShared sh;
    __shared__ qiht_problem P;                 // the current problem's descriptor
    __shared__ int s_pid;
    const BSm sm = bsm_layout(smem);
    for (;;) {
        if (threadIdx.x == 0) {
            s_pid = (int)atomicAdd(next, 1u);
            if (s_pid < nprob) P = probs[order[s_pid]];
        }
        __syncthreads();
        const int w = s_pid;
        __syncthreads();
        if (w >= nprob) return;
        solve_one<BITS, LPC>(P, iters, kk, cc, max_bt, sm, sh);
    }
}

}  // namespace

size_t batched_smem() { return batched_smem_bytes(); }

template <int BITS>
static void* batched_fn(int lpc)
{
    switch (lpc) {
    case 4: return (void*)k_batched<BITS, 4>;
    case 8: return (void*)k_batched<BITS, 8>;
    case 16: return (void*)k_batched<BITS, 16>;
    default: return (void*)k_batched<BITS, 32>;
    }
}

cudaError_t launch_batched(const qiht_problem* probs, const int* order, int nprob, int bits, int lpc, int iters,
                           double k, double c, int max_bt, unsigned* next, cudaStream_t s)
{
    const size_t smem = batched_smem_bytes();
    void* fn = bits == 8 ? batched_fn<8>(lpc) : bits == 4 ? batched_fn<4>(lpc) : batched_fn<2>(lpc);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(next, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    int grid = num_sms();
    if (grid > nprob) grid = nprob;
    void* args[] = {(void*)&probs, (void*)&order, (void*)&nprob, (void*)&iters, (void*)&k, (void*)&c, (void*)&max_bt,
                    (void*)&next};
    return cudaLaunchKernel(fn, dim3(grid), dim3(kBT), args, smem, s);
}

}  // namespace qiht
