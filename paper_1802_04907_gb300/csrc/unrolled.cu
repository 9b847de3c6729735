// K unrolled QIHT iterations and their adjoint, for many problems at once.
//
// For each problem (codes Q1, Q2 of Phi, m x n; observation y of 2m entries; per-row complex
// gain a + i b) the operator is the stacked real system A_i = [diag(a); diag(b)] Phi-hat_i.
// With x_0 = 0, step t computes
//     h_t = A1^T r_t,  r_t = y - A2 x_t,
//     G_t = supp H_s(h_0) (t = 0) or the support of x_t,
//     mu_t = ||P h_t||^2 / ||A2 P h_t||^2 (P: restriction to G_t),
//     x_{t+1} = P_{t+1}(x_t + mu_t h_t),  G_{t+1} = supp H_s(x_t + mu_t h_t),
// i.e. the iteration of Algorithm 2 without the backtracking test, and the adjoint maps
// dL/dx_K to dL/dy, dL/da, dL/db with the supports held fixed. The adjoint of a step is
//     v = P_{t+1} xbar_{t+1},  mubar = <v, h_t>,
//     hbar = mu v + mubar (2/D)(P h - mu P A2^T A2 P h)      (sparse: on G_{t+1} u G_t),
//     rbar = A1 hbar,  ybar += rbar,  xbar_t = v - A2^T rbar,
// and the gains collect r hbar^T, -rbar x^T and -(2 mubar mu / D) (A2 P h)(P h)^T through
// the rows they scale.
//
// Kernels: a batched dense product out = base + sign A^T v (persistent, one CTA per SM, a warp
// per group of four columns, exact integer sums of the codes with v in 24-bit fixed point), and
// one CTA (1024 threads) per problem for everything else of a
// step (column-subset products of the s columns, FP64 sums, H_s over all n keys in shared
// memory). The forward keeps the state every ceil(sqrt K) steps; the adjoint recomputes each
// segment from its checkpoint, recording what the reverse steps need.
#include <cmath>

#include "cta_ops.cuh"

namespace qiht {
namespace {

using namespace cta;


__device__ __forceinline__ uint32_t ud_dp4a_uu(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("dp4a.u32.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

__device__ __forceinline__ int32_t ud_dp4a_us(uint32_t a, uint32_t b, int32_t c)
{
    int32_t d;
    asm("dp4a.u32.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

// v (m floats in global memory, written by this CTA before a barrier) -> the operand of the
// batched dense product: 24-bit block fixed point (|v| 2^sh < 2^22, sh from max |v|) as three
// byte planes laid out by code plane (plane e of word w at e * ld + w: limb group g = rows
// 4g .. 4g + 3 is plane g % E of word g / E), its shift and the integer sum of its entries.
template <int BITS>
__device__ void ud_planes(const float* v, int m, int ld, uint32_t* planes, int* shift_out, long long* rsum_out)
{
    constexpr int G = 32 / BITS;
    constexpr int E = G / 4;
    __shared__ unsigned s_mx[32];
    __shared__ long long s_rs[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = (blockDim.x + 31) >> 5;
    unsigned mx = 0;
    for (int i = tid; i < m; i += blockDim.x) mx = max(mx, __float_as_uint(v[i]) & 0x7fffffffu);
    mx = __reduce_max_sync(0xffffffffu, mx);
    if (lane == 0) s_mx[warp] = mx;
    __syncthreads();
    mx = 0;
    for (int w = 0; w < nw; ++w) mx = max(mx, s_mx[w]);
    int sh = 0;
    const float M = __uint_as_float(mx);
    if (M > 0.0f && isfinite(M)) {
        int ex;
        frexpf(M, &ex);
        sh = 22 - ex;
    }
    long long rsum = 0;
    for (int g = tid; g < E * ld; g += blockDim.x) {
        uint32_t b0 = 0, b1 = 0, b2 = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = 4 * g + q;
            const int vi = i < m ? __float2int_rn(ldexpf(v[i], sh)) : 0;
            rsum += vi;
            b0 |= (uint32_t)(vi & 255) << (8 * q);
            b1 |= (uint32_t)((vi >> 8) & 255) << (8 * q);
            b2 |= (uint32_t)((vi >> 16) & 255) << (8 * q);
        }
        const int idx = (g % E) * ld + g / E;
        planes[idx] = b0;
        planes[E * ld + idx] = b1;
        planes[2 * E * ld + idx] = b2;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) rsum += __shfl_xor_sync(0xffffffffu, rsum, o);
    if (lane == 0) s_rs[warp] = rsum;
    __syncthreads();
    if (tid == 0) {
        long long R = 0;
        for (int w = 0; w < nw; ++w) R += s_rs[w];
        *shift_out = sh;
        *rsum_out = R;
    }
}

template <int BITS>
__global__ void __launch_bounds__(256) k_ud_planes(const float* __restrict__ v, UdArgs a)
{
    const int p = blockIdx.x;
    const int ld = a.q1[p].ld_words;
    ud_planes<BITS>(v + (size_t)p * a.m, a.m, ld, a.pl + (size_t)p * a.pl_stride, a.pl_sh + p, a.pl_rs + p);
}

// out[p][j] = (base ? base[p][j] : 0) + sign * alpha * sum_i (2 c_ij - (L-1)) v[p][i], in exact
// integer sums. The three byte planes of v (written once per problem by its producer) sit in
// shared memory; the codes of a column multiply them by dp4a and T = 2 sum c v~ - (L-1) sum v~
// is scaled by alpha 2^-sh in FP32 only (scale2f_apply).
// Persistent grid, one CTA of 16 warps per SM: the (problem, group of kUdC adjacent columns)
// items are split into one contiguous range per CTA, so a CTA sees one or two problems and
// copies their planes once each. A warp owns whole groups and streams the kUdC columns of a
// group together, 512 bytes of each per batch (one 16-byte piece per lane), kUdDepth register
// buffers in rotation (two batches in flight while one is used); one plane load serves the
// kUdC columns. Codes of position e are shifted down to the bytes (x = (w >> b e) & mask), so
// one set of three sums per column covers every position. Measured against two CTAs of 16
// warps per SM with one column per warp and per-position sums (two loads in flight): 6 % less
// time per forward + backward; shapes with 2 columns per warp or more CTAs per SM were slower.
constexpr int kUdThreads = 512;
constexpr int kUdMinBlocks = 1;
constexpr int kUdC = 4;
constexpr int kUdDepth = 3;
constexpr bool kUdMasked = false;

template <int BITS>
__global__ void __launch_bounds__(kUdThreads, kUdMinBlocks) k_ud_gemvt(const qiht_codes* __restrict__ Qs,
    const uint32_t* __restrict__ pl, size_t pl_stride, const int* __restrict__ pl_sh, const long long* __restrict__ pl_rs,
    const float* __restrict__ base, float sign, float* __restrict__ out, int P, int n)
{
    constexpr int G = 32 / BITS;
    constexpr int E = G / 4;
    constexpr int EA = kUdMasked ? E : 1;
    constexpr uint32_t MASK = 0x01010101u * ((1u << BITS) - 1);
    constexpr int NWARP = kUdThreads / 32;
    extern __shared__ __align__(16) uint32_t planes[];
    __shared__ Scale2f s_outscale;
    __shared__ long long s_R;
    const int ld = Qs[0].ld_words;
    const int P4 = ld / 4;
    const int nb = (P4 + 31) / 32;
    const int ngrp = (n + kUdC - 1) / kUdC;
    const long long total = (long long)P * ngrp;
    const long long i0 = total * blockIdx.x / gridDim.x;
    const long long i1 = total * (blockIdx.x + 1) / gridDim.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint64_t policy;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(policy));
    const uint4* L0 = reinterpret_cast<const uint4*>(planes);
    const uint4* L1 = L0 + (size_t)E * P4;
    const uint4* L2 = L0 + (size_t)2 * E * P4;
    for (long long seg = i0; seg < i1;) {
        const int p = (int)(seg / ngrp);
        const long long segend = min(i1, (long long)(p + 1) * ngrp);
        const int g1 = (int)(segend - (long long)p * ngrp);
        const uint32_t* words = Qs[p].words;
        __syncthreads();
        {
            const uint4* srcp = reinterpret_cast<const uint4*>(pl + (size_t)p * pl_stride);
            uint4* dst = reinterpret_cast<uint4*>(planes);
            for (int i = threadIdx.x; i < 3 * E * P4; i += kUdThreads) dst[i] = __ldcg(srcp + i);
        }
        if (threadIdx.x == 0) {
            const long long lm1 = grid_levels(BITS, Qs[p].levels) - 1;
            s_outscale = scale2f_make(ldexp((double)(*Qs[p].scale) / (double)lm1, -pl_sh[p]) * (double)sign);
            s_R = lm1 * pl_rs[p];
        }
        __syncthreads();
        auto load = [&](uint4 (&cv)[kUdC], int g, int b) {
            const int piece = b * 32 + lane;
#pragma unroll
            for (int c = 0; c < kUdC; ++c) {
                const int j = g * kUdC + c;
                if (g < g1 && j < n && piece < P4) {
                    const uint4* col = reinterpret_cast<const uint4*>(words + (size_t)j * ld);
                    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
                                 : "=r"(cv[c].x), "=r"(cv[c].y), "=r"(cv[c].z), "=r"(cv[c].w)
                                 : "l"(col + piece), "l"(policy));
                } else {
                    cv[c] = make_uint4(0u, 0u, 0u, 0u);
                }
            }
        };
        uint32_t s0[kUdC][EA], s1[kUdC][EA];
        int32_t s2[kUdC][EA];
#pragma unroll
        for (int c = 0; c < kUdC; ++c)
#pragma unroll
            for (int e = 0; e < EA; ++e) { s0[c][e] = 0; s1[c][e] = 0; s2[c][e] = 0; }
        auto use = [&](const uint4 (&cv)[kUdC], int b) {
            const int piece = b * 32 + lane;
            if (piece >= P4) return;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const uint4 A0 = L0[(size_t)e * P4 + piece];
                const uint4 A1 = L1[(size_t)e * P4 + piece];
                const uint4 A2 = L2[(size_t)e * P4 + piece];
                const uint32_t y0[4] = {A0.x, A0.y, A0.z, A0.w};
                const uint32_t y1[4] = {A1.x, A1.y, A1.z, A1.w};
                const uint32_t y2[4] = {A2.x, A2.y, A2.z, A2.w};
#pragma unroll
                for (int c = 0; c < kUdC; ++c) {
                    const uint32_t wv[4] = {cv[c].x, cv[c].y, cv[c].z, cv[c].w};
                    const int ea = kUdMasked ? e : 0;
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const uint32_t x = kUdMasked ? (wv[t] & (MASK << (BITS * e))) : ((wv[t] >> (BITS * e)) & MASK);
                        s0[c][ea] = ud_dp4a_uu(x, y0[t], s0[c][ea]);
                        s1[c][ea] = ud_dp4a_uu(x, y1[t], s1[c][ea]);
                        s2[c][ea] = ud_dp4a_us(x, y2[t], s2[c][ea]);
                    }
                }
            }
        };
        auto finish = [&](int g) {
#pragma unroll
            for (int c = 0; c < kUdC; ++c) {
                long long S = 0;
#pragma unroll
                for (int e = 0; e < EA; ++e) {
                    const long long t0 = (long long)(uint32_t)__reduce_add_sync(0xffffffffu, s0[c][e]);
                    const long long t1 = (long long)(uint32_t)__reduce_add_sync(0xffffffffu, s1[c][e]);
                    const long long t2 = (long long)__reduce_add_sync(0xffffffffu, s2[c][e]);
                    S += (t0 + (t1 << 8) + (t2 << 16)) >> (kUdMasked ? BITS * e : 0);
                    s0[c][e] = 0; s1[c][e] = 0; s2[c][e] = 0;
                }
                const int j = g * kUdC + c;
                if (lane == c && j < n) {
                    const long long T = 2 * S - s_R;
                    const float b0 = base ? base[(size_t)p * n + j] : 0.0f;
                    out[(size_t)p * n + j] = scale2f_apply(T, s_outscale, b0);
                }
            }
        };
        auto next = [&](int& g, int& b) { if (++b == nb) { b = 0; g += NWARP; } };
        uint4 buf[kUdDepth][kUdC];
        int gs[kUdDepth], bs[kUdDepth];
        gs[0] = (int)(seg - (long long)p * ngrp) + warp;
        bs[0] = 0;
        load(buf[0], gs[0], bs[0]);
#pragma unroll
        for (int k = 1; k + 1 < kUdDepth; ++k) {
            gs[k] = gs[k - 1]; bs[k] = bs[k - 1]; next(gs[k], bs[k]); load(buf[k], gs[k], bs[k]);
        }
        bool go = true;
        while (go) {
#pragma unroll
            for (int k = 0; k < kUdDepth; ++k) {
                if (go) {
                    if (gs[k] >= g1) {
                        go = false;
                    } else {
                        constexpr int D = kUdDepth;
                        const int ls = (k + D - 1) % D, prev = (k + D - 2) % D;
                        gs[ls] = gs[prev]; bs[ls] = bs[prev]; next(gs[ls], bs[ls]);
                        load(buf[ls], gs[ls], bs[ls]);
                        use(buf[k], bs[k]);
                        if (bs[k] == nb - 1) finish(gs[k]);
                    }
                }
            }
        }
        seg = segend;
    }
}

// dot products of the columns in `list` with a vector held transposed in shared memory
// (entry k of word w at k * ld + w, zero past the rows): out[e] = alpha * sum_i
// (2 c_{i, list_e} - (L-1)) vec_i, one warp per column, one 32-bit word per lane
template <int BITS>
__device__ void ucol_dots(const Codes& Q, const int* list, int count, const float* vecT, float* out)
{
    constexpr int G = 32 / BITS;
    constexpr uint32_t MASK = (1u << BITS) - 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float alpha = __fdiv_rn(*Q.scale, (float)Q.lm1);     // = the double quotient rounded to float
    const float lm1f = (float)Q.lm1;
    for (int e = warp; e < count; e += kST / 32) {
        const uint32_t* col = Q.words + (size_t)list[e] * Q.ld;
        float acc = 0.0f;
        for (int w = lane; w < Q.ld; w += 32) {
            const uint32_t wd = __ldg(col + w);
#pragma unroll
            for (int k = 0; k < G; ++k) {
                const uint32_t code = (wd >> (8 * (k & 3) + BITS * (k >> 2))) & MASK;
                const float cf = __uint_as_float(0x4B000000u | code) - 8388608.0f;
                acc = fmaf(fmaf(cf, 2.0f, -lm1f), vecT[k * Q.ld + w], acc);
            }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) out[e] = alpha * acc;
    }
    __syncthreads();
}

struct UdSh {
    double d[34];
    int i[36];
    double mu, N, D, mubar;
    float muf;
    int code;
};

__device__ Codes codes_of(const qiht_codes& q)
{
    return Codes{q.words, q.scale, q.rows, q.cols, q.bits, q.ld_words, grid_levels(q.bits, q.levels) - 1};
}

// One forward step for problem blockIdx.x: h_t is in a.h (from the batched product).
template <int BITS>
__global__ void __launch_bounds__(kST, 1) k_ud_fwd(UdArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ SSh sh;
    __shared__ UdSh us;
    const int p = blockIdx.x, tid = threadIdx.x;
    const int m = a.m, n = a.n, s = a.s;
    const MSm sm = msm_layout(smem, n, a.mk, s);
    const Codes Q2 = codes_of(a.q2[p]);
    const float* h = a.h + (size_t)p * n;
    const float* ga = a.ga + (size_t)p * m;
    const float* gb = a.gb + (size_t)p * m;
    int32_t* gsup = a.sup + (size_t)p * s;
    float* gxs = a.xs + (size_t)p * s;
    const int nbw = (n + 31) / 32;
    for (int w = tid; w < nbw; w += kST) sm.gbit[w] = 0u;
    __syncthreads();
    int uc = 0;
    if (a.t == 0) {
        // initial support H_s(h_0) (x_0 = 0)
        mkeys(n, 0, 1.0f, h, sm);
        mselect(n, s, 1.0f, h, sm, sh, &uc, false, reinterpret_cast<int*>(sm.z), a.mk);
        for (int q = tid; q < s; q += kST) { sm.sup[q] = sm.sel[q]; sm.xs[q] = 0.0f; }
    } else {
        for (int q = tid; q < s; q += kST) { sm.sup[q] = gsup[q]; sm.xs[q] = gxs[q]; }
    }
    __syncthreads();
    for (int q = tid; q < s; q += kST) atomicOr(&sm.gbit[sm.sup[q] >> 5], 1u << (sm.sup[q] & 31));
    // P h on G_t, N, u = Phi2 P h, D = sum (a^2 + b^2) u^2, mu
    for (int q = tid; q < s; q += kST) sm.val[q] = __ldg(h + sm.sup[q]);
    __syncthreads();
    double N = 0.0;
    if (tid < 32) {
        for (int q = tid; q < s; q += 32) N += (double)sm.val[q] * (double)sm.val[q];
#pragma unroll
        for (int o = 16; o; o >>= 1) N += __shfl_xor_sync(0xffffffffu, N, o);
    }
    mcols<BITS>(Q2, sm.sup, sm.val, s, sm.z, reinterpret_cast<float*>(sm.keys));
    const float alpha2 = __fdiv_rn(*Q2.scale, (float)Q2.lm1);  // FP32: every thread computes it
    // D: each thread's <= 16 terms in FP32, the CTA sum of the partials in FP64 (a per-element
    // FP64 sum keeps the narrow FP64 pipe of this GPU busy for microseconds)
    float Df = 0.0f;
    for (int i = tid; i < m; i += kST) {
        const float ui = alpha2 * sm.z[i];
        sm.z[i] = ui;
        const float g2 = fmaf(ga[i], ga[i], gb[i] * gb[i]);
        Df = fmaf(g2 * ui, ui, Df);
    }
    const double D = ssum((double)Df, sh.d);
    if (tid == 0) {
        us.N = N;
        us.D = D;
        us.mu = D > 0.0 ? N / D : 0.0;
        us.muf = (float)us.mu;
    }
    __syncthreads();
    if (a.rec_r) {
        const size_t slot = (size_t)p * a.c + a.slot;
        for (int i = tid; i < m; i += kST) {
            a.rec_u[slot * m + i] = sm.z[i];
            a.rec_q[slot * m + i] = a.q[(size_t)p * m + i];
        }
        for (int i = tid; i < 2 * m; i += kST) a.rec_r[slot * 2 * m + i] = a.r[(size_t)p * 2 * m + i];
        for (int q = tid; q < s; q += kST) {
            a.rec_G[slot * s + q] = sm.sup[q];
            a.rec_hG[slot * s + q] = sm.val[q];
        }
        if (tid == 0) {
            a.rec_sc[slot * 4 + 0] = us.mu;
            a.rec_sc[slot * 4 + 1] = us.N;
            a.rec_sc[slot * 4 + 2] = us.D;
        }
    }
    // x_{t+1} = H_s(x_t + mu h_t)
    mkeys(n, s, us.muf, h, sm);
    mselect(n, s, us.muf, h, sm, sh, &uc, false, reinterpret_cast<int*>(sm.z), a.mk);
    if (a.rec_r) {
        const size_t slot = (size_t)p * a.c + a.slot;
        for (int q = tid; q < s; q += kST) {
            a.rec_Gn[slot * s + q] = sm.sel[q];
            a.rec_hGn[slot * s + q] = __ldg(h + sm.sel[q]);
        }
    }
    for (int q = tid; q < s; q += kST) {
        gsup[q] = sm.sel[q];
        gxs[q] = sm.val[q];
    }
    // the next step's q = Phi2 x, r = y - [a q; b q] and v = a r_top + b r_bot
    mcols<BITS>(Q2, sm.sel, sm.val, s, sm.z, reinterpret_cast<float*>(sm.keys));
    const float* y = a.y + (size_t)p * 2 * m;
    for (int i = tid; i < m; i += kST) {
        const float qi = alpha2 * sm.z[i];
        const float rt = fmaf(-ga[i], qi, y[i]);
        const float rb = fmaf(-gb[i], qi, y[m + i]);
        a.q[(size_t)p * m + i] = qi;
        a.r[(size_t)p * 2 * m + i] = rt;
        a.r[(size_t)p * 2 * m + m + i] = rb;
        a.vin[(size_t)p * m + i] = fmaf(ga[i], rt, gb[i] * rb);
    }
    __syncthreads();
    ud_planes<BITS>(a.vin + (size_t)p * m, m, Q2.ld, a.pl + (size_t)p * a.pl_stride, a.pl_sh + p, a.pl_rs + p);
}

// One adjoint step for problem blockIdx.x from the record of its forward step.
template <int BITS>
__global__ void __launch_bounds__(kST, 1) k_ud_bwd(UdArgs a, const float* __restrict__ xbar, float* __restrict__ vbase,
                                                   float* __restrict__ vv, float* ybar, float* gabar, float* gbbar)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ SSh sh;
    __shared__ UdSh us;
    const int p = blockIdx.x, tid = threadIdx.x;
    const int m = a.m, n = a.n, s = a.s;
    const MSm sm = msm_layout(smem, n, a.mk, s);
    float* w2 = reinterpret_cast<float*>(smem + msm_bytes(n, a.mk, s));     // (a^2 + b^2) u, transposed by word
    float* cG = w2 + a.mk + 64;                                              // s: (A2^T A2 P h) on G
    const Codes Q1 = codes_of(a.q1[p]);
    const Codes Q2 = codes_of(a.q2[p]);
    const float* ga = a.ga + (size_t)p * m;
    const float* gb = a.gb + (size_t)p * m;
    const size_t slot = (size_t)p * a.c + a.slot;
    const float* ru = a.rec_u + slot * m;
    const float* rq = a.rec_q + slot * m;
    const float* rr = a.rec_r + slot * 2 * m;
    const int nbw = (n + 31) / 32;
    for (int w = tid; w < nbw; w += kST) sm.bitmap[w] = 0u;
    if (tid == 0) {
        us.mu = a.rec_sc[slot * 4 + 0];
        us.N = a.rec_sc[slot * 4 + 1];
        us.D = a.rec_sc[slot * 4 + 2];
    }
    __syncthreads();
    // v on G_{t+1} (sel) and mubar = <v, h>
    const float* xb = xbar + (size_t)p * n;
    for (int q = tid; q < s; q += kST) {
        const int j = a.rec_Gn[slot * s + q];
        sm.sel[q] = j;
        sm.val[q] = __ldg(xb + j);                        // v_j
        sm.sup[q] = a.rec_G[slot * s + q];
        sm.xs[q] = a.rec_hG[slot * s + q];                // h on G_t
        atomicOr(&sm.bitmap[j >> 5], 1u << (j & 31));
    }
    __syncthreads();
    double mb = 0.0;
    if (tid < 32) {
        for (int q = tid; q < s; q += 32) mb += (double)sm.val[q] * (double)a.rec_hGn[slot * s + q];
#pragma unroll
        for (int o = 16; o; o >>= 1) mb += __shfl_xor_sync(0xffffffffu, mb, o);
        if (tid == 0) us.mubar = mb;
    }
    // c = (A2^T A2 P h) on G_t = Phi2^T ((a^2 + b^2) u) there
    {
        constexpr int G = 32 / BITS;
        const int ldw = Q2.ld;
        for (int i = tid; i < ldw * G; i += kST) {
            const float g2 = i < m ? fmaf(ga[i], ga[i], gb[i] * gb[i]) : 0.0f;
            w2[(i % G) * ldw + i / G] = i < m ? g2 * ru[i] : 0.0f;
        }
    }
    __syncthreads();
    ucol_dots<BITS>(Q2, sm.sup, s, w2, cG);
    // hbar on G_{t+1} u G_t: the union list (G_{t+1}, then G_t \ G_{t+1}) with its coefficients
    const double mu = us.mu, D = us.D, mubar = us.mubar;
    const double k2 = D > 0.0 ? mubar * 2.0 / D : 0.0;
    for (int q = tid; q < s; q += kST) {
        sm.uni[q] = sm.sel[q];
        sm.dlt[q] = (float)(mu * (double)sm.val[q]);
    }
    __syncthreads();
    // G_t entries: inside G_{t+1} they add to that entry, outside they are appended in order
    {
        const int sper = (s + kST - 1) / kST;
        const int q0 = min(s, tid * sper), q1 = min(s, q0 + sper);
        int cnt = 0;
        for (int q = q0; q < q1; ++q) {
            const int j = sm.sup[q];
            cnt += !((sm.bitmap[j >> 5] >> (j & 31)) & 1u);
        }
        int extra;
        int pos = sscan(cnt, sh.i, &extra);
        for (int q = q0; q < q1; ++q) {
            const int j = sm.sup[q];
            const float add = (float)(k2 * ((double)sm.xs[q] - mu * (double)cG[q]));
            if ((sm.bitmap[j >> 5] >> (j & 31)) & 1u) {
                // position of j in G_{t+1} (ascending): binary search
                int lo = 0, hi = s - 1;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (sm.sel[mid] < j) lo = mid + 1;
                    else hi = mid;
                }
                atomicAdd(&sm.dlt[lo], add);
            } else {
                sm.uni[s + pos] = j;
                sm.dlt[s + pos] = add;
                ++pos;
            }
        }
        if (tid == 0) us.code = s + extra;
    }
    __syncthreads();
    const int uc = us.code;
    // p = Phi1 hbar; rbar = [a p; b p]
    mcols<BITS>(Q1, sm.uni, sm.dlt, uc, sm.z, reinterpret_cast<float*>(sm.keys));
    const float alpha1 = __fdiv_rn(*Q1.scale, (float)Q1.lm1);  // FP32: every thread computes it
    const float c3 = D > 0.0 ? (float)(-2.0 * mubar * mu / D) : 0.0f;
    float* yb = ybar + (size_t)p * 2 * m;
    float* gab = gabar + (size_t)p * m;
    float* gbb = gbbar + (size_t)p * m;
    for (int i = tid; i < m; i += kST) {
        const float pi = alpha1 * sm.z[i];
        const float rbt = ga[i] * pi, rbb = gb[i] * pi;
        yb[i] += rbt;
        yb[m + i] += rbb;
        const float ui = ru[i];
        gab[i] += rr[i] * pi - rbt * rq[i] + c3 * ga[i] * ui * ui;
        gbb[i] += rr[m + i] * pi - rbb * rq[i] + c3 * gb[i] * ui * ui;
        vv[(size_t)p * m + i] = fmaf(ga[i], rbt, gb[i] * rbb);
    }
    __syncthreads();
    ud_planes<BITS>(vv + (size_t)p * m, m, Q2.ld, a.pl + (size_t)p * a.pl_stride, a.pl_sh + p, a.pl_rs + p);
    // the base of xbar_t: v on G_{t+1}, zero elsewhere
    float* vb = vbase + (size_t)p * n;
    for (int j = tid; j < n; j += kST) vb[j] = 0.0f;
    __syncthreads();
    for (int q = tid; q < s; q += kST) vb[sm.sel[q]] = sm.val[q];
}

// x_0 = 0: q = 0, r = y, v = a y_top + b y_bot; a valid placeholder support
__global__ void __launch_bounds__(256) k_ud_init(UdArgs a)
{
    const int p = blockIdx.x, m = a.m;
    const float* y = a.y + (size_t)p * 2 * m;
    for (int i = threadIdx.x; i < m; i += 256) {
        a.q[(size_t)p * m + i] = 0.0f;
        a.r[(size_t)p * 2 * m + i] = y[i];
        a.r[(size_t)p * 2 * m + m + i] = y[m + i];
        a.vin[(size_t)p * m + i] = fmaf(a.ga[(size_t)p * m + i], y[i], a.gb[(size_t)p * m + i] * y[m + i]);
    }
    for (int q = threadIdx.x; q < a.s; q += 256) {
        a.sup[(size_t)p * a.s + q] = q;
        a.xs[(size_t)p * a.s + q] = 0.0f;
    }
}

__global__ void __launch_bounds__(256) k_ud_xout(UdArgs a, float* X)
{
    const int p = blockIdx.x;
    float* x = X + (size_t)p * a.n;
    for (int j = threadIdx.x; j < a.n; j += 256) x[j] = 0.0f;
    __syncthreads();
    for (int q = threadIdx.x; q < a.s; q += 256) x[a.sup[(size_t)p * a.s + q]] = a.xs[(size_t)p * a.s + q];
}

template <typename F>
cudaError_t set_smem(F* fn, size_t bytes)
{
    return cudaFuncSetAttribute(reinterpret_cast<const void*>(fn), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)bytes);
}

}  // namespace

size_t ud_fwd_smem(int n, int mk, int s) { return msm_bytes(n, mk, s); }
size_t ud_bwd_smem(int n, int mk, int s) { return msm_bytes(n, mk, s) + (size_t)(mk + 64) * 4 + (size_t)s * 4 + 64; }

cudaError_t launch_ud_init(const UdArgs& a, cudaStream_t s)
{
    k_ud_init<<<a.P, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_ud_xout(const UdArgs& a, float* X, cudaStream_t s)
{
    k_ud_xout<<<a.P, 256, 0, s>>>(a, X);
    return cudaGetLastError();
}

cudaError_t launch_ud_planes(const UdArgs& a, int bits, const float* v, cudaStream_t s)
{
    switch (bits) {
    case 8: k_ud_planes<8><<<a.P, 256, 0, s>>>(v, a); break;
    case 4: k_ud_planes<4><<<a.P, 256, 0, s>>>(v, a); break;
    default: k_ud_planes<2><<<a.P, 256, 0, s>>>(v, a); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_ud_gemvt(const UdArgs& a, const qiht_codes* Qs, int bits, const float* base, float sign, float* out,
                            int ldw, cudaStream_t s)
{
    const size_t smem = (size_t)3 * (32 / bits / 4) * ldw * 4;
    const long long items = (long long)a.P * ((a.n + kUdC - 1) / kUdC);
    const long long want = (items + kUdThreads / 32 - 1) / (kUdThreads / 32);
    const long long gx = (long long)num_sms() * kUdMinBlocks;
    const unsigned grid = (unsigned)(want < gx ? want : gx);
    cudaError_t e;
    switch (bits) {
    case 8:
        if ((e = set_smem(k_ud_gemvt<8>, smem)) != cudaSuccess) return e;
        k_ud_gemvt<8><<<grid, kUdThreads, smem, s>>>(Qs, a.pl, a.pl_stride, a.pl_sh, a.pl_rs, base, sign, out, a.P, a.n);
        break;
    case 4:
        if ((e = set_smem(k_ud_gemvt<4>, smem)) != cudaSuccess) return e;
        k_ud_gemvt<4><<<grid, kUdThreads, smem, s>>>(Qs, a.pl, a.pl_stride, a.pl_sh, a.pl_rs, base, sign, out, a.P, a.n);
        break;
    default:
        if ((e = set_smem(k_ud_gemvt<2>, smem)) != cudaSuccess) return e;
        k_ud_gemvt<2><<<grid, kUdThreads, smem, s>>>(Qs, a.pl, a.pl_stride, a.pl_sh, a.pl_rs, base, sign, out, a.P, a.n);
        break;
    }
    return cudaGetLastError();
}

cudaError_t launch_ud_fwd(const UdArgs& a, int bits, cudaStream_t s)
{
    const size_t smem = ud_fwd_smem(a.n, a.mk, a.s);
    cudaError_t e;
    switch (bits) {
    case 8:
        if ((e = set_smem(k_ud_fwd<8>, smem)) != cudaSuccess) return e;
        k_ud_fwd<8><<<a.P, kST, smem, s>>>(a);
        break;
    case 4:
        if ((e = set_smem(k_ud_fwd<4>, smem)) != cudaSuccess) return e;
        k_ud_fwd<4><<<a.P, kST, smem, s>>>(a);
        break;
    default:
        if ((e = set_smem(k_ud_fwd<2>, smem)) != cudaSuccess) return e;
        k_ud_fwd<2><<<a.P, kST, smem, s>>>(a);
        break;
    }
    return cudaGetLastError();
}

cudaError_t launch_ud_bwd(const UdArgs& a, int bits, const float* xbar, float* vbase, float* vv, float* ybar,
                          float* gabar, float* gbbar, cudaStream_t s)
{
    const size_t smem = ud_bwd_smem(a.n, a.mk, a.s);
    cudaError_t e;
    switch (bits) {
    case 8:
        if ((e = set_smem(k_ud_bwd<8>, smem)) != cudaSuccess) return e;
        k_ud_bwd<8><<<a.P, kST, smem, s>>>(a, xbar, vbase, vv, ybar, gabar, gbbar);
        break;
    case 4:
        if ((e = set_smem(k_ud_bwd<4>, smem)) != cudaSuccess) return e;
        k_ud_bwd<4><<<a.P, kST, smem, s>>>(a, xbar, vbase, vv, ybar, gabar, gbbar);
        break;
    default:
        if ((e = set_smem(k_ud_bwd<2>, smem)) != cudaSuccess) return e;
        k_ud_bwd<2><<<a.P, kST, smem, s>>>(a, xbar, vbase, vv, ybar, gabar, gbbar);
        break;
    }
    return cudaGetLastError();
}

}  // namespace qiht

// ---------------------------------------------------------------------------
// entry points
// ---------------------------------------------------------------------------
using namespace qiht;

namespace {

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

int ud_ckpt_every(int K)
{
    int c = 1;
    while (c * c < K) ++c;
    return c;
}

struct UdLayout {
    size_t q1, q2, sup, xs, vin, r, q, h, ck, rec_r, rec_q, rec_u, rec_G, rec_Gn, rec_hG, rec_hGn, rec_sc, xa, xb,
        vbase, vv, pl, pl_sh, pl_rs, total;
    size_t pl_stride;           // words of one problem's planes
    int c, nseg;
    size_t ck_stride;           // bytes of one checkpoint
};

UdLayout ud_layout(int P, int m, int n, int s, int K)
{
    UdLayout L{};
    L.c = ud_ckpt_every(K > 0 ? K : 1);
    L.nseg = (K + L.c - 1) / L.c;
    const size_t Ps = (size_t)P * s, Pm = (size_t)P * m, Pn = (size_t)P * n, Pc = (size_t)P * L.c;
    size_t o = 0;
    L.q1 = o; o += al256((size_t)P * sizeof(qiht_codes));
    L.q2 = o; o += al256((size_t)P * sizeof(qiht_codes));
    L.sup = o; o += al256(Ps * 4);
    L.xs = o; o += al256(Ps * 4);
    L.vin = o; o += al256(Pm * 4);
    L.r = o; o += al256(Pm * 8);
    L.q = o; o += al256(Pm * 4);
    L.h = o; o += al256(Pn * 4);
    L.ck_stride = al256(Ps * 4) * 2 + al256(Pm * 4) * 2 + al256(Pm * 8);
    L.ck = o; o += L.ck_stride * (size_t)(L.nseg > 0 ? L.nseg : 1);
    L.rec_r = o; o += al256(Pc * m * 8);
    L.rec_q = o; o += al256(Pc * m * 4);
    L.rec_u = o; o += al256(Pc * m * 4);
    L.rec_G = o; o += al256(Pc * s * 4);
    L.rec_Gn = o; o += al256(Pc * s * 4);
    L.rec_hG = o; o += al256(Pc * s * 4);
    L.rec_hGn = o; o += al256(Pc * s * 4);
    L.rec_sc = o; o += al256(Pc * 4 * 8);
    L.xa = o; o += al256(Pn * 4);
    L.xb = o; o += al256(Pn * 4);
    L.vbase = o; o += al256(Pn * 4);
    L.vv = o; o += al256(Pm * 4);
    L.pl_stride = (size_t)3 * qiht_ld_words(m, 2) * 16 / 4;      // the widest padding of the three widths
    L.pl = o; o += al256((size_t)P * L.pl_stride * 4);
    L.pl_sh = o; o += al256((size_t)P * 4);
    L.pl_rs = o; o += al256((size_t)P * 8);
    L.total = o;
    return L;
}

bool ud_sizes_ok(int P, int m, int n, int s, int K)
{
    return P >= 1 && m >= 1 && n >= 1 && s >= 1 && s <= m && s <= n && K >= 0 && m <= QIHT_MULTI_MAX_ROWS &&
           n <= QIHT_MULTI_MAX_COLS && s <= QIHT_MULTI_MAX_S;
}

#define UCK(x)                                \
    do {                                      \
        cudaError_t ck_e_ = (x);              \
        if (ck_e_ != cudaSuccess) {           \
            note_cuda_error(#x, ck_e_);       \
            return QIHT_ERR_CUDA;             \
        }                                     \
    } while (0)

qiht_status ud_check(const qiht_codes* Q1, const qiht_codes* Q2, int P, int s, int K)
{
    if (!Q1 || !Q2 || P < 1) return QIHT_ERR_ARG;
    const int m = Q1[0].rows, n = Q1[0].cols, bits = Q1[0].bits;
    for (int p = 0; p < P; ++p) {
        qiht_status e = check_codes(&Q1[p]);
        if (e != QIHT_OK) return e;
        if ((e = check_codes(&Q2[p])) != QIHT_OK) return e;
        if (Q1[p].rows != m || Q1[p].cols != n || Q2[p].rows != m || Q2[p].cols != n) return QIHT_ERR_ARG;
        if (Q1[p].bits != bits || Q2[p].bits != bits) return QIHT_ERR_ARG;
    }
    if (!ud_sizes_ok(P, m, n, s, K)) return QIHT_ERR_ARG;
    const int mk = mrhs_pad_rows(m);
    if (ud_bwd_smem(n, mk, s) > (size_t)227 * 1024 - 2048) return QIHT_ERR_ARG;
    return QIHT_OK;
}

// the state arrays of checkpoint k (sup, xs, vin, q, r)
struct UdCk {
    int32_t* sup;
    float *xs, *vin, *q, *r;
};

UdCk ud_ck(char* w, const UdLayout& L, int P, int m, int s, int k)
{
    char* b = w + L.ck + L.ck_stride * (size_t)k;
    const size_t Ps = (size_t)P * s, Pm = (size_t)P * m;
    UdCk c;
    c.sup = reinterpret_cast<int32_t*>(b);
    c.xs = reinterpret_cast<float*>(b + al256(Ps * 4));
    c.vin = reinterpret_cast<float*>(b + al256(Ps * 4) * 2);
    c.q = reinterpret_cast<float*>(b + al256(Ps * 4) * 2 + al256(Pm * 4));
    c.r = reinterpret_cast<float*>(b + al256(Ps * 4) * 2 + al256(Pm * 4) * 2);
    return c;
}

cudaError_t ud_copy_state(const UdArgs& a, const UdCk& c, bool save, cudaStream_t s)
{
    const size_t Ps = (size_t)a.P * a.s * 4, Pm = (size_t)a.P * a.m * 4;
    auto cp = [&](void* ck, void* st, size_t bytes) {
        return save ? cudaMemcpyAsync(ck, st, bytes, cudaMemcpyDeviceToDevice, s)
                    : cudaMemcpyAsync(st, ck, bytes, cudaMemcpyDeviceToDevice, s);
    };
    cudaError_t e;
    if ((e = cp(c.sup, a.sup, Ps)) != cudaSuccess) return e;
    if ((e = cp(c.xs, a.xs, Ps)) != cudaSuccess) return e;
    if ((e = cp(c.vin, a.vin, Pm)) != cudaSuccess) return e;
    if ((e = cp(c.q, a.q, Pm)) != cudaSuccess) return e;
    return cp(c.r, a.r, 2 * Pm);
}

UdArgs ud_args(char* w, const UdLayout& L, const qiht_codes* Q1, int P, int s, const float* y, const float* ga,
               const float* gb)
{
    UdArgs a{};
    a.q1 = reinterpret_cast<const qiht_codes*>(w + L.q1);
    a.q2 = reinterpret_cast<const qiht_codes*>(w + L.q2);
    a.y = y;
    a.ga = ga;
    a.gb = gb;
    a.P = P;
    a.m = Q1[0].rows;
    a.n = Q1[0].cols;
    a.s = s;
    a.mk = mrhs_pad_rows(a.m);
    a.sup = reinterpret_cast<int32_t*>(w + L.sup);
    a.xs = reinterpret_cast<float*>(w + L.xs);
    a.vin = reinterpret_cast<float*>(w + L.vin);
    a.r = reinterpret_cast<float*>(w + L.r);
    a.q = reinterpret_cast<float*>(w + L.q);
    a.h = reinterpret_cast<float*>(w + L.h);
    a.c = L.c;
    a.pl = reinterpret_cast<uint32_t*>(w + L.pl);
    a.pl_stride = L.pl_stride;
    a.pl_sh = reinterpret_cast<int*>(w + L.pl_sh);
    a.pl_rs = reinterpret_cast<long long*>(w + L.pl_rs);
    return a;
}

}  // namespace

extern "C" {

size_t qiht_unrolled_workspace_size(int32_t nprob, int32_t m, int32_t n, int32_t s, int32_t K)
{
    if (!ud_sizes_ok(nprob, m, n, s, K)) return 0;
    return ud_layout(nprob, m, n, s, K).total;
}

qiht_status qiht_unrolled_forward(const qiht_codes* Q1, const qiht_codes* Q2, int32_t nprob, const float* y,
                                  const float* gain_re, const float* gain_im, int32_t s, int32_t K, float* X,
                                  void* workspace, size_t workspace_bytes, qiht_stream_t stream)
{
    qiht_status e = ud_check(Q1, Q2, nprob, s, K);
    if (e != QIHT_OK) return e;
    if (!y || !gain_re || !gain_im || !X) return QIHT_ERR_ARG;
    const int m = Q1[0].rows, n = Q1[0].cols, bits = Q1[0].bits;
    const UdLayout L = ud_layout(nprob, m, n, s, K);
    if (!workspace || workspace_bytes < L.total || (reinterpret_cast<uintptr_t>(workspace) & 255))
        return QIHT_ERR_WORKSPACE;
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    char* w = reinterpret_cast<char*>(workspace);
    UCK(cudaMemcpyAsync(w + L.q1, Q1, (size_t)nprob * sizeof(qiht_codes), cudaMemcpyHostToDevice, cs));
    UCK(cudaMemcpyAsync(w + L.q2, Q2, (size_t)nprob * sizeof(qiht_codes), cudaMemcpyHostToDevice, cs));
    UdArgs a = ud_args(w, L, Q1, nprob, s, y, gain_re, gain_im);
    UCK(launch_ud_init(a, cs));
    UCK(launch_ud_planes(a, bits, a.vin, cs));
    for (int t = 0; t < K; ++t) {
        if (t % L.c == 0) UCK(ud_copy_state(a, ud_ck(w, L, nprob, m, s, t / L.c), true, cs));
        a.t = t;
        UCK(launch_ud_gemvt(a, a.q1, bits, nullptr, 1.0f, a.h, Q1[0].ld_words, cs));
        UCK(launch_ud_fwd(a, bits, cs));
    }
    UCK(launch_ud_xout(a, X, cs));
    return QIHT_OK;
}

qiht_status qiht_unrolled_backward(const qiht_codes* Q1, const qiht_codes* Q2, int32_t nprob, const float* y,
                                   const float* gain_re, const float* gain_im, int32_t s, int32_t K, const float* Xbar,
                                   float* ybar, float* gain_re_bar, float* gain_im_bar, void* workspace,
                                   size_t workspace_bytes, qiht_stream_t stream)
{
    qiht_status e = ud_check(Q1, Q2, nprob, s, K);
    if (e != QIHT_OK) return e;
    if (!y || !gain_re || !gain_im || !Xbar || !ybar || !gain_re_bar || !gain_im_bar) return QIHT_ERR_ARG;
    const int m = Q1[0].rows, n = Q1[0].cols, bits = Q1[0].bits;
    const UdLayout L = ud_layout(nprob, m, n, s, K);
    if (!workspace || workspace_bytes < L.total || (reinterpret_cast<uintptr_t>(workspace) & 255))
        return QIHT_ERR_WORKSPACE;
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    char* w = reinterpret_cast<char*>(workspace);
    UCK(cudaMemcpyAsync(w + L.q1, Q1, (size_t)nprob * sizeof(qiht_codes), cudaMemcpyHostToDevice, cs));
    UCK(cudaMemcpyAsync(w + L.q2, Q2, (size_t)nprob * sizeof(qiht_codes), cudaMemcpyHostToDevice, cs));
    UdArgs a = ud_args(w, L, Q1, nprob, s, y, gain_re, gain_im);
    a.rec_r = reinterpret_cast<float*>(w + L.rec_r);
    a.rec_q = reinterpret_cast<float*>(w + L.rec_q);
    a.rec_u = reinterpret_cast<float*>(w + L.rec_u);
    a.rec_G = reinterpret_cast<int32_t*>(w + L.rec_G);
    a.rec_Gn = reinterpret_cast<int32_t*>(w + L.rec_Gn);
    a.rec_hG = reinterpret_cast<float*>(w + L.rec_hG);
    a.rec_hGn = reinterpret_cast<float*>(w + L.rec_hGn);
    a.rec_sc = reinterpret_cast<double*>(w + L.rec_sc);
    float* xa = reinterpret_cast<float*>(w + L.xa);
    float* xb = reinterpret_cast<float*>(w + L.xb);
    float* vbase = reinterpret_cast<float*>(w + L.vbase);
    float* vv = reinterpret_cast<float*>(w + L.vv);
    const size_t Pn = (size_t)nprob * n, Pm = (size_t)nprob * m;
    UCK(cudaMemsetAsync(ybar, 0, Pm * 2 * 4, cs));
    UCK(cudaMemsetAsync(gain_re_bar, 0, Pm * 4, cs));
    UCK(cudaMemsetAsync(gain_im_bar, 0, Pm * 4, cs));
    UCK(cudaMemcpyAsync(xa, Xbar, Pn * 4, cudaMemcpyDeviceToDevice, cs));
    for (int seg = L.nseg - 1; seg >= 0; --seg) {
        const int t0 = seg * L.c, t1 = (t0 + L.c < K) ? t0 + L.c : K;
        // recompute the segment from its checkpoint, recording every step
        UCK(ud_copy_state(a, ud_ck(w, L, nprob, m, s, seg), false, cs));
        UCK(launch_ud_planes(a, bits, a.vin, cs));
        for (int t = t0; t < t1; ++t) {
            a.t = t;
            a.slot = t - t0;
            UCK(launch_ud_gemvt(a, a.q1, bits, nullptr, 1.0f, a.h, Q1[0].ld_words, cs));
            UCK(launch_ud_fwd(a, bits, cs));
        }
        // reverse steps: xbar_t = v - A2^T rbar
        for (int t = t1 - 1; t >= t0; --t) {
            a.t = t;
            a.slot = t - t0;
            UCK(launch_ud_bwd(a, bits, xa, vbase, vv, ybar, gain_re_bar, gain_im_bar, cs));
            UCK(launch_ud_gemvt(a, a.q2, bits, vbase, -1.0f, xb, Q1[0].ld_words, cs));
            float* tmp = xa;
            xa = xb;
            xb = tmp;
        }
    }
    return QIHT_OK;
}

}  // extern "C"
