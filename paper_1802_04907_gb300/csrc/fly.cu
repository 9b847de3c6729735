// Phi computed on the fly (Section IV-C) for the gridded interferometry matrix of Section IV-B:
// the entries are an integer phase index into a table of 2g values, quantized as they are made
// and, in the fused product, multiplied at once; no m x n array exists.
//
// Entry (i, p), p = ix * g + iy, row i = k (real part) or K + k (imaginary part):
//   t = (u_k (ix - g/2) + v_k (iy - g/2)) mod g,  value = table[t] (real) or table[g + t].
// The codes follow the quantizer exactly (same Philox counters: element e = p * m + i, counter
// e >> 2, word e & 3; same binary32 decision), so they equal the stored path's codes of the
// materialized matrix bit for bit. The decision depends only on the value, so it is computed
// once per table entry: code = fi + ((w >> 8) < thr) with thr = ceil(f 2^24), which is the
// quantizer's test u < f for u = (w >> 8) 2^-24 (f 2^24 is exact, and for an integer k,
// k < x exactly when k < ceil(x)).
#include "internal.cuh"
#include "quant_rng.cuh"

namespace qiht {
namespace {

struct FlyDec {
    int fi;
    uint32_t thr;
};

struct FlyCtx {
    const int32_t* uv;
    const float* table;
    int K, g, lg, m, n;           // lg = log2 g
    int lm1;
    PhiloxKeys keys;              // round keys of the seed
};

__device__ __forceinline__ FlyDec fly_decision(float v, float c, float half, int lm1)
{
    const Decision d = quant_decide(v, qscale(c), half, lm1);
    return FlyDec{(int)d.fi, (uint32_t)ceilf(d.f * 16777216.0f)};
}

__device__ __forceinline__ int fly_code(const FlyDec& d, uint32_t w)
{
    return d.fi + ((w >> 8) < d.thr ? 1 : 0);
}

// max |table| as the quantizer's max-abs key, by every CTA on its own (2g values)
__device__ __forceinline__ float fly_scale(const float* table, int g, unsigned* s_red)
{
    unsigned mx = 0;
    for (int t = threadIdx.x; t < 2 * g; t += blockDim.x) mx = max(mx, __float_as_uint(table[t]) & 0x7fffffffu);
    mx = __reduce_max_sync(0xffffffffu, mx);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = mx;
    __syncthreads();
    unsigned M = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) M = max(M, s_red[w]);
    __syncthreads();
    return __uint_as_float(M);
}

// the decisions of the table's 2g values
__device__ __forceinline__ void fly_stage_dec(const FlyCtx& f, float c, FlyDec* s_dec)
{
    const float half = (float)f.lm1 * 0.5f;
    for (int t = threadIdx.x; t < 2 * f.g; t += blockDim.x) s_dec[t] = fly_decision(f.table[t], c, half, f.lm1);
}

// Codes of one or two quantizations (streams s0, s1). A warp makes one column at a time
// (its lanes the column's words, so the column's offsets are uniform and the stores
// coalesced); words past the codes of the m rows (the column padding) are written as zero,
// as the quantizer writes them. s_uv holds each row's (u mod g) | (v mod g) << 8, plus g << 16
// on the imaginary rows, so that the row's table offset is part of the same word.
template <int BITS, int NS>
__global__ void __launch_bounds__(256) k_fly_quantize(FlyCtx f, uint32_t s0, uint32_t s1, uint32_t* __restrict__ w0,
                                                      uint32_t* __restrict__ w1, int ldw, float* __restrict__ scale_out)
{
    constexpr int G = 32 / BITS;
    extern __shared__ __align__(16) unsigned char fly_smem[];
    FlyDec* s_dec = reinterpret_cast<FlyDec*>(fly_smem);
    uint32_t* s_uv = reinterpret_cast<uint32_t*>(s_dec + 2 * f.g);
    __shared__ unsigned s_red[8];
    const float c = fly_scale(f.table, f.g, s_red);
    if (blockIdx.x == 0 && threadIdx.x == 0) *scale_out = c;
    fly_stage_dec(f, c, s_dec);
    const int gm = f.g - 1, hg = f.g >> 1;
    for (int i = threadIdx.x; i < f.m; i += blockDim.x) {
        const int k = i < f.K ? i : i - f.K;
        const uint32_t u = (uint32_t)f.uv[2 * k] & (uint32_t)gm, v = (uint32_t)f.uv[2 * k + 1] & (uint32_t)gm;
        s_uv[i] = u | (v << 8) | (i < f.K ? 0u : (uint32_t)f.g << 16);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < f.n; j += warps) {
        const int dx = (j >> f.lg) - hg, dy = (j & gm) - hg;
        const uint64_t e0 = (uint64_t)j * (uint64_t)f.m;
        uint32_t* c0 = w0 + (size_t)j * ldw;
        uint32_t* c1 = w1 + (size_t)j * ldw;
        for (int q = lane; q < ldw; q += 32) {
            const int i0 = q * G;
            uint32_t word[NS];
#pragma unroll
            for (int st = 0; st < NS; ++st) word[st] = 0;
#pragma unroll
            for (int a = 0; a < G / 4; ++a) {
                const int i = i0 + 4 * a;                       // m % 8 == 0: whole quads
                if (i < f.m) {
                    const uint64_t qq = (e0 + (uint64_t)i) >> 2;
                    uint4 rnd[NS];
#pragma unroll
                    for (int st = 0; st < NS; ++st)
                        rnd[st] = philox4x32_10_keys(make_uint4((uint32_t)qq, (uint32_t)(qq >> 32), st == 0 ? s0 : s1, 0u),
                                                     f.keys);
#pragma unroll
                    for (int p = 0; p < 4; ++p) {
                        const uint32_t rw = s_uv[i + p];
                        const int t = (((int)(rw & 0xffu) * dx + (int)((rw >> 8) & 0xffu) * dy) & gm) | (int)(rw >> 16);
                        const FlyDec d = s_dec[t];
                        const int kk = 4 * a + p;                   // position of the row in the word
#pragma unroll
                        for (int st = 0; st < NS; ++st) {
                            const uint32_t w = p == 0 ? rnd[st].x : p == 1 ? rnd[st].y : p == 2 ? rnd[st].z : rnd[st].w;
                            word[st] |= (uint32_t)fly_code(d, w) << (8 * (kk & 3) + BITS * (kk >> 2));
                        }
                    }
                }
            }
            c0[q] = word[0];
            if (NS == 2) c1[q] = word[NS - 1];
        }
    }
}

// Fused generate + quantize + g = Q^T r. A CTA takes tiles of 32 columns (one per lane, so a
// lane's sum never leaves it) and splits the rows over its warps by quads of baselines: the
// rows 4q .. 4q + 3 of the real part and K + 4q .. K + 4q + 3 of the imaginary part, which
// share (u, v) and so the phase index (K % 4 == 0 keeps both quads aligned to the random
// numbers' groups of four). The quads' (u, v) and fixed-point residual sit in shared memory
// (read as broadcasts); the warps' 64-bit sums meet in shared memory once per tile. The
// residual arithmetic and the final scaling are those of the stored-codes product:
// rf_i = rn(r_i 2^sh), sh = 22 - exponent of max |r|, S = sum_i c_i rf_i exactly,
// g_j = (float)((2 S - (L-1) sum rf) * alpha 2^-sh) in FP64.
constexpr int kFlyWarps = 16;

struct FlyQuad {
    int4 u, v, rre, rim;
};

__global__ void __launch_bounds__(kFlyWarps * 32) k_fly_gemv_t(FlyCtx f, uint32_t stream_id, const float* __restrict__ r,
                                                               float* __restrict__ g, float* __restrict__ scale_out)
{
    extern __shared__ __align__(16) unsigned char fly_smem[];
    FlyQuad* s_quad = reinterpret_cast<FlyQuad*>(fly_smem);
    FlyDec* s_dec = reinterpret_cast<FlyDec*>(s_quad + f.K / 4);
    __shared__ unsigned s_red[kFlyWarps];
    __shared__ long long s_rsum[kFlyWarps];
    __shared__ long long s_part[2][kFlyWarps][32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float c = fly_scale(f.table, f.g, s_red);
    if (blockIdx.x == 0 && tid == 0) *scale_out = c;
    fly_stage_dec(f, c, s_dec);
    // max |r| -> the fixed-point shift (as the stored-codes product computes it)
    unsigned mx = 0;
    for (int i = tid; i < f.m; i += blockDim.x) mx = max(mx, __float_as_uint(r[i]) & 0x7fffffffu);
    mx = __reduce_max_sync(0xffffffffu, mx);
    if (lane == 0) s_red[warp] = mx;
    __syncthreads();
    unsigned M = 0;
    for (int w = 0; w < kFlyWarps; ++w) M = max(M, s_red[w]);
    int sh = 0;
    {
        const float Mf = __uint_as_float(M);
        if (Mf > 0.0f && isfinite(Mf)) {
            int ex;
            frexpf(Mf, &ex);
            sh = 22 - ex;
        }
    }
    const int gm = f.g - 1, hg = f.g >> 1;
    const int nquad = f.K / 4;
    long long rs = 0;
    for (int qd = tid; qd < nquad; qd += blockDim.x) {
        int u[4], v[4], a[4], b[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const int k = 4 * qd + p;
            u[p] = f.uv[2 * k] & gm;
            v[p] = f.uv[2 * k + 1] & gm;
            a[p] = __float2int_rn(ldexpf(r[k], sh));
            b[p] = __float2int_rn(ldexpf(r[f.K + k], sh));
            rs += (long long)a[p] + b[p];
        }
        s_quad[qd] = FlyQuad{make_int4(u[0], u[1], u[2], u[3]), make_int4(v[0], v[1], v[2], v[3]),
                             make_int4(a[0], a[1], a[2], a[3]), make_int4(b[0], b[1], b[2], b[3])};
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) rs += __shfl_xor_sync(0xffffffffu, rs, o);
    if (lane == 0) s_rsum[warp] = rs;
    __syncthreads();
    long long R = 0;
    for (int w = 0; w < kFlyWarps; ++w) R += s_rsum[w];
    R *= f.lm1;
    const double outscale = ldexp((double)c / (double)f.lm1, -sh);
    const uint64_t mq = (uint64_t)(f.m >> 2), kq = (uint64_t)(f.K >> 2);
    // this warp's quads
    const int per = (nquad + kFlyWarps - 1) / kFlyWarps;
    const int q_lo = warp * per, q_hi = min(nquad, q_lo + per);
    const FlyDec* s_dim = s_dec + f.g;
    const int tiles = (f.n + 31) / 32;
    int buf = 0;
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int j = tile * 32 + lane;
        const int jj = j < f.n ? j : f.n - 1;             // lanes past n repeat the last column, unused
        const int dx = (jj >> f.lg) - hg, dy = (jj & gm) - hg;
        const uint64_t qb = (uint64_t)jj * mq;
        long long acc = 0;
        for (int qd = q_lo; qd < q_hi; ++qd) {
            const FlyQuad Qd = s_quad[qd];
            const uint64_t q0 = qb + (uint64_t)qd, q1 = q0 + kq;
            const uint4 ra = philox4x32_10_keys(make_uint4((uint32_t)q0, (uint32_t)(q0 >> 32), stream_id, 0u), f.keys);
            const uint4 rb = philox4x32_10_keys(make_uint4((uint32_t)q1, (uint32_t)(q1 >> 32), stream_id, 0u), f.keys);
            const int uu[4] = {Qd.u.x, Qd.u.y, Qd.u.z, Qd.u.w}, vv[4] = {Qd.v.x, Qd.v.y, Qd.v.z, Qd.v.w};
            const int fa[4] = {Qd.rre.x, Qd.rre.y, Qd.rre.z, Qd.rre.w}, fb[4] = {Qd.rim.x, Qd.rim.y, Qd.rim.z, Qd.rim.w};
            const uint32_t wa[4] = {ra.x, ra.y, ra.z, ra.w}, wb[4] = {rb.x, rb.y, rb.z, rb.w};
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const int t = (uu[p] * dx + vv[p] * dy) & gm;
                acc += (long long)fly_code(s_dec[t], wa[p]) * fa[p];
                acc += (long long)fly_code(s_dim[t], wb[p]) * fb[p];
            }
        }
        s_part[buf][warp][lane] = acc;
        __syncthreads();
        if (warp == 0 && j < f.n) {
            long long S = 0;
#pragma unroll
            for (int w = 0; w < kFlyWarps; ++w) S += s_part[buf][w][lane];
            g[j] = (float)((double)(2 * S - R) * outscale);
        }
        buf ^= 1;                    // the next tile writes the other half: one barrier per tile
    }
}

size_t fly_quant_smem(int K, int g) { return (size_t)2 * g * sizeof(FlyDec) + (size_t)2 * K * 4; }
size_t fly_gemv_smem(int K, int g) { return (size_t)(K / 4) * sizeof(FlyQuad) + (size_t)2 * g * sizeof(FlyDec); }

}  // namespace

bool fly_op_ok(const qiht_fly_op* op)
{
    if (!op || !op->uv || !op->table) return false;
    const int g = op->grid, K = op->baselines;
    if (g < 2 || g > QIHT_FLY_MAX_GRID || (g & (g - 1))) return false;
    if (K < 4 || (K & 3) || 2 * K > kMaxRows) return false;
    return true;
}

static FlyCtx fly_ctx(const qiht_fly_op* op, int levels, uint64_t seed)
{
    FlyCtx f;
    f.uv = op->uv;
    f.table = op->table;
    f.K = op->baselines;
    f.g = op->grid;
    f.lg = 0;
    while ((1 << f.lg) < f.g) ++f.lg;
    f.m = 2 * op->baselines;
    f.n = op->grid * op->grid;
    f.lm1 = levels - 1;
    f.keys = philox_keys(seed);
    return f;
}

cudaError_t launch_fly_quantize(const qiht_fly_op* op, int bits, int levels, uint64_t seed, uint32_t s0, uint32_t s1,
                                uint32_t* w0, uint32_t* w1, int ldw, float* scale, cudaStream_t s)
{
    const FlyCtx f = fly_ctx(op, levels, seed);
    const size_t smem = fly_quant_smem(f.K, f.g);
    long long blocks = ((long long)f.n + 7) / 8;          // eight warps (columns at a time) per CTA
    const long long cap = (long long)num_sms() * 8;
    if (blocks > cap) blocks = cap;
    const bool two = w1 != nullptr;
    void* fn = nullptr;
    switch (bits) {
    case 2: fn = two ? (void*)k_fly_quantize<2, 2> : (void*)k_fly_quantize<2, 1>; break;
    case 4: fn = two ? (void*)k_fly_quantize<4, 2> : (void*)k_fly_quantize<4, 1>; break;
    case 8: fn = two ? (void*)k_fly_quantize<8, 2> : (void*)k_fly_quantize<8, 1>; break;
    default: return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    uint32_t* w1p = two ? w1 : w0;
    void* args[] = {(void*)&f, (void*)&s0, (void*)&s1, (void*)&w0, (void*)&w1p, (void*)&ldw, (void*)&scale};
    return cudaLaunchKernel(fn, dim3((unsigned)blocks), dim3(256), args, smem, s);
}

cudaError_t launch_fly_gemv_t(const qiht_fly_op* op, int bits, int levels, uint64_t seed, uint32_t stream_id,
                              const float* r, float* g, float* scale, cudaStream_t s)
{
    (void)bits;                                     // the codes never leave registers: one kernel for every width
    const FlyCtx f = fly_ctx(op, levels, seed);
    const size_t smem = fly_gemv_smem(f.K, f.g);
    void* fn = (void*)k_fly_gemv_t;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kFlyWarps * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int tiles = (f.n + 31) / 32;
    const int grid = std::min(tiles, per_sm * num_sms());
    void* args[] = {(void*)&f, (void*)&stream_id, (void*)&r, (void*)&g, (void*)&scale};
    return cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(kFlyWarps * 32), args, smem, s);
}

}  // namespace qiht

using namespace qiht;

extern "C" {

qiht_status qiht_fly_quantize(const qiht_fly_op* op, int32_t bits, uint64_t seed, uint32_t stream_a,
                              uint32_t stream_b, int32_t flags, uint32_t* words_a, uint32_t* words_b,
                              int32_t ld_words, float* scale, qiht_stream_t stream)
{
    if (bits != 2 && bits != 4 && bits != 8) return QIHT_ERR_BITS;
    if (!fly_op_ok(op) || !words_a || !scale || (flags & ~QIHT_ODD_LEVELS) || words_a == words_b) return QIHT_ERR_ARG;
    const int m = 2 * op->baselines;
    if (ld_words != qiht_ld_words(m, bits)) return QIHT_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(words_a) & 15) || (reinterpret_cast<uintptr_t>(words_b) & 15)) return QIHT_ERR_ARG;
    const int levels = (flags & QIHT_ODD_LEVELS) ? (1 << (bits - 1)) + 1 : (1 << bits);
    const cudaError_t e = launch_fly_quantize(op, bits, levels, seed, stream_a, stream_b, words_a, words_b, ld_words,
                                              scale, reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? QIHT_OK : QIHT_ERR_CUDA;
}

qiht_status qiht_gemv_t_fly(const qiht_fly_op* op, int32_t bits, uint64_t seed, uint32_t stream_id, int32_t flags,
                            const float* r, float* g, float* scale, qiht_stream_t stream)
{
    if (bits != 2 && bits != 4 && bits != 8) return QIHT_ERR_BITS;
    if (!fly_op_ok(op) || !r || !g || !scale || (flags & ~QIHT_ODD_LEVELS)) return QIHT_ERR_ARG;
    const int levels = (flags & QIHT_ODD_LEVELS) ? (1 << (bits - 1)) + 1 : (1 << bits);
    const cudaError_t e = launch_fly_gemv_t(op, bits, levels, seed, stream_id, r, g, scale,
                                            reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? QIHT_OK : QIHT_ERR_CUDA;
}

}  // extern "C"
