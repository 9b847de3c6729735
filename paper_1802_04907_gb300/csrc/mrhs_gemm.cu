// Gradient of many right-hand sides at once on the tensor cores: G = Q^T R.
//
// With nrhs residual vectors r_k sharing one quantized matrix (Algorithm 2 run for
// many observations y_k of the same Phi), the products g_k = Q1^T r_k of one iteration
// form a dense contraction: G (n x nrhs) = W^T R with W = 2c - (L-1) the centred codes
// (odd integers, |W| <= 255) and R (m x nrhs). It runs as an f16 tcgen05 GEMM:
//   - W is exact in f16 (at most 8 significant bits). The codes are read from the
//     column-packed layout and expanded in shared memory by converter warps.
//   - each residual is scaled by a power of two 2^-e_k (max |r_k| 2^-e_k in [2^14, 2^15))
//     and split into two f16 parts, hi = f16(r'), lo = f16(r' - hi), so hi + lo carries
//     about 22 significant bits; both parts are multiplied by the same W tile and
//     accumulated into one FP32 accumulator in tensor memory.
//   - the epilogue multiplies by alpha 2^e_k (alpha = scale / (L-1)).
// Products of an f16 code and an f16 part are exact; the only roundings are the FP32
// accumulation and the final scaling.
//
// Tile: 256 columns of Q (two MMA tiles of M = 128 sharing every R tile, two accumulators
// filling the 512 tensor-memory columns) x 256 right-hand sides (N), K steps of 32 rows in a
// 4-stage ring; operands in shared memory in the K-major layout with 64-byte swizzle.
// Warp roles: warp 0 loads the R tiles with TMA, warp 1 allocates tensor memory and
// issues the MMAs (one thread), warps 2..9 expand the codes (one column of Q each) and,
// at the end, read the accumulators out of tensor memory. Every wait is bounded by %globaltimer; a timeout
// records QIHT_ERR_TIMEOUT, stops the CTA's roles, waits for the copies and MMAs it
// issued and frees its tensor memory before returning.
#include <cuda.h>
#include <cuda_fp16.h>

#include <cstring>

#include "internal.cuh"

namespace qiht {
namespace {

constexpr int kTM = 128;                       // columns of Q per MMA tile (MMA M)
constexpr int kMT = 2;                         // MMA tiles per CTA (they share the R tiles)
constexpr int kTN = 256;                       // right-hand sides per tile (MMA N)
constexpr int kTK = 32;                        // rows of Q per stage: 64 bytes of f16
constexpr int kStages = 4;
constexpr int kConvWarps = kMT * 4;            // one thread per column of Q
constexpr int kGemmThreads = 64 + 32 * kConvWarps;
constexpr uint32_t kABytes = kTM * kTK * 2;    // 8 KB per MMA tile
constexpr uint32_t kBBytes = kTN * kTK * 2;    // 16 KB (hi or lo)
constexpr uint32_t kStageBytes = kMT * kABytes + 2 * kBBytes;
constexpr uint32_t kTmemCols = kMT * kTN;      // FP32 accumulators: 128 lanes x 512 columns
constexpr unsigned long long kGemmWaitNs = 250ull * 1000 * 1000;

// FP8 variant (codes of at most 4 bits): the centred codes are exact in e4m3, and the residual
// is split into three e4m3 terms (about 12 significant bits). A stage holds 64 rows of Q, still
// 64 bytes per operand row, so the layouts and descriptors are those of the f16 kernel;
// tcgen05.mma kind::f8f6f4 takes K = 32 per instruction, so 64 rows take 2 x 2 x 3 MMAs
// (12, against 16 for 64 rows of the f16 split).
constexpr int kTK8 = 64;                       // rows of Q per stage: 64 bytes of e4m3
constexpr int kTerms8 = 3;                     // e4m3 terms of the residual
constexpr int kStages8 = 3;
constexpr uint32_t kBBytes8 = kTN * kTK8;      // 16 KB per term
constexpr uint32_t kStageBytes8 = kMT * kABytes + kTerms8 * kBBytes8;

template <bool F8> struct GemmShape {
    static constexpr int tk = F8 ? kTK8 : kTK;
    static constexpr int stages = F8 ? kStages8 : kStages;
    static constexpr int terms = F8 ? kTerms8 : 2;
    static constexpr uint32_t bbytes = F8 ? kBBytes8 : kBBytes;
    static constexpr uint32_t stage_bytes = F8 ? kStageBytes8 : kStageBytes;
};

// instruction descriptor of tcgen05.mma kind::f16: D FP32, A and B f16, both K-major,
// N = 256, M = 128
constexpr uint32_t kIdesc = (1u << 4) | ((uint32_t)(kTN >> 3) << 17) | ((uint32_t)(kTM >> 4) << 24);

__device__ __forceinline__ uint32_t s_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long g_now()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// shared-memory matrix descriptor: K-major, 64-byte swizzle, 8-row groups 512 bytes apart
__device__ __forceinline__ uint64_t sw64_desc(uint32_t saddr)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(512 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
}

__device__ __forceinline__ void bar_init(uint64_t* b, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s_u32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void bar_arrive(uint64_t* b)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(s_u32(b)) : "memory");
}

__device__ __forceinline__ void bar_expect(uint64_t* b, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s_u32(b)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool bar_test(uint64_t* b, unsigned parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(s_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase of the given parity; false if the CTA aborted or the wait ran out
// (which aborts the CTA and records the timeout).
__device__ __forceinline__ bool bar_wait(uint64_t* b, unsigned parity, volatile int* abort_flag, int* status)
{
    if (bar_test(b, parity)) return true;
    const unsigned long long t0 = g_now();
    for (;;) {
        if (bar_test(b, parity)) return true;
        if (*abort_flag) return false;
        if (g_now() - t0 > kGemmWaitNs) {
            *abort_flag = 1;
            atomicExch(status, (int)QIHT_ERR_TIMEOUT);
            return false;
        }
    }
}

// the same wait, unconditional on the abort flag (draining what this CTA issued)
__device__ __forceinline__ bool bar_drain(uint64_t* b, unsigned parity)
{
    const unsigned long long t0 = g_now();
    while (!bar_test(b, parity))
        if (g_now() - t0 > kGemmWaitNs) return false;
    return true;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(s_u32(bar))
        : "memory");
}

__device__ __forceinline__ void mma_f16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
        : "memory");
}

// the same with e4m3 operands (the descriptor's format fields: 0 = e4m3 for A and B)
__device__ __forceinline__ void mma_f8(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
        : "memory");
}

// one f16 value (the low 16 bits of h) -> its e4m3 byte; the pair converted holds the value
// twice, so the result does not depend on which half goes to which byte
__device__ __forceinline__ uint32_t h_to_e4m3(uint32_t h)
{
    const uint32_t hh = (h & 0xffffu) * 0x00010001u;
    uint16_t r;
    asm("cvt.rn.satfinite.e4m3x2.f16x2 %0, %1;" : "=h"(r) : "r"(hh));
    return (uint32_t)r & 0xffu;
}

// two f16 values that are exact in e4m3 -> two e4m3 bytes in the same order (low 16 bits)
__device__ __forceinline__ uint32_t h2_to_e4m3x2(uint32_t h2)
{
    return h_to_e4m3(h2) | (h_to_e4m3(h2 >> 16) << 8);
}

__device__ __forceinline__ void mma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(s_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// four codes (one per byte, < 256) -> two half2 holding 2c - lm1, exactly: the bytes become
// the f16 values 1024 + c, then (x - 1024) * 2 - lm1
__device__ __forceinline__ void codes4_to_h2(uint32_t bytes4, __half2 two, __half2 m2048, __half2 lm1h,
                                             uint32_t& out01, uint32_t& out23)
{
    uint32_t a, b;
    asm("prmt.b32 %0, %1, %2, 0x4140;" : "=r"(a) : "r"(bytes4), "r"(0x64646464u));
    asm("prmt.b32 %0, %1, %2, 0x4342;" : "=r"(b) : "r"(bytes4), "r"(0x64646464u));
    __half2 ha = *reinterpret_cast<__half2*>(&a), hb = *reinterpret_cast<__half2*>(&b);
    ha = __hsub2(__hfma2(ha, two, m2048), lm1h);
    hb = __hsub2(__hfma2(hb, two, m2048), lm1h);
    out01 = *reinterpret_cast<uint32_t*>(&ha);
    out23 = *reinterpret_cast<uint32_t*>(&hb);
}

struct GemmArgs {
    Codes Q;                  // m x n codes (column-packed)
    const float* sc;          // nrhs_pad: alpha 2^e_k per right-hand side
    float* G;                 // nrhs x ldg
    long long ldg;
    int nrhs;                 // right-hand sides stored (columns of D beyond are dropped)
    int nk;                   // K stages: ceil(m / 32)
    int ntn;                  // N tiles
    int rhi;                  // row of the first lo part in the R tensor (= nrhs_pad)
    int* status;
    // tiles [0, nfull) take one CTA each over all nk stages; every later tile takes two, one per
    // half of the stages ([0, khalf) and [khalf, nk)), whose products add into G (zeroed first)
    int nfull;
    int khalf;
};

template <int BITS, bool F8>
__global__ void __launch_bounds__(kGemmThreads, 1) k_mrhs_gemm(const __grid_constant__ CUtensorMap rmap, GemmArgs a)
{
    using Sh = GemmShape<F8>;
    constexpr int WPS = Sh::tk * BITS / 32;    // code words per column per stage (32 or 64 codes)
    constexpr uint32_t MASK8 = 0x01010101u * ((1u << BITS) - 1);
    constexpr int PD = 3;                      // stages of codes a converter has in flight
    constexpr int PL = 8 / BITS;               // 4-code planes per word
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full_a[kStages], full_b[kStages], empty[kStages], done;
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_abort;

    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int tile = blockIdx.x, kb = 0, ke = a.nk;
    const bool part = (int)blockIdx.x >= a.nfull;
    if (part) {
        const int u = (int)blockIdx.x - a.nfull;
        tile = a.nfull + (u >> 1);
        if (u & 1) kb = a.khalf;
        else ke = a.khalf;
    }
    const int tm = tile / a.ntn, tn = tile % a.ntn;
    const int m0 = tm * kTM * kMT, n0 = tn * kTN;

    if (tid == 0) {
        for (int i = 0; i < Sh::stages; ++i) {
            bar_init(&full_a[i], kConvWarps);
            bar_init(&full_b[i], 1);
            bar_init(&empty[i], 1);
        }
        bar_init(&done, 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_u32(&s_tmem)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    auto stage_a = [&](int s) { return smem + (size_t)s * Sh::stage_bytes; };
    auto stage_b = [&](int s, int t) { return smem + (size_t)s * Sh::stage_bytes + kMT * kABytes + (size_t)t * Sh::bbytes; };

    if (warp == 0) {
        // ---- TMA producer of the R tiles (hi and lo parts) ----
        if (lane == 0) {
            int issued = 0;
            for (int it = kb; it < ke; ++it) {
                const int rr = it - kb;             // stages are counted from this CTA's first
                const int s = rr % Sh::stages;
                const unsigned u = (unsigned)(rr / Sh::stages);
                if (rr >= Sh::stages && !bar_wait(&empty[s], (u & 1u) ^ 1u, &s_abort, a.status)) break;
                bar_expect(&full_b[s], Sh::terms * Sh::bbytes);
#pragma unroll
                for (int t = 0; t < Sh::terms; ++t)
                    tma_load_2d(s_u32(stage_b(s, t)), &rmap, it * Sh::tk, t * a.rhi + n0, &full_b[s]);
                ++issued;
            }
            // no copy may still be in flight when the CTA leaves
            for (int s = 0; s < Sh::stages && s < issued; ++s) {
                const int last = s + ((issued - 1 - s) / Sh::stages) * Sh::stages;
                bar_drain(&full_b[s], (unsigned)(last / Sh::stages) & 1u);
            }
        }
    } else if (warp == 1) {
        // ---- MMA issuer ----
        if (lane == 0) {
            for (int it = kb; it < ke; ++it) {
                const int s = (it - kb) % Sh::stages;
                const unsigned par = (unsigned)((it - kb) / Sh::stages) & 1u;
                if (!bar_wait(&full_a[s], par, &s_abort, a.status)) break;
                if (!bar_wait(&full_b[s], par, &s_abort, a.status)) break;
                tc_fence_after();
                const uint32_t ab = s_u32(stage_a(s));
                // 32 bytes of every operand row per MMA: K = 16 f16 or K = 32 e4m3
#pragma unroll
                for (int kk = 0; kk < 2; ++kk) {
#pragma unroll
                    for (int t = 0; t < kMT; ++t) {
                        const uint64_t ad = sw64_desc(ab + t * kABytes + 32 * kk);
#pragma unroll
                        for (int u = 0; u < Sh::terms; ++u) {
                            const uint64_t bd = sw64_desc(s_u32(stage_b(s, u)) + 32 * kk);
                            const uint32_t acc = ((it - kb) | kk | u) != 0;
                            if (F8) mma_f8(tmem + (uint32_t)(t * kTN), ad, bd, acc);
                            else mma_f16(tmem + (uint32_t)(t * kTN), ad, bd, acc);
                        }
                    }
                }
                mma_commit(&empty[s]);
            }
            mma_commit(&done);                 // tracks every MMA issued above
        }
        __syncwarp();
    } else {
        // ---- converters (A tiles), then the epilogue ----
        const int ct = tid - 64;               // column m0 + ct of Q: row ct % 128 of A tile ct / 128
        const int j = m0 + ct;
        const bool colok = j < a.Q.cols;
        const uint32_t* col = a.Q.words + (size_t)(colok ? j : 0) * a.Q.ld;
        const int ldw = a.Q.ld;
        const __half2 two = __float2half2_rn(2.0f), m2048 = __float2half2_rn(-2048.0f);
        const __half2 lm1h = __float2half2_rn((float)a.Q.lm1);
        uint32_t ring[PD][WPS];
        auto fetch = [&](int it, uint32_t (&w)[WPS]) {
#pragma unroll
            for (int q = 0; q < WPS; q += (WPS >= 4 ? 4 : WPS)) {
                const int wo = it * WPS + q;
                if (WPS >= 4) {
                    uint4 v = make_uint4(0, 0, 0, 0);
                    if (colok && it < ke && wo + 4 <= ldw)
                        v = __ldg(reinterpret_cast<const uint4*>(col + wo));
                    w[q] = v.x; w[q + 1] = v.y; w[q + 2] = v.z; w[q + 3] = v.w;
                } else {
                    uint2 v = make_uint2(0, 0);
                    if (colok && it < ke && wo + 2 <= ldw)
                        v = __ldg(reinterpret_cast<const uint2*>(col + wo));
                    w[q] = v.x; w[q + 1] = v.y;
                }
            }
        };
#pragma unroll
        for (int p = 0; p < PD; ++p) fetch(kb + p, ring[p]);
        for (int it = kb; it < ke; ++it) {
            const int s = (it - kb) % Sh::stages;
            const unsigned u = (unsigned)((it - kb) / Sh::stages);
            uint32_t cur[WPS];
#pragma unroll
            for (int q = 0; q < WPS; ++q) {
                cur[q] = ring[0][q];
#pragma unroll
                for (int p = 0; p + 1 < PD; ++p) ring[p][q] = ring[p + 1][q];
            }
            fetch(it + PD, ring[PD - 1]);
            // the whole warp leaves together (the arrive and the epilogue's loads are warp-wide)
            if (it - kb >= Sh::stages && !__all_sync(0xffffffffu, bar_wait(&empty[s], (u & 1u) ^ 1u, &s_abort, a.status)))
                break;
            // the stage's codes of column j in K order -> f16 values (then e4m3), 64 bytes per row
            uint32_t h[Sh::tk / 2];
#pragma unroll
            for (int q = 0; q < WPS; ++q) {
#pragma unroll
                for (int e = 0; e < PL; ++e) {
                    // plane e of word q: rows q*G + 4e .. + 3 (G = 32 / BITS codes per word)
                    const uint32_t plane = (cur[q] >> (BITS * e)) & MASK8;
                    const int k = q * (32 / BITS) + 4 * e;      // first K index of the plane
                    codes4_to_h2(plane, two, m2048, lm1h, h[k / 2], h[k / 2 + 1]);
                }
            }
            unsigned char* A = stage_a(s) + (ct / kTM) * kABytes;
            const int row = ct % kTM, sw = (row >> 1) & 3;
            if (F8) {
#pragma unroll
                for (int i = 0; i < Sh::tk / 4; ++i) h[i] = h2_to_e4m3x2(h[2 * i]) | (h2_to_e4m3x2(h[2 * i + 1]) << 16);
            }
#pragma unroll
            for (int c = 0; c < 4; ++c)
                *reinterpret_cast<uint4*>(A + row * 64 + ((c ^ sw) << 4)) =
                    make_uint4(h[4 * c], h[4 * c + 1], h[4 * c + 2], h[4 * c + 3]);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) bar_arrive(&full_a[s]);
        }
        // ---- epilogue: the rows of this warp's lane quarter of accumulator (warp - 2) / 4 ----
        const bool fin = __all_sync(0xffffffffu, bar_drain(&done, 0u));
        tc_fence_after();
        if (__all_sync(0xffffffffu, fin && !s_abort)) {
            const int quarter = warp & 3, t = (warp - 2) / 4;
            const int row = 32 * quarter + lane;
            const int jj = m0 + t * kTM + row;
            for (int c0 = 0; c0 < kTN; c0 += 16) {
                uint32_t v[16];
                tmem_ld16(tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(t * kTN + c0), v);
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int k = n0 + c0 + i;
                    if (jj < a.Q.cols && k < a.nrhs) {
                        const float gv = __uint_as_float(v[i]) * a.sc[k];
                        if (part) atomicAdd(a.G + (size_t)k * a.ldg + jj, gv);   // two terms onto zero: order-free
                        else a.G[(size_t)k * a.ldg + jj] = gv;
                    }
                }
            }
        } else if (!fin) {
            atomicExch(a.status, (int)QIHT_ERR_TIMEOUT);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

// Residuals -> scaled f16 parts: one CTA per right-hand side (rows k >= nrhs of the padded
// tensor become zeros). e_k puts max |r_k| 2^-e_k in [2^14, 2^15); sc_k = alpha 2^e_k.
__global__ void __launch_bounds__(256) k_mrhs_split(const float* __restrict__ R, long long ldr, int m, int nrhs,
                                                    int mk, int rhi, __half* __restrict__ R16,
                                                    float* __restrict__ sc, const float* __restrict__ scale, int lm1)
{
    const int k = blockIdx.x;
    __shared__ unsigned s_max[8];
    unsigned mx = 0;
    const float* r = R + (size_t)k * ldr;
    if (k < nrhs)
        for (int i = threadIdx.x; i < m; i += 256) mx = max(mx, __float_as_uint(r[i]) & 0x7fffffffu);
    mx = __reduce_max_sync(0xffffffffu, mx);
    if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = mx;
    __syncthreads();
    unsigned M = 0;
    for (int w = 0; w < 8; ++w) M = max(M, s_max[w]);
    int e = 0;
    const float Mf = __uint_as_float(M);
    if (Mf > 0.0f && isfinite(Mf)) {
        int ex;
        frexpf(Mf, &ex);
        e = ex - 15;
    }
    __half* hi = R16 + (size_t)k * mk;
    __half* lo = R16 + (size_t)(rhi + k) * mk;
    for (int i = threadIdx.x; i < mk; i += 256) {
        const float v = (k < nrhs && i < m) ? ldexpf(r[i], -e) : 0.0f;
        const __half h = __float2half_rn(v);
        hi[i] = h;
        lo[i] = __float2half_rn(v - __half2float(h));
    }
    if (threadIdx.x == 0) sc[k] = (float)ldexp((double)*scale / (double)lm1, e);
}

// Residuals -> three scaled e4m3 terms (FP8 variant): e_k puts max |r_k| 2^-e_k in [2^7, 2^8)
// (e4m3 reaches 448); term 1 = e4m3(r'), term 2 = e4m3(r' - term 1), term 3 = e4m3 of what is
// left, each a row of bytes (term t of right-hand side k at row t * rhi + k).
__global__ void __launch_bounds__(256) k_mrhs_split8(const float* __restrict__ R, long long ldr, int m, int nrhs,
                                                     int mk, int rhi, unsigned char* __restrict__ R8,
                                                     float* __restrict__ sc, const float* __restrict__ scale, int lm1)
{
    const int k = blockIdx.x;
    __shared__ unsigned s_max[8];
    unsigned mx = 0;
    const float* r = R + (size_t)k * ldr;
    if (k < nrhs)
        for (int i = threadIdx.x; i < m; i += 256) mx = max(mx, __float_as_uint(r[i]) & 0x7fffffffu);
    mx = __reduce_max_sync(0xffffffffu, mx);
    if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = mx;
    __syncthreads();
    unsigned M = 0;
    for (int w = 0; w < 8; ++w) M = max(M, s_max[w]);
    int e = 0;
    const float Mf = __uint_as_float(M);
    if (Mf > 0.0f && isfinite(Mf)) {
        int ex;
        frexpf(Mf, &ex);
        e = ex - 8;
    }
    for (int i = threadIdx.x; i < mk; i += 256) {
        float v = (k < nrhs && i < m) ? ldexpf(r[i], -e) : 0.0f;
#pragma unroll
        for (int t = 0; t < kTerms8; ++t) {
            const uint32_t b = f_to_e4m3(v);
            R8[(size_t)(t * rhi + k) * mk + i] = (unsigned char)b;
            v -= e4m3_to_f(b);                     // exact: v and the term are close
        }
    }
    if (threadIdx.x == 0) sc[k] = (float)ldexp((double)*scale / (double)lm1, e);
}

// G = 0 on the tiles [t0, t0 + gridDim.x / kTN) that two CTAs add into: one block per (tile,
// right-hand side), one thread per column
__global__ void __launch_bounds__(kTM * kMT) k_mrhs_zero_tiles(float* __restrict__ G, long long ldg, int n, int nrhs,
                                                               int ntn, int t0)
{
    const int tile = t0 + (int)blockIdx.x / kTN, kk = (int)blockIdx.x % kTN;
    const int tm = tile / ntn, tn = tile % ntn;
    const int k = tn * kTN + kk, jj = tm * kTM * kMT + (int)threadIdx.x;
    if (k < nrhs && jj < n) G[(size_t)k * ldg + jj] = 0.0f;
}
}  // namespace

size_t mrhs_gemm_smem() { return (size_t)kStages * kStageBytes + 1024; }
size_t mrhs_gemm_smem8() { return (size_t)kStages8 * kStageBytes8 + 1024; }

int mrhs_pad_rhs(int nrhs) { return (nrhs + kTN - 1) / kTN * kTN; }
int mrhs_pad_rows(int m) { return (m + kTK - 1) / kTK * kTK; }
int mrhs_pad_rows8(int m) { return (m + kTK8 - 1) / kTK8 * kTK8; }

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link against libcuda)
static EncodeFn tensor_map_encoder()
{
    static EncodeFn encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return nullptr;
        encode = reinterpret_cast<EncodeFn>(fn);
    }
    return encode;
}

// Tensor map of the e4m3 residual terms: rows of mk bytes (K), 3 * nrhs_pad rows.
cudaError_t mrhs_make_map8(void* map, const void* R8, int mk, int rows)
{
    EncodeFn encode = tensor_map_encoder();
    if (!encode) return cudaErrorNotSupported;
    const cuuint64_t dims[2] = {(cuuint64_t)mk, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)mk};
    const cuuint32_t box[2] = {(cuuint32_t)kTK8, (cuuint32_t)kTN};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = encode(reinterpret_cast<CUtensorMap*>(map), CU_TENSOR_MAP_DATA_TYPE_UINT8, 2,
                              const_cast<void*>(R8), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_mrhs_split8(const float* R, long long ldr, int m, int nrhs, void* R8, float* sc,
                               const float* scale, int lm1, cudaStream_t s)
{
    const int np = mrhs_pad_rhs(nrhs), mk = mrhs_pad_rows8(m);
    k_mrhs_split8<<<np, 256, 0, s>>>(R, ldr, m, nrhs, mk, np, reinterpret_cast<unsigned char*>(R8), sc, scale, lm1);
    return cudaGetLastError();
}

// Tensor map of the f16 residual parts: rows of mk halves (K), 2 * nrhs_pad rows (hi, then lo).
cudaError_t mrhs_make_map(void* map, const void* R16, int mk, int rows)
{
    EncodeFn encode = tensor_map_encoder();
    if (!encode) return cudaErrorNotSupported;
    const cuuint64_t dims[2] = {(cuuint64_t)mk, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)mk * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kTK, (cuuint32_t)kTN};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = encode(reinterpret_cast<CUtensorMap*>(map), CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
                              const_cast<void*>(R16), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_mrhs_split(const float* R, long long ldr, int m, int nrhs, void* R16, float* sc,
                              const float* scale, int lm1, cudaStream_t s)
{
    const int np = mrhs_pad_rhs(nrhs), mk = mrhs_pad_rows(m);
    k_mrhs_split<<<np, 256, 0, s>>>(R, ldr, m, nrhs, mk, np, reinterpret_cast<__half*>(R16), sc, scale, lm1);
    return cudaGetLastError();
}

cudaError_t launch_mrhs_gemm(const Codes& Q, const void* map, const float* sc, float* G, long long ldg, int nrhs,
                             int* status, cudaStream_t s, bool fp8)
{
    GemmArgs a;
    a.Q = Q;
    a.sc = sc;
    a.G = G;
    a.ldg = ldg;
    a.nrhs = nrhs;
    a.nk = mrhs_pad_rows(Q.rows) / kTK;
    a.ntn = mrhs_pad_rhs(nrhs) / kTN;
    a.rhi = mrhs_pad_rhs(nrhs);
    a.status = status;
    const int ntm = (Q.cols + kTM * kMT - 1) / (kTM * kMT);
    const size_t smem = fp8 ? mrhs_gemm_smem8() : mrhs_gemm_smem();
    if (fp8) a.nk = mrhs_pad_rows8(Q.rows) / kTK8;
    if (fp8 && Q.bits == 8) return cudaErrorInvalidValue;     // 8-bit codes are not exact in e4m3
    void* fn = fp8 ? (Q.bits == 4 ? (void*)k_mrhs_gemm<4, true> : (void*)k_mrhs_gemm<2, true>)
                   : (Q.bits == 8 ? (void*)k_mrhs_gemm<8, false>
                                  : Q.bits == 4 ? (void*)k_mrhs_gemm<4, false> : (void*)k_mrhs_gemm<2, false>);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // One CTA per SM: a last wave of few tiles would keep most SMs idle for a whole tile's time.
    // When it holds at most half the SMs, each of its tiles is split into two halves of the
    // stages (two CTAs adding into G), so the wave takes about half as long.
    const int ntiles = ntm * a.ntn, nsm = num_sms();
    const int tail = ntiles % nsm;
    const bool split = ntiles > nsm && tail > 0 && 2 * tail <= nsm && a.nk >= 2;
    a.nfull = split ? ntiles - tail : ntiles;
    a.khalf = a.nk / 2;
    if (split) {
        k_mrhs_zero_tiles<<<(unsigned)(tail * kTN), kTM * kMT, 0, s>>>(G, ldg, Q.cols, nrhs, a.ntn, a.nfull);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    CUtensorMap m;
    memcpy(&m, map, sizeof(m));
    void* args[] = {(void*)&m, (void*)&a};
    return cudaLaunchKernel(fn, dim3((unsigned)(split ? a.nfull + 2 * tail : ntiles)), dim3(kGemmThreads), args, smem, s);
}

}  // namespace qiht
