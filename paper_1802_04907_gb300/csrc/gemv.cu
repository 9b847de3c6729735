// g = Q^T r over column-packed b-bit codes: the gradient product of Algorithm 2
// (g = Q1^T (Q(y) - Q2 x)), one full pass over the codes per call.
//
// Arithmetic. On a grid of L levels (2^b, or 2^(b-1) + 1 on the odd grid) the value of
// code c is alpha * (2c - (L-1)), alpha = scale / (L-1),
// so  g_j = alpha * (2 * sum_i c_ij r_i - (L-1) * sum_i r_i).
// r is converted once per call to 24-bit block fixed point, r_i ~ rf_i * 2^-sh
// with a power-of-two scale from max |r| (|rf_i| < 2^22), and rf_i is split into
// three bytes (two unsigned, the top one signed). Codes are multiplied with the
// byte limbs by dp4a (four 8-bit products summed into 32 bits), so every inner
// sum is an exact integer; only the final per-column scaling rounds. The result
// is independent of the summation order (deterministic).
//
// Mapping. A CTA holds the fixed-point residual in registers: thread t owns rows
// [t*RPT, t*RPT + RPT) of the padded column (TPC threads span a column). The
// CTA walks a contiguous range of column groups (CPW columns each); a slot of
// TPC threads reads CPW columns at a time with coalesced vector loads, and the
// per-column integer sums are reduced across the slot with warp reductions.
#include <cstdlib>

#include "internal.cuh"

namespace qiht {

__device__ __forceinline__ uint32_t dp4a_uu(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("dp4a.u32.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

__device__ __forceinline__ int32_t dp4a_us(uint32_t a, uint32_t b, int32_t c)
{
    int32_t d;
    asm("dp4a.u32.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

// Load this thread's NW words of one column (word offset w0 of a column of ld
// words, ld a multiple of 4). Pieces past the column end read as zero codes.
template <int NW>
__device__ __forceinline__ void load_words(const uint32_t* __restrict__ col, int w0, int ld, uint32_t (&w)[NW])
{
    if constexpr (NW % 4 == 0) {
#pragma unroll
        for (int v = 0; v < NW / 4; ++v) {
            if (w0 + 4 * v + 4 <= ld) {
                asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                             : "=r"(w[4 * v]), "=r"(w[4 * v + 1]), "=r"(w[4 * v + 2]), "=r"(w[4 * v + 3])
                             : "l"(col + w0 + 4 * v));
            } else {
                w[4 * v] = w[4 * v + 1] = w[4 * v + 2] = w[4 * v + 3] = 0u;
            }
        }
    } else if constexpr (NW == 2) {
        if (w0 + 2 <= ld)
            asm volatile("ld.global.nc.L1::no_allocate.v2.u32 {%0,%1}, [%2];" : "=r"(w[0]), "=r"(w[1]) : "l"(col + w0));
        else
            w[0] = w[1] = 0u;
    } else {
        static_assert(NW == 1, "words per thread");
        if (w0 + 1 <= ld)
            asm volatile("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(w[0]) : "l"(col + w0));
        else
            w[0] = 0u;
    }
}

// Power-of-two exponent sh so that |r| * 2^sh < 2^22 for all r (0 if r == 0).
__device__ __forceinline__ int fixed_shift(unsigned rmax_bits)
{
    const float M = __uint_as_float(rmax_bits);
    if (!(M > 0.0f) || !isfinite(M)) return 0;
    int ex;
    frexpf(M, &ex);          // M = f * 2^ex, 0.5 <= f < 1, so M < 2^ex
    return 22 - ex;
}

template <int BITS, int CPW, int RPT>
__global__ void __launch_bounds__(256) k_gemv_t(GemvTArgs a, int tpc)
{
    constexpr int G = 32 / BITS;          // codes per word
    constexpr int E = G / 4;              // 4-code extractions per word
    constexpr uint32_t MASK = 0x01010101u * ((1u << BITS) - 1);
    constexpr int NW = RPT / G;           // words per thread per column
    constexpr int NL = RPT / 4;           // limb words per limb per thread

    griddep_wait();
    if (a.h_outer && blockIdx.x == 0 && threadIdx.x == 0) {
        // the solver's outer loop continues while not stopped, and never more than
        // iters + 1 times even if a stop were missed
        const int guard = ++a.st->outer_guard;
        cudaGraphSetConditional((cudaGraphConditionalHandle)a.h_outer,
                                (!a.st->stop && guard < a.guard_limit) ? 1u : 0u);
    }
    if (a.st && a.st->stop) return;
    const int m = a.Q.rows, n = a.Q.cols, ld = a.Q.ld;
    const int slots = 256 / tpc;
    const int slot = threadIdx.x / tpc;
    const int t = threadIdx.x % tpc;              // thread within the slot
    const int w0 = t * NW;                        // first word of this thread in a column
    const bool active = w0 < ld;
    const int sh = fixed_shift(*a.rmax_bits);

    // fixed-point residual limbs of rows [t*RPT, t*RPT + RPT)
    uint32_t l0[NL], l1[NL], l2[NL];
    long long rsum = 0;
#pragma unroll
    for (int q = 0; q < NL; ++q) {
        uint32_t b0 = 0, b1 = 0, b2 = 0;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const int i = t * RPT + 4 * q + p;
            int v = 0;
            if (i < m) v = __float2int_rn(ldexpf(a.r[i], sh));
            rsum += v;
            b0 |= (uint32_t)(v & 255) << (8 * p);
            b1 |= (uint32_t)((v >> 8) & 255) << (8 * p);
            b2 |= (uint32_t)((v >> 16) & 255) << (8 * p);
        }
        l0[q] = b0; l1[q] = b1; l2[q] = b2;
    }

    // sum of the fixed-point residual over the slot's rows (every slot holds all rows)
    __shared__ long long red_r[8];
    __shared__ long long red_c[2][8][CPW * 3];
    {
        long long v = rsum;
#pragma unroll
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) red_r[threadIdx.x >> 5] = v;
    }
    __syncthreads();
    const int wps = tpc >> 5;                     // warps per slot (tpc >= 32)
    long long R = 0;
    for (int w = 0; w < wps; ++w) R += red_r[w];  // slot 0's rows = all rows
    R *= a.Q.lm1;                                 // (L-1) sum_i r_i

    const double alpha = (double)(*a.Q.scale) / (double)a.Q.lm1;
    const double outscale = ldexp(alpha, -sh);

    const int ncg = (n + CPW - 1) / CPW;
    // contiguous range of column groups for this CTA, split over its slots
    const long long per = ((long long)ncg + gridDim.x - 1) / gridDim.x;
    const int cg_begin = (int)min((long long)ncg, per * blockIdx.x);
    const int cg_end = (int)min((long long)ncg, per * (blockIdx.x + 1));
    int buf = 0;
    for (int cgb = cg_begin; cgb < cg_end; cgb += slots) {
        const int cg = cgb + slot;
        uint32_t a0[CPW], a1[CPW];
        int32_t a2[CPW];
#pragma unroll
        for (int c = 0; c < CPW; ++c) { a0[c] = 0; a1[c] = 0; a2[c] = 0; }
        if (cg < cg_end && active) {
            uint32_t cw[CPW][NW];
#pragma unroll
            for (int c = 0; c < CPW; ++c) {
                const int j = min(cg * CPW + c, n - 1);
                load_words<NW>(a.Q.words + (size_t)j * ld, w0, ld, cw[c]);
            }
#pragma unroll
            for (int c = 0; c < CPW; ++c) {
#pragma unroll
                for (int q = 0; q < NW; ++q) {
#pragma unroll
                    for (int k = 0; k < E; ++k) {
                        const uint32_t x = (cw[c][q] >> (BITS * k)) & MASK;
                        const int li = q * E + k;
                        a0[c] = dp4a_uu(x, l0[li], a0[c]);
                        a1[c] = dp4a_uu(x, l1[li], a1[c]);
                        a2[c] = dp4a_us(x, l2[li], a2[c]);
                    }
                }
            }
        }
        // reduce over the slot: warp sums, then the slot's warps in shared memory
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
        for (int c = 0; c < CPW; ++c) {
            const uint32_t s0 = __reduce_add_sync(0xffffffffu, a0[c]);
            const uint32_t s1 = __reduce_add_sync(0xffffffffu, a1[c]);
            const int32_t s2 = __reduce_add_sync(0xffffffffu, a2[c]);
            if (lane == 0) {
                red_c[buf][warp][3 * c + 0] = (long long)s0;
                red_c[buf][warp][3 * c + 1] = (long long)s1;
                red_c[buf][warp][3 * c + 2] = (long long)s2;
            }
        }
        __syncthreads();
        if (t < CPW && cg < cg_end) {
            const int c = t;
            const int j = cg * CPW + c;
            if (j < n) {
                long long S0 = 0, S1 = 0, S2 = 0;
                for (int w = 0; w < wps; ++w) {
                    S0 += red_c[buf][slot * wps + w][3 * c + 0];
                    S1 += red_c[buf][slot * wps + w][3 * c + 1];
                    S2 += red_c[buf][slot * wps + w][3 * c + 2];
                }
                const long long S = S0 + (S1 << 8) + (S2 << 16);
                const long long T = 2 * S - R;
                a.g[j] = (float)((double)T * outscale);
            }
        }
        buf ^= 1;   // double-buffered partials: the next group's writes do not race these reads
    }
}

// ---------------------------------------------------------------------------
// TMA-staged variant. One CTA per SM walks a contiguous range of columns (its
// bytes are contiguous in the column-packed layout). A producer warp streams
// stages of CPSL*slots columns into a ring of shared-memory buffers with
// cp.async.bulk (completion counted in bytes on an mbarrier); 16 consumer warps
// hold the fixed-point residual in registers and read each code once from
// shared memory (16-byte pieces, consecutive threads on consecutive pieces).
// Every wait is bounded by %globaltimer; a timeout sets the status and the CTA
// drains its own copies before leaving.
// ---------------------------------------------------------------------------
constexpr int kTmaConsumers = 512;
constexpr int kTmaThreads = kTmaConsumers + 32;
constexpr int kTmaWarps = kTmaConsumers / 32;
constexpr int kTmaRingBytes = 196608;        // stage ring (192 KiB)
constexpr unsigned long long kWaitBudgetNs = 200ull * 1000 * 1000;   // 0.2 s per wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase of the given parity to complete; false after the time budget.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (globaltimer_ns() - t0 > kWaitBudgetNs) return false;
    }
    return true;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void consumer_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kTmaConsumers) : "memory"); }

__device__ __forceinline__ void report_timeout(const GemvTArgs& a)
{
    if (a.st) {
        a.st->status = QIHT_ERR_TIMEOUT;
        a.st->stop = 1;
    }
    if (a.err) atomicExch(a.err, 1u);
}

template <int BITS, int PPT, int CPSL>
__global__ void __launch_bounds__(kTmaThreads, 1) k_gemv_t_tma(GemvTArgs a, int tpc, int nstage_buf)
{
    constexpr int G = 32 / BITS;
    constexpr int E = G / 4;
    constexpr uint32_t MASK = 0x01010101u * ((1u << BITS) - 1);
    constexpr int NLW = PPT * 4 * E;            // limb words per limb per thread

    extern __shared__ __align__(128) unsigned char smem[];
    griddep_wait();
    if (a.h_outer && blockIdx.x == 0 && threadIdx.x == 0) {
        const int guard = ++a.st->outer_guard;
        cudaGraphSetConditional((cudaGraphConditionalHandle)a.h_outer,
                                (!a.st->stop && guard < a.guard_limit) ? 1u : 0u);
    }
    if (a.st && a.st->stop) return;

    const int n = a.Q.cols, ld = a.Q.ld, m = a.Q.rows;
    const int P = ld / 4;                        // 16-byte pieces per column
    const unsigned colbytes = (unsigned)ld * 4u;
    const int slots = kTmaConsumers / tpc;
    const int cps = CPSL * slots;                // columns per stage
    const unsigned stage_bytes = (unsigned)cps * colbytes;
    const int NS = nstage_buf;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)NS * stage_bytes);
    uint64_t* empty = full + NS;
    unsigned long long* acc = reinterpret_cast<unsigned long long*>(empty + NS);   // [NS][cps][3]
    unsigned* cnt = reinterpret_cast<unsigned*>(acc + (size_t)NS * cps * 3);       // [NS][cps]
    long long* red_r = reinterpret_cast<long long*>(cnt + (((size_t)NS * cps + 1) & ~(size_t)1));  // [warps]
    __shared__ int s_abort;

    const int c0 = (int)((long long)n * blockIdx.x / gridDim.x);
    const int c1 = (int)((long long)n * (blockIdx.x + 1) / gridDim.x);
    const int ncols = c1 - c0;
    const int nst = (ncols + cps - 1) / cps;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    for (int i = threadIdx.x; i < NS * cps * 3; i += blockDim.x) acc[i] = 0ull;
    for (int i = threadIdx.x; i < NS * cps; i += blockDim.x) cnt[i] = 0u;
    if (threadIdx.x == 0) {
        s_abort = 0;
        for (int i = 0; i < NS; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], kTmaWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == kTmaWarps) {
        // producer
        if (lane == 0) {
            int issued = 0;
            bool ok = true;
            for (int it = 0; it < nst; ++it) {
                const int sb = it % NS;
                const unsigned ph = (unsigned)(it / NS) & 1u;
                if (*(volatile int*)&s_abort) { ok = false; break; }
                if (it >= NS && !mbar_wait(&empty[sb], ph ^ 1u)) { ok = false; break; }
                const int cols_here = min(cps, ncols - it * cps);
                const unsigned bytes = (unsigned)cols_here * colbytes;
                mbar_expect_tx(&full[sb], bytes);
                bulk_g2s(smem + (size_t)sb * stage_bytes,
                         reinterpret_cast<const unsigned char*>(a.Q.words) + (size_t)(c0 + it * cps) * colbytes,
                         bytes, &full[sb]);
                ++issued;
            }
            if (!ok) {
                report_timeout(a);
                // drain this CTA's own copies (bounded) before leaving
                for (int it = max(0, issued - NS); it < issued; ++it)
                    mbar_wait(&full[it % NS], (unsigned)(it / NS) & 1u);
            }
        }
        return;
    }

    // consumers: fixed-point residual limbs of this thread's pieces
    const int slot = threadIdx.x / tpc;
    const int t = threadIdx.x % tpc;
    const int wps = tpc >> 5;                    // warps per slot
    (void)wps;
    const int sh = fixed_shift(*a.rmax_bits);
    uint32_t l0[NLW], l1[NLW], l2[NLW];
    long long rsum = 0;
#pragma unroll
    for (int pp = 0; pp < PPT; ++pp) {
        const int piece = t + pp * tpc;
#pragma unroll
        for (int q = 0; q < 4 * E; ++q) {
            uint32_t b0 = 0, b1 = 0, b2 = 0;
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const int i = piece * 4 * G + 4 * q + p;
                int v = 0;
                if (piece < P && i < m) v = __float2int_rn(ldexpf(__ldcg(a.r + i), sh));
                rsum += v;
                b0 |= (uint32_t)(v & 255) << (8 * p);
                b1 |= (uint32_t)((v >> 8) & 255) << (8 * p);
                b2 |= (uint32_t)((v >> 16) & 255) << (8 * p);
            }
            l0[pp * 4 * E + q] = b0;
            l1[pp * 4 * E + q] = b1;
            l2[pp * 4 * E + q] = b2;
        }
    }
    {
        long long v = (slot == 0) ? rsum : 0;
#pragma unroll
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red_r[warp] = v;
    }
    consumer_sync();
    long long R = 0;
    for (int w = 0; w < wps; ++w) R += red_r[w];
    R *= a.Q.lm1;                                 // (L-1) sum_i r_i
    const double alpha = (double)(*a.Q.scale) / (double)a.Q.lm1;
    const double outscale = ldexp(alpha, -sh);

    // Steady state: no CTA-wide barrier. Each warp adds its per-column integer sums
    // to shared accumulators with 64-bit atomics (exact, so order does not matter);
    // the last warp of the slot to arrive at a column finishes it and clears the
    // accumulator. A warp releases a stage only after that, so the producer cannot
    // refill a stage (and no warp can reuse its accumulators) before it is finished.
    for (int it = 0; it < nst; ++it) {
        const int sb = it % NS;
        const unsigned ph = (unsigned)(it / NS) & 1u;
        if (!mbar_wait(&full[sb], ph)) {
            if (lane == 0) { s_abort = 1; report_timeout(a); }
            break;
        }
        if (*(volatile int*)&s_abort) break;
        const int cols_here = min(cps, ncols - it * cps);
        const unsigned char* stage = smem + (size_t)sb * stage_bytes;
        uint32_t a0[CPSL], a1[CPSL];
        int32_t a2[CPSL];
#pragma unroll
        for (int cl = 0; cl < CPSL; ++cl) {
            a0[cl] = 0; a1[cl] = 0; a2[cl] = 0;
            const int col = slot * CPSL + cl;
            if (col < cols_here) {
                const uint4* cp = reinterpret_cast<const uint4*>(stage + (size_t)col * colbytes);
#pragma unroll
                for (int pp = 0; pp < PPT; ++pp) {
                    const int piece = t + pp * tpc;
                    if (piece < P) {
                        const uint4 v = cp[piece];
                        const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                        for (int w = 0; w < 4; ++w)
#pragma unroll
                            for (int k = 0; k < E; ++k) {
                                const uint32_t x = (wv[w] >> (BITS * k)) & MASK;
                                const int li = pp * 4 * E + w * E + k;
                                a0[cl] = dp4a_uu(x, l0[li], a0[cl]);
                                a1[cl] = dp4a_uu(x, l1[li], a1[cl]);
                                a2[cl] = dp4a_us(x, l2[li], a2[cl]);
                            }
                    }
                }
            }
        }
        unsigned long long v0 = 0, v1 = 0, v2 = 0;
#pragma unroll
        for (int cl = 0; cl < CPSL; ++cl) {
            const uint32_t s0 = __reduce_add_sync(0xffffffffu, a0[cl]);
            const uint32_t s1 = __reduce_add_sync(0xffffffffu, a1[cl]);
            const int32_t s2 = __reduce_add_sync(0xffffffffu, a2[cl]);
            if (lane == cl) { v0 = s0; v1 = s1; v2 = (unsigned long long)(long long)s2; }
        }
        if (lane < CPSL) {
            const int col = slot * CPSL + lane;
            if (col < cols_here) {
                unsigned long long* ac = acc + ((size_t)sb * cps + col) * 3;
                atomicAdd(ac + 0, v0);
                atomicAdd(ac + 1, v1);
                atomicAdd(ac + 2, v2);
                __threadfence_block();
                const unsigned prev = atomicAdd(&cnt[sb * cps + col], 1u);
                if (prev == (unsigned)wps - 1) {
                    __threadfence_block();
                    volatile unsigned long long* vac = ac;
                    const long long S0 = (long long)vac[0], S1 = (long long)vac[1], S2 = (long long)vac[2];
                    const long long S = S0 + (S1 << 8) + (S2 << 16);
                    const long long T = 2 * S - R;
                    a.g[c0 + it * cps + col] = (float)((double)T * outscale);
                    vac[0] = 0ull; vac[1] = 0ull; vac[2] = 0ull;
                    cnt[sb * cps + col] = 0u;
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[sb]);     // this warp is done with the stage
    }
    // on an abort the producer stops issuing and drains its own copies before the CTA ends
}

// ---------------------------------------------------------------------------
// Column-owning TMA variant (the default). A CTA owns a contiguous range of
// columns and walks it in groups of 32 columns; each group is streamed in row
// chunks of 32 * RC * b / 8 bytes (one cp.async.bulk per column chunk, issued
// by the 32 lanes of the producer warp). Consumer warp w owns columns
// 2w, 2w+1 of every group for the whole group, so its integer sums stay in
// registers across the row chunks and no two warps ever share a column.
// The fixed-point residual lives in shared memory as three byte planes in a
// lane-interleaved layout ([E][piece][4 words]), read with conflict-free 16-byte
// loads and reused for both columns of the warp.
// ---------------------------------------------------------------------------
constexpr int kColsPerGroup = 32;
constexpr int kCpw = 2;                        // columns per consumer warp (16 warps x 2 = 32)
constexpr int kChunkBytes = 1024;              // bytes of one column chunk (32 chunks = 32 KiB per stage)

template <int BITS>
__global__ void __launch_bounds__(kTmaThreads, 1) k_gemv_t_col(GemvTArgs a, int nstage_buf)
{
    constexpr int G = 32 / BITS;
    constexpr int E = G / 4;                   // 16-byte limb loads per limb per piece
    constexpr uint32_t MASK = 0x01010101u * ((1u << BITS) - 1);
    constexpr int PPC = kChunkBytes / 16;      // pieces per column chunk
    constexpr int PPL = PPC / 32;              // pieces per lane per column chunk

    extern __shared__ __align__(128) unsigned char smem[];
    griddep_wait();
    if (a.h_outer && blockIdx.x == 0 && threadIdx.x == 0) {
        const int guard = ++a.st->outer_guard;
        cudaGraphSetConditional((cudaGraphConditionalHandle)a.h_outer,
                                (!a.st->stop && guard < a.guard_limit) ? 1u : 0u);
    }
    if (a.st && a.st->stop) return;

    const int n = a.Q.cols, ld = a.Q.ld, m = a.Q.rows;
    const int P = ld / 4;                              // 16-byte pieces per column
    const unsigned colbytes = (unsigned)ld * 4u;
    const int nchunk = (int)((colbytes + kChunkBytes - 1) / kChunkBytes);
    const int NS = nstage_buf;
    const unsigned stage_bytes = (unsigned)kColsPerGroup * kChunkBytes;
    uint32_t* limb = reinterpret_cast<uint32_t*>(smem + (size_t)NS * stage_bytes);   // [3][E][P][4]
    uint64_t* full = reinterpret_cast<uint64_t*>(limb + (size_t)3 * E * P * 4);
    uint64_t* empty = full + NS;
    long long* red_r = reinterpret_cast<long long*>(empty + NS);
    __shared__ int s_abort;

    const int c0 = (int)((long long)n * blockIdx.x / gridDim.x);
    const int c1 = (int)((long long)n * (blockIdx.x + 1) / gridDim.x);
    const int ncols = c1 - c0;
    const int ngroups = (ncols + kColsPerGroup - 1) / kColsPerGroup;
    const int nst = ngroups * nchunk;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        s_abort = 0;
        for (int i = 0; i < NS; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], kTmaWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == kTmaWarps) {
        // producer warp: stage it = (group it / nchunk, chunk it % nchunk)
        int issued = 0;
        bool ok = true;
        for (int it = 0; it < nst; ++it) {
            const int sb = it % NS;
            const unsigned ph = (unsigned)(it / NS) & 1u;
            const int grp = it / nchunk, ch = it - grp * nchunk;
            const int gc0 = c0 + grp * kColsPerGroup;
            const int gcols = min(kColsPerGroup, c1 - gc0);
            const unsigned off = (unsigned)ch * kChunkBytes;
            const unsigned cb = min((unsigned)kChunkBytes, colbytes - off);
            int stop = 0;
            if (lane == 0) {
                if (*(volatile int*)&s_abort) stop = 1;
                else if (it >= NS && !mbar_wait(&empty[sb], ph ^ 1u)) stop = 1;
                else mbar_expect_tx(&full[sb], (unsigned)gcols * cb);
            }
            stop = __shfl_sync(0xffffffffu, stop, 0);
            if (stop) { ok = false; break; }
            if (lane < gcols)
                bulk_g2s(smem + (size_t)sb * stage_bytes + (size_t)lane * kChunkBytes,
                         reinterpret_cast<const unsigned char*>(a.Q.words) + (size_t)(gc0 + lane) * colbytes + off,
                         cb, &full[sb]);
            ++issued;
        }
        if (!ok && lane == 0) {
            report_timeout(a);
            for (int it = max(0, issued - NS); it < issued; ++it)
                mbar_wait(&full[it % NS], (unsigned)(it / NS) & 1u);
        }
        return;
    }

    // consumers: residual -> fixed point byte planes in shared memory
    const int sh = fixed_shift(*a.rmax_bits);
    long long rsum = 0;
    for (int lw = threadIdx.x; lw < P * G; lw += kTmaConsumers) {      // limb word lw covers rows 4lw..4lw+3
        uint32_t b0 = 0, b1 = 0, b2 = 0;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const int i = 4 * lw + p;
            int v = 0;
            if (i < m) v = __float2int_rn(ldexpf(__ldcg(a.r + i), sh));
            rsum += v;
            b0 |= (uint32_t)(v & 255) << (8 * p);
            b1 |= (uint32_t)((v >> 8) & 255) << (8 * p);
            b2 |= (uint32_t)((v >> 16) & 255) << (8 * p);
        }
        // limb word lw = piece * G + q*4 + w  ->  index ((q * P + piece) * 4 + w)
        const int piece = lw / G, rem = lw - piece * G, q = rem >> 2, w = rem & 3;
        const size_t idx = ((size_t)q * P + piece) * 4 + w;
        limb[idx] = b0;
        limb[(size_t)E * P * 4 + idx] = b1;
        limb[(size_t)2 * E * P * 4 + idx] = b2;
    }
    {
        long long v = rsum;
#pragma unroll
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red_r[warp] = v;
    }
    consumer_sync();
    long long R = 0;
    for (int w = 0; w < kTmaWarps; ++w) R += red_r[w];
    R *= a.Q.lm1;                                 // (L-1) sum_i r_i
    const double alpha = (double)(*a.Q.scale) / (double)a.Q.lm1;
    const double outscale = ldexp(alpha, -sh);
    const uint4* L0 = reinterpret_cast<const uint4*>(limb);
    const uint4* L1 = L0 + (size_t)E * P;
    const uint4* L2 = L0 + (size_t)2 * E * P;

    uint32_t a0[kCpw], a1[kCpw];
    int32_t a2[kCpw];
    for (int it = 0; it < nst; ++it) {
        const int sb = it % NS;
        const unsigned ph = (unsigned)(it / NS) & 1u;
        const int grp = it / nchunk, ch = it - grp * nchunk;
        const int gc0 = c0 + grp * kColsPerGroup;
        const int gcols = min(kColsPerGroup, c1 - gc0);
        if (ch == 0) {
#pragma unroll
            for (int c = 0; c < kCpw; ++c) { a0[c] = 0; a1[c] = 0; a2[c] = 0; }
        }
        if (!mbar_wait(&full[sb], ph)) {
            if (lane == 0) { s_abort = 1; report_timeout(a); }
            break;
        }
        if (*(volatile int*)&s_abort) break;
        const unsigned char* stage = smem + (size_t)sb * stage_bytes;
        const int pbase = ch * PPC;                    // first piece of this chunk in the column
#pragma unroll
        for (int pl = 0; pl < PPL; ++pl) {
            const int pc = lane + 32 * pl;             // piece within the chunk
            const int piece = pbase + pc;
            if (piece < P) {
                uint4 l0v[E], l1v[E], l2v[E];
#pragma unroll
                for (int q = 0; q < E; ++q) {
                    l0v[q] = L0[(size_t)q * P + piece];
                    l1v[q] = L1[(size_t)q * P + piece];
                    l2v[q] = L2[(size_t)q * P + piece];
                }
#pragma unroll
                for (int c = 0; c < kCpw; ++c) {
                    const int col = warp * kCpw + c;
                    if (col < gcols) {
                        const uint4 v = reinterpret_cast<const uint4*>(stage + (size_t)col * kChunkBytes)[pc];
                        const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                        for (int w = 0; w < 4; ++w)
#pragma unroll
                            for (int k = 0; k < E; ++k) {
                                const uint32_t x = (wv[w] >> (BITS * k)) & MASK;
                                // limb word w*E + k of the piece -> plane q = (w*E+k)/4, word (w*E+k)%4
                                const int lw = w * E + k;
                                const uint4& A0 = l0v[lw >> 2];
                                const uint4& A1 = l1v[lw >> 2];
                                const uint4& A2 = l2v[lw >> 2];
                                const int sel = lw & 3;
                                const uint32_t y0 = sel == 0 ? A0.x : sel == 1 ? A0.y : sel == 2 ? A0.z : A0.w;
                                const uint32_t y1 = sel == 0 ? A1.x : sel == 1 ? A1.y : sel == 2 ? A1.z : A1.w;
                                const uint32_t y2 = sel == 0 ? A2.x : sel == 1 ? A2.y : sel == 2 ? A2.z : A2.w;
                                a0[c] = dp4a_uu(x, y0, a0[c]);
                                a1[c] = dp4a_uu(x, y1, a1[c]);
                                a2[c] = dp4a_us(x, y2, a2[c]);
                            }
                    }
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[sb]);
        if (ch == nchunk - 1) {
#pragma unroll
            for (int c = 0; c < kCpw; ++c) {
                const uint32_t s0 = __reduce_add_sync(0xffffffffu, a0[c]);
                const uint32_t s1 = __reduce_add_sync(0xffffffffu, a1[c]);
                const int32_t s2 = __reduce_add_sync(0xffffffffu, a2[c]);
                const int col = warp * kCpw + c;
                if (lane == c && col < gcols) {
                    const long long S = (long long)s0 + ((long long)s1 << 8) + ((long long)s2 << 16);
                    const long long T = 2 * S - R;
                    a.g[gc0 + col] = (float)((double)T * outscale);
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Warp-per-column variant (the default). Many warps per SM (2 CTAs x 16 warps),
// each warp owns whole columns (static round-robin over the columns), so its
// integer sums never leave the warp. A lane loads NPL 16-byte pieces of the
// column at once (coalesced: consecutive lanes, consecutive pieces), which keeps
// ~128 KB of loads in flight per SM. The fixed-point residual is held once per
// CTA in shared memory as three byte planes in a lane-interleaved layout
// ([E][piece][4 words], conflict-free 16-byte loads).
// Codes are extracted with one mask per four codes: (w & (mask << b k)) gives
// the codes of position k times 2^(b k); products are summed per position and
// the positions are combined at the end with exact right shifts.
// In the solver's loop the epilogue also prepares the next threshold: g on the
// support goes to its support position, and a column outside the support with
// |g| >= tau_g is appended to the candidate list (the largest |g| below tau_g is
// kept per CTA and merged with one atomic).
// ---------------------------------------------------------------------------
constexpr int kWarpThreads = 512;           // 16 warps per CTA, two CTAs per SM

// Warp 0 of a GEMV^T CTA: stop flag, max |r| (fast path: from the iteration kernel's
// residual partials, whose non-finite maximum stops the solve), candidate threshold, the
// loop condition (CTA 0) and, after the last iteration, its ||r||^2 (CTA 0). Kept out of
// line: it runs once per CTA and its registers would otherwise crowd the streaming loop.
__device__ __noinline__ void warp_prologue(const GemvTArgs& a, unsigned* s_st)
{
    // max |r|: from the iteration kernel's residual partials (fast path) or the state
    unsigned rmx = 0;
    if (a.rpart) rmx = (unsigned)slot_max_complete(a.rpart, kSlotRmax, a.rgrid);
    if (threadIdx.x == 0) {
        int stop = a.st ? a.st->stop : 0;
        if (!a.rpart) rmx = *a.rmax_bits;
        if (a.rpart && !stop && rmx >= 0x7f800000u) {
            // a residual entry is not finite: the solve stops (the CTAs all see it)
            stop = 1;
            if (blockIdx.x == 0) {
                a.st->status = QIHT_ERR_NONFINITE;
                a.st->stop = 1;
                if (a.report) a.report->status = QIHT_ERR_NONFINITE;
            }
        }
        s_st[0] = (unsigned)stop;
        s_st[1] = rmx;
        s_st[2] = (a.pos && a.st) ? a.st->tau_g_bits : 0u;
        if (a.h_outer && blockIdx.x == 0) {
            const int guard = ++a.st->outer_guard;
            cudaGraphSetConditional((cudaGraphConditionalHandle)a.h_outer,
                                    (!stop && guard < a.guard_limit) ? 1u : 0u);
        }
    }
    // ||r||^2 of the iteration the iteration kernel just completed (it leaves the record to
    // this kernel, so that none of its CTAs waits for the others at the end)
    if (a.rpart && blockIdx.x == 0) {
        const int st_iter = __shfl_sync(0xffffffffu, a.st->iter, 0);
        const int logged = __shfl_sync(0xffffffffu, a.st->resid_logged, 0);
        if (st_iter > logged) {
            const double r2 = slot_sum_complete(a.rpart, kSlotResid, a.rgrid);
            if (threadIdx.x == 0) {
                a.st->resid2 = r2;
                a.st->resid_logged = st_iter;
                if (a.trace_resid2) a.trace_resid2[st_iter] = r2;
                if (a.report) a.report->resid_norm2 = r2;
            }
        }
    }
}

template <int BITS, int NPL>
__global__ void __launch_bounds__(kWarpThreads, 2) k_gemv_t_warp(GemvTArgs a)
{
    constexpr int G = 32 / BITS;
    constexpr int E = G / 4;
    constexpr uint32_t MASK = 0x01010101u * ((1u << BITS) - 1);
    extern __shared__ __align__(16) uint32_t limb[];    // [3][E][P][4]
    __shared__ long long red_r[16];
    __shared__ unsigned bmax_cta;
    __shared__ double outscale_sh;

    const int n = a.Q.cols, ld = a.Q.ld, m = a.Q.rows;
    const int P = ld / 4;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // Software pipeline over the warp's sequence of batches (column j, batch pb of NPL
    // pieces per lane): the loads of the next batch are in flight while this one is used.
    // The first batch is requested before the residual is staged, so its DRAM latency
    // overlaps the staging.
    const int W = gridDim.x * (blockDim.x >> 5);
    const int nb = (P + 32 * NPL - 1) / (32 * NPL);     // batches per column
    int j = blockIdx.x * (blockDim.x >> 5) + warp;
    int pb = 0;
    // the code stream is read once per call: mark it first to leave L2, so that the small
    // working set of the rest of the iteration (support columns of Q2, g, x, r) stays there
    uint64_t stream_policy;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(stream_policy));
    auto load_batch = [&](uint4 (&cv)[NPL], int jj, int bb) {
        const uint4* col = reinterpret_cast<const uint4*>(a.Q.words + (size_t)jj * ld);
#pragma unroll
        for (int u = 0; u < NPL; ++u) {
            const int piece = bb * 32 * NPL + lane + 32 * u;
            if (piece < P)
                asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
                             : "=r"(cv[u].x), "=r"(cv[u].y), "=r"(cv[u].z), "=r"(cv[u].w)
                             : "l"(col + piece), "l"(stream_policy));
            else
                cv[u] = make_uint4(0u, 0u, 0u, 0u);
        }
    };
    uint4 cA[NPL], cB[NPL];
    if (j < n) load_batch(cA, j, pb);

    // everything above reads only the codes; r, max |r| and the solver state come from
    // the previous kernel. The state words are read by one thread per CTA and shared (all
    // threads reading them would pile requests onto one L2 line); the first chunk of r is
    // requested at the same time.
    griddep_wait();
    griddep_launch();
    __shared__ unsigned s_st[3];
    if (threadIdx.x < 32) warp_prologue(a, s_st);
    // residual to 24-bit fixed point, as three byte planes; four rows (one float4) per limb
    // word, UR words of a thread in flight at once
    constexpr int UR = 4;
    const bool r_vec = (reinterpret_cast<uintptr_t>(a.r) & 15) == 0;
    const int nlw = P * G;
    auto load_r = [&](float (&rv)[UR][4], int lw0) {
#pragma unroll
        for (int u = 0; u < UR; ++u) {
            const int lw = lw0 + u * (int)blockDim.x;
            const int i = 4 * lw;
            if (lw < nlw && r_vec && i + 3 < m) {
                const float4 t = __ldcg(reinterpret_cast<const float4*>(a.r) + lw);
                rv[u][0] = t.x; rv[u][1] = t.y; rv[u][2] = t.z; rv[u][3] = t.w;
            } else {
#pragma unroll
                for (int p = 0; p < 4; ++p) rv[u][p] = (lw < nlw && i + p < m) ? __ldcg(a.r + i + p) : 0.0f;
            }
        }
    };
    float rv[UR][4];
    load_r(rv, threadIdx.x);
    __syncthreads();
    if (s_st[0]) return;                        // uniform
    const int sh = fixed_shift(s_st[1]);
    long long rsum = 0;
    for (int lw0 = threadIdx.x; lw0 < nlw; lw0 += blockDim.x * UR) {
        if (lw0 != (int)threadIdx.x) load_r(rv, lw0);
#pragma unroll
        for (int u = 0; u < UR; ++u) {
            const int lw = lw0 + u * (int)blockDim.x;
            if (lw < nlw) {
                uint32_t b0 = 0, b1 = 0, b2 = 0;
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    const int v = __float2int_rn(ldexpf(rv[u][p], sh));   // rows past m are 0
                    rsum += v;
                    b0 |= (uint32_t)(v & 255) << (8 * p);
                    b1 |= (uint32_t)((v >> 8) & 255) << (8 * p);
                    b2 |= (uint32_t)((v >> 16) & 255) << (8 * p);
                }
                const int piece = lw / G, rem = lw - piece * G, q = rem >> 2, w = rem & 3;
                const size_t idx = ((size_t)q * P + piece) * 4 + w;
                limb[idx] = b0;
                limb[(size_t)E * P * 4 + idx] = b1;
                limb[(size_t)2 * E * P * 4 + idx] = b2;
            }
        }
    }
    {
        long long v = rsum;
#pragma unroll
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red_r[warp] = v * a.Q.lm1;    // (L-1) times the warp's sum of r
    }
    if (threadIdx.x == 0) bmax_cta = 0u;
    if (threadIdx.x == 32) {
        // alpha 2^-sh, once per CTA: FP64 division is slow on this GPU, and every warp
        // that did it would hold back its first loads
        const double alpha = (double)(*a.Q.scale) / (double)a.Q.lm1;
        outscale_sh = ldexp(alpha, -sh);
    }
    __syncthreads();
    // candidate filter of the solver's next threshold (off: tau_g == 0 or no position map)
    const uint32_t tau_g = s_st[2];
    unsigned bmax = 0;
    int pos_cur = -1;
    long long R = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) R += red_r[w];
    const uint4* L0 = reinterpret_cast<const uint4*>(limb);
    const uint4* L1 = L0 + (size_t)E * P;
    const uint4* L2 = L0 + (size_t)2 * E * P;

    uint32_t s0[E], s1[E];
    int32_t s2[E];
#pragma unroll
    for (int k = 0; k < E; ++k) { s0[k] = 0; s1[k] = 0; s2[k] = 0; }

    auto use_batch = [&](const uint4 (&cv)[NPL], int bb) {
#pragma unroll
        for (int u = 0; u < NPL; ++u) {
            const int piece = min(bb * 32 * NPL + lane + 32 * u, P - 1);   // past the end: zero codes
            const uint32_t wv[4] = {cv[u].x, cv[u].y, cv[u].z, cv[u].w};
#pragma unroll
            for (int q = 0; q < E; ++q) {
                const uint4 A0 = L0[(size_t)q * P + piece];
                const uint4 A1 = L1[(size_t)q * P + piece];
                const uint4 A2 = L2[(size_t)q * P + piece];
                const uint32_t y0[4] = {A0.x, A0.y, A0.z, A0.w};
                const uint32_t y1[4] = {A1.x, A1.y, A1.z, A1.w};
                const uint32_t y2[4] = {A2.x, A2.y, A2.z, A2.w};
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    // limb word lw = q*4 + t of the piece = word w = lw / E, position k = lw % E
                    const int lw = q * 4 + t, w = lw / E, k = lw - w * E;
                    const uint32_t x = wv[w] & (MASK << (BITS * k));
                    s0[k] = dp4a_uu(x, y0[t], s0[k]);
                    s1[k] = dp4a_uu(x, y1[t], s1[k]);
                    s2[k] = dp4a_us(x, y2[t], s2[k]);
                }
            }
        }
    };
    auto finish_column = [&](int jj) {
        long long S = 0;
#pragma unroll
        for (int k = 0; k < E; ++k) {
            // position k sums carry the factor 2^(b k): exact, so shift it out after the warp sum
            const long long t0 = (long long)(uint32_t)__reduce_add_sync(0xffffffffu, s0[k]);
            const long long t1 = (long long)(uint32_t)__reduce_add_sync(0xffffffffu, s1[k]);
            const long long t2 = (long long)__reduce_add_sync(0xffffffffu, s2[k]);
            S += (t0 + (t1 << 8) + (t2 << 16)) >> (BITS * k);
            s0[k] = 0; s1[k] = 0; s2[k] = 0;
        }
        if (lane == 0) {
            const long long T = 2 * S - R;
            const float gv = (float)((double)T * outscale_sh);
            a.g[jj] = gv;
            if (pos_cur >= 0) {
                a.gsup[pos_cur] = gv;
            } else if (tau_g) {
                const uint32_t kb = __float_as_uint(gv) & 0x7fffffffu;
                if (kb >= tau_g) {
                    const unsigned slot = atomicAdd(&a.st->gcand_count, 1u);
                    if (slot < (unsigned)a.gcap)
                        a.gcand[slot] = ((unsigned long long)__float_as_uint(gv) << 32) | (unsigned)jj;
                } else {
                    bmax = max(bmax, kb);
                }
            }
        }
    };
    // support position of column jj (lane 0 only; read early, used by finish_column)
    auto fetch_pos = [&](int jj) {
        if (a.pos && lane == 0) pos_cur = __ldg(a.pos + jj);
    };
    auto advance = [&](int& jj, int& bb) {
        if (++bb == nb) { bb = 0; jj += W; }
    };

    while (j < n) {
        int jB = j, pB = pb;
        advance(jB, pB);
        if (jB < n) load_batch(cB, jB, pB);
        if (pb == 0) fetch_pos(j);
        use_batch(cA, pb);
        if (pb == nb - 1) finish_column(j);
        j = jB; pb = pB;
        if (j >= n) break;
        int jA = j, pA = pb;
        advance(jA, pA);
        if (jA < n) load_batch(cA, jA, pA);
        if (pb == 0) fetch_pos(j);
        use_batch(cB, pb);
        if (pb == nb - 1) finish_column(j);
        j = jA; pb = pA;
    }
    if (tau_g) {
        if (lane == 0 && bmax) atomicMax(&bmax_cta, bmax);
        __syncthreads();
        if (threadIdx.x == 0 && bmax_cta) atomicMax(&a.st->bmax_g, bmax_cta);
    }
}

struct WarpPlan {
    void* fn;
    size_t smem;
    unsigned grid;
    bool ok;
};

static WarpPlan plan_warp(const Codes& Q, int nsm)
{
    WarpPlan p{};
    const int G = 32 / Q.bits, E = G / 4;
    const size_t P = (size_t)Q.ld / 4;
    p.smem = 3 * (size_t)E * P * 16;
    if (p.smem > 48 * 1024 * 2) return p;          // keep at least two CTAs per SM
    if (Q.bits == 8) p.fn = (void*)k_gemv_t_warp<8, 4>;
    else if (Q.bits == 4) p.fn = (void*)k_gemv_t_warp<4, 2>;
    else p.fn = (void*)k_gemv_t_warp<2, 1>;
    cudaFuncSetAttribute(p.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, p.fn, kWarpThreads, p.smem);
    if (occ < 1) return p;
    long long grid = (long long)nsm * occ;
    const long long want = ((long long)Q.cols + kWarpThreads / 32 - 1) / (kWarpThreads / 32);
    if (grid > want) grid = want;
    p.grid = (unsigned)(grid < 1 ? 1 : grid);
    p.ok = true;
    return p;
}

struct TmaPlan {
    void* fn;
    int tpc;
    int ns;
    size_t smem;
    unsigned grid;
    bool ok;
};

template <int BITS, int PPT, int CPSL>
static void* tma_fn() { return (void*)k_gemv_t_tma<BITS, PPT, CPSL>; }

static TmaPlan plan_tma(const Codes& Q, int nsm)
{
    TmaPlan p{};
    const int P = Q.ld / 4;
    int tpc = 32;
    while (tpc < P && tpc < kTmaConsumers) tpc <<= 1;
    const int ppt = (P + tpc - 1) / tpc;
    const int slots = kTmaConsumers / tpc;
    const size_t colbytes = (size_t)Q.ld * 4;
    int cpsl = 4;
    while (cpsl > 1 && (size_t)cpsl * slots * colbytes > 49152) cpsl >>= 1;
    const size_t stage = (size_t)cpsl * slots * colbytes;
    int ns = (int)(kTmaRingBytes / stage);
    if (ns > 8) ns = 8;
    if (ppt > 2 || ns < 2 || (Q.bits != 8 && ppt > 1)) return p;
    void* fn = nullptr;
#define QIHT_TMA_CASE(B, PP, C) if (Q.bits == B && ppt == PP && cpsl == C) fn = tma_fn<B, PP, C>();
    QIHT_TMA_CASE(8, 1, 4) QIHT_TMA_CASE(8, 1, 2) QIHT_TMA_CASE(8, 1, 1)
    QIHT_TMA_CASE(8, 2, 4) QIHT_TMA_CASE(8, 2, 2) QIHT_TMA_CASE(8, 2, 1)
    QIHT_TMA_CASE(4, 1, 4) QIHT_TMA_CASE(4, 1, 2) QIHT_TMA_CASE(4, 1, 1)
    QIHT_TMA_CASE(2, 1, 4) QIHT_TMA_CASE(2, 1, 2) QIHT_TMA_CASE(2, 1, 1)
#undef QIHT_TMA_CASE
    if (!fn) return p;
    p.fn = fn;
    p.tpc = tpc;
    p.ns = ns;
    const size_t cps = (size_t)cpsl * slots;
    p.smem = (size_t)ns * stage + 2 * (size_t)ns * 8 + (size_t)ns * cps * 3 * 8 + ((((size_t)ns * cps + 1) & ~(size_t)1) * 4) +
             kTmaWarps * 8;
    int grid = nsm;
    if (grid > Q.cols) grid = Q.cols;
    p.grid = (unsigned)grid;
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
    p.ok = true;
    return p;
}

struct ColPlan {
    void* fn;
    int ns;
    size_t smem;
    unsigned grid;
    bool ok;
};

static ColPlan plan_col(const Codes& Q, int nsm)
{
    ColPlan p{};
    const int G = 32 / Q.bits, E = G / 4;
    const size_t P = (size_t)Q.ld / 4;
    const size_t limb_bytes = 3 * (size_t)E * P * 16;
    const size_t stage = (size_t)kColsPerGroup * kChunkBytes;
    const size_t budget = 220 * 1024;
    if (limb_bytes + 2 * stage + 1024 > budget) return p;
    int ns = (int)((budget - limb_bytes - 1024) / stage);
    if (ns > 6) ns = 6;
    p.ns = ns;
    p.smem = (size_t)ns * stage + limb_bytes + 2 * (size_t)ns * 8 + kTmaWarps * 8;
    p.fn = Q.bits == 8 ? (void*)k_gemv_t_col<8> : Q.bits == 4 ? (void*)k_gemv_t_col<4> : (void*)k_gemv_t_col<2>;
    int grid = nsm;
    if (grid > Q.cols) grid = Q.cols;
    p.grid = (unsigned)grid;
    cudaFuncSetAttribute(p.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
    p.ok = true;
    return p;
}

static int gemv_variant()
{
    // QIHT_GEMV selects a kernel for measurement: "warp" (default), "col", "tma", "ldg"
    static int v = -1;
    if (v < 0) {
        const char* e = getenv("QIHT_GEMV");
        v = (e && e[0] == 'l') ? 0 : (e && e[0] == 't') ? 1 : (e && e[0] == 'c') ? 2 : 3;
    }
    return v;
}

static bool use_warp() { return gemv_variant() == 3; }

static bool use_tma() { return gemv_variant() == 1; }
static bool use_col() { return gemv_variant() == 2; }

template <int BITS>
static void pick(int rows_pad, int& rpt, int& tpc, void** fn)
{
    // smallest rows-per-thread that covers the column with 256 threads
    if (rows_pad <= 256 * 16) rpt = 16;
    else if (rows_pad <= 256 * 32) rpt = 32;
    else rpt = 64;
    int need = (rows_pad + rpt - 1) / rpt;
    tpc = 32;
    while (tpc < need) tpc <<= 1;
    if (BITS == 8) {
        if (rpt == 16) *fn = (void*)k_gemv_t<8, 8, 16>;
        else if (rpt == 32) *fn = (void*)k_gemv_t<8, 4, 32>;
        else *fn = (void*)k_gemv_t<8, 2, 64>;
    } else if (BITS == 4) {
        if (rpt == 16) *fn = (void*)k_gemv_t<4, 8, 16>;
        else if (rpt == 32) *fn = (void*)k_gemv_t<4, 8, 32>;
        else *fn = (void*)k_gemv_t<4, 4, 64>;
    } else {
        if (rpt == 16) *fn = (void*)k_gemv_t<2, 8, 16>;
        else if (rpt == 32) *fn = (void*)k_gemv_t<2, 8, 32>;
        else *fn = (void*)k_gemv_t<2, 8, 64>;
    }
}

static int cpw_of(int bits, int rpt)
{
    if (bits == 8) return rpt == 16 ? 8 : rpt == 32 ? 4 : 2;
    if (bits == 4) return rpt == 64 ? 4 : 8;
    return 8;
}

struct GemvPlan {
    void* fn;
    int tpc;
    unsigned grid;
};

static GemvPlan plan_gemv_t(const Codes& Q, int nsm)
{
    GemvPlan p{};
    const int G = 32 / Q.bits;
    const int rows_pad = Q.ld * G;
    int rpt = 16;
    if (Q.bits == 8) pick<8>(rows_pad, rpt, p.tpc, &p.fn);
    else if (Q.bits == 4) pick<4>(rows_pad, rpt, p.tpc, &p.fn);
    else pick<2>(rows_pad, rpt, p.tpc, &p.fn);
    const int cpw = cpw_of(Q.bits, rpt);
    const int slots = 256 / p.tpc;
    const long long ncg = (Q.cols + cpw - 1) / cpw;
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, p.fn, 256, 0);
    if (occ < 1) occ = 1;
    long long grid = (long long)nsm * occ;
    const long long want = (ncg + slots - 1) / slots;
    if (grid > want) grid = want;
    if (grid < 1) grid = 1;
    p.grid = (unsigned)grid;
    return p;
}

void gemv_t_node(const GemvTArgs& a, int nsm, cudaKernelNodeParams* p, void** argbuf)
{
    if (use_warp()) {
        WarpPlan wp = plan_warp(a.Q, nsm);
        if (wp.ok) {
            p->func = wp.fn;
            p->gridDim = dim3(wp.grid);
            p->blockDim = dim3(kWarpThreads);
            p->sharedMemBytes = (unsigned)wp.smem;
            p->kernelParams = argbuf;        // (GemvTArgs)
            p->extra = nullptr;
            return;
        }
    }
    if (use_col()) {
        ColPlan cp = plan_col(a.Q, nsm);
        if (cp.ok) {
            // kernel arguments: (GemvTArgs, int stages) -> argbuf[0], argbuf[2]
            *reinterpret_cast<int*>(argbuf[2]) = cp.ns;
            argbuf[1] = argbuf[2];
            p->func = cp.fn;
            p->gridDim = dim3(cp.grid);
            p->blockDim = dim3(kTmaThreads);
            p->sharedMemBytes = (unsigned)cp.smem;
            p->kernelParams = argbuf;
            p->extra = nullptr;
            return;
        }
    }
    if (use_tma()) {
        TmaPlan tp = plan_tma(a.Q, nsm);
        if (tp.ok) {
            // argbuf[0] -> GemvTArgs, argbuf[1] -> int tpc, argbuf[2] -> int stages (owned by the caller)
            *reinterpret_cast<int*>(argbuf[1]) = tp.tpc;
            *reinterpret_cast<int*>(argbuf[2]) = tp.ns;
            p->func = tp.fn;
            p->gridDim = dim3(tp.grid);
            p->blockDim = dim3(kTmaThreads);
            p->sharedMemBytes = (unsigned)tp.smem;
            p->kernelParams = argbuf;
            p->extra = nullptr;
            return;
        }
    }
    GemvPlan pl = plan_gemv_t(a.Q, nsm);
    // argbuf[0] -> GemvTArgs copy, argbuf[1] -> int tpc (owned by the caller)
    *reinterpret_cast<int*>(argbuf[1]) = pl.tpc;
    p->func = pl.fn;
    p->gridDim = dim3(pl.grid);
    p->blockDim = dim3(256);
    p->sharedMemBytes = 0;
    p->kernelParams = argbuf;
    p->extra = nullptr;
}

cudaError_t launch_gemv_t(const GemvTArgs& a, int nsm, cudaStream_t s)
{
    if (use_warp()) {
        WarpPlan wp = plan_warp(a.Q, nsm);
        if (wp.ok) {
            GemvTArgs copy = a;
            void* args[1] = {&copy};
            return cudaLaunchKernel(wp.fn, dim3(wp.grid), dim3(kWarpThreads), args, wp.smem, s);
        }
    }
    if (use_col()) {
        ColPlan cp = plan_col(a.Q, nsm);
        if (cp.ok) {
            GemvTArgs copy = a;
            int ns = cp.ns;
            void* args[2] = {&copy, &ns};
            return cudaLaunchKernel(cp.fn, dim3(cp.grid), dim3(kTmaThreads), args, cp.smem, s);
        }
    }
    if (use_tma()) {
        TmaPlan tp = plan_tma(a.Q, nsm);
        if (tp.ok) {
            GemvTArgs copy = a;
            int tpc = tp.tpc, ns = tp.ns;
            void* args[3] = {&copy, &tpc, &ns};
            return cudaLaunchKernel(tp.fn, dim3(tp.grid), dim3(kTmaThreads), args, tp.smem, s);
        }
    }
    GemvPlan pl = plan_gemv_t(a.Q, nsm);
    GemvTArgs copy = a;
    int tpc = pl.tpc;
    void* args[2] = {&copy, &tpc};
    return cudaLaunchKernel(pl.fn, dim3(pl.grid), dim3(256), args, 0, s);
}

}  // namespace qiht
