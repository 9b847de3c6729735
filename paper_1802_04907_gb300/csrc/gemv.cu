// g = Q^T r over column-packed b-bit codes: the gradient product of Algorithm 2
// (g = Q1^T (Q(y) - Q2 x)), one full pass over the codes per call.
//
// Arithmetic. The value of code c is alpha * (2c - (L-1)), alpha = scale / (L-1),
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
    constexpr int L = 1 << BITS;
    constexpr uint32_t MASK = 0x01010101u * (uint32_t)(L - 1);
    constexpr int NW = RPT / G;           // words per thread per column
    constexpr int NL = RPT / 4;           // limb words per limb per thread

    if (a.h_outer && blockIdx.x == 0 && threadIdx.x == 0) {
        // the solver's outer loop continues while not stopped, and never more than
        // iters + 1 times even if a stop were missed
        const int guard = ++a.st->outer_guard;
        cudaGraphSetConditional((cudaGraphConditionalHandle)a.h_outer,
                                (!a.st->stop && guard < a.st->iters + 1) ? 1u : 0u);
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

    const double alpha = (double)(*a.Q.scale) / (double)(L - 1);
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
                const long long T = 2 * S - (long long)(L - 1) * R;
                a.g[j] = (float)((double)T * outscale);
            }
        }
        buf ^= 1;   // double-buffered partials: the next group's writes do not race these reads
    }
}

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
    GemvPlan pl = plan_gemv_t(a.Q, nsm);
    GemvTArgs copy = a;
    int tpc = pl.tpc;
    void* args[2] = {&copy, &tpc};
    return cudaLaunchKernel(pl.fn, dim3(pl.grid), dim3(256), args, 0, s);
}

}  // namespace qiht
