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
// Mapping (k_gemv_t_warp). Each warp owns whole columns, so its integer sums never
// leave the warp; the fixed-point residual is held once per CTA in shared memory.
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

// Power-of-two exponent sh so that |r| * 2^sh < 2^22 for all r (0 if r == 0).
__device__ __forceinline__ int fixed_shift(unsigned rmax_bits)
{
    const float M = __uint_as_float(rmax_bits);
    if (!(M > 0.0f) || !isfinite(M)) return 0;
    int ex;
    frexpf(M, &ex);          // M = f * 2^ex, 0.5 <= f < 1, so M < 2^ex
    return 22 - ex;
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
constexpr int kWarpThreads = 512;           // 16 warps per CTA, two CTAs per SM (one at C = 4)
constexpr int kColsPerWarp = 4;             // columns a warp streams together at 2 bits (measured: 30.8 vs
                                            // 33.0 us at 8192 x 32768 with one column)
constexpr int kColsPerWarp4 = 2;            // at 4 bits, one piece per lane (measured: 33.0 us, against
                                            // 34.9 with one column and two pieces, 37.1 with four columns)

// Warp 0 of a GEMV^T CTA: stop flag, max |r| (fast path: from the iteration kernel's
// residual partials, whose non-finite maximum stops the solve), candidate threshold, the
// loop condition (CTA 0) and, after the last iteration, its ||r||^2 (CTA 0). Kept out of
// line: it runs once per CTA and its registers would otherwise crowd the streaming loop.
__device__ __noinline__ void warp_prologue(const GemvTArgs& a, unsigned* s_st)
{
    // max |r|: from the iteration kernel's residual partials (fast path) or the state
    unsigned rmx = 0;
    if (a.rpart) rmx = (unsigned)slot_max_complete(a.rpart, kSlotRmax, a.rgrid);
    // ||r||^2 of the iteration the iteration kernel just completed (it leaves the record to
    // this kernel, so that none of its CTAs waits for the others at the end), and the
    // residual tolerance: a run whose ||r||^2 reached tol stops after this iteration
    bool tol_stop = false;
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
            tol_stop = a.tol > 0.0 && r2 <= a.tol;
        }
    }
    if (threadIdx.x == 0) {
        int stop = a.st ? a.st->stop : 0;
        if (tol_stop && !stop) {
            stop = 1;                       // CTA 0 only; the other CTAs' products are not used
            a.st->stop = 1;
        }
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
}

// C = 1: a warp streams one column, NPL 16-byte pieces per lane at once (8 bits).
// C = 2, 4: a warp streams C adjacent columns together, one piece of each per lane, so that
// every load of the residual's planes from shared memory serves C columns (4 and 2 bits,
// where the per-code work and the planes' shared-memory reads, not HBM, bound the pass).
template <int BITS, int NPL, int C>
__global__ void __launch_bounds__(kWarpThreads, C <= 2 ? 2 : 1) k_gemv_t_warp(GemvTArgs a)
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
    const int ngc = (n + C - 1) / C;                    // groups of C adjacent columns
    int j = blockIdx.x * (blockDim.x >> 5) + warp;      // the warp's current column group
    int pb = 0;
    // the code stream is read once per call: mark it first to leave L2, so that the small
    // working set of the rest of the iteration (support columns of Q2, g, x, r) stays there
    uint64_t stream_policy;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(stream_policy));
    auto load_batch = [&](uint4 (&cv)[C][NPL], int jg, int bb) {
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const int jj = jg * C + c;
            const uint4* col = reinterpret_cast<const uint4*>(a.Q.words + (size_t)jj * ld);
#pragma unroll
            for (int u = 0; u < NPL; ++u) {
                const int piece = bb * 32 * NPL + lane + 32 * u;
                if (piece < P && jj < n)
                    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
                                 : "=r"(cv[c][u].x), "=r"(cv[c][u].y), "=r"(cv[c][u].z), "=r"(cv[c][u].w)
                                 : "l"(col + piece), "l"(stream_policy));
                else
                    cv[c][u] = make_uint4(0u, 0u, 0u, 0u);
            }
        }
    };
    uint4 cA[C][NPL], cB[C][NPL];
    if (j < ngc) load_batch(cA, j, pb);

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

    uint32_t s0[C][E], s1[C][E];
    int32_t s2[C][E];
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
        for (int k = 0; k < E; ++k) { s0[c][k] = 0; s1[c][k] = 0; s2[c][k] = 0; }

    auto use_batch = [&](const uint4 (&cv)[C][NPL], int bb) {
#pragma unroll
        for (int u = 0; u < NPL; ++u) {
            const int piece = min(bb * 32 * NPL + lane + 32 * u, P - 1);   // past the end: zero codes
#pragma unroll
            for (int q = 0; q < E; ++q) {
                const uint4 A0 = L0[(size_t)q * P + piece];
                const uint4 A1 = L1[(size_t)q * P + piece];
                const uint4 A2 = L2[(size_t)q * P + piece];
                const uint32_t y0[4] = {A0.x, A0.y, A0.z, A0.w};
                const uint32_t y1[4] = {A1.x, A1.y, A1.z, A1.w};
                const uint32_t y2[4] = {A2.x, A2.y, A2.z, A2.w};
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const uint32_t wv[4] = {cv[c][u].x, cv[c][u].y, cv[c][u].z, cv[c][u].w};
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        // limb word lw = q*4 + t of the piece = word w = lw / E, position k = lw % E
                        const int lw = q * 4 + t, w = lw / E, k = lw - w * E;
                        const uint32_t x = wv[w] & (MASK << (BITS * k));
                        s0[c][k] = dp4a_uu(x, y0[t], s0[c][k]);
                        s1[c][k] = dp4a_uu(x, y1[t], s1[c][k]);
                        s2[c][k] = dp4a_us(x, y2[t], s2[c][k]);
                    }
                }
            }
        }
    };
    auto finish_column = [&](int jg) {
#pragma unroll
        for (int c = 0; c < C; ++c) {
        long long S = 0;
#pragma unroll
        for (int k = 0; k < E; ++k) {
            // position k sums carry the factor 2^(b k): exact, so shift it out after the warp sum
            const long long t0 = (long long)(uint32_t)__reduce_add_sync(0xffffffffu, s0[c][k]);
            const long long t1 = (long long)(uint32_t)__reduce_add_sync(0xffffffffu, s1[c][k]);
            const long long t2 = (long long)__reduce_add_sync(0xffffffffu, s2[c][k]);
            S += (t0 + (t1 << 8) + (t2 << 16)) >> (BITS * k);
            s0[c][k] = 0; s1[c][k] = 0; s2[c][k] = 0;
        }
        const int jj = jg * C + c;
        if (lane == c && jj < n) {                  // lane c finishes column c of the group
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
        }
    };
    // support position of column c of group jg (lane c; read early, used by finish_column)
    auto fetch_pos = [&](int jg) {
        if (a.pos && lane < C) pos_cur = jg * C + lane < n ? __ldg(a.pos + jg * C + lane) : -1;
    };
    auto advance = [&](int& jj, int& bb) {
        if (++bb == nb) { bb = 0; jj += W; }
    };

    while (j < ngc) {
        int jB = j, pB = pb;
        advance(jB, pB);
        if (jB < ngc) load_batch(cB, jB, pB);
        if (pb == 0) fetch_pos(j);
        use_batch(cA, pb);
        if (pb == nb - 1) finish_column(j);
        j = jB; pb = pB;
        if (j >= ngc) break;
        int jA = j, pA = pb;
        advance(jA, pA);
        if (jA < ngc) load_batch(cA, jA, pA);
        if (pb == 0) fetch_pos(j);
        use_batch(cB, pb);
        if (pb == nb - 1) finish_column(j);
        j = jA; pb = pA;
    }
    if (tau_g) {
        if (lane < C && bmax) atomicMax(&bmax_cta, bmax);
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
    if (Q.bits == 8) p.fn = (void*)k_gemv_t_warp<8, 4, 1>;
    else if (Q.bits == 4) p.fn = (void*)k_gemv_t_warp<4, 1, kColsPerWarp4>;
    else p.fn = (void*)k_gemv_t_warp<2, 1, kColsPerWarp>;
    cudaFuncSetAttribute(p.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, p.fn, kWarpThreads, p.smem);
    if (occ < 1) return p;
    long long grid = (long long)nsm * occ;
    const int cpw = Q.bits == 2 ? kColsPerWarp : Q.bits == 4 ? kColsPerWarp4 : 1;
    const long long want = (((long long)Q.cols + cpw - 1) / cpw + kWarpThreads / 32 - 1) / (kWarpThreads / 32);
    if (grid > want) grid = want;
    if (Q.bits == 8) {
        // HBM-bound: no fewer CTAs than needed for the busiest warp's rounds of columns, so that
        // every warp runs that many (32768 columns: 293 CTAs, ~7 columns per warp, in place of
        // 304 CTAs with 6 or 7; measured 45.27 -> 44.7 us). At 4 and 2 bits the pass is bound by
        // per-code work and wants every SM full (4 bits: 33.0 -> 38.8 us with the same rule).
        const long long ngc = ((long long)Q.cols + cpw - 1) / cpw;
        const long long w0 = grid * (kWarpThreads / 32);
        const long long rounds = (ngc + w0 - 1) / w0;
        const long long wneed = (ngc + rounds - 1) / rounds;
        const long long gb = (wneed + kWarpThreads / 32 - 1) / (kWarpThreads / 32);
        if (gb < grid) grid = gb;
    }
    p.grid = (unsigned)(grid < 1 ? 1 : grid);
    p.ok = true;
    return p;
}

void gemv_t_node(const GemvTArgs& a, int nsm, cudaKernelNodeParams* p, void** argbuf)
{
    // argbuf[0] -> the GemvTArgs (owned by the caller). A plan that does not fit (rows beyond
    // the library's limit) leaves func null, which the graph builder reports as an error.
    const WarpPlan wp = plan_warp(a.Q, nsm);
    p->func = wp.ok ? wp.fn : nullptr;
    p->gridDim = dim3(wp.ok ? wp.grid : 1u);
    p->blockDim = dim3(kWarpThreads);
    p->sharedMemBytes = (unsigned)wp.smem;
    p->kernelParams = argbuf;
    p->extra = nullptr;
}

cudaError_t launch_gemv_t(const GemvTArgs& a, int nsm, cudaStream_t s)
{
    const WarpPlan wp = plan_warp(a.Q, nsm);
    if (!wp.ok) return cudaErrorInvalidConfiguration;
    GemvTArgs copy = a;
    void* args[1] = {&copy};
    return cudaLaunchKernel(wp.fn, dim3(wp.grid), dim3(kWarpThreads), args, wp.smem, s);
}

}  // namespace qiht
