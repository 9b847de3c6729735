// z = Q[:, list] coef: products of the quantized matrix with a column subset.
// In one QIHT iteration (Algorithm 2) this kernel serves three uses, each with
// its own epilogue:
//   Mu     z = Q2_G g_G on the current support; mu = ||g_G||^2 / ||z||^2   (Eq. step_size)
//   Omega  z = Q2 (x' - x) on G' u G; omega = ||x'-x||^2 / ||z||^2, and the
//          backtracking test mu <= (1-c) omega (Section II-A); shrink mu by k(1-c) if it fails
//   Resid  z = Q2_G' x'; r = Q(y) - z, ||r||^2, max |r|; commit x <- x', G <- G'
// Grid: (row blocks of 256 words) x (chunks of 8 list entries). Each CTA sums its
// chunk for its rows into a partial buffer; the last CTA of a row block (arrival
// counter) adds the chunks in chunk order, and the last row block finishes the
// scalars. Sums are in a fixed order, so results are deterministic. No CTA ever
// waits on another one.
#include <cfloat>
#include <cmath>
#include <mutex>
#include <vector>

#include "internal.cuh"

namespace qiht {

__device__ __forceinline__ void set_cond(unsigned long long h, unsigned v)
{
    if (h) cudaGraphSetConditional((cudaGraphConditionalHandle)h, v);
}

// Deterministic block sum of one double per thread (fixed shuffle tree, then warps in order).
__device__ double block_sum_d(double v, double* sh)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sh[i];
        sh[32] = t;
    }
    __syncthreads();
    return sh[32];
}

__device__ unsigned block_max_u(unsigned v, unsigned* sh)
{
    v = __reduce_max_sync(0xffffffffu, v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t = max(t, sh[i]);
        sh[32] = t;
    }
    __syncthreads();
    return sh[32];
}

// Sum of squares of a list (g[idx[q]] when idx != nullptr, else v[q]) in a fixed order.
__device__ void write_report(const GatherArgs& a, const State* st)
{
    if (!a.report) return;
    a.report->iters_run = st->iter;
    a.report->backtracks = st->backtracks_total;
    a.report->support_changes = st->support_changes_total;
    a.report->status = st->status;
    a.report->resid_norm2 = st->resid2;
    a.report->mu = st->mu_accepted;
    a.report->full_selects = st->full_selects;
}

template <int BITS>
__global__ void __launch_bounds__(kGatherThreads) k_gather(GatherArgs a)
{
    constexpr int G = 32 / BITS;
    const int lm1 = a.Q.lm1;
    __shared__ double shd[33];
    __shared__ unsigned shu[33];
    __shared__ int flag;
    State* st = a.st;
    const bool first = blockIdx.x == 0 && blockIdx.y == 0;

    if (st) {
        if (st->stop) {
            if (first && threadIdx.x == 0) {
                if (a.mode == kGatherOmega) { st->again = 0; set_cond(a.h_bt, 0); }
                if (a.mode == kGatherResid) write_report(a, st);
            }
            return;
        }
        if (a.mode == kGatherOmega && !st->changed) {
            if (first && threadIdx.x == 0) { st->again = 0; set_cond(a.h_bt, 0); }
            return;
        }
    }

    const int count = (a.mode == kGatherOmega) ? st->union_count : (a.mode == kGatherPlain ? a.count : a.s);
    const int nchunks = (count + kGatherCols - 1) / kGatherCols;
    const int ld = a.Q.ld;
    const int rows_pad = ld * G;
    const int m = a.Q.rows;
    const int rb = blockIdx.x, jc = blockIdx.y;
    const int q = rb * kGatherThreads + threadIdx.x;       // word index in every column
    const int32_t* list = (a.mode == kGatherMu) ? a.support : (a.mode == kGatherResid ? a.new_sel : a.cols);
    const float* coefs = (a.mode == kGatherResid) ? a.new_val : a.coef;
    __shared__ int s_col[kGatherCols];
    __shared__ float s_cf[kGatherCols];
    __shared__ int s_bad;

    if (jc < nchunks) {
        // this chunk's columns and coefficients, loaded once for the CTA. A column index
        // outside [0, cols) (possible only in a caller's list) is not read: the entry is
        // dropped and the chunk's partial sums become NaN, so every entry of z is NaN
        if (threadIdx.x == 0) s_bad = 0;
        __syncthreads();
        if (threadIdx.x < kGatherCols) {
            const int jj = jc * kGatherCols + threadIdx.x;
            int col = -1;
            float cf = 0.0f;
            if (jj < count) {
                col = __ldcg(list + jj);
                if ((unsigned)col >= (unsigned)a.Q.cols) {
                    s_bad = 1;
                    col = -1;
                } else {
                    cf = (a.mode == kGatherMu || a.coef_from_g) ? __ldcg(a.g + col) : __ldcg(coefs + jj);
                }
            }
            s_col[threadIdx.x] = col;
            s_cf[threadIdx.x] = cf;
        }
        __syncthreads();
        if (rb == 0 && threadIdx.x == 0 && a.chunk_partial) {
            double acc2 = 0.0;
            for (int c = 0; c < kGatherCols; ++c) acc2 += (double)s_cf[c] * (double)s_cf[c];
            a.chunk_partial[jc] = acc2;
        }
        if (q < ld) {
            uint32_t w[kGatherCols];
#pragma unroll
            for (int c = 0; c < kGatherCols; ++c) {
                const int col = s_col[c];
                w[c] = col >= 0 ? __ldg(a.Q.words + (size_t)col * ld + q) : 0u;
            }
            float z[G];
#pragma unroll
            for (int k = 0; k < G; ++k) z[k] = 0.0f;
#pragma unroll
            for (int c = 0; c < kGatherCols; ++c) {
                if (s_col[c] >= 0) {
                    const float cf = s_cf[c];
#pragma unroll
                    for (int k = 0; k < G; ++k) {
                        const int code = (int)((w[c] >> (8 * (k & 3) + BITS * (k >> 2))) & ((1u << BITS) - 1));
                        z[k] = fmaf((float)(2 * code - lm1), cf, z[k]);
                    }
                }
            }
            if (s_bad) {
#pragma unroll
                for (int k = 0; k < G; ++k) z[k] = __int_as_float(0x7fc00000);
            }
            float* dst = a.partial + (size_t)jc * rows_pad + (size_t)q * G;
#pragma unroll
            for (int k = 0; k < G; k += 4) __stcg(reinterpret_cast<float4*>(dst + k), make_float4(z[k], z[k + 1], z[k + 2], z[k + 3]));
        }
    }

    // arrival of this CTA in its row block
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) flag = (atomicAdd(&a.counters[rb], 1u) == gridDim.y - 1);
    __syncthreads();
    if (!flag) return;
    __threadfence();

    const float alpha = __fdiv_rn(*a.Q.scale, (float)a.Q.lm1);   // = the double quotient rounded to float
    const bool cross = a.mode == kGatherMu && a.zx;                // QIHT_MU_CROSS: also zx . z
    double acc = 0.0, accx = 0.0;
    unsigned mx = 0;
    if (q < ld) {
        float zz[G];
#pragma unroll
        for (int k = 0; k < G; ++k) zz[k] = 0.0f;
        const float* src0 = a.partial + (size_t)q * G;
        int ch = 0;
        for (; ch + 4 <= nchunks; ch += 4) {
            float4 v[4][G / 4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int k = 0; k < G; k += 4)
                    v[u][k / 4] = __ldcg(reinterpret_cast<const float4*>(src0 + (size_t)(ch + u) * rows_pad + k));
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int k = 0; k < G; k += 4) {
                    zz[k] += v[u][k / 4].x; zz[k + 1] += v[u][k / 4].y;
                    zz[k + 2] += v[u][k / 4].z; zz[k + 3] += v[u][k / 4].w;
                }
        }
        for (; ch < nchunks; ++ch) {
#pragma unroll
            for (int k = 0; k < G; k += 4) {
                const float4 v = __ldcg(reinterpret_cast<const float4*>(src0 + (size_t)ch * rows_pad + k));
                zz[k] += v.x; zz[k + 1] += v.y; zz[k + 2] += v.z; zz[k + 3] += v.w;
            }
        }
#pragma unroll
        for (int k = 0; k < G; ++k) {
            const int i = q * G + k;
            if (i < m) {
                if (a.mode == kGatherPlain) {
                    a.z[i] = alpha * zz[k];
                } else if (a.mode == kGatherResid) {
                    const float ri = fmaf(-alpha, zz[k], __ldcg(a.yhat + i));
                    a.r[i] = ri;
                    acc += (double)ri * (double)ri;
                    mx = max(mx, __float_as_uint(ri) & 0x7fffffffu);
                } else {
                    acc += (double)zz[k] * (double)zz[k];
                    if (cross) accx += (double)__ldcg(a.zx + i) * (double)zz[k];
                }
            }
        }
    }
    if (a.mode == kGatherPlain) {
        __syncthreads();
        if (threadIdx.x == 0) a.counters[rb] = 0;
        return;
    }
    acc = block_sum_d(acc, shd);
    mx = block_max_u(mx, shu);
    if (cross) accx = block_sum_d(accx, shd);
    if (threadIdx.x == 0) {
        a.rb_partial[2 * rb] = acc;
        a.rb_partial[2 * rb + 1] = cross ? accx : (double)mx;   // exact: mx < 2^32
        a.counters[rb] = 0;
    }
    // arrival of this row block
    __threadfence();
    __syncthreads();
    const int nrb = gridDim.x;
    if (threadIdx.x == 0) flag = (atomicAdd(&a.counters[nrb], 1u) == (unsigned)nrb - 1);
    __syncthreads();
    if (!flag) return;
    __threadfence();

    // final scalars (one CTA): the partials are read in parallel by warp 0 and summed with a
    // fixed tree, so the result is deterministic
    if (threadIdx.x < 32) {
        double t = 0.0, mxl = 0.0, cs = 0.0;
        for (int b = threadIdx.x; b < nrb; b += 32) {
            t += __ldcg(a.rb_partial + 2 * b);
            if (cross) mxl += __ldcg(a.rb_partial + 2 * b + 1);        // the sum of zx . z
            else mxl = fmax(mxl, __ldcg(a.rb_partial + 2 * b + 1));
        }
        if (a.chunk_partial && (a.mode == kGatherMu || a.mode == kGatherOmega))
            for (int c = threadIdx.x; c < nchunks; c += 32) cs += __ldcg(a.chunk_partial + c);
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            t += __shfl_xor_sync(0xffffffffu, t, o);
            const double om = __shfl_xor_sync(0xffffffffu, mxl, o);
            mxl = cross ? mxl + om : fmax(mxl, om);
            cs += __shfl_xor_sync(0xffffffffu, cs, o);
        }
        if (threadIdx.x == 0) {
            a.counters[nrb] = 0;
            shd[32] = t;
            shd[31] = mxl;
            shd[30] = cs;
        }
    }
    __syncthreads();
    const double total = shd[32];
    const double mxd = shd[31];
    const double coef_norm2 = shd[30];
    const double alpha_d = (double)(*a.Q.scale) / (double)a.Q.lm1;

    if (a.mode == kGatherMu) {
        if (threadIdx.x == 0) {
            const double num = coef_norm2;
            const double den_f = alpha_d * alpha_d * total;
            double den = den_f;
            if (cross) {
                const double den_c = alpha_d * mxd;         // zx holds alpha Q1_G g_G
                if (den_c > 0.0) den = den_c;              // else the forward square
            }
            st->num = num;
            st->bt = 0;
            if (!isfinite(num) || !isfinite(den_f)) {
                st->status = QIHT_ERR_NONFINITE;
                st->stop = 1;
            } else if (num == 0.0 || den_f == 0.0) {
                st->stop = 1;                      // converged: x stays
            } else {
                st->mu = num / den;
            }
        }
    } else if (a.mode == kGatherOmega) {
        if (threadIdx.x == 0) {
            const double dn = coef_norm2;
            const double dd = alpha_d * alpha_d * total;
            unsigned again = 0;
            if (dn > 0.0) {
                const double omega = dd > 0.0 ? dn / dd : INFINITY;
                const double bound = (1.0 - a.c) * omega;
                const double mu = st->mu;
                if (!(mu <= bound)) {
                    if (st->bt >= a.max_bt) {
                        st->status = QIHT_ERR_BACKTRACK_CAP;
                        st->stop = 1;
                    } else {
                        st->mu = mu / (a.k * (1.0 - a.c));
                        st->bt += 1;
                        again = 1;
                    }
                }
            }
            st->again = (int)again;
            set_cond(a.h_bt, again);
        }
    } else {  // Resid: commit the accepted proposal
        const int s = a.s;
        // zero the old support, then write the new one
        for (int q2 = threadIdx.x; q2 < s; q2 += blockDim.x) a.x[__ldcg(a.support_out + q2)] = 0.0f;
        __syncthreads();
        for (int q2 = threadIdx.x; q2 < s; q2 += blockDim.x) {
            const int j = __ldcg(a.new_sel + q2);
            a.x[j] = __ldcg(a.new_val + q2);
            a.support_out[q2] = j;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const int it = st->iter + 1;
            st->iter = it;
            st->resid2 = total;
            st->rmax_bits = (unsigned)mxd;
            st->mu_accepted = st->mu;
            st->backtracks_total += st->bt;
            st->support_changes_total += st->changed;
            if (!isfinite(total)) {
                st->status = QIHT_ERR_NONFINITE;
                st->stop = 1;
            }
            if (a.trace.kth) { a.trace.kth[2 * it] = st->kth0; a.trace.kth[2 * it + 1] = st->kth1; }
            if (a.trace.mu) a.trace.mu[it] = st->mu;
            if (a.trace.bt) a.trace.bt[it] = st->bt;
            if (a.trace.resid2) a.trace.resid2[it] = total;
            if (it >= st->iters) st->stop = 1;
            if (a.tol > 0.0 && total <= a.tol) st->stop = 1;      // the residual reached tol
            write_report(a, st);
        }
        __syncthreads();
        if (a.trace.support) {
            const int it = st->iter;
            for (int q2 = threadIdx.x; q2 < s; q2 += blockDim.x)
                a.trace.support[(size_t)it * s + q2] = __ldcg(a.new_sel + q2);
        }
    }
}

int gather_row_blocks(int rows, int bits)
{
    const int G = 32 / bits;
    const int words = (rows + G - 1) / G;
    return (words + kGatherThreads - 1) / kGatherThreads;
}

int gather_chunks(int count) { return (count + kGatherCols - 1) / kGatherCols; }

size_t gather_partial_floats(int rows, int bits, int count)
{
    const int G = 32 / bits;
    const int ld = qiht_ld_words(rows, bits);
    return (size_t)gather_chunks(count) * (size_t)ld * (size_t)G;
}

static void* gather_fn(int bits)
{
    switch (bits) {
    case 2: return (void*)k_gather<2>;
    case 4: return (void*)k_gather<4>;
    default: return (void*)k_gather<8>;
    }
}

void gather_node(const GatherArgs& a, cudaKernelNodeParams* p, void** argbuf)
{
    const int maxcount = (a.mode == kGatherOmega) ? 2 * a.s : (a.mode == kGatherPlain ? a.count : a.s);
    p->func = gather_fn(a.Q.bits);
    p->gridDim = dim3(gather_row_blocks(a.Q.rows, a.Q.bits), gather_chunks(maxcount));
    p->blockDim = dim3(kGatherThreads);
    p->sharedMemBytes = 0;
    p->kernelParams = argbuf;
    p->extra = nullptr;
}

// Residual of a fresh realization: the observation codes Y (one column) are dequantized
// into yhat, r = yhat - z with z = alpha Q2_G x_G already formed, and max |r| is folded into
// *rmax_bits (reset by the caller) for the next gradient product.
__global__ void __launch_bounds__(256) k_fresh_resid(Codes Y, const float* __restrict__ z, float* __restrict__ yhat,
                                                     float* __restrict__ r, int m, unsigned* rmax_bits)
{
    __shared__ unsigned wmax[8];
    const int Gy = 32 / Y.bits;
    const double alpha_y = (double)(*Y.scale) / (double)Y.lm1;
    unsigned mx = 0;
    for (int i = blockIdx.x * 256 + threadIdx.x; i < m; i += gridDim.x * 256) {
        const uint32_t w = __ldg(Y.words + i / Gy);
        const int k = i % Gy;
        const int code = (int)((w >> (8 * (k & 3) + Y.bits * (k >> 2))) & ((1u << Y.bits) - 1));
        const float v = (float)(alpha_y * (double)(2 * code - Y.lm1));
        yhat[i] = v;
        const float ri = v - z[i];
        r[i] = ri;
        mx = max(mx, __float_as_uint(ri) & 0x7fffffffu);
    }
    mx = __reduce_max_sync(0xffffffffu, mx);
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned b = 0;
        for (int w = 0; w < 8; ++w) b = max(b, wmax[w]);
        atomicMax(rmax_bits, b);
    }
}

cudaError_t launch_fresh_resid(const Codes& Y, const float* z, float* yhat, float* r, int m, unsigned* rmax_bits,
                               cudaStream_t s)
{
    int blocks = (m + 255) / 256;
    if (blocks > 152) blocks = 152;
    k_fresh_resid<<<blocks, 256, 0, s>>>(Y, z, yhat, r, m, rmax_bits);
    return cudaGetLastError();
}

cudaError_t launch_gather(const GatherArgs& a, cudaStream_t s)
{
    cudaKernelNodeParams p{};
    GatherArgs copy = a;
    void* args[1] = {&copy};
    gather_node(a, &p, args);
    return cudaLaunchKernel(p.func, p.gridDim, p.blockDim, args, 0, s);
}

// ---------------------------------------------------------------------------
// Allocation-free column-subset product (qiht_gemv_cols_static).
//
// Some callers cannot call cudaMalloc at the moment they need this product:
// code that runs while its stream is being captured into a CUDA graph, real-time
// loops that forbid device allocation once they are running, or plug-ins whose
// host application owns every device allocation and hands out no workspace.
// For them the scratch of the product (chunk partial sums, per-row-block sums and
// arrival counters) lives in one fixed array of this library's device memory.
// Every GPU that loads the library holds the array until the process exits.
// ---------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_static_scratch[QIHT_STATIC_SCRATCH_BYTES];

namespace {
// Device address of g_static_scratch, per CUDA context: the array has its own address in
// every context that loads the library (the primary context of each device, or a context
// the caller made current through the driver API). Contexts are told apart by their
// unique id, which is never reused within a process.
struct StaticAddr {
    unsigned long long ctx_id;
    void* addr;
};
std::mutex g_static_mu;
std::vector<StaticAddr> g_static_addr;

typedef int (*CtxGetCurrentFn)(void**);
typedef int (*CtxGetIdFn)(void*, unsigned long long*);

// Unique id of the current context (0 when no context is current yet).
cudaError_t current_context_id(unsigned long long* id)
{
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    if (!get_current || !get_id) {
        void* f1 = nullptr;
        void* f2 = nullptr;
        cudaDriverEntryPointQueryResult q1{}, q2{};
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
        if (e != cudaSuccess || q1 != cudaDriverEntryPointSuccess || !f1) return cudaErrorNotSupported;
        e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
        if (e != cudaSuccess || q2 != cudaDriverEntryPointSuccess || !f2) return cudaErrorNotSupported;
        get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
        get_id = reinterpret_cast<CtxGetIdFn>(f2);
    }
    void* ctx = nullptr;
    *id = 0;
    if (get_current(&ctx) != 0) return cudaErrorDeviceUninitialized;
    if (ctx && get_id(ctx, id) != 0) return cudaErrorDeviceUninitialized;
    return cudaSuccess;
}
}  // namespace

// Device address of the static scratch in the current context. The host-side name
// g_static_scratch is only a stand-in; its device address comes from
// cudaGetSymbolAddress, taken once per context while that context is current.
static cudaError_t static_scratch_address(void** out)
{
    unsigned long long id = 0;
    cudaError_t e = current_context_id(&id);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (id != 0)
        for (const StaticAddr& sa : g_static_addr)
            if (sa.ctx_id == id) {
                *out = sa.addr;
                return cudaSuccess;
            }
    // first call in this context (the lookup also makes the device's primary context
    // current when the thread had none)
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    if (id == 0) {
        e = current_context_id(&id);
        if (e != cudaSuccess) return e;
        if (id == 0) return cudaErrorDeviceUninitialized;
    }
    g_static_addr.push_back(StaticAddr{id, p});
    *out = p;
    return cudaSuccess;
}

}  // namespace qiht

extern "C" qiht_status qiht_gemv_cols_static(const qiht_codes* Q, const int32_t* cols, const float* coef,
                                             int32_t count, float* z, qiht_stream_t stream)
{
    using namespace qiht;
    const qiht_status ce = check_codes(Q);     // the same checks as qiht_gemv_cols
    if (ce != QIHT_OK) return ce;
    if (!cols || !coef || !z || count < 1) return QIHT_ERR_ARG;
    // same scratch layout as qiht_gemv_cols; it must fit the fixed array
    const size_t need = qiht_gemv_cols_workspace_size(Q->rows, count);
    if (need > QIHT_STATIC_SCRATCH_BYTES) return QIHT_ERR_WORKSPACE;
    void* base = nullptr;
    if (static_scratch_address(&base) != cudaSuccess) return QIHT_ERR_CUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    char* w = reinterpret_cast<char*>(base);
    size_t fl = 0;
    for (int b : {2, 4, 8}) {
        const size_t f = gather_partial_floats(Q->rows, b, count);
        if (f > fl) fl = f;
    }
    const int rbmax = gather_row_blocks(Q->rows, 2) > gather_row_blocks(Q->rows, 8) ? gather_row_blocks(Q->rows, 2)
                                                                                  : gather_row_blocks(Q->rows, 8);
    const size_t a256 = 255;
    const size_t off_rb = (fl * 4 + a256) & ~a256;
    const size_t off_cnt = off_rb + (((size_t)rbmax * 2 * 8 + a256) & ~a256);
    GatherArgs a{};
    a.Q = view(Q);
    a.cols = cols;
    a.coef = coef;
    a.count = count;
    a.z = z;
    a.partial = reinterpret_cast<float*>(w);
    a.rb_partial = reinterpret_cast<double*>(w + off_rb);
    a.counters = reinterpret_cast<unsigned*>(w + off_cnt);
    a.mode = kGatherPlain;
    // the array keeps the previous call's contents: the arrival counters must start at zero
    if (cudaMemsetAsync(a.counters, 0, (size_t)(gather_row_blocks(Q->rows, Q->bits) + 1) * 4, s) != cudaSuccess)
        return QIHT_ERR_CUDA;
    if (launch_gather(a, s) != cudaSuccess) return QIHT_ERR_CUDA;
    return QIHT_OK;
}

