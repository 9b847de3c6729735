// C ABI of the QIHT library and the iteration driver of Algorithm 2.
//
// One call of qiht_niht_solve launches one CUDA graph:
//   init:  Q(y) dequantized, r = Q(y), x = 0        (k_init)
//          g = Q1^T r                              (gemv_t)
//          G = supp H_s(g)                         (top, init mode)
//   WHILE (not done):                              conditional node, set by Resid
//          mu = ||g_G||^2 / ||Q2_G g_G||^2          (gather, Mu)
//          x' = H_s(x + mu g), G'                   (top)
//          backtracking test on G' u G              (gather, Omega)
//          WHILE (test failed): shrink mu; top; Omega   conditional node, set by Omega
//          r = Q(y) - Q2_G' x', commit x, G          (gather, Resid)
//          g = Q1^T r                              (gemv_t)
// Control stays on the device for the whole solve. Graphs are cached per
// argument set (pointers, sizes, parameters, device).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "internal.cuh"

namespace qiht {

thread_local char g_last_error[256] = "";

void note_cuda_error(const char* what, cudaError_t e)
{
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s", what, cudaGetErrorString(e));
}

int num_sms()
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

__device__ __forceinline__ void set_cond_init(unsigned long long h, unsigned v)
{
    if (h) cudaGraphSetConditional((cudaGraphConditionalHandle)h, v);
}

struct InitKernelArgs {
    InitArgs a;
    unsigned long long h_outer;
};

// Initial state: dequantized observation Q(y), r = Q(y), x = 0, scalars reset.
__global__ void __launch_bounds__(1024) k_init(InitKernelArgs ka)
{
    const InitArgs& a = ka.a;
    State* st = a.st;
    __shared__ double shd[33];
    __shared__ unsigned shu[33];
    const uint32_t ymask = (1u << a.Y.bits) - 1;
    const int lm1y = a.Y.lm1;
    const int Gy = 32 / a.Y.bits;
    const float sy = *a.Y.scale, s1 = *a.scale_q1, s2 = *a.scale_q2;
    const bool finite = isfinite(sy) && isfinite(s1) && isfinite(s2);
    const double alpha_y = (double)sy / (double)lm1y;
    double acc = 0.0;
    unsigned mx = 0;
    for (int i = threadIdx.x; i < a.m; i += blockDim.x) {
        const uint32_t w = a.Y.words[i / Gy];
        const int k = i % Gy;
        const int code = (int)((w >> (8 * (k & 3) + a.Y.bits * (k >> 2))) & ymask);
        const float v = (float)(alpha_y * (double)(2 * code - lm1y));
        a.yhat[i] = v;
        a.r[i] = v;
        acc += (double)v * (double)v;
        mx = max(mx, __float_as_uint(v) & 0x7fffffffu);
    }
    for (int j = threadIdx.x; j < a.n; j += blockDim.x) a.x[j] = 0.0f;
    if (a.pos)
        for (int j = threadIdx.x; j < a.n; j += blockDim.x) a.pos[j] = -1;
    if (a.part)       // -0.0: tag bit set, value 0 (the first writes carry tag 0)
        for (int i = threadIdx.x; i < kPartSlots * kSlotCtas; i += blockDim.x) a.part[i] = -0.0;
    // deterministic block reductions
#pragma unroll
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    mx = __reduce_max_sync(0xffffffffu, mx);
    if ((threadIdx.x & 31) == 0) { shd[threadIdx.x >> 5] = acc; shu[threadIdx.x >> 5] = mx; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        unsigned b = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { t += shd[w]; b = max(b, shu[w]); }
        memset(st, 0, sizeof(State));
        st->iters = a.iters;
        st->dec_word = 1ull << 63;     // tag 1: the first decision carries tag 0
        st->resid2 = t;
        st->rmax_bits = b;
        st->status = finite ? QIHT_OK : QIHT_ERR_NONFINITE;
        st->stop = finite ? 0 : 1;     // iters == 0 still selects the initial support
        if (a.trace.mu) a.trace.mu[0] = 0.0;
        if (a.trace.bt) a.trace.bt[0] = 0;
        if (a.trace.resid2) a.trace.resid2[0] = t;
        if (a.report) {
            a.report->iters_run = 0;
            a.report->backtracks = 0;
            a.report->support_changes = 0;
            a.report->status = st->status;
            a.report->resid_norm2 = t;
            a.report->mu = 0.0;
            a.report->full_selects = 0;
            a.report->reserved = 0;
            for (int i = 0; i < 8; ++i) a.report->phase_us[i] = 0.0f;
        }
        set_cond_init(ka.h_outer, (finite && a.iters > 0) ? 1u : 0u);
    }
}

void init_node(const InitArgs&, cudaKernelNodeParams*, void**) {}

}  // namespace qiht

using namespace qiht;

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static bool bits_ok(int b) { return b == 2 || b == 4 || b == 8; }

static bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

qiht_status qiht::check_codes(const qiht_codes* Q)
{
    if (!Q || !Q->words || !Q->scale) return QIHT_ERR_ARG;
    if (!bits_ok(Q->bits)) return QIHT_ERR_BITS;
    if (Q->rows < 1 || Q->cols < 1) return QIHT_ERR_ARG;
    if (Q->ld_words != qiht_ld_words(Q->rows, Q->bits)) return QIHT_ERR_ARG;
    if (grid_levels(Q->bits, Q->levels) < 0) return QIHT_ERR_ARG;
    if (!aligned(Q->words, 16)) return QIHT_ERR_ARG;
    return QIHT_OK;
}

Codes qiht::view(const qiht_codes* Q)
{
    Codes c;
    c.words = Q->words;
    c.scale = Q->scale;
    c.rows = Q->rows;
    c.cols = Q->cols;
    c.bits = Q->bits;
    c.ld = Q->ld_words;
    c.lm1 = grid_levels(Q->bits, Q->levels) - 1;
    return c;
}

extern "C" {

const char* qiht_status_string(int32_t status)
{
    switch (status) {
    case QIHT_OK: return "QIHT_OK";
    case QIHT_ERR_ARG: return "QIHT_ERR_ARG";
    case QIHT_ERR_BITS: return "QIHT_ERR_BITS";
    case QIHT_ERR_NONFINITE: return "QIHT_ERR_NONFINITE";
    case QIHT_ERR_TIMEOUT: return "QIHT_ERR_TIMEOUT";
    case QIHT_ERR_BACKTRACK_CAP: return "QIHT_ERR_BACKTRACK_CAP";
    case QIHT_ERR_CUDA: return "QIHT_ERR_CUDA";
    case QIHT_ERR_WORKSPACE: return "QIHT_ERR_WORKSPACE";
    default: return "QIHT_UNKNOWN_STATUS";
    }
}

int32_t qiht_abi_version(void) { return QIHT_ABI_VERSION; }

const char* qiht_last_error(void) { return g_last_error; }

int32_t qiht_ld_words(int32_t rows, int32_t bits)
{
    if (!bits_ok(bits) || rows < 1) return -1;
    const int G = 32 / bits;
    const int w = (rows + G - 1) / G;
    return (w + 3) & ~3;
}

static qiht_status quantize_impl(const float* in, int32_t rows, int32_t cols, int64_t ld_in, int32_t bits,
                                 uint64_t seed, uint32_t stream_id, uint32_t stream_id2, int32_t flags,
                                 uint32_t* words, uint32_t* words2, int32_t ld_words, float* scale,
                                 qiht_stream_t stream)
{
    if (!bits_ok(bits)) return QIHT_ERR_BITS;
    if (!in || !words || !scale || rows < 1 || cols < 1 || ld_in < cols) return QIHT_ERR_ARG;
    if (ld_words != qiht_ld_words(rows, bits) || !aligned(words, 16)) return QIHT_ERR_ARG;
    if (words2 && (!aligned(words2, 16) || words2 == words)) return QIHT_ERR_ARG;
    if (flags & ~(QIHT_SCALE_GIVEN | QIHT_CHECK_FINITE | QIHT_ODD_LEVELS)) return QIHT_ERR_ARG;
    const int levels = (flags & QIHT_ODD_LEVELS) ? (1 << (bits - 1)) + 1 : (1 << bits);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (!(flags & QIHT_SCALE_GIVEN)) {
        if (launch_absmax(in, rows, cols, ld_in, scale, s) != cudaSuccess) return QIHT_ERR_CUDA;
    }
    if (launch_quantize(in, rows, cols, ld_in, bits, seed, stream_id, words, ld_words, scale, s, stream_id2,
                        words2, levels) != cudaSuccess)
        return QIHT_ERR_CUDA;
    if (flags & QIHT_CHECK_FINITE) {
        float h = 0.0f;
        if (cudaMemcpyAsync(&h, scale, sizeof(float), cudaMemcpyDeviceToHost, s) != cudaSuccess) return QIHT_ERR_CUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return QIHT_ERR_CUDA;
        if (!std::isfinite(h)) return QIHT_ERR_NONFINITE;
    }
    return QIHT_OK;
}

qiht_status qiht_quantize(const float* in, int32_t rows, int32_t cols, int64_t ld_in, int32_t bits,
                          uint64_t seed, uint32_t stream_id, int32_t flags,
                          uint32_t* words, int32_t ld_words, float* scale, qiht_stream_t stream)
{
    return quantize_impl(in, rows, cols, ld_in, bits, seed, stream_id, 0u, flags, words, nullptr, ld_words, scale,
                         stream);
}

qiht_status qiht_quantize_pair(const float* in, int32_t rows, int32_t cols, int64_t ld_in, int32_t bits,
                               uint64_t seed, uint32_t stream_a, uint32_t stream_b, int32_t flags,
                               uint32_t* words_a, uint32_t* words_b, int32_t ld_words, float* scale,
                               qiht_stream_t stream)
{
    if (!words_b) return QIHT_ERR_ARG;
    return quantize_impl(in, rows, cols, ld_in, bits, seed, stream_a, stream_b, flags, words_a, words_b, ld_words,
                         scale, stream);
}

size_t qiht_gemv_t_workspace_size(void) { return 256; }

qiht_status qiht_gemv_t(const qiht_codes* Q, const float* r, float* g, void* workspace, size_t workspace_bytes,
                        qiht_stream_t stream)
{
    qiht_status e = check_codes(Q);
    if (e != QIHT_OK) return e;
    if (!r || !g) return QIHT_ERR_ARG;
    if (Q->rows > kMaxRows) return QIHT_ERR_ARG;
    if (!workspace || workspace_bytes < qiht_gemv_t_workspace_size() || !aligned(workspace, 256))
        return QIHT_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    float* rmax = reinterpret_cast<float*>(workspace);
    if (launch_absmax(r, Q->rows, 1, 1, rmax, s) != cudaSuccess) return QIHT_ERR_CUDA;
    GemvTArgs a{};
    a.Q = view(Q);
    a.r = r;
    a.rmax_bits = reinterpret_cast<const unsigned*>(rmax);
    a.g = g;
    a.st = nullptr;
    a.err = reinterpret_cast<unsigned*>(reinterpret_cast<char*>(workspace) + 4);
    if (launch_gemv_t(a, num_sms(), s) != cudaSuccess) return QIHT_ERR_CUDA;
    return QIHT_OK;
}

qiht_status qiht_gemv_t_prescaled(const qiht_codes* Q, const float* r, const float* rmax, float* g,
                                  qiht_stream_t stream)
{
    qiht_status e = check_codes(Q);
    if (e != QIHT_OK) return e;
    if (!r || !g || !rmax) return QIHT_ERR_ARG;
    if (Q->rows > kMaxRows) return QIHT_ERR_ARG;
    GemvTArgs a{};
    a.Q = view(Q);
    a.r = r;
    a.rmax_bits = reinterpret_cast<const unsigned*>(rmax);
    a.g = g;
    a.st = nullptr;
    if (launch_gemv_t(a, num_sms(), reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess) return QIHT_ERR_CUDA;
    return QIHT_OK;
}

size_t qiht_gemv_cols_workspace_size(int32_t rows, int32_t count)
{
    if (rows < 1 || count < 1) return 0;
    const int rb = gather_row_blocks(rows, 2) > gather_row_blocks(rows, 8) ? gather_row_blocks(rows, 2)
                                                                            : gather_row_blocks(rows, 8);
    size_t fl = 0;
    for (int b : {2, 4, 8}) {
        const size_t f = gather_partial_floats(rows, b, count);
        if (f > fl) fl = f;
    }
    return align256(fl * 4) + align256((size_t)rb * 2 * 8) + align256((size_t)(rb + 1) * 4);
}

qiht_status qiht_gemv_cols(const qiht_codes* Q, const int32_t* cols, const float* coef, int32_t count, float* z,
                           void* workspace, size_t workspace_bytes, qiht_stream_t stream)
{
    qiht_status e = check_codes(Q);
    if (e != QIHT_OK) return e;
    if (!cols || !coef || !z || count < 1) return QIHT_ERR_ARG;
    const size_t need = qiht_gemv_cols_workspace_size(Q->rows, count);
    if (!workspace || workspace_bytes < need || !aligned(workspace, 256)) return QIHT_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    char* w = reinterpret_cast<char*>(workspace);
    const int rb = gather_row_blocks(Q->rows, Q->bits);
    size_t fl = 0;
    for (int b : {2, 4, 8}) {
        const size_t f = gather_partial_floats(Q->rows, b, count);
        if (f > fl) fl = f;
    }
    const int rbmax = gather_row_blocks(Q->rows, 2) > gather_row_blocks(Q->rows, 8) ? gather_row_blocks(Q->rows, 2)
                                                                                  : gather_row_blocks(Q->rows, 8);
    GatherArgs a{};
    a.Q = view(Q);
    a.cols = cols;
    a.coef = coef;
    a.count = count;
    a.z = z;
    a.partial = reinterpret_cast<float*>(w);
    a.rb_partial = reinterpret_cast<double*>(w + align256(fl * 4));
    a.counters = reinterpret_cast<unsigned*>(w + align256(fl * 4) + align256((size_t)rbmax * 2 * 8));
    a.mode = kGatherPlain;
    if (cudaMemsetAsync(a.counters, 0, (size_t)(rb + 1) * 4, s) != cudaSuccess) return QIHT_ERR_CUDA;
    if (launch_gather(a, s) != cudaSuccess) return QIHT_ERR_CUDA;
    return QIHT_OK;
}

size_t qiht_top_s_workspace_size(int32_t n)
{
    return (n > kMaxTopN && n <= kMaxBigTopN) ? big_top_workspace(n) : 0;
}

qiht_status qiht_top_s(const float* a, int32_t n, int32_t s, int32_t* idx, float* val, float* kth, void* workspace,
                       size_t workspace_bytes, qiht_stream_t stream)
{
    if (!a || !idx || n < 1 || s < 1 || s > n || n > kMaxBigTopN) return QIHT_ERR_ARG;
    if (n > kMaxTopN) {
        // more keys than one CTA holds: the multi-CTA select (same result)
        if (!workspace || workspace_bytes < big_top_workspace(n) || !aligned(workspace, 256)) return QIHT_ERR_WORKSPACE;
        if (launch_big_top(a, nullptr, nullptr, n, s, idx, val, kth, workspace, reinterpret_cast<cudaStream_t>(stream)) !=
            cudaSuccess)
            return QIHT_ERR_CUDA;
        return QIHT_OK;
    }
    TopArgs t{};
    t.g = a;
    t.x = nullptr;
    t.mu = nullptr;
    t.n = n;
    t.s = s;
    t.sel = idx;
    t.val = val;
    t.kth = kth;
    t.st = nullptr;
    if (launch_top(t, reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess) return QIHT_ERR_CUDA;
    return QIHT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// solver workspace plan
// ---------------------------------------------------------------------------
namespace {

struct Plan {
    size_t off_state, off_yhat, off_r, off_g, off_sel, off_val, off_uni, off_delta, off_partial, off_rbp, off_chunk,
        off_cand, off_keys, off_part, off_pos, off_xs, off_gsup, off_gcand, off_z1, total;
};

Plan plan_solve(int m, int n, int s)
{
    Plan p{};
    size_t o = 0;
    const size_t rows_pad = (size_t)qiht_ld_words(m, 2) * 16;   // the largest padding over b in {2, 4, 8}
    p.off_state = o; o += align256(sizeof(State));
    p.off_yhat = o; o += align256(rows_pad * 4);
    p.off_r = o; o += align256(rows_pad * 4);
    p.off_g = o; o += align256((size_t)n * 4);
    p.off_sel = o; o += align256((size_t)s * 4);
    p.off_val = o; o += align256((size_t)s * 4);
    p.off_uni = o; o += align256((size_t)2 * s * 4);
    p.off_delta = o; o += align256((size_t)2 * s * 4);
    size_t fl = 0;
    for (int b : {2, 4, 8}) {
        const size_t f = gather_partial_floats(m, b, 2 * s);
        if (f > fl) fl = f;
    }
    p.off_partial = o; o += align256(fl * 4);
    const int rb = gather_row_blocks(m, 2) > gather_row_blocks(m, 8) ? gather_row_blocks(m, 2) : gather_row_blocks(m, 8);
    p.off_rbp = o; o += align256((size_t)rb * 2 * 8);
    p.off_chunk = o; o += align256((size_t)gather_chunks(2 * s) * 8);
    p.off_cand = o; o += align256((size_t)kTopCandCap * 16);     // keys, then values and old x
    p.off_keys = o; o += align256((size_t)n * 4);
    p.off_part = o; o += align256((size_t)kPartSlots * kSlotCtas * 8);
    p.off_pos = o; o += align256((size_t)n * 4);
    p.off_xs = o; o += align256((size_t)s * 4);
    p.off_gsup = o; o += align256((size_t)s * 4);
    p.off_gcand = o; o += align256((size_t)kTopCandCap * 8);
    p.off_z1 = o; o += align256(rows_pad * 4);                   // alpha Q1_G g_G (QIHT_MU_CROSS)
    p.total = o;
    return p;
}

struct Key {
    std::vector<uint64_t> v;
    bool operator<(const Key& o) const { return v < o.v; }
};

struct Cached {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

std::mutex g_mu;
std::map<Key, Cached> g_cache;

uint64_t dbits(double d)
{
    uint64_t u;
    std::memcpy(&u, &d, 8);
    return u;
}

void push_codes(std::vector<uint64_t>& v, const qiht_codes* Q)
{
    v.push_back(reinterpret_cast<uint64_t>(Q->words));
    v.push_back(reinterpret_cast<uint64_t>(Q->scale));
    v.push_back((uint64_t)Q->rows);
    v.push_back((uint64_t)Q->cols);
    v.push_back((uint64_t)Q->bits);
    v.push_back((uint64_t)Q->ld_words);
    v.push_back((uint64_t)grid_levels(Q->bits, Q->levels));
}

#define CK(x)                                       \
    do {                                            \
        cudaError_t ck_e_ = (x);                    \
        if (ck_e_ != cudaSuccess) {                 \
            note_cuda_error(#x, ck_e_);             \
            return QIHT_ERR_CUDA;                   \
        }                                           \
    } while (0)

qiht_status add_kernel(cudaGraph_t g, cudaGraphNode_t* out, const cudaGraphNode_t* dep, int ndep,
                       const cudaKernelNodeParams& p)
{
    CK(cudaGraphAddKernelNode(out, g, dep, ndep, &p));
    return QIHT_OK;
}

qiht_status add_while(cudaGraph_t g, cudaGraphNode_t* out, const cudaGraphNode_t* dep, int ndep,
                      cudaGraphConditionalHandle h, cudaGraph_t* body)
{
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    CK(cudaGraphAddNode(out, g, dep, nullptr, ndep, &cp));
    *body = cp.conditional.phGraph_out[0];
    return QIHT_OK;
}

#define TRY(x)                          \
    do {                                \
        qiht_status _e = (x);           \
        if (_e != QIHT_OK) return _e;   \
    } while (0)

static bool multi_kernel_iteration();

// QIHT_PDL=0 turns the programmatic edges of the loop body off; QIHT_UNROLL sets the
// iterations per body execution with them (default 8). For measurement.
static bool use_pdl()
{
    static int v = -1;
    if (v < 0) {
        const char* e = getenv("QIHT_PDL");
        v = (e && e[0] == '0') ? 0 : 1;
    }
    return v == 1;
}

static int body_unroll()
{
    static int v = -1;
    if (v < 0) {
        const char* e = getenv("QIHT_UNROLL");
        v = e ? atoi(e) : 8;
        if (v < 1) v = 1;
        if (v > 16) v = 16;
    }
    return v;
}

// The solver's kernels and their arguments, shared by the graph driver and the eager driver.
struct SolveKernels {
    InitKernelArgs ia;
    GemvTArgs g0, gb;
    TopArgs t0, tt;
    GatherArgs gmu, gom, gre, gz1;
    void* a_tf[1];
    cudaKernelNodeParams p_tf;
    alignas(16) unsigned char iter_store[kIterArgsMax];
    void* a_it[1];
    cudaKernelNodeParams p_it;
    void* a_init[1];
    void* a_g0[1];
    void* a_gb[1];
    void* a_t0[1];
    void* a_tt[1];
    void* a_mu[1];
    void* a_om[1];
    void* a_re[1];
    void* a_z1[1];
    cudaKernelNodeParams p_init, p_g0, p_gb, p_t0, p_tt, p_mu, p_om, p_re, p_z1;
    bool cross;                 // QIHT_MU_CROSS: p_z1 (z1 = alpha Q1_G g_G) runs before p_mu
    State* st;
};

static void make_kernels(SolveKernels& K, const qiht_codes* Q1, const qiht_codes* Q2, const qiht_codes* Y, int s,
                         int iters, const qiht_params* prm, float* x, int32_t* support, qiht_report* report,
                         const qiht_trace* trace, char* ws, unsigned long long h_outer, unsigned long long h_bt,
                         bool force_multi = false)
{
    const int m = Q1->rows, n = Q1->cols;
    const Plan pl = plan_solve(m, n, s);
    State* st = reinterpret_cast<State*>(ws + pl.off_state);
    K.st = st;
    float* yhat = reinterpret_cast<float*>(ws + pl.off_yhat);
    float* r = reinterpret_cast<float*>(ws + pl.off_r);
    float* g = reinterpret_cast<float*>(ws + pl.off_g);
    int32_t* sel = reinterpret_cast<int32_t*>(ws + pl.off_sel);
    float* val = reinterpret_cast<float*>(ws + pl.off_val);
    int32_t* uni = reinterpret_cast<int32_t*>(ws + pl.off_uni);
    float* delta = reinterpret_cast<float*>(ws + pl.off_delta);
    float* partial = reinterpret_cast<float*>(ws + pl.off_partial);
    double* rbp = reinterpret_cast<double*>(ws + pl.off_rbp);
    double* chunkp = reinterpret_cast<double*>(ws + pl.off_chunk);
    unsigned long long* cand = reinterpret_cast<unsigned long long*>(ws + pl.off_cand);
    qiht_trace tr{};
    if (trace) tr = *trace;
    const int nsm = num_sms();
    const bool fast = !force_multi && !multi_kernel_iteration() && iter_fast(s);
    IterFastBufs fb{};
    if (fast) {
        fb.pos = reinterpret_cast<int32_t*>(ws + pl.off_pos);
        fb.xs = reinterpret_cast<float*>(ws + pl.off_xs);
        fb.gsup = reinterpret_cast<float*>(ws + pl.off_gsup);
        fb.gcand = reinterpret_cast<unsigned long long*>(ws + pl.off_gcand);
        fb.gcap = kTopCandCap;
    }

    K.ia = InitKernelArgs{};
    K.ia.a.Y = view(Y);
    K.ia.a.scale_q1 = Q1->scale;
    K.ia.a.scale_q2 = Q2->scale;
    K.ia.a.yhat = yhat;
    K.ia.a.r = r;
    K.ia.a.x = x;
    K.ia.a.pos = fb.pos;
    K.ia.a.part = fast ? reinterpret_cast<double*>(ws + pl.off_part) : nullptr;
    K.ia.a.n = n;
    K.ia.a.m = m;
    K.ia.a.s = s;
    K.ia.a.iters = iters;
    K.ia.a.st = st;
    K.ia.a.report = report;
    K.ia.a.trace = tr;
    K.ia.h_outer = h_outer;
    K.a_init[0] = &K.ia;
    K.p_init = cudaKernelNodeParams{};
    K.p_init.func = (void*)k_init;
    K.p_init.gridDim = dim3(1);
    K.p_init.blockDim = dim3(1024);
    K.p_init.kernelParams = K.a_init;

    K.g0 = GemvTArgs{};
    K.g0.Q = view(Q1);
    K.g0.r = r;
    K.g0.rmax_bits = &st->rmax_bits;
    K.g0.g = g;
    K.g0.st = st;
    K.g0.h_outer = 0;               // the set-up product does not steer the loop
    K.a_g0[0] = &K.g0;
    gemv_t_node(K.g0, nsm, &K.p_g0, K.a_g0);
    K.gb = K.g0;
    K.gb.h_outer = h_outer;         // the loop body's product decides whether to go on
    K.gb.guard_limit = iters + 1;
    K.gb.pos = fb.pos;              // and prepares the fast path's next threshold
    K.gb.gsup = fb.gsup;
    K.gb.gcand = fb.gcand;
    K.gb.gcap = fb.gcap;
    if (fast) {                     // max |r| from the iteration kernel's partials; final ||r||^2
        K.gb.rpart = reinterpret_cast<const double*>(ws + pl.off_part);
        K.gb.rgrid = iter_grid();
        K.gb.report = report;
        K.gb.trace_resid2 = tr.resid2;
        K.gb.tol = prm->tol;        // ... and the residual tolerance test
    }
    K.a_gb[0] = &K.gb;
    gemv_t_node(K.gb, nsm, &K.p_gb, K.a_gb);

    K.t0 = TopArgs{};
    K.t0.g = g;
    K.t0.n = n;
    K.t0.s = s;
    K.t0.sel = sel;
    K.t0.val = val;
    K.t0.st = st;
    K.t0.init = 1;
    K.t0.support_init = support;
    K.t0.trace = tr;
    K.t0.cand = cand;
    K.t0.cap = kTopCandCap;
    K.a_t0[0] = &K.t0;
    top_node(K.t0, &K.p_t0, K.a_t0);

    K.tt = TopArgs{};
    K.tt.g = g;
    K.tt.x = x;
    K.tt.mu = &st->mu;
    K.tt.n = n;
    K.tt.s = s;
    K.tt.sel = sel;
    K.tt.val = val;
    K.tt.st = st;
    K.tt.support = support;
    K.tt.uni = uni;
    K.tt.delta = delta;
    K.tt.trace = tr;
    K.tt.h_bt = h_bt;
    K.tt.cand = cand;
    K.tt.cap = kTopCandCap;
    K.a_tt[0] = &K.tt;
    top_node(K.tt, &K.p_tt, K.a_tt);
    K.a_tf[0] = &K.tt;
    top_filter_node(K.tt, &K.p_tf, K.a_tf);
    iter_node(view(Q2), st, g, x, support, sel, val, uni, delta, yhat, r,
              reinterpret_cast<uint32_t*>(ws + pl.off_keys), cand, reinterpret_cast<double*>(ws + pl.off_part), fb, n, m, s,
              prm->k, prm->c, prm->max_backtrack, prm->flags, report, tr, &K.p_it, K.iter_store, K.a_it, Q1->words,
              prm->mu_mode, prm->tol);

    GatherArgs base{};
    base.Q = view(Q2);
    base.partial = partial;
    base.rb_partial = rbp;
    base.chunk_partial = chunkp;
    base.st = st;
    base.g = g;
    base.support = support;
    base.yhat = yhat;
    base.r = r;
    base.x = x;
    base.support_out = support;
    base.new_sel = sel;
    base.new_val = val;
    base.s = s;
    base.k = prm->k;
    base.c = prm->c;
    base.max_bt = prm->max_backtrack;
    base.h_outer = h_outer;
    base.h_bt = h_bt;
    base.report = report;
    base.trace = tr;
    K.cross = prm->mu_mode == QIHT_MU_CROSS;
    float* z1 = reinterpret_cast<float*>(ws + pl.off_z1);
    K.gz1 = base;                   // z1 = alpha Q1_G g_G (plain product with the first quantization)
    K.gz1.Q = view(Q1);
    K.gz1.mode = kGatherPlain;
    K.gz1.cols = support;
    K.gz1.coef_from_g = 1;
    K.gz1.count = s;
    K.gz1.z = z1;
    K.gz1.counters = st->counters[0] + 96;
    K.a_z1[0] = &K.gz1;
    gather_node(K.gz1, &K.p_z1, K.a_z1);
    K.gmu = base;
    K.gmu.mode = kGatherMu;
    K.gmu.counters = st->counters[0];
    K.gmu.zx = K.cross ? z1 : nullptr;
    K.a_mu[0] = &K.gmu;
    gather_node(K.gmu, &K.p_mu, K.a_mu);
    K.gom = base;
    K.gom.mode = kGatherOmega;
    K.gom.cols = uni;
    K.gom.coef = delta;
    K.gom.counters = st->counters[0] + 32;
    K.a_om[0] = &K.gom;
    gather_node(K.gom, &K.p_om, K.a_om);
    K.gre = base;
    K.gre.mode = kGatherResid;
    K.gre.tol = prm->tol;
    K.gre.counters = st->counters[0] + 64;
    K.a_re[0] = &K.gre;
    gather_node(K.gre, &K.p_re, K.a_re);
}

static cudaError_t launch_node(const cudaKernelNodeParams& p, cudaStream_t s)
{
    return cudaLaunchKernel(p.func, p.gridDim, p.blockDim, p.kernelParams, p.sharedMemBytes, s);
}

// The iteration kernel waits on grid barriers, so all its CTAs must be resident at once.
static cudaError_t launch_cooperative(const cudaKernelNodeParams& p, cudaStream_t s)
{
    return cudaLaunchCooperativeKernel(p.func, p.gridDim, p.blockDim, p.kernelParams, p.sharedMemBytes, s);
}

static bool multi_kernel_iteration()
{
    // QIHT_SOLVER=multi runs an iteration as separate kernels (step size, filter, select,
    // backtracking test, residual) instead of the persistent iteration kernel
    static int v = -1;
    if (v < 0) {
        const char* e = getenv("QIHT_SOLVER");
        v = (e && e[0] == 'm') ? 1 : 0;
    }
    return v == 1;
}

// Host-driven run of the same kernels (QIHT_SOLVE_EAGER): reads the device state
// after every iteration and after every backtracking test.
qiht_status run_eager(const qiht_codes* Q1, const qiht_codes* Q2, const qiht_codes* Y, int s, int iters,
                      const qiht_params* prm, float* x, int32_t* support, qiht_report* report,
                      const qiht_trace* trace, char* ws, cudaStream_t cs)
{
    SolveKernels K;
    make_kernels(K, Q1, Q2, Y, s, iters, prm, x, support, report, trace, ws, 0, 0);
    State h{};
    auto read_state = [&]() -> bool {
        if (cudaMemcpyAsync(&h, K.st, sizeof(State), cudaMemcpyDeviceToHost, cs) != cudaSuccess) return false;
        return cudaStreamSynchronize(cs) == cudaSuccess;
    };
    CK(launch_node(K.p_init, cs));
    CK(launch_node(K.p_g0, cs));
    CK(launch_node(K.p_t0, cs));
    if (!read_state()) return QIHT_ERR_CUDA;
    if (!multi_kernel_iteration()) {
        for (int t = 0; t < iters && !h.stop; ++t) {
            CK(launch_cooperative(K.p_it, cs));
            CK(launch_node(K.p_gb, cs));
            if (!read_state()) return QIHT_ERR_CUDA;
        }
        return QIHT_OK;
    }
    for (int t = 0; t < iters && !h.stop; ++t) {
        if (K.cross) CK(launch_node(K.p_z1, cs));
        CK(launch_node(K.p_mu, cs));
        CK(launch_node(K.p_tf, cs));
        CK(launch_node(K.p_tt, cs));
        CK(launch_node(K.p_om, cs));
        if (!read_state()) return QIHT_ERR_CUDA;
        for (int b = 0; b <= prm->max_backtrack && h.again && !h.stop; ++b) {
            CK(launch_node(K.p_tf, cs));
            CK(launch_node(K.p_tt, cs));
            CK(launch_node(K.p_om, cs));
            if (!read_state()) return QIHT_ERR_CUDA;
        }
        CK(launch_node(K.p_re, cs));
        CK(launch_node(K.p_gb, cs));
        if (!read_state()) return QIHT_ERR_CUDA;
    }
    return QIHT_OK;
}

// cooperative: mark the iteration kernel's node as a cooperative launch. Without it
// the kernel still finds all its CTAs resident (one CTA per SM, one per SM launched,
// the node starts after the previous one has finished); its bounded barriers turn
// any other case into QIHT_ERR_TIMEOUT.
qiht_status build_graph(const qiht_codes* Q1, const qiht_codes* Q2, const qiht_codes* Y, int s, int iters,
                        const qiht_params* prm, float* x, int32_t* support, qiht_report* report,
                        const qiht_trace* trace, char* ws, bool cooperative, bool pdl, int unroll, cudaGraph_t* out)
{
    cudaGraph_t top;
    CK(cudaGraphCreate(&top, 0));
    cudaGraphConditionalHandle h_outer;
    CK(cudaGraphConditionalHandleCreate(&h_outer, top, 1, cudaGraphCondAssignDefault));
    // the body graph (and its handle) exist only after the outer node is added; the
    // kernel arguments need both handles, so add the set-up nodes first with
    // provisional arguments and fill the loop afterwards
    SolveKernels K0;
    make_kernels(K0, Q1, Q2, Y, s, iters, prm, x, support, report, trace, ws, (unsigned long long)h_outer, 0);
    cudaGraphNode_t n_init, n_g0, n_t0;
    TRY(add_kernel(top, &n_init, nullptr, 0, K0.p_init));
    TRY(add_kernel(top, &n_g0, &n_init, 1, K0.p_g0));
    TRY(add_kernel(top, &n_t0, &n_g0, 1, K0.p_t0));

    cudaGraphNode_t n_w;
    cudaGraph_t body;
    TRY(add_while(top, &n_w, &n_t0, 1, h_outer, &body));
    // the inner (backtracking) loop handle exists only when a conditional node uses it
    cudaGraphConditionalHandle h_bt = 0;
    if (multi_kernel_iteration()) CK(cudaGraphConditionalHandleCreate(&h_bt, body, 0, 0));
    SolveKernels K;
    make_kernels(K, Q1, Q2, Y, s, iters, prm, x, support, report, trace, ws, (unsigned long long)h_outer,
                 (unsigned long long)h_bt);

    if (!multi_kernel_iteration()) {
        // `unroll` iterations per body execution; with `pdl`, programmatic edges let each
        // kernel start (and issue its loads that do not depend on the previous kernel)
        // while the previous one finishes
        GemvTArgs inner = K.gb;
        inner.h_outer = 0;                           // only the body's last product steers the loop
        void* inner_args[1] = {&inner};
        cudaKernelNodeParams p_inner = K.p_gb;
        p_inner.kernelParams = inner_args;
        GemvTArgs last = K.gb;
        last.guard_limit = (iters + unroll - 1) / unroll + 1;
        void* last_args[1] = {&last};
        cudaKernelNodeParams p_last = K.p_gb;
        p_last.kernelParams = last_args;
        cudaGraphEdgeData prog{};
        prog.from_port = cudaGraphKernelNodePortProgrammatic;
        prog.to_port = cudaGraphKernelNodePortDefault;
        prog.type = cudaGraphDependencyTypeProgrammatic;
        cudaGraphNode_t prev = nullptr;
        for (int u = 0; u < unroll; ++u) {
            cudaGraphNode_t b_it, b_gk;
            TRY(add_kernel(body, &b_it, pdl || !prev ? nullptr : &prev, pdl || !prev ? 0 : 1, K.p_it));
            if (pdl && prev) CK(cudaGraphAddDependencies(body, &prev, &b_it, &prog, 1));
            if (cooperative) {
                cudaLaunchAttributeValue coop{};
                coop.cooperative = 1;
                CK(cudaGraphKernelNodeSetAttribute(b_it, cudaLaunchAttributeCooperative, &coop));
            }
            const cudaKernelNodeParams& pg = u == unroll - 1 ? p_last : p_inner;
            TRY(add_kernel(body, &b_gk, pdl ? nullptr : &b_it, pdl ? 0 : 1, pg));
            if (pdl) CK(cudaGraphAddDependencies(body, &b_it, &b_gk, &prog, 1));
            prev = b_gk;
        }
        *out = top;
        return QIHT_OK;
    }

    cudaGraphNode_t b_mu, b_tf, b_top, b_om, b_w, b_re, b_g, b_z1;
    if (K.cross) {
        TRY(add_kernel(body, &b_z1, nullptr, 0, K.p_z1));
        TRY(add_kernel(body, &b_mu, &b_z1, 1, K.p_mu));
    } else {
        TRY(add_kernel(body, &b_mu, nullptr, 0, K.p_mu));
    }
    TRY(add_kernel(body, &b_tf, &b_mu, 1, K.p_tf));
    TRY(add_kernel(body, &b_top, &b_tf, 1, K.p_tt));
    TRY(add_kernel(body, &b_om, &b_top, 1, K.p_om));
    cudaGraph_t inner;
    TRY(add_while(body, &b_w, &b_om, 1, h_bt, &inner));
    cudaGraphNode_t i_tf, i_top, i_om;
    TRY(add_kernel(inner, &i_tf, nullptr, 0, K.p_tf));
    TRY(add_kernel(inner, &i_top, &i_tf, 1, K.p_tt));
    TRY(add_kernel(inner, &i_om, &i_top, 1, K.p_om));
    TRY(add_kernel(body, &b_re, &b_w, 1, K.p_re));
    TRY(add_kernel(body, &b_g, &b_re, 1, K.p_gb));
    *out = top;
    return QIHT_OK;
}

}  // namespace

extern "C" {

size_t qiht_solve_workspace_size(int32_t m, int32_t n, int32_t s)
{
    if (m < 1 || n < 1 || s < 1) return 0;
    return plan_solve(m, n, s).total;
}

qiht_status qiht_niht_solve(const qiht_codes* Q1, const qiht_codes* Q2, const qiht_codes* y, int32_t s, int32_t iters,
                            const qiht_params* params, float* x, int32_t* support, qiht_report* report,
                            const qiht_trace* trace, void* workspace, size_t workspace_bytes, qiht_stream_t stream)
{
    TRY(check_codes(Q1));
    TRY(check_codes(Q2));
    TRY(check_codes(y));
    const int m = Q1->rows, n = Q1->cols;
    if (Q2->rows != m || Q2->cols != n || Q2->bits != Q1->bits) return QIHT_ERR_ARG;
    if (y->rows != m || y->cols != 1) return QIHT_ERR_ARG;
    if (s < 1 || s > m || s > n || iters < 0) return QIHT_ERR_ARG;
    if (m > kMaxRows || n > kMaxTopN) return QIHT_ERR_ARG;
    if (!x || !support || !report) return QIHT_ERR_ARG;
    qiht_params prm{2.0, 0.01, 32, 0, 0.0, QIHT_MU_FORWARD_SQ, 0};
    if (params) prm = *params;
    if (!(prm.c > 0.0 && prm.c < 1.0) || !(prm.k * (1.0 - prm.c) > 1.0) || prm.max_backtrack < 0 ||
        (prm.flags & ~(QIHT_SOLVE_EAGER | QIHT_SOLVE_TEST_TIMEOUT)) != 0)
        return QIHT_ERR_ARG;
    if (!(prm.tol >= 0.0 && std::isfinite(prm.tol)) || (prm.mu_mode != QIHT_MU_FORWARD_SQ && prm.mu_mode != QIHT_MU_CROSS))
        return QIHT_ERR_ARG;
    if (prm.mu_mode == QIHT_MU_CROSS && grid_levels(Q1->bits, Q1->levels) != grid_levels(Q2->bits, Q2->levels))
        return QIHT_ERR_ARG;
    if (!workspace || workspace_bytes < qiht_solve_workspace_size(m, n, s) || !aligned(workspace, 256))
        return QIHT_ERR_WORKSPACE;

    if (prm.flags & QIHT_SOLVE_EAGER)
        return run_eager(Q1, Q2, y, s, iters, &prm, x, support, report, trace, reinterpret_cast<char*>(workspace),
                         reinterpret_cast<cudaStream_t>(stream));

    int dev = 0;
    CK(cudaGetDevice(&dev));
    Key key;
    key.v.push_back((uint64_t)dev);
    push_codes(key.v, Q1);
    push_codes(key.v, Q2);
    push_codes(key.v, y);
    key.v.push_back((uint64_t)s);
    key.v.push_back((uint64_t)iters);
    key.v.push_back(dbits(prm.k));
    key.v.push_back(dbits(prm.c));
    key.v.push_back((uint64_t)prm.max_backtrack);
    key.v.push_back((uint64_t)prm.flags);
    key.v.push_back(dbits(prm.tol));
    key.v.push_back((uint64_t)prm.mu_mode);
    key.v.push_back(reinterpret_cast<uint64_t>(x));
    key.v.push_back(reinterpret_cast<uint64_t>(support));
    key.v.push_back(reinterpret_cast<uint64_t>(report));
    key.v.push_back(reinterpret_cast<uint64_t>(workspace));
    qiht_trace tr{};
    if (trace) tr = *trace;
    key.v.push_back(reinterpret_cast<uint64_t>(tr.support));
    key.v.push_back(reinterpret_cast<uint64_t>(tr.kth));
    key.v.push_back(reinterpret_cast<uint64_t>(tr.mu));
    key.v.push_back(reinterpret_cast<uint64_t>(tr.bt));
    key.v.push_back(reinterpret_cast<uint64_t>(tr.resid2));

    cudaGraphExec_t exec = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        auto it = g_cache.find(key);
        if (it != g_cache.end()) {
            exec = it->second.exec;
        } else {
            cudaGraph_t graph = nullptr;
            qiht_status st = QIHT_ERR_CUDA;
            // preferred first: programmatic edges with the cooperative attribute, then without
            // either; the kernels are correct under all four
            const int unroll = body_unroll();
            for (int attempt = 0; attempt < 4 && st != QIHT_OK; ++attempt) {
                const bool pdl = attempt < 2 && use_pdl();
                const bool coop = (attempt & 1) == 0;
                if (!use_pdl() && attempt < 2) continue;
                if (graph) { cudaGraphDestroy(graph); graph = nullptr; }
                st = build_graph(Q1, Q2, y, s, iters, &prm, x, support, report, trace ? &tr : nullptr,
                                 reinterpret_cast<char*>(workspace), coop, pdl, pdl ? unroll : 1, &graph);
                if (st == QIHT_OK) {
                    const cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
                    if (e != cudaSuccess) {
                        note_cuda_error("cudaGraphInstantiate", e);
                        st = QIHT_ERR_CUDA;
                    }
                }
                if (st != QIHT_OK) cudaGetLastError();       // clear the error before the retry
            }
            if (st != QIHT_OK) {
                if (graph) cudaGraphDestroy(graph);
                return st;
            }
            g_cache[key] = Cached{graph, exec};
        }
    }
    CK(cudaGraphLaunch(exec, reinterpret_cast<cudaStream_t>(stream)));
    return QIHT_OK;
}

// ---- fresh realizations per iteration (Algorithm 2 as written) ----

static int phi_stream(int k) { return k <= 2 ? k - 1 : 0x1000 + k; }
static int y_stream(int t) { return t == 1 ? 2 : 0x2000 + t; }

struct FreshLayout {
    size_t solve, q1, q2, qy, scales, z, total;
};

static FreshLayout fresh_layout(int m, int n, int s, int bits_phi, int bits_y)
{
    FreshLayout L{};
    size_t o = 0;
    L.solve = o; o += align256(plan_solve(m, n, s).total);
    const size_t wq = (size_t)n * qiht_ld_words(m, bits_phi) * 4;
    L.q1 = o; o += align256(wq);
    L.q2 = o; o += align256(wq);
    L.qy = o; o += align256((size_t)qiht_ld_words(m, bits_y) * 4);
    L.scales = o; o += 256;
    L.z = o; o += align256((size_t)qiht_ld_words(m, 2) * 16 * 4);
    L.total = o;
    return L;
}

size_t qiht_solve_fresh_workspace_size(int32_t m, int32_t n, int32_t s, int32_t bits_phi, int32_t bits_y)
{
    if (m < 1 || n < 1 || s < 1 || s > m || s > n || m > kMaxRows || n > kMaxTopN || !bits_ok(bits_phi) ||
        !bits_ok(bits_y))
        return 0;
    return fresh_layout(m, n, s, bits_phi, bits_y).total;
}

// Where the fresh solve's realizations of Q(Phi) come from: a stored FP32 matrix (quantized
// every iteration), or the on-the-fly operator (its codes generated every iteration).
struct FreshSource {
    const float* phi;
    int64_t ld_phi;
    const qiht_fly_op* op;
};

static qiht_status fresh_solve(const FreshSource& src, const float* y, int32_t m, int32_t n, int32_t bits_phi,
                               int32_t bits_y, uint64_t seed, int32_t quant_flags, int32_t s, int32_t iters,
                               const qiht_params* params, float* x, int32_t* support, qiht_report* report,
                               const qiht_trace* trace, void* workspace, size_t workspace_bytes, qiht_stream_t stream)
{
    if (!bits_ok(bits_phi) || !bits_ok(bits_y)) return QIHT_ERR_BITS;
    if (!y || !x || !support || !report || m < 1 || n < 1) return QIHT_ERR_ARG;
    if (src.op ? !fly_op_ok(src.op) : (!src.phi || src.ld_phi < n)) return QIHT_ERR_ARG;
    if (s < 1 || s > m || s > n || iters < 0 || m > kMaxRows || n > kMaxTopN) return QIHT_ERR_ARG;
    if (quant_flags & ~QIHT_ODD_LEVELS) return QIHT_ERR_ARG;
    qiht_params prm{2.0, 0.01, 32, 0, 0.0, QIHT_MU_FORWARD_SQ, 0};
    if (params) prm = *params;
    if (!(prm.c > 0.0 && prm.c < 1.0) || !(prm.k * (1.0 - prm.c) > 1.0) || prm.max_backtrack < 0 || prm.flags != 0)
        return QIHT_ERR_ARG;
    if (!(prm.tol >= 0.0 && std::isfinite(prm.tol)) || (prm.mu_mode != QIHT_MU_FORWARD_SQ && prm.mu_mode != QIHT_MU_CROSS))
        return QIHT_ERR_ARG;
    const FreshLayout L = fresh_layout(m, n, s, bits_phi, bits_y);
    if (!workspace || workspace_bytes < L.total || !aligned(workspace, 256)) return QIHT_ERR_WORKSPACE;
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    char* w = reinterpret_cast<char*>(workspace);
    uint32_t* w1 = reinterpret_cast<uint32_t*>(w + L.q1);
    uint32_t* w2 = reinterpret_cast<uint32_t*>(w + L.q2);
    uint32_t* wy = reinterpret_cast<uint32_t*>(w + L.qy);
    float* sc = reinterpret_cast<float*>(w + L.scales);          // [0] max |Phi|, [1] max |y|
    float* z = reinterpret_cast<float*>(w + L.z);
    const bool odd = (quant_flags & QIHT_ODD_LEVELS) != 0;
    const int lev_phi = odd ? (1 << (bits_phi - 1)) + 1 : (1 << bits_phi);
    const int lev_y = odd ? (1 << (bits_y - 1)) + 1 : (1 << bits_y);
    const int ldp = qiht_ld_words(m, bits_phi), ldy = qiht_ld_words(m, bits_y);
    const qiht_codes q1{w1, sc, m, n, bits_phi, ldp, lev_phi, 0};
    const qiht_codes q2{w2, sc, m, n, bits_phi, ldp, lev_phi, 0};
    const qiht_codes qy{wy, sc + 1, m, 1, bits_y, ldy, lev_y, 0};
    auto quantize_iteration = [&](int t) -> cudaError_t {
        cudaError_t e = src.op ? launch_fly_quantize(src.op, bits_phi, lev_phi, seed, (uint32_t)phi_stream(2 * t - 1),
                                                     (uint32_t)phi_stream(2 * t), w1, w2, ldp, sc, cs)
                               : launch_quantize(src.phi, m, n, src.ld_phi, bits_phi, seed,
                                                 (uint32_t)phi_stream(2 * t - 1), w1, ldp, sc, cs,
                                                 (uint32_t)phi_stream(2 * t), w2, lev_phi);
        if (e != cudaSuccess) return e;
        return launch_quantize(y, m, 1, 1, bits_y, seed, (uint32_t)y_stream(t), wy, ldy, sc + 1, cs, 0, nullptr,
                               lev_y);
    };
    if (!src.op) CK(launch_absmax(src.phi, m, n, src.ld_phi, sc, cs));   // the operator's kernels write max |table|
    CK(launch_absmax(y, m, 1, 1, sc + 1, cs));
    CK(quantize_iteration(1));

    char* ws = w + L.solve;
    SolveKernels K;
    make_kernels(K, &q1, &q2, &qy, s, iters, &prm, x, support, report, trace, ws, 0, 0, true);
    const Plan pl = plan_solve(m, n, s);
    GatherArgs ga{};
    ga.Q = view(&q2);
    ga.cols = support;                   // the committed support and the values on it
    ga.coef = reinterpret_cast<const float*>(ws + pl.off_val);
    ga.count = s;
    ga.z = z;
    ga.partial = reinterpret_cast<float*>(ws + pl.off_partial);
    ga.rb_partial = reinterpret_cast<double*>(ws + pl.off_rbp);
    ga.counters = K.st->counters[1];
    ga.mode = kGatherPlain;
    CK(cudaMemsetAsync(ga.counters, 0, sizeof(unsigned) * 1024, cs));
    float* yhat = reinterpret_cast<float*>(ws + pl.off_yhat);
    float* r = reinterpret_cast<float*>(ws + pl.off_r);

    State h{};
    auto read_state = [&]() -> bool {
        if (cudaMemcpyAsync(&h, K.st, sizeof(State), cudaMemcpyDeviceToHost, cs) != cudaSuccess) return false;
        return cudaStreamSynchronize(cs) == cudaSuccess;
    };
    CK(launch_node(K.p_init, cs));
    CK(launch_node(K.p_g0, cs));
    CK(launch_node(K.p_t0, cs));
    if (!read_state()) return QIHT_ERR_CUDA;
    for (int t = 1; t <= iters && !h.stop; ++t) {
        if (t >= 2) {
            // this iteration's realizations, its residual y-hat_t - Phi-hat_{2t} x, the gradient
            CK(quantize_iteration(t));
            CK(launch_gather(ga, cs));
            CK(cudaMemsetAsync(&K.st->rmax_bits, 0, sizeof(unsigned), cs));
            CK(launch_fresh_resid(view(&qy), z, yhat, r, m, &K.st->rmax_bits, cs));
            CK(launch_node(K.p_gb, cs));
        }
        if (K.cross) CK(launch_node(K.p_z1, cs));
        CK(launch_node(K.p_mu, cs));
        CK(launch_node(K.p_tf, cs));
        CK(launch_node(K.p_tt, cs));
        CK(launch_node(K.p_om, cs));
        if (!read_state()) return QIHT_ERR_CUDA;
        for (int b = 0; b <= prm.max_backtrack && h.again && !h.stop; ++b) {
            CK(launch_node(K.p_tf, cs));
            CK(launch_node(K.p_tt, cs));
            CK(launch_node(K.p_om, cs));
            if (!read_state()) return QIHT_ERR_CUDA;
        }
        CK(launch_node(K.p_re, cs));
        if (!read_state()) return QIHT_ERR_CUDA;
    }
    return QIHT_OK;
}

qiht_status qiht_niht_solve_fresh(const float* phi, int64_t ld_phi, const float* y, int32_t m, int32_t n,
                                  int32_t bits_phi, int32_t bits_y, uint64_t seed, int32_t quant_flags, int32_t s,
                                  int32_t iters, const qiht_params* params, float* x, int32_t* support,
                                  qiht_report* report, const qiht_trace* trace, void* workspace,
                                  size_t workspace_bytes, qiht_stream_t stream)
{
    if (!phi) return bits_ok(bits_phi) && bits_ok(bits_y) ? QIHT_ERR_ARG : QIHT_ERR_BITS;
    return fresh_solve(FreshSource{phi, ld_phi, nullptr}, y, m, n, bits_phi, bits_y, seed, quant_flags, s, iters,
                       params, x, support, report, trace, workspace, workspace_bytes, stream);
}

qiht_status qiht_niht_solve_fresh_fly(const qiht_fly_op* op, const float* y, int32_t bits_phi, int32_t bits_y,
                                      uint64_t seed, int32_t quant_flags, int32_t s, int32_t iters,
                                      const qiht_params* params, float* x, int32_t* support, qiht_report* report,
                                      const qiht_trace* trace, void* workspace, size_t workspace_bytes,
                                      qiht_stream_t stream)
{
    if (!fly_op_ok(op)) return bits_ok(bits_phi) && bits_ok(bits_y) ? QIHT_ERR_ARG : QIHT_ERR_BITS;
    return fresh_solve(FreshSource{nullptr, 0, op}, y, 2 * op->baselines, op->grid * op->grid, bits_phi, bits_y,
                       seed, quant_flags, s, iters, params, x, support, report, trace, workspace, workspace_bytes,
                       stream);
}

size_t qiht_solve_batched_workspace_size(int32_t nprob)
{
    if (nprob < 1) return 0;
    return align256((size_t)nprob * sizeof(qiht_problem)) + align256((size_t)nprob * 4) + 256;
}

// ---- tile shape of the batched gradient product: lanes per column, picked per size bucket ----

// bucket of a problem: ceil(log2(16-byte pieces per column of Q1))
static int shape_bucket(const qiht_problem& P)
{
    const int pieces = P.Q1.ld_words / 4;
    int b = 0;
    while ((1 << b) < pieces) ++b;
    return b;
}

// without tuning: the smallest group that covers a column's pieces (4 to 32 lanes)
static int shape_default(int bucket)
{
    const int p2 = 1 << bucket;
    return p2 < 4 ? 4 : p2 > 32 ? 32 : p2;
}

static std::mutex g_shape_mu;
static std::map<std::pair<int, int>, int> g_shape;           // (bits, bucket) -> lanes per column

static int shape_forced()
{
    const char* e = getenv("QIHT_BATCH_SHAPE");             // measurement and tests: one shape for all
    if (!e) return 0;
    const int v = atoi(e);
    return (v == 4 || v == 8 || v == 16 || v == 32) ? v : 0;
}

static bool shape_tuning()
{
    const char* e = getenv("QIHT_BATCH_TUNE");
    return !(e && e[0] == '0');
}

// side streams of this device for the concurrent shape groups (created once, never destroyed)
static cudaStream_t side_stream(int k)
{
    static std::mutex mu;
    static std::map<std::pair<int, int>, cudaStream_t> streams;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    auto it = streams.find({dev, k});
    if (it != streams.end()) return it->second;
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
    streams[{dev, k}] = st;
    return st;
}

qiht_status qiht_niht_solve_batched(const qiht_problem* problems, int32_t nprob, int32_t iters,
                                    const qiht_params* params, void* workspace, size_t workspace_bytes,
                                    qiht_stream_t stream)
{
    if (!problems || nprob < 1 || iters < 0) return QIHT_ERR_ARG;
    qiht_params prm{2.0, 0.01, 32, 0, 0.0, QIHT_MU_FORWARD_SQ, 0};
    if (params) prm = *params;
    if (!(prm.c > 0.0 && prm.c < 1.0) || !(prm.k * (1.0 - prm.c) > 1.0) || prm.max_backtrack < 0 || prm.flags != 0)
        return QIHT_ERR_ARG;
    if (prm.tol != 0.0 || prm.mu_mode != QIHT_MU_FORWARD_SQ) return QIHT_ERR_ARG;   // the defaults only
    const int bits = problems[0].Q1.bits;
    for (int i = 0; i < nprob; ++i) {
        const qiht_problem& P = problems[i];
        TRY(check_codes(&P.Q1));
        TRY(check_codes(&P.Q2));
        TRY(check_codes(&P.y));
        const int m = P.Q1.rows, n = P.Q1.cols;
        if (P.Q1.bits != bits || P.Q2.bits != bits) return QIHT_ERR_ARG;
        if (P.Q2.rows != m || P.Q2.cols != n || P.y.rows != m || P.y.cols != 1) return QIHT_ERR_ARG;
        if (m > QIHT_BATCH_MAX_ROWS || n > QIHT_BATCH_MAX_COLS) return QIHT_ERR_ARG;
        if (P.s < 1 || P.s > m || P.s > n || P.s > QIHT_BATCH_MAX_S) return QIHT_ERR_ARG;
        if (!P.x || !P.support || !P.report) return QIHT_ERR_ARG;
    }
    if (!workspace || workspace_bytes < qiht_solve_batched_workspace_size(nprob) || !aligned(workspace, 256))
        return QIHT_ERR_WORKSPACE;
    // largest problems first (m n, then index): the persistent CTAs take them in this order
    std::vector<int> order((size_t)nprob);
    for (int i = 0; i < nprob; ++i) order[(size_t)i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return (long long)problems[a].Q1.rows * problems[a].Q1.cols > (long long)problems[b].Q1.rows * problems[b].Q1.cols;
    });
    char* ws = reinterpret_cast<char*>(workspace);
    qiht_problem* d_probs = reinterpret_cast<qiht_problem*>(ws);
    int* d_order = reinterpret_cast<int*>(ws + align256((size_t)nprob * sizeof(qiht_problem)));
    unsigned* d_next = reinterpret_cast<unsigned*>(ws + align256((size_t)nprob * sizeof(qiht_problem)) +
                                                   align256((size_t)nprob * 4));      // one counter per group
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    // host -> device from pageable memory: the copies are staged before the calls return
    CK(cudaMemcpyAsync(d_probs, problems, (size_t)nprob * sizeof(qiht_problem), cudaMemcpyHostToDevice, cs));

    // tile shapes: forced, tuned (first batch with a new (bits, size bucket): every shape is
    // timed on up to 64 of the bucket's problems for a few iterations and the fastest kept; all
    // shapes give bit-identical results, the problems' outputs are overwritten below), or the
    // default covering a column's pieces
    const int forced = shape_forced();
    std::map<int, std::vector<int>> by_bucket;
    for (int i = 0; i < nprob; ++i) by_bucket[shape_bucket(problems[order[(size_t)i]])].push_back(order[(size_t)i]);
    std::map<int, int> pick;
    for (auto& kv : by_bucket) {
        const int b = kv.first;
        int lpc = forced ? forced : shape_default(b);
        if (!forced && shape_tuning() && iters > 0) {
            int cached = 0;
            {
                std::lock_guard<std::mutex> lock(g_shape_mu);
                auto it = g_shape.find({bits, b});
                if (it != g_shape.end()) cached = it->second;
            }
            if (cached) {
                lpc = cached;
            } else {
                const int cnt = (int)std::min<size_t>(kv.second.size(), 64);
                const int titers = std::min(iters, 8);
                cudaEvent_t e0, e1;
                CK(cudaEventCreate(&e0));
                CK(cudaEventCreate(&e1));
                float best = 0.0f;
                CK(cudaMemcpyAsync(d_order, kv.second.data(), (size_t)cnt * 4, cudaMemcpyHostToDevice, cs));
                for (int cand : {4, 8, 16, 32}) {
                    CK(cudaEventRecord(e0, cs));
                    CK(launch_batched(d_probs, d_order, cnt, bits, cand, titers, prm.k, prm.c, prm.max_backtrack,
                                      d_next, cs));
                    CK(cudaEventRecord(e1, cs));
                    CK(cudaEventSynchronize(e1));
                    float ms = 0.0f;
                    CK(cudaEventElapsedTime(&ms, e0, e1));
                    if (best == 0.0f || ms < best) { best = ms; lpc = cand; }
                }
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                std::lock_guard<std::mutex> lock(g_shape_mu);
                g_shape[{bits, b}] = lpc;
            }
        }
        pick[b] = lpc;
    }
    // one persistent launch per shape (each kernel compiled for its shape), largest problems first
    // within a group; the groups run concurrently on streams forked from `stream`
    std::map<int, std::vector<int>> groups;
    for (int i = 0; i < nprob; ++i) {
        const int p = order[(size_t)i];
        groups[pick[shape_bucket(problems[p])]].push_back(p);
    }
    std::vector<int> flat;
    std::vector<std::pair<int, std::pair<int, int>>> seg;   // (shape, (offset, count))
    for (auto& g : groups) {
        seg.push_back({g.first, {(int)flat.size(), (int)g.second.size()}});
        flat.insert(flat.end(), g.second.begin(), g.second.end());
    }
    std::sort(seg.begin(), seg.end(), [&](const auto& a, const auto& b) {
        const qiht_problem& pa = problems[flat[(size_t)a.second.first]];
        const qiht_problem& pb = problems[flat[(size_t)b.second.first]];
        return (long long)pa.Q1.rows * pa.Q1.cols > (long long)pb.Q1.rows * pb.Q1.cols;
    });
    CK(cudaMemcpyAsync(d_order, flat.data(), (size_t)nprob * 4, cudaMemcpyHostToDevice, cs));
    if (seg.size() == 1) {
        CK(launch_batched(d_probs, d_order, nprob, bits, seg[0].first, iters, prm.k, prm.c, prm.max_backtrack,
                          d_next, cs));
        return QIHT_OK;
    }
    cudaEvent_t fork;
    CK(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    CK(cudaEventRecord(fork, cs));
    std::vector<cudaEvent_t> joins;
    for (size_t g = 0; g < seg.size(); ++g) {
        cudaStream_t gs = g == 0 ? cs : side_stream((int)g);    // cs may be the legacy stream (NULL)
        if (g > 0 && !gs) {
            note_cuda_error("cudaStreamCreateWithFlags", cudaErrorUnknown);
            return QIHT_ERR_CUDA;
        }
        if (g > 0) CK(cudaStreamWaitEvent(gs, fork, 0));
        CK(launch_batched(d_probs, d_order + seg[g].second.first, seg[g].second.second, bits, seg[g].first, iters,
                          prm.k, prm.c, prm.max_backtrack, d_next + g, gs));
        if (g > 0) {
            cudaEvent_t j;
            CK(cudaEventCreateWithFlags(&j, cudaEventDisableTiming));
            CK(cudaEventRecord(j, gs));
            CK(cudaStreamWaitEvent(cs, j, 0));
            joins.push_back(j);
        }
    }
    cudaEventDestroy(fork);
    for (cudaEvent_t j : joins) cudaEventDestroy(j);
    return QIHT_OK;
}

void qiht_clear_graph_cache(void)
{
    std::lock_guard<std::mutex> lock(g_mu);
    for (auto& kv : g_cache) {
        cudaGraphExecDestroy(kv.second.exec);
        cudaGraphDestroy(kv.second.graph);
    }
    g_cache.clear();
}

}  // extern "C"
