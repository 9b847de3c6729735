// Entry points for many right-hand sides sharing one quantized matrix: the tensor-core
// gradient product (qiht_gemv_t_multi) and the solver built on it (qiht_niht_solve_multi).
#include <cstring>

#include "internal.cuh"

using namespace qiht;

namespace {

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
bool aligned256(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 255) == 0; }

}  // namespace

#define CK(x)                                 \
    do {                                      \
        cudaError_t ck_e_ = (x);              \
        if (ck_e_ != cudaSuccess) {           \
            note_cuda_error(#x, ck_e_);       \
            return QIHT_ERR_CUDA;             \
        }                                     \
    } while (0)

extern "C" {

// bytes of the residual operand: two f16 parts (mk halves per row), or three e4m3 terms
// (mk8 bytes per row) of the FP8 variant, which reuses the same memory
static size_t operand_bytes(int rows, int nrhs)
{
    const size_t np = (size_t)mrhs_pad_rhs(nrhs), mk = (size_t)mrhs_pad_rows(rows), mk8 = (size_t)mrhs_pad_rows8(rows);
    const size_t f16 = 2 * np * mk * 2, f8 = (size_t)kMrhsTerms8 * np * mk8;
    return f16 > f8 ? f16 : f8;
}

size_t qiht_gemv_t_multi_workspace_size(int32_t rows, int32_t nrhs)
{
    if (rows < 1 || nrhs < 1) return 0;
    const size_t np = (size_t)mrhs_pad_rhs(nrhs);
    return align256(operand_bytes(rows, nrhs)) + align256(np * 4) + 256;
}

static qiht_status gemv_t_multi_impl(const qiht_codes* Q, const float* R, int64_t ldr, int32_t nrhs, float* G,
                                     int64_t ldg, int32_t* status, void* workspace, size_t workspace_bytes,
                                     qiht_stream_t stream, bool fp8)
{
    qiht_status e = check_codes(Q);
    if (e != QIHT_OK) return e;
    if (fp8 && Q->bits == 8) return QIHT_ERR_BITS;           // 8-bit centred codes are not exact in e4m3
    if (!R || !G || nrhs < 1 || ldr < Q->rows || ldg < Q->cols) return QIHT_ERR_ARG;
    if (Q->rows > kMaxRows) return QIHT_ERR_ARG;
    if (!workspace || workspace_bytes < qiht_gemv_t_multi_workspace_size(Q->rows, nrhs) || !aligned256(workspace))
        return QIHT_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int np = mrhs_pad_rhs(nrhs), mk = mrhs_pad_rows(Q->rows), mk8 = mrhs_pad_rows8(Q->rows);
    char* w = reinterpret_cast<char*>(workspace);
    void* rop = w;
    const size_t ob = align256(operand_bytes(Q->rows, nrhs));
    float* sc = reinterpret_cast<float*>(w + ob);
    int* st = reinterpret_cast<int*>(w + ob + align256((size_t)np * 4));
    if (!status) {
        CK(cudaMemsetAsync(st, 0, sizeof(int), s));
        status = st;
    }
    const Codes c = view(Q);
    alignas(64) unsigned char map[kMrhsMapBytes];
    if (fp8) {
        CK(launch_mrhs_split8(R, ldr, Q->rows, nrhs, rop, sc, Q->scale, c.lm1, s));
        CK(mrhs_make_map8(map, rop, mk8, kMrhsTerms8 * np));
    } else {
        CK(launch_mrhs_split(R, ldr, Q->rows, nrhs, rop, sc, Q->scale, c.lm1, s));
        CK(mrhs_make_map(map, rop, mk, 2 * np));
    }
    CK(launch_mrhs_gemm(c, map, sc, G, ldg, nrhs, status, s, fp8));
    return QIHT_OK;
}

qiht_status qiht_gemv_t_multi(const qiht_codes* Q, const float* R, int64_t ldr, int32_t nrhs, float* G,
                              int64_t ldg, int32_t* status, void* workspace, size_t workspace_bytes,
                              qiht_stream_t stream)
{
    return gemv_t_multi_impl(Q, R, ldr, nrhs, G, ldg, status, workspace, workspace_bytes, stream, false);
}

qiht_status qiht_gemv_t_multi_fp8(const qiht_codes* Q, const float* R, int64_t ldr, int32_t nrhs, float* G,
                                  int64_t ldg, int32_t* status, void* workspace, size_t workspace_bytes,
                                  qiht_stream_t stream)
{
    return gemv_t_multi_impl(Q, R, ldr, nrhs, G, ldg, status, workspace, workspace_bytes, stream, true);
}

// the residual is formed directly every kMultiRefresh iterations (and on the last), else
// updated from the step's product
constexpr int kMultiRefresh = 32;

struct MultiLayout {
    size_t ydesc, yhat, resid, zmu, r16, sc, g, xs, st, status, total;
};

static MultiLayout multi_layout(int m, int n, int s, int nrhs)
{
    const size_t np = (size_t)mrhs_pad_rhs(nrhs);
    MultiLayout L;
    size_t o = 0;
    L.ydesc = o; o += align256((size_t)nrhs * sizeof(qiht_codes));
    L.yhat = o; o += align256((size_t)nrhs * m * 4);
    L.resid = o; o += align256((size_t)nrhs * m * 4);
    L.zmu = o; o += align256((size_t)nrhs * m * 4);
    L.r16 = o; o += align256(operand_bytes(m, nrhs));
    L.sc = o; o += align256(np * 4);
    L.g = o; o += align256((size_t)nrhs * n * 4);
    L.xs = o; o += align256((size_t)nrhs * s * 4);
    L.st = o; o += align256((size_t)nrhs * sizeof(MrhsState));
    L.status = o; o += 256;
    L.total = o;
    return L;
}

static bool multi_sizes_ok(int m, int n, int s, int nrhs)
{
    return m >= 1 && n >= 1 && nrhs >= 1 && s >= 1 && s <= m && s <= n && m <= QIHT_MULTI_MAX_ROWS &&
           n <= QIHT_MULTI_MAX_COLS && s <= QIHT_MULTI_MAX_S;
}

size_t qiht_solve_multi_workspace_size(int32_t m, int32_t n, int32_t s, int32_t nrhs)
{
    if (!multi_sizes_ok(m, n, s, nrhs)) return 0;
    return multi_layout(m, n, s, nrhs).total;
}

qiht_status qiht_niht_solve_multi(const qiht_codes* Q1, const qiht_codes* Q2, const qiht_codes* y, int32_t nrhs,
                                  int32_t s, int32_t iters, const qiht_params* params, float* X,
                                  int32_t* support, qiht_report* reports, void* workspace, size_t workspace_bytes,
                                  qiht_stream_t stream)
{
    qiht_status e = check_codes(Q1);
    if (e != QIHT_OK) return e;
    if ((e = check_codes(Q2)) != QIHT_OK) return e;
    const int m = Q1->rows, n = Q1->cols;
    if (Q2->rows != m || Q2->cols != n || Q2->bits != Q1->bits) return QIHT_ERR_ARG;
    if (!y || !X || !support || !reports || iters < 0) return QIHT_ERR_ARG;
    if (!multi_sizes_ok(m, n, s, nrhs)) return QIHT_ERR_ARG;
    for (int k = 0; k < nrhs; ++k) {
        if ((e = check_codes(&y[k])) != QIHT_OK) return e;
        if (y[k].rows != m || y[k].cols != 1) return QIHT_ERR_ARG;
    }
    qiht_params prm{2.0, 0.01, 32, 0, 0.0, QIHT_MU_FORWARD_SQ, 0};
    if (params) prm = *params;
    if (!(prm.c > 0.0 && prm.c < 1.0) || !(prm.k * (1.0 - prm.c) > 1.0) || prm.max_backtrack < 0 ||
        (prm.flags & ~QIHT_SOLVE_FP8) != 0)
        return QIHT_ERR_ARG;
    if (prm.tol != 0.0 || prm.mu_mode != QIHT_MU_FORWARD_SQ) return QIHT_ERR_ARG;   // the defaults only
    const bool fp8 = (prm.flags & QIHT_SOLVE_FP8) != 0;
    if (fp8 && Q1->bits == 8) return QIHT_ERR_BITS;
    const MultiLayout L = multi_layout(m, n, s, nrhs);
    if (!workspace || workspace_bytes < L.total || !aligned256(workspace)) return QIHT_ERR_WORKSPACE;
    const int mk = mrhs_pad_rows(m), np = mrhs_pad_rhs(nrhs);
    if (mrhs_step_smem(n, mk, s) > (size_t)227 * 1024 - 1024) return QIHT_ERR_ARG;
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    char* w = reinterpret_cast<char*>(workspace);
    qiht_codes* d_y = reinterpret_cast<qiht_codes*>(w + L.ydesc);
    int* gstatus = reinterpret_cast<int*>(w + L.status);
    CK(cudaMemcpyAsync(d_y, y, (size_t)nrhs * sizeof(qiht_codes), cudaMemcpyHostToDevice, cs));
    CK(cudaMemsetAsync(gstatus, 0, sizeof(int), cs));

    MrhsStepArgs a{};
    a.Q2 = view(Q2);
    a.scale1 = Q1->scale;
    a.lm1_1 = view(Q1).lm1;
    a.ydesc = d_y;
    a.yhat = reinterpret_cast<float*>(w + L.yhat);
    a.resid = reinterpret_cast<float*>(w + L.resid);
    a.zmu = reinterpret_cast<float*>(w + L.zmu);
    a.G = reinterpret_cast<float*>(w + L.g);
    a.sup = support;
    a.xs = reinterpret_cast<float*>(w + L.xs);
    a.R16 = reinterpret_cast<__half*>(w + L.r16);
    a.sc = reinterpret_cast<float*>(w + L.sc);
    a.mk = mk;
    a.rhi = np;
    a.st = reinterpret_cast<MrhsState*>(w + L.st);
    a.n = n;
    a.m = m;
    a.s = s;
    a.nrhs = nrhs;
    a.kk = prm.k;
    a.cc = prm.c;
    a.max_bt = prm.max_backtrack;
    a.fp8 = fp8 ? 1 : 0;
    a.mk8 = mrhs_pad_rows8(m);
    alignas(64) unsigned char map[kMrhsMapBytes];
    if (fp8) CK(mrhs_make_map8(map, a.R16, a.mk8, kMrhsTerms8 * np));
    else CK(mrhs_make_map(map, a.R16, mk, 2 * np));
    const Codes c1 = view(Q1);
    float* G = reinterpret_cast<float*>(w + L.g);

    CK(launch_mrhs_init(a, cs));
    CK(launch_mrhs_gemm(c1, map, a.sc, G, n, nrhs, gstatus, cs, fp8));
    a.mode = 0;
    a.last = iters == 0;
    CK(launch_mrhs_step(a, Q1->bits, cs));
    for (int it = 1; it <= iters; ++it) {
        a.mode = 1;
        a.last = it == iters;
        a.refresh = a.last || it % kMultiRefresh == 0;
        CK(launch_mrhs_step(a, Q1->bits, cs));
        if (!a.last) CK(launch_mrhs_gemm(c1, map, a.sc, G, n, nrhs, gstatus, cs, fp8));
    }
    CK(launch_mrhs_final(a, X, reports, gstatus, cs));
    return QIHT_OK;
}

}  // extern "C"
