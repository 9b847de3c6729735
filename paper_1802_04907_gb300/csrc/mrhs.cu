// Entry points for many right-hand sides sharing one quantized matrix: the tensor-core
// gradient product (qiht_gemv_t_multi).
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

size_t qiht_gemv_t_multi_workspace_size(int32_t rows, int32_t nrhs)
{
    if (rows < 1 || nrhs < 1) return 0;
    const size_t np = (size_t)mrhs_pad_rhs(nrhs), mk = (size_t)mrhs_pad_rows(rows);
    return align256(2 * np * mk * 2) + align256(np * 4) + 256;
}

qiht_status qiht_gemv_t_multi(const qiht_codes* Q, const float* R, int64_t ldr, int32_t nrhs, float* G,
                              int64_t ldg, int32_t* status, void* workspace, size_t workspace_bytes,
                              qiht_stream_t stream)
{
    qiht_status e = check_codes(Q);
    if (e != QIHT_OK) return e;
    if (!R || !G || nrhs < 1 || ldr < Q->rows || ldg < Q->cols) return QIHT_ERR_ARG;
    if (Q->rows > kMaxRows) return QIHT_ERR_ARG;
    if (!workspace || workspace_bytes < qiht_gemv_t_multi_workspace_size(Q->rows, nrhs) || !aligned256(workspace))
        return QIHT_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int np = mrhs_pad_rhs(nrhs), mk = mrhs_pad_rows(Q->rows);
    char* w = reinterpret_cast<char*>(workspace);
    void* r16 = w;
    float* sc = reinterpret_cast<float*>(w + align256((size_t)2 * np * mk * 2));
    int* st = reinterpret_cast<int*>(w + align256((size_t)2 * np * mk * 2) + align256((size_t)np * 4));
    if (!status) {
        CK(cudaMemsetAsync(st, 0, sizeof(int), s));
        status = st;
    }
    const Codes c = view(Q);
    CK(launch_mrhs_split(R, ldr, Q->rows, nrhs, r16, sc, Q->scale, c.lm1, s));
    alignas(64) unsigned char map[kMrhsMapBytes];
    CK(mrhs_make_map(map, r16, mk, 2 * np));
    CK(launch_mrhs_gemm(c, map, sc, G, ldg, nrhs, status, s));
    return QIHT_OK;
}

}  // extern "C"
