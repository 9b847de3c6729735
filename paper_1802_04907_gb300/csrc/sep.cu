// Separable operator with quantized transform factors (Section IV-B, MRI): Phi = S (A (x) A),
// stacked real, with the N x N complex 1D transform A (the DFT times the Haar synthesis)
// quantized as one stacked real matrix [Re A; Im A]. The operator is applied as dense
// transforms of the N x N image, never as an m x n matrix:
//   forward  x -> [Re B; Im B] at the mask,  B = A X A^T  (X = x as N x N, row-major)
//            T1 = [Ar; Ai] X                      (2N x N)
//            T2 = T1 [Ar; Ai]^T                   (2N x 2N) = [[P Ar^T, P Ai^T], [Q Ar^T, Q Ai^T]]
//            Re B = P Ar^T - Q Ai^T, Im B = P Ai^T + Q Ar^T  (read at the mask only)
//   adjoint  r -> Re(A^T conj(Z) A), Z = r_re + i r_im scattered to the mask (zero elsewhere)
//            [P; Q] = [[Ar^T, Ai^T], [Ai^T, -Ar^T]] [Zr; Zi]     (2N x N)
//            G = P Ar - Q Ai                      (N x N)
// The products are FP32 GEMMs of a plain tiled kernel (each output one thread's sum in a fixed
// order, so results are deterministic). The solve (Algorithm 2) runs on the host around these
// kernels and the one-CTA threshold, reading the scalars it decides on after each product.
#include "internal.cuh"
#include "quant_rng.cuh"

#include <vector>

namespace qiht {
namespace {

// ---- C = alpha op(A) op(B) + beta C, row-major FP32 ----
// Tiles of T x T outputs (T = 64, or 32 when a 64-tile grid would leave most SMs idle), K in
// steps of 16, 256 threads with (T/16)^2 outputs each. SA: A is two stacked blocks read side by
// side, A(i, k) = A[i][k] for k < K/2 and A[K/2 + i][k - K/2] after (the adjoint's [P | Q]).
constexpr int kGK = 16;

template <int T, bool TA, bool TB, bool SA>
__global__ void __launch_bounds__(256) k_sgemm(int M, int N, int K, const float* __restrict__ A, int lda,
                                               const float* __restrict__ B, int ldb, float* __restrict__ C, int ldc,
                                               float alpha, float beta)
{
    constexpr int R = T / 16;                          // outputs per thread along each dimension
    __shared__ __align__(16) float As[kGK][T + 4];
    __shared__ __align__(16) float Bs[kGK][T + 4];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * T, n0 = blockIdx.x * T;
    const int kh = K >> 1;
    float acc[R][R] = {};
    for (int k0 = 0; k0 < K; k0 += kGK) {
#pragma unroll
        for (int l = 0; l < T * kGK / 256; ++l) {
            const int e = tid + 256 * l;
            {
                const int kk = e & 15, ii = e >> 4;        // A tile: T rows x 16 k
                const int i = m0 + ii, k = k0 + kk;
                float v = 0.0f;
                if (i < M && k < K) {
                    if (SA) v = k < kh ? A[(size_t)i * lda + k] : A[(size_t)(kh + i) * lda + (k - kh)];
                    else v = TA ? A[(size_t)k * lda + i] : A[(size_t)i * lda + k];
                }
                As[kk][ii] = v;
            }
            {
                const int jj = e % T, kk = e / T;          // B tile: 16 k x T columns
                const int j = n0 + jj, k = k0 + kk;
                Bs[kk][jj] = (j < N && k < K) ? (TB ? B[(size_t)j * ldb + k] : B[(size_t)k * ldb + j]) : 0.0f;
            }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kGK; ++kk) {
            // a thread's R consecutive rows and R consecutive columns: vector loads, and the
            // lanes of a warp read one contiguous run of B (no bank conflicts) and broadcast A
            float a[R], b[R];
            if (R == 4) {
                const float4 va = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
                const float4 vb = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
                a[0] = va.x; a[R > 1 ? 1 : 0] = va.y; a[R > 2 ? 2 : 0] = va.z; a[R > 3 ? 3 : 0] = va.w;
                b[0] = vb.x; b[R > 1 ? 1 : 0] = vb.y; b[R > 2 ? 2 : 0] = vb.z; b[R > 3 ? 3 : 0] = vb.w;
            } else {
                const float2 va = *reinterpret_cast<const float2*>(&As[kk][ty * 2]);
                const float2 vb = *reinterpret_cast<const float2*>(&Bs[kk][tx * 2]);
                a[0] = va.x; a[R > 1 ? 1 : 0] = va.y;
                b[0] = vb.x; b[R > 1 ? 1 : 0] = vb.y;
            }
#pragma unroll
            for (int u = 0; u < R; ++u)
#pragma unroll
                for (int v = 0; v < R; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < R; ++u)
#pragma unroll
        for (int v = 0; v < R; ++v) {
            const int i = m0 + ty * R + u, j = n0 + tx * R + v;
            if (i < M && j < N) {
                float* c = C + (size_t)i * ldc + j;
                *c = beta != 0.0f ? fmaf(alpha, acc[u][v], beta * *c) : alpha * acc[u][v];
            }
        }
}

template <bool TA, bool TB, bool SA = false>
cudaError_t sgemm(int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C, int ldc,
                  float alpha, float beta, cudaStream_t s)
{
    const long long tiles64 = (long long)((N + 63) / 64) * ((M + 63) / 64);
    if (tiles64 >= num_sms()) {
        const dim3 grid((N + 63) / 64, (M + 63) / 64);
        k_sgemm<64, TA, TB, SA><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, alpha, beta);
    } else {
        const dim3 grid((N + 31) / 32, (M + 31) / 32);
        k_sgemm<32, TA, TB, SA><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, alpha, beta);
    }
    return cudaGetLastError();
}

// ---- the quantized factor: codes and dequantized values of one realization ----
// Element (i, j) of the rows x cols matrix has the quantizer's number e = j * rows + i.
__global__ void __launch_bounds__(256) k_sep_quantize(const float* __restrict__ v, int rows, int cols,
                                                      const float* __restrict__ scale, int lm1, uint64_t seed,
                                                      uint32_t stream_id, uint16_t* __restrict__ codes,
                                                      float* __restrict__ out)
{
    const float c = *scale;
    const QScale qs = qscale(c);
    const float half = (float)lm1 * 0.5f;
    const double alpha = (double)c / (double)lm1;
    const uint32_t key0 = (uint32_t)seed, key1 = (uint32_t)(seed >> 32);
    const long long total = (long long)rows * cols;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t / cols), j = (int)(t - (long long)i * cols);     // row-major position
        const uint64_t e = (uint64_t)j * (uint64_t)rows + (uint64_t)i;
        const uint64_t qq = e >> 2;
        const uint4 rnd = philox4x32_10(make_uint4((uint32_t)qq, (uint32_t)(qq >> 32), stream_id, 0u), key0, key1);
        const uint32_t sel = (uint32_t)(e & 3);
        const uint32_t rw = sel == 0 ? rnd.x : sel == 1 ? rnd.y : sel == 2 ? rnd.z : rnd.w;
        const Decision d = quant_decide(v[t], qs, half, lm1);
        const uint32_t code = quant_code(d, lm1, (float)(rw >> 8) * 0x1p-24f);
        if (codes) codes[t] = (uint16_t)code;
        out[t] = (float)(alpha * (double)(2 * (int)code - lm1));
    }
}

// adjoint factors from the stacked factor F = [Ar; Ai]: M2 = [[Ar^T, Ai^T], [Ai^T, -Ar^T]] (2N x 2N)
// and Fn = [Ar; -Ai] (2N x N)
__global__ void __launch_bounds__(256) k_sep_adjoint_factor(const float* __restrict__ F, int N, float* __restrict__ M2,
                                                            float* __restrict__ Fn)
{
    const int n2 = 2 * N;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n2 * N; t += gridDim.x * blockDim.x)
        Fn[t] = t < N * N ? F[t] : -F[t];
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n2 * n2; t += gridDim.x * blockDim.x) {
        const int a = t / n2, b = t - a * n2;          // output row a, column b
        const int ra = a % N, rb = b % N;
        const bool top = a < N, left = b < N;
        // block (top, left) = Ar^T, (top, right) = Ai^T, (bottom, left) = Ai^T, (bottom, right) = -Ar^T
        const bool imag = top != left;
        const float v = F[(size_t)((imag ? N : 0) + rb) * N + ra];
        M2[t] = (!top && !left) ? -v : v;
    }
}

// forward: read B at the mask from T2 (2N x 2N)
__global__ void k_sep_sample(const float* __restrict__ T2, int N, const int32_t* __restrict__ mask, int M,
                             float* __restrict__ out)
{
    const int n2 = 2 * N;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < M; k += gridDim.x * blockDim.x) {
        const int pos = mask[k], p = pos / N, q = pos - p * N;
        if (pos < 0 || pos >= N * N) {                 // a position off the grid samples nothing
            out[k] = 0.0f;
            out[M + k] = 0.0f;
            continue;
        }
        out[k] = T2[(size_t)p * n2 + q] - T2[(size_t)(N + p) * n2 + N + q];
        out[M + k] = T2[(size_t)p * n2 + N + q] + T2[(size_t)(N + p) * n2 + q];
    }
}

// adjoint: Z = [Zr; Zi] (2N x N) with r at the mask (the buffer was cleared)
__global__ void k_sep_scatter(const float* __restrict__ r, int N, const int32_t* __restrict__ mask, int M,
                              float* __restrict__ Z)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < M; k += gridDim.x * blockDim.x) {
        const int pos = mask[k];
        if (pos < 0 || pos >= N * N) continue;
        Z[pos] = r[k];
        Z[(size_t)N * N + pos] = r[M + k];
    }
}

// sum of squares in FP64 (one CTA; the vectors here are at most 2 N^2 long)
__global__ void __launch_bounds__(256) k_sep_norm2(const float* __restrict__ v, int n, double* __restrict__ out)
{
    __shared__ double s[8];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += 256) acc += (double)v[i] * (double)v[i];
#pragma unroll
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += s[w];
        *out = t;
    }
}

// d = v on the support list, zero elsewhere (d was cleared); sum of squares of the kept values
__global__ void __launch_bounds__(256) k_sep_masked(const float* __restrict__ v, const int32_t* __restrict__ sup,
                                                    int s, float* __restrict__ d, double* __restrict__ out)
{
    __shared__ double sh[8];
    double acc = 0.0;
    for (int q = threadIdx.x; q < s; q += 256) {
        const float g = v[sup[q]];
        d[sup[q]] = g;
        acc += (double)g * (double)g;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += sh[w];
        *out = t;
    }
}

// r = yhat - z, and its sum of squares (one CTA)
__global__ void __launch_bounds__(256) k_sep_resid(const float* __restrict__ yhat, const float* __restrict__ z, int m,
                                                   float* __restrict__ r, double* __restrict__ out)
{
    __shared__ double sh[8];
    double acc = 0.0;
    for (int i = threadIdx.x; i < m; i += 256) {
        const float v = yhat[i] - z[i];
        r[i] = v;
        acc += (double)v * (double)v;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += sh[w];
        *out = t;
    }
}

// x' - x over the dense vectors (x' is zero off its support): d = xn - x, ||d||^2
__global__ void __launch_bounds__(256) k_sep_diff(const float* __restrict__ xn, const float* __restrict__ x, int n,
                                                  float* __restrict__ d, double* __restrict__ out)
{
    __shared__ double sh[8];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += 256) {
        const float v = xn[i] - x[i];
        d[i] = v;
        acc += (double)v * (double)v;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += sh[w];
        *out = t;
    }
}

// dense x' from the selection (xn was cleared)
__global__ void k_sep_place(const int32_t* __restrict__ sel, const float* __restrict__ val, int s, float* __restrict__ xn)
{
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < s; q += gridDim.x * blockDim.x) xn[sel[q]] = val[q];
}

// ---- workspace ----
struct SepPlan {
    size_t f1, f2, m2, fn, t1, t2, z, pq, yhat, x, xn, g, d, r, zv, sel, val, kth, scal, sc, big, total;
};

size_t al(size_t b) { return (b + 255) & ~(size_t)255; }

SepPlan sep_plan(int N, int M, int s)
{
    SepPlan p{};
    const size_t n = (size_t)N * N, fN = 2 * n, m = 2 * (size_t)M;
    size_t o = 0;
    p.f1 = o; o += al(fN * 4);
    p.f2 = o; o += al(fN * 4);
    p.m2 = o; o += al(4 * n * 4);
    p.fn = o; o += al(fN * 4);
    p.t1 = o; o += al(fN * 4);
    p.t2 = o; o += al(4 * n * 4);
    p.z = o; o += al(fN * 4);
    p.pq = o; o += al(fN * 4);
    p.yhat = o; o += al(m * 4);
    p.x = o; o += al(n * 4);
    p.xn = o; o += al(n * 4);
    p.g = o; o += al(n * 4);
    p.d = o; o += al(n * 4);
    p.r = o; o += al(m * 4);
    p.zv = o; o += al(m * 4);
    p.sel = o; o += al((size_t)s * 4);
    p.val = o; o += al((size_t)s * 4);
    p.kth = o; o += al(8);
    p.scal = o; o += al(8 * 8);
    p.sc = o; o += al(16);
    p.big = o; o += (int)n > kMaxTopN ? al(big_top_workspace((int)n)) : 0;
    p.total = o;
    return p;
}

bool sep_ok(const qiht_sep_op* op)
{
    return op && op->factor && op->mask && op->N >= 2 && op->N <= QIHT_SEP_MAX_N && op->M >= 1 &&
           op->M <= op->N * op->N;
}

int levels_of(int bits, int flags) { return (flags & QIHT_ODD_LEVELS) ? (1 << (bits - 1)) + 1 : (1 << bits); }

// forward: out (2M) = Phi-hat x, F the dequantized stacked factor
cudaError_t sep_forward(int N, int M, const int32_t* mask, const float* F, const float* x, float* out, float* T1,
                        float* T2, cudaStream_t s)
{
    cudaError_t e = sgemm<false, false>(2 * N, N, N, F, N, x, N, T1, N, 1.0f, 0.0f, s);          // [P; Q] = F X
    if (e != cudaSuccess) return e;
    e = sgemm<false, true>(2 * N, 2 * N, N, T1, N, F, N, T2, 2 * N, 1.0f, 0.0f, s);             // T1 F^T
    if (e != cudaSuccess) return e;
    k_sep_sample<<<(M + 255) / 256, 256, 0, s>>>(T2, N, mask, M, out);
    return cudaGetLastError();
}

// adjoint: out (N^2) = Phi-hat^T r, M2 and Fn = [Ar; -Ai] the adjoint factors
cudaError_t sep_adjoint(int N, int M, const int32_t* mask, const float* Fn, const float* M2, const float* r, float* out,
                        float* Z, float* PQ, cudaStream_t s)
{
    const size_t n = (size_t)N * N;
    cudaError_t e = cudaMemsetAsync(Z, 0, 2 * n * sizeof(float), s);
    if (e != cudaSuccess) return e;
    k_sep_scatter<<<(M + 255) / 256, 256, 0, s>>>(r, N, mask, M, Z);
    e = sgemm<false, false>(2 * N, N, 2 * N, M2, 2 * N, Z, N, PQ, N, 1.0f, 0.0f, s);          // [P; Q]
    if (e != cudaSuccess) return e;
    return sgemm<false, false, true>(N, N, 2 * N, PQ, N, Fn, N, out, N, 1.0f, 0.0f, s);        // [P | Q] [Ar; -Ai]
}

cudaError_t sep_quantize(const qiht_sep_op* op, const float* v, int rows, int cols, float* scale, int lm1,
                         uint64_t seed, uint32_t stream_id, uint16_t* codes, float* out, cudaStream_t s)
{
    cudaError_t e = launch_absmax(v, rows, cols, cols, scale, s);
    if (e != cudaSuccess) return e;
    (void)op;
    const long long total = (long long)rows * cols;
    long long blocks = (total + 255) / 256;
    if (blocks > (long long)num_sms() * 8) blocks = (long long)num_sms() * 8;
    k_sep_quantize<<<(unsigned)blocks, 256, 0, s>>>(v, rows, cols, scale, lm1, seed, stream_id, codes, out);
    return cudaGetLastError();
}

}  // namespace
}  // namespace qiht

using namespace qiht;

#define SEP_CK(x)                                                \
    do {                                                         \
        if ((x) != cudaSuccess) return QIHT_ERR_CUDA;            \
    } while (0)

extern "C" {

size_t qiht_solve_separable_workspace_size(int32_t N, int32_t M, int32_t s)
{
    if (N < 2 || N > QIHT_SEP_MAX_N || M < 1 || M > N * N || s < 1 || s > N * N) return 0;
    return sep_plan(N, M, s).total;
}

qiht_status qiht_sep_quantize_factor(const qiht_sep_op* op, int32_t bits, uint64_t seed, uint32_t stream_id,
                                     int32_t quant_flags, uint16_t* codes, float* factor_hat, float* scale,
                                     qiht_stream_t stream)
{
    if (bits < 2 || bits > 16) return QIHT_ERR_BITS;
    if (!sep_ok(op) || !factor_hat || !scale || (quant_flags & ~QIHT_ODD_LEVELS)) return QIHT_ERR_ARG;
    SEP_CK(sep_quantize(op, op->factor, 2 * op->N, op->N, scale, levels_of(bits, quant_flags) - 1, seed, stream_id,
                        codes, factor_hat, reinterpret_cast<cudaStream_t>(stream)));
    return QIHT_OK;
}

qiht_status qiht_sep_apply(const qiht_sep_op* op, const float* factor_hat, int32_t adjoint, const float* in, float* out,
                           void* workspace, size_t workspace_bytes, qiht_stream_t stream)
{
    if (!sep_ok(op) || !factor_hat || !in || !out) return QIHT_ERR_ARG;
    const SepPlan P = sep_plan(op->N, op->M, 1);
    if (!workspace || workspace_bytes < P.total || (reinterpret_cast<uintptr_t>(workspace) & 255))
        return QIHT_ERR_WORKSPACE;
    char* w = reinterpret_cast<char*>(workspace);
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    const int N = op->N, M = op->M;
    if (adjoint) {
        float* M2 = reinterpret_cast<float*>(w + P.m2);
        float* Fn = reinterpret_cast<float*>(w + P.fn);
        k_sep_adjoint_factor<<<(4 * N * N + 255) / 256, 256, 0, cs>>>(factor_hat, N, M2, Fn);
        SEP_CK(cudaGetLastError());
        SEP_CK(sep_adjoint(N, M, op->mask, Fn, M2, in, out, reinterpret_cast<float*>(w + P.z),
                           reinterpret_cast<float*>(w + P.pq), cs));
    } else {
        SEP_CK(sep_forward(N, M, op->mask, factor_hat, in, out, reinterpret_cast<float*>(w + P.t1),
                           reinterpret_cast<float*>(w + P.t2), cs));
    }
    return QIHT_OK;
}

qiht_status qiht_niht_solve_separable(const qiht_sep_op* op, const float* y, int32_t bits_factor, int32_t bits_y,
                                      uint64_t seed, int32_t quant_flags, int32_t s, int32_t iters,
                                      const qiht_params* params, float* x, int32_t* support, qiht_report* report,
                                      const qiht_trace* trace, void* workspace, size_t workspace_bytes,
                                      qiht_stream_t stream)
{
    if (bits_factor < 2 || bits_factor > 16 || bits_y < 2 || bits_y > 16) return QIHT_ERR_BITS;
    if (!sep_ok(op) || !y || !x || !support || !report || iters < 0 || (quant_flags & ~QIHT_ODD_LEVELS))
        return QIHT_ERR_ARG;
    const int N = op->N, M = op->M, n = N * N, m = 2 * M;
    if (s < 1 || s > n || s > m) return QIHT_ERR_ARG;
    qiht_params prm{2.0, 0.01, 32, 0, 0.0, QIHT_MU_FORWARD_SQ, 0};
    if (params) prm = *params;
    if (!(prm.c > 0.0 && prm.c < 1.0) || !(prm.k * (1.0 - prm.c) > 1.0) || prm.max_backtrack < 0 || prm.flags != 0 ||
        prm.mu_mode != QIHT_MU_FORWARD_SQ || !(prm.tol >= 0.0 && std::isfinite(prm.tol)))
        return QIHT_ERR_ARG;
    const SepPlan P = sep_plan(N, M, s);
    if (!workspace || workspace_bytes < P.total || (reinterpret_cast<uintptr_t>(workspace) & 255))
        return QIHT_ERR_WORKSPACE;
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    char* w = reinterpret_cast<char*>(workspace);
    auto F = [&](size_t off) { return reinterpret_cast<float*>(w + off); };
    float *F1 = F(P.f1), *F2 = F(P.f2), *M2 = F(P.m2), *Fn1 = F(P.fn), *T1 = F(P.t1), *T2 = F(P.t2), *Z = F(P.z),
          *PQ = F(P.pq);
    float *yhat = F(P.yhat), *xd = F(P.x), *xn = F(P.xn), *g = F(P.g), *d = F(P.d), *r = F(P.r), *zv = F(P.zv);
    int32_t* sel = reinterpret_cast<int32_t*>(w + P.sel);
    float* val = F(P.val);
    float* kth = F(P.kth);
    double* scal = reinterpret_cast<double*>(w + P.scal);    // [0] num, [1] den, [2] dn, [3] dd, [4] rr, [5] mu
    float* sc = F(P.sc);                                      // [0] factor scale, [1] y scale
    const int lmf = levels_of(bits_factor, quant_flags) - 1, lmy = levels_of(bits_y, quant_flags) - 1;

    // the two realizations of the factor, the adjoint factor of the first, and y-hat
    SEP_CK(sep_quantize(op, op->factor, 2 * N, N, sc, lmf, seed, 0, nullptr, F1, cs));
    SEP_CK(sep_quantize(op, op->factor, 2 * N, N, sc, lmf, seed, 1, nullptr, F2, cs));
    k_sep_adjoint_factor<<<(4 * n + 255) / 256, 256, 0, cs>>>(F1, N, M2, Fn1);
    SEP_CK(cudaGetLastError());
    SEP_CK(sep_quantize(op, y, m, 1, sc + 1, lmy, seed, 2, nullptr, yhat, cs));

    std::vector<int32_t> h_sup(s), h_sel(s);
    double h_scal[6];
    auto read = [&](void* dst, const void* src, size_t bytes) -> bool {
        if (cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, cs) != cudaSuccess) return false;
        return cudaStreamSynchronize(cs) == cudaSuccess;
    };
    qiht_report rep{};
    rep.status = QIHT_OK;
    auto finish = [&](int status) -> qiht_status {
        rep.status = status;
        if (cudaMemcpyAsync(report, &rep, sizeof(rep), cudaMemcpyHostToDevice, cs) != cudaSuccess) return QIHT_ERR_CUDA;
        if (cudaMemcpyAsync(x, xd, (size_t)n * 4, cudaMemcpyDeviceToDevice, cs) != cudaSuccess) return QIHT_ERR_CUDA;
        if (cudaMemcpyAsync(support, sel, (size_t)s * 4, cudaMemcpyDeviceToDevice, cs) != cudaSuccess)
            return QIHT_ERR_CUDA;
        return cudaStreamSynchronize(cs) == cudaSuccess ? QIHT_OK : QIHT_ERR_CUDA;
    };
    auto record = [&](int t, double mu, int bt) -> bool {
        if (!trace) return true;
        if (trace->support &&
            cudaMemcpyAsync(trace->support + (size_t)t * s, sel, (size_t)s * 4, cudaMemcpyDeviceToDevice, cs) != cudaSuccess)
            return false;
        if (trace->mu && cudaMemcpyAsync(trace->mu + t, &mu, 8, cudaMemcpyHostToDevice, cs) != cudaSuccess) return false;
        if (trace->bt && cudaMemcpyAsync(trace->bt + t, &bt, 4, cudaMemcpyHostToDevice, cs) != cudaSuccess) return false;
        if (trace->resid2 && cudaMemcpyAsync(trace->resid2 + t, scal + 4, 8, cudaMemcpyDeviceToDevice, cs) != cudaSuccess)
            return false;
        if (trace->kth && cudaMemcpyAsync(trace->kth + 2 * t, kth, 8, cudaMemcpyDeviceToDevice, cs) != cudaSuccess)
            return false;
        return cudaStreamSynchronize(cs) == cudaSuccess;
    };
    auto top = [&](const double* mu_dev) -> cudaError_t {
        if (n > kMaxTopN)
            return launch_big_top(g, mu_dev ? xd : nullptr, mu_dev, n, s, sel, val, kth, w + P.big, cs);
        TopArgs t{};
        t.g = g;
        t.x = mu_dev ? xd : nullptr;
        t.mu = mu_dev;
        t.n = n;
        t.s = s;
        t.sel = sel;
        t.val = val;
        t.kth = kth;
        t.st = nullptr;
        return launch_top(t, cs);
    };

    // initial state: x = 0, r = y-hat, support of H_s(Phi-hat_1^T y-hat)
    SEP_CK(cudaMemsetAsync(xd, 0, (size_t)n * 4, cs));
    SEP_CK(cudaMemcpyAsync(r, yhat, (size_t)m * 4, cudaMemcpyDeviceToDevice, cs));
    k_sep_norm2<<<1, 256, 0, cs>>>(r, m, scal + 4);
    SEP_CK(sep_adjoint(N, M, op->mask, Fn1, M2, r, g, Z, PQ, cs));
    SEP_CK(top(nullptr));
    SEP_CK(cudaMemsetAsync(val, 0, (size_t)s * 4, cs));
    if (!read(h_sup.data(), sel, (size_t)s * 4)) return QIHT_ERR_CUDA;
    if (!record(0, 0.0, 0)) return QIHT_ERR_CUDA;
    const double shrink = prm.k * (1.0 - prm.c);
    for (int t = 1; t <= iters; ++t) {
        // g = Phi-hat_1^T r (r is the residual of the current x)
        if (t > 1) SEP_CK(sep_adjoint(N, M, op->mask, Fn1, M2, r, g, Z, PQ, cs));
        // mu = ||g_G||^2 / ||Phi-hat_2 g_G||^2 on the current support (still in sel)
        SEP_CK(cudaMemsetAsync(d, 0, (size_t)n * 4, cs));
        k_sep_masked<<<1, 256, 0, cs>>>(g, sel, s, d, scal + 0);
        SEP_CK(sep_forward(N, M, op->mask, F2, d, zv, T1, T2, cs));
        k_sep_norm2<<<1, 256, 0, cs>>>(zv, m, scal + 1);
        if (!read(h_scal, scal, 16)) return QIHT_ERR_CUDA;
        const double num = h_scal[0], den = h_scal[1];
        if (!std::isfinite(num) || !std::isfinite(den)) return finish(QIHT_ERR_NONFINITE);
        if (num == 0.0 || den == 0.0) break;                     // converged: x stays
        double mu = num / den;
        int bt = 0, status = QIHT_OK;
        bool changed = false;
        for (;;) {
            SEP_CK(cudaMemcpyAsync(scal + 5, &mu, 8, cudaMemcpyHostToDevice, cs));
            SEP_CK(top(scal + 5));                               // x' = H_s(x + mu g): sel, val
            if (!read(h_sel.data(), sel, (size_t)s * 4)) return QIHT_ERR_CUDA;
            changed = h_sel != h_sup;
            if (!changed) break;
            // backtracking test on x' - x
            SEP_CK(cudaMemsetAsync(xn, 0, (size_t)n * 4, cs));
            k_sep_place<<<(s + 255) / 256, 256, 0, cs>>>(sel, val, s, xn);
            k_sep_diff<<<1, 256, 0, cs>>>(xn, xd, n, d, scal + 2);
            SEP_CK(sep_forward(N, M, op->mask, F2, d, zv, T1, T2, cs));
            k_sep_norm2<<<1, 256, 0, cs>>>(zv, m, scal + 3);
            if (!read(h_scal, scal, 32)) return QIHT_ERR_CUDA;
            const double dn = h_scal[2], dd = h_scal[3];
            if (dn == 0.0) break;
            const double omega = dd > 0.0 ? dn / dd : INFINITY;
            if (mu <= (1.0 - prm.c) * omega) break;
            if (bt >= prm.max_backtrack) { status = QIHT_ERR_BACKTRACK_CAP; break; }
            mu = mu / shrink;
            ++bt;
        }
        if (status != QIHT_OK) {
            // restore the committed support for the outputs
            SEP_CK(cudaMemcpyAsync(sel, h_sup.data(), (size_t)s * 4, cudaMemcpyHostToDevice, cs));
            return finish(status);
        }
        // accept x' (sel, val): dense x, the residual of it, the record
        SEP_CK(cudaMemsetAsync(xd, 0, (size_t)n * 4, cs));
        k_sep_place<<<(s + 255) / 256, 256, 0, cs>>>(sel, val, s, xd);
        SEP_CK(sep_forward(N, M, op->mask, F2, xd, zv, T1, T2, cs));
        k_sep_resid<<<1, 256, 0, cs>>>(yhat, zv, m, r, scal + 4);
        if (changed) rep.support_changes++;
        rep.backtracks += bt;
        rep.mu = mu;
        rep.iters_run = t;
        h_sup = h_sel;
        if (!record(t, mu, bt)) return QIHT_ERR_CUDA;
        if (!read(h_scal + 4, scal + 4, 8)) return QIHT_ERR_CUDA;
        rep.resid_norm2 = h_scal[4];
        if (!std::isfinite(rep.resid_norm2)) return finish(QIHT_ERR_NONFINITE);
        if (prm.tol > 0.0 && rep.resid_norm2 <= prm.tol) break;
    }
    if (!read(h_scal + 4, scal + 4, 8)) return QIHT_ERR_CUDA;
    rep.resid_norm2 = h_scal[4];
    return finish(QIHT_OK);
}

}  // extern "C"
