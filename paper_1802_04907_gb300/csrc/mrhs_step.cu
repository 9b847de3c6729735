// Algorithm 2 for many right-hand sides sharing one quantized matrix: everything of an
// iteration except the gradient product, one CTA per right-hand side.
//
// The gradients of all right-hand sides come from one tensor-core GEMM (mrhs_gemm.cu);
// the rest of an iteration is per right-hand side and runs here: the step size
// mu = ||g_G||^2 / ||Q2_G g_G||^2 (FP64 sums of squares; the product Q2_G g_G as exact
// integer sums of the codes with the coefficients in 24-bit fixed point, rounded once to
// FP32, at 8 and 4 bits, and FP32 products summed in list order at 2 bits), H_s over the
// binary32 keys |fmaf(mu, g, x)| with ties to the lower index (a radix select over the
// support and the entries off it whose key reaches the smallest key on it, which hold the
// s largest; over all n when those do not fit), the backtracking test
// omega = ||x' - x||^2 / ||Q2 (x' - x)||^2, and the residual r = Q(y) - Q2_G' x', updated
// from the product the step already formed (Q2 (x' - x) of the backtracking test, or
// mu Q2_G g_G when the support is unchanged), and directly as Q(y) - Q2_G' x' every few
// iterations and on the last. The backtracking test's product reads only the columns that
// enter or leave the support and adds mu Q2_G g_G for the rest. The CTA then splits r into
// the scaled f16 parts the next GEMM reads.
// The iterate of a right-hand side is kept sparse (its support and the values on it).
#include <cuda_fp16.h>

#include <cmath>

#include "cta_ops.cuh"

namespace qiht {
namespace {

using namespace cta;

// dequantized observation value of row i (FP64 product, rounded once)
__device__ __forceinline__ float yhat_at(const qiht_codes& Y, int lm1y, double alpha_y, int i)
{
    const int Gy = 32 / Y.bits;
    const uint32_t w = __ldg(Y.words + i / Gy);
    const int k = i % Gy;
    const int code = (int)((w >> (8 * (k & 3) + Y.bits * (k >> 2))) & ((1u << Y.bits) - 1));
    return (float)(alpha_y * (double)(2 * code - lm1y));
}

// r (in z[0..m)) -> the scaled f16 parts of the next gradient product
__device__ void split_residual(const float* r, int m, int mk, __half* hi, __half* lo, float* sc_k, double alpha1,
                               SSh& sh)
{
    unsigned mx = 0;
    for (int i = threadIdx.x; i < m; i += kST) mx = max(mx, __float_as_uint(r[i]) & 0x7fffffffu);
    mx = smax(mx, sh.i);
    int e = 0;
    const float M = __uint_as_float(mx);
    if (M > 0.0f && isfinite(M)) {
        int ex;
        frexpf(M, &ex);
        e = ex - 15;
    }
    for (int i = threadIdx.x; i < mk; i += kST) {
        const float v = i < m ? ldexpf(r[i], -e) : 0.0f;
        const __half h = __float2half_rn(v);
        hi[i] = h;
        lo[i] = __float2half_rn(v - __half2float(h));
    }
    if (threadIdx.x == 0) *sc_k = (float)ldexp(alpha1, e);
}

// r (in z[0..m)) -> the three scaled e4m3 terms of the FP8 gradient product (max |r| 2^-e in
// [2^7, 2^8)): term t of right-hand side k at row t * rhi + k of the byte tensor, mk8 bytes each
__device__ void split_residual8(const float* r, int m, int mk8, int rhi, int k, unsigned char* R8, float* sc_k,
                                double alpha1, SSh& sh)
{
    unsigned mx = 0;
    for (int i = threadIdx.x; i < m; i += kST) mx = max(mx, __float_as_uint(r[i]) & 0x7fffffffu);
    mx = smax(mx, sh.i);
    int e = 0;
    const float M = __uint_as_float(mx);
    if (M > 0.0f && isfinite(M)) {
        int ex;
        frexpf(M, &ex);
        e = ex - 8;
    }
    for (int i = threadIdx.x; i < mk8; i += kST) {
        float v = i < m ? ldexpf(r[i], -e) : 0.0f;
#pragma unroll
        for (int t = 0; t < kMrhsTerms8; ++t) {
            const uint32_t b = f_to_e4m3(v);
            R8[(size_t)(t * rhi + k) * mk8 + i] = (unsigned char)b;
            v -= e4m3_to_f(b);                 // exact: the term is within a factor 2 of v (or v is tiny)
        }
    }
    if (threadIdx.x == 0) *sc_k = (float)ldexp(alpha1, e);
}

static_assert(2 * QIHT_MULTI_MAX_S <= kST, "the backtracking test gives each union entry its own thread");

// the products over s columns (the step size's and the refresh's): exact integer sums at 8 and
// 4 bits, FP32 at 2 bits
template <int BITS>
__device__ __forceinline__ void mcols_s(const Codes& Q, const int* list, const float* coef, int count, float* z,
                                        uint32_t* scratch, SSh& sh)
{
    if constexpr (BITS == 2) mcols<BITS>(Q, list, coef, count, z, reinterpret_cast<float*>(scratch));
    else mcols_fx<BITS>(Q, list, coef, count, z, scratch, sh);
}

template <int BITS>
__global__ void __launch_bounds__(kST, 1) k_mrhs_step(MrhsStepArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ SSh sh;
    const int k = blockIdx.x, tid = threadIdx.x;
    MrhsState* st = a.st + k;
    if (st->stop) return;
    const int n = a.n, m = a.m, s = a.s;
    const MSm sm = msm_layout(smem, n, a.mk, s);
    const float* g = a.G + (size_t)k * n;
    int32_t* gsup = a.sup + (size_t)k * s;
    float* gxs = a.xs + (size_t)k * s;
    if (tid == 0) {
        sh.alpha1 = (double)(*a.scale1) / (double)a.lm1_1;
        sh.alpha2 = (double)(*a.Q2.scale) / (double)a.Q2.lm1;
        sh.alpha2f = (float)sh.alpha2;
    }
    const int nbw = (n + 31) / 32;
    for (int w = tid; w < nbw; w += kST) sm.gbit[w] = 0u;
    __syncthreads();
    int status = QIHT_OK;
    int uc = 0;
    if (a.mode == 0) {
        // initial support H_s(g) (x = 0, keys |g|)
        for (int q = tid; q < s; q += kST) { sm.sup[q] = 0; sm.xs[q] = 0.0f; }
        __syncthreads();
        if (mkeys(n, 0, 1.0f, g, sm)) {
            status = QIHT_ERR_NONFINITE;
        } else {
            mselect(n, s, 1.0f, g, sm, sh, &uc, false, reinterpret_cast<int*>(sm.z), a.mk);
            for (int q = tid; q < s; q += kST) { gsup[q] = sm.sel[q]; gxs[q] = 0.0f; }
        }
        if (tid == 0 && status != QIHT_OK) { st->status = status; st->stop = 2; }
        return;
    }
    for (int q = tid; q < s; q += kST) {
        const int j = gsup[q];
        sm.sup[q] = j;
        sm.xs[q] = gxs[q];
        atomicOr(&sm.gbit[j >> 5], 1u << (j & 31));
    }
    __syncthreads();
    // step size mu = ||g_G||^2 / (alpha2^2 ||Q2_G g_G||^2)
    for (int q = tid; q < s; q += kST) sm.val[q] = __ldg(g + sm.sup[q]);
    __syncthreads();
    double num = 0.0;
    if (tid < 32) {
        for (int q = tid; q < s; q += 32) num += (double)sm.val[q] * (double)sm.val[q];
#pragma unroll
        for (int o = 16; o; o >>= 1) num += __shfl_xor_sync(0xffffffffu, num, o);
    }
    mcols_s<BITS>(a.Q2, sm.sup, sm.val, s, sm.z, sm.keys, sh);
    // sums of squares: each thread's <= 16 terms in FP32, the CTA sum of the partials in FP64
    // (a per-element FP64 sum keeps the narrow FP64 pipe of this GPU busy for microseconds)
    float zzf = 0.0f;
    float* zmu = a.zmu + (size_t)k * m;             // kept for the residual update
    for (int i = tid; i < m; i += kST) {
        zzf = fmaf(sm.z[i], sm.z[i], zzf);
        zmu[i] = sm.z[i];
    }
    const double zz = ssum((double)zzf, sh.d);
    if (tid == 0) {
        const double den = sh.alpha2 * sh.alpha2 * zz;
        int code = 0;
        if (!isfinite(num) || !isfinite(den)) code = 2;
        else if (num == 0.0 || den == 0.0) code = 1;      // converged: x stays
        sh.mu = code ? 0.0 : num / den;
        sh.muf = (float)sh.mu;
        sh.code = code;
    }
    __syncthreads();
    if (sh.code != 0) {
        if (tid == 0) {
            if (sh.code == 2) st->status = QIHT_ERR_NONFINITE;
            st->stop = sh.code;
        }
        return;
    }
    int bt = 0, changed = 0, ranked = 0;
    for (;;) {
        uint32_t kmin = 0, rest = 0;
        int ncand = -1;
        int* clist = reinterpret_cast<int*>(sm.z);      // free here: the step size's product is in zmu
        if (mkeys_cand(n, s, sh.muf, g, sm, sh.i, &kmin, &rest, clist, a.mk, &ncand)) { changed = -1; break; }
        if (kmin > rest) {
            // every key of G exceeds every other key: G' = G without ranking
            for (int q = tid; q < s; q += kST) {
                sm.sel[q] = sm.sup[q];
                sm.val[q] = fmaf(sh.muf, __ldg(g + sm.sup[q]), sm.xs[q]);
            }
            uc = s;
            changed = 0;
            __syncthreads();
            break;
        }
        changed = mselect(n, s, sh.muf, g, sm, sh, &uc, true, clist, a.mk, ncand >= 0 ? s + ncand : -1);
        ++ranked;
        if (!changed) break;
        // backtracking test on G' u G
        double dn = 0.0;
        if (tid < 32) {
            for (int q = tid; q < uc; q += 32) dn += (double)sm.dlt[q] * (double)sm.dlt[q];
#pragma unroll
            for (int o = 16; o; o >>= 1) dn += __shfl_xor_sync(0xffffffffu, dn, o);
        }
        // Q2 (x' - x) = mu Q2_G g_G + Q2 over the columns that enter or leave the support: on
        // G n G' the step is mu g, which the step size's own product covers; on G' \ G it is x';
        // on G \ G' it is -x, from which mu g is taken back out. So only those columns are read
        // (a few, against s for the whole union). s <= 256 leaves one union entry per thread.
        int keep = 0, jk = 0;
        float ck = 0.0f;
        if (tid < uc) {
            jk = sm.uni[tid];
            if (tid >= s) {
                keep = 1;
                ck = sm.dlt[tid] - sh.muf * __ldg(g + jk);
            } else if (!((sm.gbit[jk >> 5] >> (jk & 31)) & 1u)) {
                keep = 1;
                ck = sm.dlt[tid];
            }
        }
        int nsym;
        const int pos = sscan(keep, sh.i, &nsym);
        __syncthreads();                     // every entry (and the sum above) read before the list is rewritten
        if (keep) {
            sm.uni[pos] = jk;
            sm.dlt[pos] = ck;
        }
        __syncthreads();
        mcols<BITS>(a.Q2, sm.uni, sm.dlt, nsym, sm.z, reinterpret_cast<float*>(sm.keys));
        float dzf = 0.0f;
        for (int i = tid; i < m; i += kST) {
            const float v = fmaf(sh.muf, __ldcg(zmu + i), sm.z[i]);
            sm.z[i] = v;
            dzf = fmaf(v, v, dzf);
        }
        const double dz = ssum((double)dzf, sh.d);
        if (tid == 0) {
            const double dd = sh.alpha2 * sh.alpha2 * dz;
            int code = 0;                                   // 0 accept, 1 shrink, 2 give up
            if (dn > 0.0) {
                const double omega = dd > 0.0 ? dn / dd : INFINITY;
                if (!(sh.mu <= (1.0 - a.cc) * omega)) {
                    if (bt >= a.max_bt) code = 2;
                    else {
                        code = 1;
                        sh.mu = sh.mu / (a.kk * (1.0 - a.cc));
                        sh.muf = (float)sh.mu;
                    }
                }
            }
            sh.code = code;
        }
        __syncthreads();
        if (sh.code == 0) break;
        if (sh.code == 2) { changed = -2; break; }
        ++bt;
    }
    if (changed < 0) {
        if (tid == 0) {
            st->status = changed == -1 ? QIHT_ERR_NONFINITE : QIHT_ERR_BACKTRACK_CAP;
            st->stop = 2;
        }
        return;
    }
    // commit G' and x'
    for (int q = tid; q < s; q += kST) {
        gsup[q] = sm.sel[q];
        gxs[q] = sm.val[q];
    }
    // residual: r - alpha2 Q2 (x' - x) with the product already formed for this step (the
    // backtracking test's Q2 (x' - x) if G' != G, else mu Q2_G g_G of the step size), or
    // directly r = Q(y) - alpha2 Q2_G' x' on refresh iterations (periodically and on the last)
    float rrf = 0.0f;
    float* rk = a.resid + (size_t)k * m;
    // r_i = base_i - c prod_i for this thread's rows i = tid + kST u, in groups of RU whose loads
    // are issued before any of their stores (a store to rk may alias a later load, so the
    // compiler would otherwise wait on each load in turn); the sum of squares keeps row order
    constexpr int RU = 8;
    auto resid_rows = [&](const float* base, const float* prod, bool prod_shared, float c) {
        for (int i0 = tid; i0 < m; i0 += RU * kST) {
            float bv[RU], pv[RU];
#pragma unroll
            for (int u = 0; u < RU; ++u) {
                const int i = i0 + u * kST;
                if (i < m) {
                    bv[u] = __ldcg(base + i);
                    pv[u] = prod_shared ? sm.z[i] : __ldcg(prod + i);
                }
            }
#pragma unroll
            for (int u = 0; u < RU; ++u) {
                const int i = i0 + u * kST;
                if (i < m) {
                    const float ri = fmaf(-c, pv[u], bv[u]);
                    sm.z[i] = ri;
                    rk[i] = ri;
                    rrf = fmaf(ri, ri, rrf);
                }
            }
        }
    };
    if (a.refresh) {
        mcols_s<BITS>(a.Q2, sm.sel, sm.val, s, sm.z, sm.keys, sh);
        resid_rows(a.yhat + (size_t)k * m, nullptr, true, sh.alpha2f);
    } else if (changed) {
        resid_rows(rk, nullptr, true, sh.alpha2f);
    } else {
        resid_rows(rk, zmu, false, sh.alpha2f * sh.muf);
    }
    const double rr = ssum((double)rrf, sh.d);
    if (tid == 0) {
        st->iters_run += 1;
        st->backtracks += bt;
        st->changes += changed;
        st->full_selects += ranked;
        st->mu = sh.mu;
        st->resid2 = rr;
        if (!isfinite(rr)) { st->status = QIHT_ERR_NONFINITE; st->stop = 2; }
    }
    if (!a.last && isfinite(rr)) {
        if (a.fp8)
            split_residual8(sm.z, m, a.mk8, a.rhi, k, reinterpret_cast<unsigned char*>(a.R16), a.sc + k, sh.alpha1, sh);
        else
            split_residual(sm.z, m, a.mk, a.R16 + (size_t)k * a.mk, a.R16 + (size_t)(a.rhi + k) * a.mk, a.sc + k,
                           sh.alpha1, sh);
    }
}

// Q(y_k) -> r = Q(y_k), its f16 parts, ||Q(y_k)||^2; the state of every right-hand side reset.
// Rows of the padded tensor past nrhs become zeros.
__global__ void __launch_bounds__(kST) k_mrhs_init(MrhsStepArgs a)
{
    __shared__ SSh sh;
    extern __shared__ __align__(16) unsigned char smem[];
    float* r = reinterpret_cast<float*>(smem);
    const int k = blockIdx.x, tid = threadIdx.x, m = a.m;
    __half* hi = a.R16 + (size_t)k * a.mk;
    __half* lo = a.R16 + (size_t)(a.rhi + k) * a.mk;
    unsigned char* R8 = reinterpret_cast<unsigned char*>(a.R16);
    if (k >= a.nrhs) {
        if (a.fp8) {
            for (int t = 0; t < kMrhsTerms8; ++t)
                for (int i = tid; i < a.mk8; i += kST) R8[(size_t)(t * a.rhi + k) * a.mk8 + i] = 0;
        } else {
            for (int i = tid; i < a.mk; i += kST) { hi[i] = __float2half_rn(0.0f); lo[i] = __float2half_rn(0.0f); }
        }
        if (tid == 0) a.sc[k] = 0.0f;
        return;
    }
    const qiht_codes Y = a.ydesc[k];
    const int lm1y = grid_levels(Y.bits, Y.levels) - 1;
    if (tid == 0) {
        const float c1 = *a.scale1, c2 = *a.Q2.scale, cy = *Y.scale;
        sh.code = (isfinite(c1) && isfinite(c2) && isfinite(cy)) ? 0 : 1;
        sh.alpha1 = (double)c1 / (double)a.lm1_1;
        sh.alpha_y = (double)cy / (double)lm1y;
    }
    __syncthreads();
    double acc = 0.0;
    for (int i = tid; i < m; i += kST) {
        const float v = yhat_at(Y, lm1y, sh.alpha_y, i);
        r[i] = v;
        a.yhat[(size_t)k * m + i] = v;
        a.resid[(size_t)k * m + i] = v;
        acc += (double)v * (double)v;
    }
    acc = ssum(acc, sh.d);
    MrhsState* st = a.st + k;
    // a valid support until the first selection (a right-hand side stopped here keeps x = 0)
    for (int q = tid; q < a.s; q += kST) {
        a.sup[(size_t)k * a.s + q] = q;
        a.xs[(size_t)k * a.s + q] = 0.0f;
    }
    if (tid == 0) {
        st->mu = 0.0;
        st->resid2 = acc;
        st->stop = sh.code ? 2 : 0;
        st->status = sh.code ? QIHT_ERR_NONFINITE : QIHT_OK;
        st->iters_run = 0;
        st->backtracks = 0;
        st->changes = 0;
        st->full_selects = 1;             // the initial support
    }
    if (a.fp8)
        split_residual8(r, m, a.mk8, a.rhi, k, R8, a.sc + k, sh.alpha1, sh);
    else
        split_residual(r, m, a.mk, hi, lo, a.sc + k, sh.alpha1, sh);
}

// dense x, the support and the report of every right-hand side
__global__ void __launch_bounds__(256) k_mrhs_final(MrhsStepArgs a, float* X, qiht_report* reports,
                                                    const int* gemm_status)
{
    const int k = blockIdx.x;
    const MrhsState* st = a.st + k;
    float* x = X + (size_t)k * a.n;
    for (int j = threadIdx.x; j < a.n; j += 256) x[j] = 0.0f;
    __syncthreads();
    for (int q = threadIdx.x; q < a.s; q += 256) x[a.sup[(size_t)k * a.s + q]] = a.xs[(size_t)k * a.s + q];
    if (threadIdx.x == 0) {
        qiht_report* rp = reports + k;
        rp->iters_run = st->iters_run;
        rp->backtracks = st->backtracks;
        rp->support_changes = st->changes;
        rp->status = *gemm_status ? *gemm_status : st->status;
        rp->resid_norm2 = st->resid2;
        rp->mu = st->mu;
        rp->full_selects = st->full_selects;
        rp->reserved = 0;
        for (int i = 0; i < 8; ++i) rp->phase_us[i] = 0.0f;
    }
}

}  // namespace

size_t mrhs_step_smem(int n, int mk, int s) { return mrhs_step_smem_bytes(n, mk, s); }

cudaError_t launch_mrhs_init(const MrhsStepArgs& a, cudaStream_t s)
{
    const size_t smem = (size_t)a.mk * 4;
    cudaError_t e = cudaFuncSetAttribute(k_mrhs_init, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_mrhs_init<<<a.rhi, kST, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_mrhs_step(const MrhsStepArgs& a, int bits, cudaStream_t s)
{
    const size_t smem = mrhs_step_smem_bytes(a.n, a.mk, a.s);
    void* fn = bits == 8 ? (void*)k_mrhs_step<8> : bits == 4 ? (void*)k_mrhs_step<4> : (void*)k_mrhs_step<2>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    MrhsStepArgs b = a;
    void* args[] = {(void*)&b};
    return cudaLaunchKernel(fn, dim3((unsigned)a.nrhs), dim3(kST), args, smem, s);
}

cudaError_t launch_mrhs_final(const MrhsStepArgs& a, float* X, qiht_report* reports, const int* gemm_status,
                              cudaStream_t s)
{
    k_mrhs_final<<<a.nrhs, 256, 0, s>>>(a, X, reports, gemm_status);
    return cudaGetLastError();
}

}  // namespace qiht
