// Internal declarations shared by the translation units of the QIHT CUDA library.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cmath>
#include <cstddef>
#include <cstdint>

#include "../../include/qiht.h"

namespace qiht {

constexpr int kMaxRows = 16384;   // m limit of the integer GEMV^T (32-bit lane sums cannot overflow)
constexpr int kMaxTopN = 49152;   // n limit of the one-CTA radix select (keys held in shared memory)
constexpr int kGatherCols = 32;   // list entries (columns) per CTA in the column-subset product
constexpr int kGatherThreads = 256;

// Programmatic dependent launch: a kernel launched with a programmatic edge may start
// while its upstream kernel still runs; griddep_wait() returns once the upstream grid
// has completed and its memory is visible (a no-op for an ordinary launch), and
// griddep_launch() lets the downstream kernel start early.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

constexpr int kPartSlots = 8;             // kinds of per-CTA partials of the iteration kernel
constexpr int kSlotCtas = 256;            // CTAs per partial kind (largest iteration grid)
constexpr int kSlotPerLane = kSlotCtas / 32;
constexpr int kSlotResid = 4;             // ||r||^2 of the CTA's rows
constexpr int kSlotRmax = 5;              // max |r| (float bits) of the CTA's rows

// Value of a tagged partial slot word (the sign bit carries the tag).
__device__ __forceinline__ double slot_value(unsigned long long b)
{
    return __longlong_as_double((long long)(b & 0x7fffffffffffffffull));
}

// Warp 0 (all 32 lanes call it): sum (kind ks) or maximum (kind km) over the first `grid`
// CTAs of complete partial slots (no tag check: the kernel that wrote them has finished),
// lane l taking CTAs l, l + 32, ... in order, then a fixed shuffle tree.
__device__ __forceinline__ double slot_sum_complete(const double* part, int ks, int grid)
{
    const int lane = threadIdx.x & 31;
    double v = 0.0;
#pragma unroll
    for (int u = 0; u < kSlotPerLane; ++u) {
        const int c = lane + 32 * u;
        const double t = c < grid ? slot_value(__ldcg(reinterpret_cast<const unsigned long long*>(part) +
                                                      (size_t)ks * kSlotCtas + c))
                                  : 0.0;
        v += t;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double slot_max_complete(const double* part, int km, int grid)
{
    const int lane = threadIdx.x & 31;
    double v = 0.0;
#pragma unroll
    for (int u = 0; u < kSlotPerLane; ++u) {
        const int c = lane + 32 * u;
        if (c < grid)
            v = fmax(v, slot_value(__ldcg(reinterpret_cast<const unsigned long long*>(part) + (size_t)km * kSlotCtas + c)));
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Device view of a quantized matrix (see the column-packed layout in qiht.h).
// lm1 = levels - 1 of its grid: 2^bits - 1 by default, 2^(bits-1) on the odd grid.
// Codes are extracted with the bits-wide mask; lm1 enters only the affine term
// 2c - lm1 of a value and the scale alpha = c / lm1.
struct Codes {
    const uint32_t* words;
    const float* scale;
    int rows, cols, bits, ld;
    int lm1;
};

// Number of levels of a grid given as in qiht_codes (0 = 2^bits); -1 unless it is
// 2^bits or 2^(bits-1) + 1.
__host__ __device__ inline int grid_levels(int bits, int levels)
{
    if (levels == 0 || levels == (1 << bits)) return 1 << bits;
    if (levels == (1 << (bits - 1)) + 1) return levels;
    return -1;
}

// Scale factors alpha = c / (L - 1) that every thread of a CTA needs are divided in FP32
// (__fdiv_rn): for float operands the double quotient rounded to float is the correctly
// rounded float quotient (the double format has more than 2 x 24 + 2 bits), so the value is the
// same, without a double division (about 15 FP64 instructions per warp) in every warp.

// ---- b0 + T d for an exact integer sum T, without the FP64 pipe ----
// The FP64 pipe of this GPU is narrow: a warp-wide FP64 instruction occupies it for ~16 SM
// clocks, so per-column epilogues that scaled their integer sums in double were bound by it.
// Scale2f holds a double constant d as (hi + lo) 2^e: hi + lo is d's significand in [0.5, 1)
// to ~48 bits, split in two floats. A power-of-two rescaling of d is an integer add to e.
struct Scale2f {
    float hi, lo;
    int e;
};

__host__ __device__ inline Scale2f scale2f_make(double d)
{
    int e = 0;
    const double m = (d == 0.0) ? 0.0 : frexp(d, &e);
    Scale2f s;
    s.hi = (float)m;
    s.lo = (float)(m - (double)s.hi);
    s.e = e;
    return s;
}

// 2^k as a float for k in [-126, 127] (integer operations only)
__device__ __forceinline__ float pow2f(int k)
{
    k = k < -126 ? -126 : (k > 127 ? 127 : k);
    return __uint_as_float((uint32_t)(k + 127) << 23);
}

// b0 + T d in FP32 arithmetic, for any T with |T| < 2^63. |T| = F2 + F1 + F0, F_k = c_k 2^(23k)
// with 0 <= c_k < 2^23 (c_2 < 2^17): exact floats. The three products with hi are formed with
// their exact FMA errors and summed by TwoSum, the lo terms are added to the error term, the
// pair is scaled by 2^e in two power-of-two steps (exact unless the result is subnormal), added to
// b0 by a last TwoSum; one final rounding. Before that rounding the value is within ~2^-44 of
// b0 + T d relative to |T d| + |b0|.
__device__ __forceinline__ float two_sum_err(float a, float b, float s)
{
    const float bb = __fsub_rn(s, a);
    return __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ float scale2f_apply(long long T, const Scale2f& s, float b0)
{
    const bool neg = T < 0;
    const unsigned long long A = neg ? 0ull - (unsigned long long)T : (unsigned long long)T;
    auto chunk = [](uint32_t c) { return __fsub_rn(__uint_as_float(0x4B000000u | c), 8388608.0f); };
    const float F0 = chunk((uint32_t)(A & 0x7fffffu));
    const float F1 = __fmul_rn(chunk((uint32_t)((A >> 23) & 0x7fffffu)), 8388608.0f);
    const float F2 = __fmul_rn(chunk((uint32_t)(A >> 46)), 70368744177664.0f);
    const float h = neg ? -s.hi : s.hi;
    const float l = neg ? -s.lo : s.lo;
    const float q2 = __fmul_rn(F2, h), r2 = __fmaf_rn(F2, h, -q2);
    const float q1 = __fmul_rn(F1, h), r1 = __fmaf_rn(F1, h, -q1);
    const float q0 = __fmul_rn(F0, h), r0 = __fmaf_rn(F0, h, -q0);
    const float u1 = __fadd_rn(q2, q1);
    float t = two_sum_err(q2, q1, u1);
    const float u = __fadd_rn(u1, q0);
    t = __fadd_rn(t, two_sum_err(u1, q0, u));
    t = __fadd_rn(t, __fadd_rn(__fadd_rn(r2, r1), r0));
    t = __fmaf_rn(F2, l, t);
    t = __fmaf_rn(F1, l, t);
    t = __fmaf_rn(F0, l, t);
    const int e1 = s.e >> 1;
    const float p1 = pow2f(e1), p2 = pow2f(s.e - e1);       // 2^e in two exact steps
    const float U = __fmul_rn(__fmul_rn(u, p1), p2);
    const float V = __fmul_rn(__fmul_rn(t, p1), p2);
    const float w = __fadd_rn(U, b0);
    return __fadd_rn(w, __fadd_rn(two_sum_err(U, b0, w), V));
}

__host__ __device__ inline int codes_per_word(int bits) { return 32 / bits; }

// Per-solve device state, placed at the start of the solver workspace.
struct State {
    double mu;             // step size of the current proposal
    double num;            // ||g_G||^2 of this iteration
    double resid2;         // ||Q(y) - Q2 x||^2 after the last accepted iterate
    double mu_accepted;    // step size of the last accepted iterate
    int iter;              // completed iterations
    int changed;           // 1 if the current proposal's support differs from G
    int bt;                // shrinks in the current iteration
    int stop;              // 1: nothing left to do (done, converged, error)
    int status;            // qiht_status
    int union_count;       // entries of the (G' u G) list of x' - x
    unsigned rmax_bits;    // float bits of max |r|
    int backtracks_total;
    int support_changes_total;
    float kth0, kth1;      // s-th and (s+1)-th |x + mu g| of the current proposal
    int iters;             // requested iterations
    int outer_guard;       // executions of the outer loop body (bounds the loop)
    int again;             // 1 if the last backtracking test asked for another shrink
    unsigned tau_bits;     // candidate threshold of the next selection (float bits, 0 = none)
    unsigned cand_count;   // keys >= tau found by the filter
    unsigned below_max;    // largest key < tau seen by the filter
    int full_selects;      // selections that ranked all n entries
    unsigned tau_g_bits;   // |g| threshold of the gradient kernel's candidates (float bits, 0 = off)
    unsigned gcand_count;  // entries outside G with |g| >= tau_g appended by the gradient kernel
    unsigned bmax_g;       // largest |g| (float bits) outside G below tau_g
    unsigned omega_uses;   // backtracking-test rounds of the fast iteration kernel so far
    unsigned dec_uses;     // uses of the fast iteration kernel's decision word so far
    int resid_logged;      // last iteration whose ||r||^2 is in resid2, the trace and the report
    unsigned long long t_phase[8];   // device clock at phase boundaries of the last iteration
    unsigned long long bar_count;    // grid-barrier arrivals of the iteration kernel (only grows)
    unsigned long long dec_word;     // fast iteration kernel: CTA 0's tagged decision (starts with tag 1)
    unsigned counters[2][1024];  // arrival counters of the column-subset products (row 0; the
                                 // iteration kernel's commit counter is word 2)
};

// Column-subset product modes (one epilogue each).
enum GatherMode { kGatherPlain = 0, kGatherMu = 1, kGatherOmega = 2, kGatherResid = 3 };

struct GatherArgs {
    Codes Q;
    const int32_t* cols;      // list of column indices
    const float* coef;        // list of coefficients
    int count;                // list length (host-known upper bound when count_dev != nullptr)
    const int* count_dev;     // device list length (nullptr: use count)
    float* z;                 // plain mode: output z (rows)
    float* partial;           // [chunks][rows_pad] partial sums
    double* rb_partial;       // [row_blocks][2] per-row-block sums
    double* chunk_partial;    // [chunks] sums of squared coefficients per chunk (Mu, Omega)
    unsigned* counters;       // [row_blocks + 1]
    int mode;
    // solver fields (modes Mu, Omega, Resid)
    State* st;
    const float* g;           // Mu: gradient
    const int32_t* support;   // Mu: current support G (s entries)
    const float* yhat;        // Resid: dequantized observation
    float* r;                 // Resid: residual output
    float* x;                 // Resid: dense iterate (committed)
    int32_t* support_out;     // Resid: support to commit into (the caller's support array)
    const int32_t* new_sel;   // Resid: G' (s entries)
    const float* new_val;     // Resid: x' values on G'
    int s;
    double k, c;              // backtracking parameters
    int max_bt;
    unsigned long long h_outer, h_bt;   // conditional graph handles (0 when not in a graph)
    qiht_report* report;
    qiht_trace trace;
    int coef_from_g;          // plain mode: coefficients g[cols[q]] instead of coef[q]
    const float* zx;          // Mu: alpha Q1_G g_G (the first quantization's image; non-null: the
                              //     cross-product step size of QIHT_MU_CROSS)
    double tol;               // Resid: stop once ||r||^2 <= tol (0: off)
};

struct GemvTArgs {
    Codes Q;
    const float* r;
    const unsigned* rmax_bits;  // float bits of max |r| (device)
    float* g;
    State* st;                  // non-null in the solver: skip when st->stop
    unsigned long long h_outer; // outer-loop handle (solver loop body only): set by thread 0 of CTA 0
    int guard_limit;            // loop-body executions allowed (bounds the outer loop)
    unsigned* err;              // optional: set to 1 when a device-side wait runs out (no solver state)
    // solver loop body with the fast-path iteration kernel (nullptr elsewhere)
    const int32_t* pos;         // position of every column in the support G, -1 outside
    float* gsup;                // out: g on G, by position
    unsigned long long* gcand;  // out: columns outside G with |g| >= st->tau_g_bits: (g bits << 32) | column
    int gcap;                   // capacity of gcand (st->gcand_count counts past it)
    // fast path: max |r| comes from the iteration kernel's residual partial slots (instead of
    // st->rmax_bits), and after the last iteration the first product records ||r||^2
    const double* rpart;        // partial slots [kPartSlots][kSlotCtas] (nullptr: use rmax_bits)
    int rgrid;                  // CTAs of the iteration kernel
    qiht_report* report;
    double* trace_resid2;       // optional
    double tol;                 // fast path: stop once the recorded ||r||^2 <= tol (0: off)
};

struct TopArgs {
    const float* g;
    const float* x;             // dense iterate (nullptr: zero)
    const double* mu;           // step (nullptr: 1)
    int n, s;
    int32_t* sel;               // G' (ascending)
    float* val;                 // x' values on G'
    float* kth;                 // optional [2]
    // solver fields
    State* st;
    const int32_t* support;     // current support G (compare / union)
    int32_t* uni;               // union list (2s)
    float* delta;               // x' - x on the union list
    int init;                   // 1: initial selection written straight into `support_init`
    int32_t* support_init;
    qiht_trace trace;
    unsigned long long h_bt;    // backtracking-loop handle: cleared on entry, set later by the Omega product
    unsigned long long* cand;   // candidate keys from the filter: (key << 32) | ~index
    int cap;                    // candidate capacity (0: no filter, always the full select)
};

struct InitArgs {
    Codes Y;
    const Codes* Q1;            // unused on device; scales are checked through these pointers
    const float* scale_q1;
    const float* scale_q2;
    float* yhat;
    float* r;
    float* x;
    int32_t* pos;               // optional: position map of the fast path, set to -1
    double* part;               // optional: tagged partial slots of the fast path, set to tag 1
    int n, m, s, iters;
    State* st;
    qiht_report* report;
    qiht_trace trace;
};

// Kernel node builders (each translation unit owns its kernels). argbuf[0] points at the
// kernel's argument struct, owned by the caller.
void gemv_t_node(const GemvTArgs& a, int num_sms, cudaKernelNodeParams* p, void** argbuf);
void gather_node(const GatherArgs& a, cudaKernelNodeParams* p, void** argbuf);
void top_node(const TopArgs& a, cudaKernelNodeParams* p, void** argbuf);
void top_filter_node(const TopArgs& a, cudaKernelNodeParams* p, void** argbuf);
constexpr int kTopCandCap = 4096;
void init_node(const InitArgs& a, cudaKernelNodeParams* p, void** argbuf);

// Direct launches (building blocks).
cudaError_t launch_absmax(const float* in, int rows, int cols, int64_t ld, float* scale, cudaStream_t s);
// words2 != nullptr: a second quantization (stream_id2) of the same input in the same pass.
cudaError_t launch_quantize(const float* in, int rows, int cols, int64_t ld, int bits, uint64_t seed,
                            uint32_t stream_id, uint32_t* words, int ld_words, const float* scale,
                            cudaStream_t s, uint32_t stream_id2 = 0, uint32_t* words2 = nullptr,
                            int levels = 0);
cudaError_t launch_gemv_t(const GemvTArgs& a, int num_sms, cudaStream_t s);
cudaError_t launch_gather(const GatherArgs& a, cudaStream_t s);
cudaError_t launch_fresh_resid(const Codes& Y, const float* z, float* yhat, float* r, int m, unsigned* rmax_bits,
                               cudaStream_t s);
cudaError_t launch_top(const TopArgs& a, cudaStream_t s);

// One iteration after the gradient product as one persistent kernel (iter.cu).
struct IterArgs;
constexpr size_t kIterArgsMax = 1024;     // bytes reserved for the iteration kernel's arguments

int iter_grid();
bool iter_fast(int s);                    // the fast-path iteration kernel serves this support size
// Buffers of the fast path (ignored by the other kernel).
struct IterFastBufs {
    int32_t* pos;                         // n
    float* xs;                            // s
    float* gsup;                          // s
    unsigned long long* gcand;            // gcap
    int gcap;
};
void iter_node(const Codes& Q2, State* st, const float* g, float* x, int32_t* support, int32_t* sel, float* val,
               int32_t* uni, float* delta, const float* yhat, float* r, uint32_t* keys, unsigned long long* cand,
               double* part, const IterFastBufs& fb, int n, int m, int s, double k, double c, int max_bt,
               int flags, qiht_report* report, const qiht_trace& trace, cudaKernelNodeParams* p, void* argstore,
               void** argbuf, const uint32_t* q1_words = nullptr, int mu_mode = 0, double tol = 0.0);
size_t iter_args_bytes();

// Many independent problems in one persistent launch (batched.cu).
size_t batched_smem();
// lpc: lanes per column (4, 8, 16 or 32) of the gradient product, the tile shape the
// autotuner picked for these problems' size.
cudaError_t launch_batched(const qiht_problem* probs, const int* order, int nprob, int bits, int lpc, int iters,
                           double k, double c, int max_bt, unsigned* next, cudaStream_t s);

// Host-side checks shared by the entry points (solve.cu).
qiht_status check_codes(const qiht_codes* Q);   // pointers, bits, sizes, ld_words, levels, alignment
Codes view(const qiht_codes* Q);
void note_cuda_error(const char* what, cudaError_t e);

// Gradient of many right-hand sides on the tensor cores (mrhs_gemm.cu).
size_t mrhs_gemm_smem();
int mrhs_pad_rhs(int nrhs);               // right-hand sides rounded up to the N tile
int mrhs_pad_rows(int m);                 // rows rounded up to the K stage
constexpr size_t kMrhsMapBytes = 128;     // a CUtensorMap
cudaError_t mrhs_make_map(void* map, const void* R16, int mk, int rows);
cudaError_t launch_mrhs_split(const float* R, long long ldr, int m, int nrhs, void* R16, float* sc,
                              const float* scale, int lm1, cudaStream_t s);
cudaError_t launch_mrhs_gemm(const Codes& Q, const void* map, const float* sc, float* G, long long ldg, int nrhs,
                             int* status, cudaStream_t s, bool fp8 = false);
// FP8 variant (codes of at most 4 bits): the residual as three e4m3 terms, rows padded to 64
size_t mrhs_gemm_smem8();
int mrhs_pad_rows8(int m);
cudaError_t mrhs_make_map8(void* map, const void* R8, int mk, int rows);
cudaError_t launch_mrhs_split8(const float* R, long long ldr, int m, int nrhs, void* R8, float* sc,
                               const float* scale, int lm1, cudaStream_t s);
constexpr int kMrhsTerms8 = 3;

// float -> e4m3 byte (round to nearest, saturating) and back; the converted pair holds the
// value twice, so the byte taken does not depend on the pair's packing order
__device__ __forceinline__ uint32_t f_to_e4m3(float v)
{
    uint16_t r;
    asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %1;" : "=h"(r) : "f"(v));
    return (uint32_t)r & 0xffu;
}

__device__ __forceinline__ float e4m3_to_f(uint32_t b)
{
    const uint16_t pair = (uint16_t)(b * 0x0101u);
    uint32_t h2;
    asm("cvt.rn.f16x2.e4m3x2 %0, %1;" : "=r"(h2) : "h"(pair));
    return __half2float(__ushort_as_half((unsigned short)(h2 & 0xffffu)));
}

// Per-right-hand-side iterations after the gradient product (mrhs_step.cu).
struct MrhsState {
    double mu;                // last accepted step size
    double resid2;            // ||Q(y) - Q2 x||^2 of the current iterate
    int stop;                 // 0 running, 1 converged, 2 stopped by an error (status)
    int status;
    int iters_run, backtracks, changes, full_selects;   // full_selects: selections that ranked all n keys
};
struct MrhsStepArgs {
    Codes Q2;
    const float* scale1;      // scale of Q1 (alpha1 of the next gradient product)
    int lm1_1;                // levels - 1 of Q1
    const qiht_codes* ydesc;  // nrhs observation codes [device]
    float* yhat;              // nrhs x m dequantized observations (written by the init kernel)
    float* resid;             // nrhs x m residuals
    float* zmu;               // nrhs x m: Q2_G g_G of the current step size (unscaled)
    const float* G;           // nrhs x n gradients
    int32_t* sup;             // nrhs x s supports (ascending)
    float* xs;                // nrhs x s values on them
    __half* R16;              // f16 residual parts: rows k (hi) and rhi + k (lo), mk halves each
    float* sc;                // alpha1 2^e_k
    int mk, rhi;
    MrhsState* st;
    int n, m, s, nrhs;
    double kk, cc;
    int max_bt;
    int mode;                 // 0: initial support, 1: an iteration
    int last;                 // 1: no gradient product follows (skip the split)
    int refresh;              // 1: form the residual directly (else update it)
    int fp8;                  // 1: the next gradient product takes e4m3 terms (R16's bytes reused:
                              //    term t of right-hand side k at row t * rhi + k, mk8 bytes each)
    int mk8;
};
size_t mrhs_step_smem(int n, int mk, int s);
cudaError_t launch_mrhs_init(const MrhsStepArgs& a, cudaStream_t s);
cudaError_t launch_mrhs_step(const MrhsStepArgs& a, int bits, cudaStream_t s);
cudaError_t launch_mrhs_final(const MrhsStepArgs& a, float* X, qiht_report* reports, const int* gemm_status,
                              cudaStream_t s);

// K unrolled iterations and their adjoint for many problems (unrolled.cu).
struct UdArgs {
    const qiht_codes* q1;     // nprob descriptors [device]
    const qiht_codes* q2;
    const float* y;           // P x 2m observations
    const float* ga;          // P x m gains (real parts)
    const float* gb;          // P x m gains (imaginary parts)
    int P, m, n, s, mk;
    int32_t* sup;             // P x s: support of the current iterate (ascending)
    float* xs;                // P x s: its values
    float* vin;               // P x m: a r_top + b r_bot of the current iterate
    float* r;                 // P x 2m: y - A2 x
    float* q;                 // P x m: Phi2 x
    float* h;                 // P x n: the current gradient A1^T r
    // record of a segment (rec_r == nullptr: not recording); slot = step - first step
    float* rec_r;             // P x c x 2m
    float* rec_q;             // P x c x m
    float* rec_u;             // P x c x m: Phi2 P h
    int32_t* rec_G;           // P x c x s
    int32_t* rec_Gn;          // P x c x s
    float* rec_hG;            // P x c x s: h on G_t
    float* rec_hGn;           // P x c x s: h on G_{t+1}
    double* rec_sc;           // P x c x 4: mu, ||P h||^2, ||A2 P h||^2
    int c, slot, t;
    // operand of the next dense product: the vector in fixed point (byte planes, shift, sum)
    uint32_t* pl;             // P x pl_stride words
    size_t pl_stride;
    int* pl_sh;               // P
    long long* pl_rs;         // P
};
size_t ud_fwd_smem(int n, int mk, int s);
size_t ud_bwd_smem(int n, int mk, int s);
cudaError_t launch_ud_init(const UdArgs& a, cudaStream_t s);
cudaError_t launch_ud_xout(const UdArgs& a, float* X, cudaStream_t s);
cudaError_t launch_ud_planes(const UdArgs& a, int bits, const float* v, cudaStream_t s);
cudaError_t launch_ud_gemvt(const UdArgs& a, const qiht_codes* Qs, int bits, const float* base, float sign, float* out,
                            int ldw, cudaStream_t s);
cudaError_t launch_ud_fwd(const UdArgs& a, int bits, cudaStream_t s);
cudaError_t launch_ud_bwd(const UdArgs& a, int bits, const float* xbar, float* vbase, float* vv, float* ybar,
                          float* gabar, float* gbbar, cudaStream_t s);

int gather_row_blocks(int rows, int bits);
int gather_chunks(int count);
size_t gather_partial_floats(int rows, int bits, int count);
size_t top_smem_bytes(int n);
int num_sms();

// H_s over more keys than one CTA holds (bigsel.cu): keys |fmaf(mu, g, x)| (|g| when x is null),
// exactly s kept, ties to the lower index, indices ascending; workspace big_top_workspace(n).
constexpr int kMaxBigTopN = 1 << 24;
size_t big_top_workspace(int n);
cudaError_t launch_big_top(const float* g, const float* x, const double* mu, int n, int s, int32_t* sel, float* val,
                           float* kth, void* ws, cudaStream_t st);

// Phi computed on the fly (fly.cu): the operator's limits, codes of one or two quantizations,
// and the fused generate + quantize + GEMV^T (scale = max |table| written by both).
bool fly_op_ok(const qiht_fly_op* op);
cudaError_t launch_fly_quantize(const qiht_fly_op* op, int bits, int levels, uint64_t seed, uint32_t s0, uint32_t s1,
                                uint32_t* w0, uint32_t* w1, int ldw, float* scale, cudaStream_t s);
cudaError_t launch_fly_gemv_t(const qiht_fly_op* op, int bits, int levels, uint64_t seed, uint32_t stream_id,
                              const float* r, float* g, float* scale, cudaStream_t s);

}  // namespace qiht
