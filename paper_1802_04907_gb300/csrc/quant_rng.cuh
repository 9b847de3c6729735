// Device pieces of the stochastic quantizer Q(v, b) (Section III-A) shared by the
// kernels that produce codes: the random numbers and the binary32 rounding decision.
// Every producer of codes goes through these, so codes of the same value, seed, stream
// and element index are identical whichever kernel makes them.
#pragma once
#include <cstdint>

namespace qiht {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel Random Numbers: As Easy
// as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplications with the
// published multipliers, the key bumped by the published Weyl constants.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        // one 32 x 32 -> 64-bit product per multiplier gives both halves
        const uint64_t p0 = (uint64_t)0xD2511F53u * c.x, p1 = (uint64_t)0xCD9E8D57u * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k1, (uint32_t)p0);
    }
    return c;
}

// The same generator with the ten round keys given (key (k0, k1) bumped r times for round r),
// for kernels that pass them as launch parameters: the rounds then take their keys as
// constant operands instead of recomputing them per call.
struct PhiloxKeys {
    uint32_t k0[10], k1[10];
};

inline PhiloxKeys philox_keys(uint64_t seed)
{
    PhiloxKeys k;
    uint32_t a = (uint32_t)seed, b = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        k.k0[r] = a;
        k.k1[r] = b;
        a += 0x9E3779B9u;
        b += 0xBB67AE85u;
    }
    return k;
}

__device__ __forceinline__ uint4 philox4x32_10_keys(uint4 c, const PhiloxKeys& k)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c.x, p1 = (uint64_t)0xCD9E8D57u * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k.k0[round], (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k.k1[round],
                       (uint32_t)p0);
    }
    return c;
}

// One rounding decision in binary32, every operation correctly rounded, on a grid of
// `levels` points (lm1 = levels - 1 intervals): t = (v / c + 1) * lm1/2, clamped to
// [0, lm1]; fi = floor(t), f = t - fi. The code is fi + (u < f) (at most lm1); the
// decision does not depend on u, so several quantizations of the same value share it.
struct Decision {
    float fi, f;
};

// The scale of a quantization with its reciprocal, for the decision's v / c by Markstein's FMA
// division: y = RN(1/c) once, then q = RN(v y), r = RN(v - c q) and RN(q + r y), each FMA
// rounded once. Against __fdiv_rn over every binary32 v in [0, c] for 16 scales c (among them
// 2^-100 and 2^100) it differed only where |v/c| < 2^-25; there 1 + v/c rounds to 1, so the
// decision is the same either way. A CPU test replays the steps in exact arithmetic on random
// pairs and checks the same. Scales outside [2^-125, 2^125] (where y could be subnormal) take
// __fdiv_rn.
struct QScale {
    float c, y;
    bool fast;
};

__device__ __forceinline__ QScale qscale(float c)
{
    const bool fast = c >= 0x1p-125f && c <= 0x1p125f;
    return QScale{c, fast ? __frcp_rn(c) : 0.0f, fast};
}

__device__ __forceinline__ Decision quant_decide(float v, const QScale& s, float half, int lm1)
{
    const float c = s.c;
    float vt = 0.0f;
    if (s.fast) {
        const float q = __fmul_rn(v, s.y);
        vt = __fmaf_rn(__fmaf_rn(-c, q, v), s.y, q);
    } else if (c > 0.0f) {
        vt = __fdiv_rn(v, c);
    }
    float t = __fmul_rn(__fadd_rn(vt, 1.0f), half);
    t = fminf(fmaxf(t, 0.0f), (float)lm1);
    const float fi = floorf(t);
    return Decision{fi, __fsub_rn(t, fi)};
}

__device__ __forceinline__ uint32_t quant_code(const Decision& d, int lm1, float u)
{
    const int code = (int)d.fi + (u < d.f ? 1 : 0);
    return (uint32_t)min(code, lm1);
}

}  // namespace qiht
