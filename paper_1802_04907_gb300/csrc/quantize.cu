// Stochastic quantizer Q(v, b) (Section III-A) with max-abs scaling c_v
// (Appendix, quantization-error lemma), emitting the column-packed code layout.
#include "internal.cuh"

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
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

__device__ __forceinline__ uint32_t abs_bits(float v)
{
    // |v| as an unsigned key: monotone for finite values, Inf above them, NaN above Inf
    return __float_as_uint(v) & 0x7fffffffu;
}

// c = max |v| over a row-major rows x cols block (row stride ld), by atomicMax on the key.
__global__ void __launch_bounds__(256) k_absmax(const float* __restrict__ in, int rows, int cols,
                                                long long ld, unsigned* __restrict__ out)
{
    unsigned mx = 0;
    const long long total = (long long)rows * cols;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    if (ld == cols && ((reinterpret_cast<uintptr_t>(in) & 15) == 0)) {
        const float4* in4 = reinterpret_cast<const float4*>(in);
        const long long n4 = total >> 2;
        for (long long i = tid; i < n4; i += stride) {
            float4 v;
            asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
                         : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(in4 + i));
            mx = max(mx, max(max(abs_bits(v.x), abs_bits(v.y)), max(abs_bits(v.z), abs_bits(v.w))));
        }
        for (long long i = (n4 << 2) + tid; i < total; i += stride) mx = max(mx, abs_bits(in[i]));
    } else {
        for (long long i = tid; i < total; i += stride) {
            const long long r = i / cols, c = i - r * cols;
            mx = max(mx, abs_bits(in[r * ld + c]));
        }
    }
    mx = __reduce_max_sync(0xffffffffu, mx);
    __shared__ unsigned wmax[8];
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned b = wmax[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) b = max(b, wmax[w]);
        atomicMax(out, b);
    }
}

// One rounding decision in binary32, every operation correctly rounded:
// t = (v / c + 1) * (L-1)/2, code = floor(t) + (u < t - floor(t)).
__device__ __forceinline__ uint32_t quant_code(float v, float c, float half, int L, float u)
{
    const float vt = (c > 0.0f) ? __fdiv_rn(v, c) : 0.0f;
    float t = __fmul_rn(__fadd_rn(vt, 1.0f), half);
    t = fminf(fmaxf(t, 0.0f), (float)(L - 1));
    const float fi = floorf(t);
    const float f = __fsub_rn(t, fi);
    int code = (int)fi + (u < f ? 1 : 0);
    return (uint32_t)min(code, L - 1);
}

constexpr int kQTileRows = 128;
constexpr int kQTileCols = 32;

// Quantize tiles of 128 rows x 32 columns: the tile is staged transposed in
// shared memory (coalesced reads of the row-major input), then every thread
// packs whole words of one column (coalesced writes of the column-packed output).
template <int BITS>
__global__ void __launch_bounds__(256) k_quantize(const float* __restrict__ in, int rows, int cols,
                                                  long long ld, uint64_t seed, uint32_t stream_id,
                                                  uint32_t* __restrict__ words, int ldw,
                                                  const float* __restrict__ scale_p)
{
    constexpr int G = 32 / BITS;
    constexpr int L = 1 << BITS;
    constexpr int WPC = kQTileRows / G;                   // words per column per tile
    constexpr int WPT = WPC * kQTileCols / 256;           // words per thread per tile
    __shared__ float tile[kQTileCols][kQTileRows + 1];

    const float c = *scale_p;
    const float half = (float)(L - 1) * 0.5f;
    const uint32_t key0 = (uint32_t)seed, key1 = (uint32_t)(seed >> 32);
    const int row_tiles = (ldw * G + kQTileRows - 1) / kQTileRows;
    const int col_tiles = (cols + kQTileCols - 1) / kQTileCols;
    const long long ntiles = (long long)row_tiles * col_tiles;

    for (long long tile_id = blockIdx.x; tile_id < ntiles; tile_id += gridDim.x) {
        const int rt = (int)(tile_id % row_tiles);
        const int ct = (int)(tile_id / row_tiles);
        const int r0 = rt * kQTileRows, c0 = ct * kQTileCols;
#pragma unroll 4
        for (int k = 0; k < kQTileRows * kQTileCols / 256; ++k) {
            const int idx = threadIdx.x + 256 * k;
            const int rr = idx >> 5, cc = idx & 31;
            const int i = r0 + rr, j = c0 + cc;
            tile[cc][rr] = (i < rows && j < cols) ? in[(long long)i * ld + j] : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < WPT; ++k) {
            const int w = threadIdx.x + 256 * k;
            const int cc = w / WPC, q = w % WPC;
            const int j = c0 + cc;
            const int qg = r0 / G + q;
            if (j < cols && qg < ldw) {
                const int i0 = qg * G;
                const uint64_t e0 = (uint64_t)j * (uint64_t)rows + (uint64_t)i0;
                uint64_t cur = ~0ull;
                uint4 rnd = make_uint4(0, 0, 0, 0);
                uint32_t word = 0;
#pragma unroll
                for (int kk = 0; kk < G; ++kk) {
                    if (i0 + kk < rows) {
                        const uint64_t e = e0 + kk;
                        const uint64_t qq = e >> 2;
                        if (qq != cur) {
                            rnd = philox4x32_10(make_uint4((uint32_t)qq, (uint32_t)(qq >> 32), stream_id, 0u),
                                                key0, key1);
                            cur = qq;
                        }
                        const uint32_t sel = e & 3;
                        const uint32_t rw = sel == 0 ? rnd.x : sel == 1 ? rnd.y : sel == 2 ? rnd.z : rnd.w;
                        const float u = (float)(rw >> 8) * 0x1p-24f;
                        const uint32_t code = quant_code(tile[cc][q * G + kk], c, half, L, u);
                        word |= code << (8 * (kk & 3) + BITS * (kk >> 2));
                    }
                }
                words[(size_t)j * ldw + qg] = word;
            }
        }
        __syncthreads();
    }
}

cudaError_t launch_absmax(const float* in, int rows, int cols, int64_t ld, float* scale, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(scale, 0, sizeof(float), s);
    if (e != cudaSuccess) return e;
    const long long total = (long long)rows * cols;
    long long blocks = (total / 4 + 255) / 256;
    const long long cap = (long long)num_sms() * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k_absmax<<<(unsigned)blocks, 256, 0, s>>>(in, rows, cols, ld, reinterpret_cast<unsigned*>(scale));
    return cudaGetLastError();
}

cudaError_t launch_quantize(const float* in, int rows, int cols, int64_t ld, int bits, uint64_t seed,
                            uint32_t stream_id, uint32_t* words, int ld_words, const float* scale,
                            cudaStream_t s)
{
    const int G = 32 / bits;
    const long long tiles = (long long)((ld_words * G + kQTileRows - 1) / kQTileRows) *
                            ((cols + kQTileCols - 1) / kQTileCols);
    long long blocks = tiles;
    const long long cap = (long long)num_sms() * 8;
    if (blocks > cap) blocks = cap;
    switch (bits) {
    case 2: k_quantize<2><<<(unsigned)blocks, 256, 0, s>>>(in, rows, cols, ld, seed, stream_id, words, ld_words, scale); break;
    case 4: k_quantize<4><<<(unsigned)blocks, 256, 0, s>>>(in, rows, cols, ld, seed, stream_id, words, ld_words, scale); break;
    case 8: k_quantize<8><<<(unsigned)blocks, 256, 0, s>>>(in, rows, cols, ld, seed, stream_id, words, ld_words, scale); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace qiht
