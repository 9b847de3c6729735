// Stochastic quantizer Q(v, b) (Section III-A) with max-abs scaling c_v
// (Appendix, quantization-error lemma), emitting the column-packed code layout.
#include "internal.cuh"
#include "quant_rng.cuh"

namespace qiht {

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

constexpr int kQTileRows = 128;
constexpr int kQTileCols = 32;

// Quantize tiles of 128 rows x 32 columns with NS independent random streams at once
// (NS = 2: the two quantizations Q1, Q2 of the same matrix in one pass). The tile is
// read as float4 (coalesced, row-major input), staged transposed in shared memory, and
// every thread packs whole words of one column (coalesced writes of the column-packed
// output); the next tile's loads are in flight while this one is packed. The rounding
// decision of an element is computed once and shared by the streams.
template <int BITS, int NS>
__global__ void __launch_bounds__(256) k_quantize(const float* __restrict__ in, int rows, int cols,
                                                  long long ld, PhiloxKeys keys, uint32_t stream0, uint32_t stream1,
                                                  uint32_t* __restrict__ words0, uint32_t* __restrict__ words1,
                                                  int ldw, const float* __restrict__ scale_p, int lm1)
{
    constexpr int G = 32 / BITS;
    constexpr int WPC = kQTileRows / G;                   // words per column per tile
    constexpr int WPT = WPC * kQTileCols / 256;           // words per thread per tile
    constexpr int F4 = kQTileRows * kQTileCols / 4 / 256; // float4 loads per thread per tile
    __shared__ float tile[kQTileCols][kQTileRows + 1];

    const float c = *scale_p;
    const QScale qs = qscale(c);
    const float half = (float)lm1 * 0.5f;
    const int row_tiles = (ldw * G + kQTileRows - 1) / kQTileRows;
    const int col_tiles = (cols + kQTileCols - 1) / kQTileCols;
    const long long ntiles = (long long)row_tiles * col_tiles;
    const bool vec = (ld % 4 == 0) && ((reinterpret_cast<uintptr_t>(in) & 15) == 0);

    // thread t reads float4 f = t + 256 k: row f / 8 of the tile, columns 4 (f % 8) .. + 3
    auto fetch = [&](long long tid, float4 (&v)[F4]) {
        const int rt = (int)(tid % row_tiles), ct = (int)(tid / row_tiles);
        const int r0 = rt * kQTileRows, c0 = ct * kQTileCols;
#pragma unroll
        for (int k = 0; k < F4; ++k) {
            const int f = threadIdx.x + 256 * k;
            const int i = r0 + (f >> 3), j = c0 + 4 * (f & 7);
            const float* src = in + (long long)i * ld + j;
            if (vec && i < rows && j + 3 < cols) {
                asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
                             : "=f"(v[k].x), "=f"(v[k].y), "=f"(v[k].z), "=f"(v[k].w) : "l"(src));
            } else {
                v[k].x = (i < rows && j < cols) ? src[0] : 0.0f;
                v[k].y = (i < rows && j + 1 < cols) ? src[1] : 0.0f;
                v[k].z = (i < rows && j + 2 < cols) ? src[2] : 0.0f;
                v[k].w = (i < rows && j + 3 < cols) ? src[3] : 0.0f;
            }
        }
    };
    float4 pre[F4];
    long long tile_id = blockIdx.x;
    if (tile_id < ntiles) fetch(tile_id, pre);
    for (; tile_id < ntiles; tile_id += gridDim.x) {
        const int rt = (int)(tile_id % row_tiles);
        const int ct = (int)(tile_id / row_tiles);
        const int r0 = rt * kQTileRows, c0 = ct * kQTileCols;
#pragma unroll
        for (int k = 0; k < F4; ++k) {
            const int f = threadIdx.x + 256 * k;
            const int rr = f >> 3, cq = 4 * (f & 7);
            tile[cq][rr] = pre[k].x;
            tile[cq + 1][rr] = pre[k].y;
            tile[cq + 2][rr] = pre[k].z;
            tile[cq + 3][rr] = pre[k].w;
        }
        __syncthreads();
        if (tile_id + gridDim.x < ntiles) fetch(tile_id + gridDim.x, pre);
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
                uint4 rnd[NS];
                uint32_t word[NS];
#pragma unroll
                for (int st = 0; st < NS; ++st) { rnd[st] = make_uint4(0, 0, 0, 0); word[st] = 0; }
#pragma unroll
                for (int kk = 0; kk < G; ++kk) {
                    if (i0 + kk < rows) {
                        const uint64_t e = e0 + kk;
                        const uint64_t qq = e >> 2;
                        if (qq != cur) {
#pragma unroll
                            for (int st = 0; st < NS; ++st)
                                rnd[st] = philox4x32_10_keys(
                                    make_uint4((uint32_t)qq, (uint32_t)(qq >> 32), st == 0 ? stream0 : stream1, 0u),
                                    keys);
                            cur = qq;
                        }
                        const uint32_t sel = e & 3;
                        const Decision d = quant_decide(tile[cc][q * G + kk], qs, half, lm1);
#pragma unroll
                        for (int st = 0; st < NS; ++st) {
                            const uint32_t rw = sel == 0 ? rnd[st].x : sel == 1 ? rnd[st].y : sel == 2 ? rnd[st].z : rnd[st].w;
                            const float u = (float)(rw >> 8) * 0x1p-24f;
                            word[st] |= quant_code(d, lm1, u) << (8 * (kk & 3) + BITS * (kk >> 2));
                        }
                    }
                }
                words0[(size_t)j * ldw + qg] = word[0];
                if (NS == 2) words1[(size_t)j * ldw + qg] = word[NS - 1];
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
                            cudaStream_t s, uint32_t stream_id2, uint32_t* words2, int levels)
{
    const PhiloxKeys keys = philox_keys(seed);   // the ten round keys, as launch constants
    if (levels <= 0) levels = 1 << bits;
    const int lm1 = levels - 1;
    const int G = 32 / bits;
    const long long tiles = (long long)((ld_words * G + kQTileRows - 1) / kQTileRows) *
                            ((cols + kQTileCols - 1) / kQTileCols);
    long long blocks = tiles;
    const long long cap = (long long)num_sms() * 8;
    if (blocks > cap) blocks = cap;
    const unsigned nb = (unsigned)blocks;
    const bool two = words2 != nullptr;
    switch (bits) {
    case 2:
        if (two) k_quantize<2, 2><<<nb, 256, 0, s>>>(in, rows, cols, ld, keys, stream_id, stream_id2, words, words2, ld_words, scale, lm1);
        else k_quantize<2, 1><<<nb, 256, 0, s>>>(in, rows, cols, ld, keys, stream_id, stream_id, words, words, ld_words, scale, lm1);
        break;
    case 4:
        if (two) k_quantize<4, 2><<<nb, 256, 0, s>>>(in, rows, cols, ld, keys, stream_id, stream_id2, words, words2, ld_words, scale, lm1);
        else k_quantize<4, 1><<<nb, 256, 0, s>>>(in, rows, cols, ld, keys, stream_id, stream_id, words, words, ld_words, scale, lm1);
        break;
    case 8:
        if (two) k_quantize<8, 2><<<nb, 256, 0, s>>>(in, rows, cols, ld, keys, stream_id, stream_id2, words, words2, ld_words, scale, lm1);
        else k_quantize<8, 1><<<nb, 256, 0, s>>>(in, rows, cols, ld, keys, stream_id, stream_id, words, words, ld_words, scale, lm1);
        break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace qiht
