// Stand-alone codec kernels: encode a device field (input generation),
// decode an explicit list of blocks, and decode a whole volume into a
// dense field (the full-volume baseline of the paper's ZFP decompression
// measurements).
#include <algorithm>
#include <cstdint>

#include "codec.cuh"
#include "kernels.cuh"

namespace bcmc {

// One thread per block: gather the 4x4x4 samples (repeating the last
// sample past the volume edge), encode, then decode what was written to
// get the block's range over its in-volume decoded samples.
__global__ void __launch_bounds__(128) encode_kernel(const float *__restrict__ field, Geom g, uint64_t *bits,
                                                     float *bmin, float *bmax) {
    __shared__ uint64_t planes[32 * 128];
    const uint32_t slab = g.nbx * g.nby;
    for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < g.nb; b += gridDim.x * blockDim.x) {
        const uint32_t bx = b % g.nbx, by = (b / g.nbx) % g.nby, bz = b / slab;
        float v[64];
#pragma unroll
        for (int k = 0; k < 4; k++)
#pragma unroll
            for (int j = 0; j < 4; j++)
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    const uint32_t x = min(4 * bx + i, g.nx - 1), y = min(4 * by + j, g.ny - 1),
                                   z = min(4 * bz + k, g.nz - 1);
                    v[i + 4 * j + 16 * k] = __ldg(field + (size_t)x + (size_t)g.nx * ((size_t)y + (size_t)g.ny * z));
                }
        uint64_t *w = bits + (size_t)b * g.rate;
        encode_block(v, g.rate, w);
        float d[64];
        decode_block<false>(w, g.rate, d, planes + threadIdx.x, blockDim.x);   // just written by this thread
        float lo = __int_as_float(0x7F800000), hi = __int_as_float(0xFF800000);   // +inf, -inf
#pragma unroll
        for (int k = 0; k < 4; k++)
#pragma unroll
            for (int j = 0; j < 4; j++)
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    if (4 * bx + i >= g.nx || 4 * by + j >= g.ny || 4 * bz + k >= g.nz) continue;
                    const float x = d[i + 4 * j + 16 * k];
                    if (x < lo) lo = x;
                    if (x > hi) hi = x;
                }
        bmin[b] = lo;
        bmax[b] = hi;
    }
}

__global__ void __launch_bounds__(128) decode_list_kernel(const uint64_t *__restrict__ bits, uint32_t rate,
                                                          const uint32_t *__restrict__ ids, uint64_t n, float *out) {
    __shared__ uint64_t planes[32 * 128];
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        float v[64];
        decode_block(bits + (size_t)ids[i] * rate, rate, v, planes + threadIdx.x, blockDim.x);
        float4 *dst = reinterpret_cast<float4 *>(out + i * 64);
#pragma unroll
        for (int q = 0; q < 16; q++) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    }
}

// One thread per block, blocks in id order: decode, then write the block's
// in-volume samples into the dense x-fastest field.  Threads of a warp hold
// consecutive blocks along x, so each row store of the warp covers one
// contiguous span of the field.
__global__ void __launch_bounds__(128) decode_volume_kernel(const uint64_t *__restrict__ bits, Geom g, float *field) {
    __shared__ uint64_t planes[32 * 128];
    const bool rows16 = (g.nx & 3u) == 0;       // every row starts 16-byte aligned
    for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < g.nb; b += gridDim.x * blockDim.x) {
        uint32_t bx, by, bz;
        block_coords(g, b, bx, by, bz);
        float v[64];
        decode_block(bits + (size_t)b * g.rate, g.rate, v, planes + threadIdx.x, blockDim.x);
        const uint32_t x0 = 4 * bx;
        const bool full_x = x0 + 4 <= g.nx;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const uint32_t z = 4 * bz + k;
            if (z >= g.nz) break;
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const uint32_t y = 4 * by + j;
                if (y >= g.ny) break;
                float *row = field + (size_t)x0 + (size_t)g.nx * ((size_t)y + (size_t)g.ny * z);
                if (rows16 && full_x) {
                    *reinterpret_cast<float4 *>(row) =
                        make_float4(v[16 * k + 4 * j], v[16 * k + 4 * j + 1], v[16 * k + 4 * j + 2], v[16 * k + 4 * j + 3]);
                } else {
#pragma unroll
                    for (int i = 0; i < 4; i++)
                        if (x0 + i < g.nx) row[i] = v[16 * k + 4 * j + i];
                }
            }
        }
    }
}

void launch_decode_volume(const uint64_t *bits, const Geom &g, float *field, cudaStream_t st) {
    const uint32_t blocks = std::max<uint32_t>(1, std::min<uint32_t>((g.nb + 127) / 128, 1u << 20));
    decode_volume_kernel<<<blocks, 128, 0, st>>>(bits, g, field);
}

void launch_encode(const float *field, const Geom &g, uint64_t *bits, float *bmin, float *bmax, cudaStream_t st) {
    const uint32_t blocks = std::max<uint32_t>(1, std::min<uint32_t>((g.nb + 127) / 128, 1u << 20));
    encode_kernel<<<blocks, 128, 0, st>>>(field, g, bits, bmin, bmax);
}

void launch_decode_list(const uint64_t *bits, uint32_t rate, const uint32_t *ids, uint64_t n, float *out,
                        cudaStream_t st) {
    if (n == 0) return;
    const uint64_t blocks = std::min<uint64_t>((n + 127) / 128, 1u << 20);
    decode_list_kernel<<<(unsigned)blocks, 128, 0, st>>>(bits, rate, ids, n, out);
}

}  // namespace bcmc
