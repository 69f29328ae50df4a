// Stand-alone codec kernels: encode a device field (input generation),
// decode an explicit list of blocks, and decode a whole volume into a
// dense field (the full-volume baseline of the paper's ZFP decompression
// measurements).
#include <algorithm>
#include <cstdint>

#include "codec.cuh"
#include "kernels.cuh"

namespace bcmc {

constexpr uint32_t kCodecThreads = 128;

// the codec kernels' dynamic shared memory (plane columns, group-step
// table, staging areas), with the table filled
__device__ __forceinline__ DecodeSmem codec_smem(uint64_t *base, uint32_t rate) {
    const DecodeSmem sm = decode_smem_layout(base, kCodecThreads, rate);
    load_group_table(sm.tab);
    __syncthreads();
    return sm;
}

// One thread per block: gather the 4x4x4 samples (repeating the last
// sample past the volume edge), encode, then decode what was written (the
// warp stages its blocks' new words) to get the block's range over its
// in-volume decoded samples.  Warps step over the blocks together.
__global__ void __launch_bounds__(kCodecThreads) encode_kernel(const float *__restrict__ field, Geom g, uint64_t *bits,
                                                               float *bmin, float *bmax) {
    extern __shared__ uint64_t dsm[];
    const DecodeSmem sm = codec_smem(dsm, g.rate);
    const uint32_t slab = g.nbx * g.nby;
    const uint32_t lane = threadIdx.x & 31u;
    for (uint32_t b0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); b0 < g.nb; b0 += gridDim.x * blockDim.x) {
        const uint32_t b = b0 + lane;
        const bool have = b < g.nb;
        if (have) {
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
                        v[i + 4 * j + 16 * k] =
                            __ldg(field + (size_t)x + (size_t)g.nx * ((size_t)y + (size_t)g.ny * z));
                    }
            encode_block(v, g.rate, bits + (size_t)b * g.rate);
        }
        __syncwarp();                                   // the words are written (and visible to the warp)
        stage_blocks<false>(bits, g.rate, b, have, sm.stage);
        if (!have) continue;
        const uint32_t bx = b % g.nbx, by = (b / g.nbx) % g.nby, bz = b / slab;
        float d[64];
        decode_staged(sm.stage + lane * (2u * g.rate + 1u), g.rate, sm.tab, d, sm.planes + threadIdx.x, blockDim.x);
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

__global__ void __launch_bounds__(kCodecThreads) decode_list_kernel(const uint64_t *__restrict__ bits, uint32_t rate,
                                                                    const uint32_t *__restrict__ ids, uint64_t n,
                                                                    float *out) {
    extern __shared__ uint64_t dsm[];
    const DecodeSmem sm = codec_smem(dsm, rate);
    const uint32_t lane = threadIdx.x & 31u;
    for (uint64_t i0 = blockIdx.x * (uint64_t)blockDim.x + (threadIdx.x & ~31u); i0 < n;
         i0 += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t i = i0 + lane;
        const bool have = i < n;
        stage_blocks<true>(bits, rate, have ? ids[i] : 0u, have, sm.stage);
        if (!have) continue;
        float v[64];
        decode_staged(sm.stage + lane * (2u * rate + 1u), rate, sm.tab, v, sm.planes + threadIdx.x, blockDim.x);
        float4 *dst = reinterpret_cast<float4 *>(out + i * 64);
#pragma unroll
        for (int q = 0; q < 16; q++) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    }
}

// One block per lane, blocks in id order: decode, then write the block's
// in-volume samples into the dense x-fastest field.  Lanes of a warp hold
// consecutive blocks along x, so each row store of the warp covers one
// contiguous span of the field, and the staging loads read one contiguous
// span of the bitstream.
__global__ void __launch_bounds__(kCodecThreads) decode_volume_kernel(const uint64_t *__restrict__ bits, Geom g,
                                                                      float *field) {
    extern __shared__ uint64_t dsm[];
    const DecodeSmem sm = codec_smem(dsm, g.rate);
    const bool rows16 = (g.nx & 3u) == 0;       // every row starts 16-byte aligned
    const uint32_t lane = threadIdx.x & 31u;
    for (uint32_t b0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); b0 < g.nb; b0 += gridDim.x * blockDim.x) {
        const uint32_t b = b0 + lane;
        const bool have = b < g.nb;
        stage_blocks<true>(bits, g.rate, b, have, sm.stage);
        if (!have) continue;
        uint32_t bx, by, bz;
        block_coords(g, b, bx, by, bz);
        float v[64];
        decode_staged(sm.stage + lane * (2u * g.rate + 1u), g.rate, sm.tab, v, sm.planes + threadIdx.x, blockDim.x);
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

template <class K>
size_t codec_smem(K kernel, uint32_t rate) {
    const size_t bytes = decode_smem_bytes(kCodecThreads, rate);
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    return bytes;
}

void launch_decode_volume(const uint64_t *bits, const Geom &g, float *field, cudaStream_t st) {
    const uint32_t blocks = std::max<uint32_t>(1, std::min<uint32_t>((g.nb + 127) / 128, 1u << 20));
    decode_volume_kernel<<<blocks, kCodecThreads, codec_smem(decode_volume_kernel, g.rate), st>>>(bits, g, field);
}

void launch_encode(const float *field, const Geom &g, uint64_t *bits, float *bmin, float *bmax, cudaStream_t st) {
    const uint32_t blocks = std::max<uint32_t>(1, std::min<uint32_t>((g.nb + 127) / 128, 1u << 20));
    encode_kernel<<<blocks, kCodecThreads, codec_smem(encode_kernel, g.rate), st>>>(field, g, bits, bmin, bmax);
}

void launch_decode_list(const uint64_t *bits, uint32_t rate, const uint32_t *ids, uint64_t n, float *out,
                        cudaStream_t st) {
    if (n == 0) return;
    const uint64_t blocks = std::min<uint64_t>((n + 127) / 128, 1u << 20);
    decode_list_kernel<<<(unsigned)blocks, kCodecThreads, codec_smem(decode_list_kernel, rate), st>>>(bits, rate, ids,
                                                                                                      n, out);
}

}  // namespace bcmc
