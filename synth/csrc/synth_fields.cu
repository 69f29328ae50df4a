// GPU versions of the seeded field generators in synth/fields.py.
//
// Input generation only (no part of the isosurface method).  Each value is
// computed with the same float64 operations in the same order as the NumPy
// code, compiled with -fmad=false, so both produce identical float32
// volumes.  Layout: x fastest, out[x + nx*(y + ny*z)].
#include <cstdint>
#include <cuda_runtime.h>

namespace {

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

__device__ __forceinline__ uint64_t lattice_hash(uint64_t seed, uint64_t octave, int64_t ix, int64_t iy, int64_t iz) {
    uint64_t h = splitmix64(seed + octave);
    h = splitmix64(h + (uint64_t)ix);
    h = splitmix64(h + (uint64_t)iy);
    return splitmix64(h + (uint64_t)iz);
}

__device__ __forceinline__ double fade(double t) {
    return __dmul_rn(__dmul_rn(__dmul_rn(t, t), t),
                     __dadd_rn(__dmul_rn(t, __dsub_rn(__dmul_rn(t, 6.0), 15.0)), 10.0));
}

__device__ __forceinline__ double lerp(double a, double b, double w) { return __dadd_rn(a, __dmul_rn(w, __dsub_rn(b, a))); }

__constant__ int kGrad[12][3] = {{1, 1, 0}, {-1, 1, 0}, {1, -1, 0}, {-1, -1, 0}, {1, 0, 1}, {-1, 0, 1},
                                 {1, 0, -1}, {-1, 0, -1}, {0, 1, 1}, {0, -1, 1}, {0, 1, -1}, {0, -1, -1}};

__global__ void noise_kernel(float *out, uint32_t nx, uint32_t ny, uint32_t nz, int64_t x0, int64_t y0, int64_t z0,
                             uint64_t seed, int octaves, int64_t base_period, double gain, double scale) {
    const uint64_t n = (uint64_t)nx * ny * nz;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const int64_t X = x0 + (int64_t)(i % nx), Y = y0 + (int64_t)((i / nx) % ny), Z = z0 + (int64_t)(i / ((uint64_t)nx * ny));
        double acc = 0.0;
        double amp = 1.0;
        for (int o = 0; o < octaves; o++) {
            const int64_t period = base_period >> o;
            const double inv = 1.0 / (double)period;
            const int64_t cx = X / period, cy = Y / period, cz = Z / period;
            const double fx = __dmul_rn((double)(X - cx * period), inv);
            const double fy = __dmul_rn((double)(Y - cy * period), inv);
            const double fz = __dmul_rn((double)(Z - cz * period), inv);
            double d[8];
            for (int k = 0; k < 2; k++)
                for (int j = 0; j < 2; j++)
                    for (int ii = 0; ii < 2; ii++) {
                        const uint64_t h = lattice_hash(seed, (uint64_t)o, cx + ii, cy + j, cz + k);
                        const int *g = kGrad[(h >> 32) % 12];
                        const double dx = __dsub_rn(fx, (double)ii), dy = __dsub_rn(fy, (double)j),
                                     dz = __dsub_rn(fz, (double)k);
                        d[ii + 2 * j + 4 * k] = __dadd_rn(__dadd_rn(__dmul_rn((double)g[0], dx), __dmul_rn((double)g[1], dy)),
                                                          __dmul_rn((double)g[2], dz));
                    }
            const double wx = fade(fx), wy = fade(fy), wz = fade(fz);
            const double x00 = lerp(d[0], d[1], wx), x10 = lerp(d[2], d[3], wx);
            const double x01 = lerp(d[4], d[5], wx), x11 = lerp(d[6], d[7], wx);
            const double yz0 = lerp(x00, x10, wy), yz1 = lerp(x01, x11, wy);
            acc = __dadd_rn(acc, __dmul_rn(amp, lerp(yz0, yz1, wz)));
            amp = __dmul_rn(amp, gain);
        }
        out[i] = __double2float_rn(__dmul_rn(acc, scale));
    }
}

__global__ void sphere_kernel(float *out, uint32_t nx, uint32_t ny, uint32_t nz, int64_t x0, int64_t y0, int64_t z0,
                              double cx, double cy, double cz, double radius) {
    const uint64_t n = (uint64_t)nx * ny * nz;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const double dx = __dsub_rn((double)(x0 + (int64_t)(i % nx)), cx);
        const double dy = __dsub_rn((double)(y0 + (int64_t)((i / nx) % ny)), cy);
        const double dz = __dsub_rn((double)(z0 + (int64_t)(i / ((uint64_t)nx * ny))), cz);
        const double s = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
        out[i] = __double2float_rn(__dsub_rn(__dsqrt_rn(s), radius));
    }
}

unsigned grid_for(uint64_t n) {
    const uint64_t b = (n + 255) / 256;
    return (unsigned)(b < 65535ull * 16 ? (b ? b : 1) : 65535ull * 16);
}

}  // namespace

extern "C" {

int synth_gradient_noise(float *out, uint32_t nx, uint32_t ny, uint32_t nz, int64_t x0, int64_t y0, int64_t z0,
                         uint64_t seed, int octaves, int64_t base_period, double gain, double scale, void *stream) {
    if (!out || !nx || !ny || !nz || octaves < 1 || (base_period >> (octaves - 1)) < 1) return 1;
    noise_kernel<<<grid_for((uint64_t)nx * ny * nz), 256, 0, (cudaStream_t)stream>>>(out, nx, ny, nz, x0, y0, z0, seed,
                                                                                       octaves, base_period, gain, scale);
    return cudaGetLastError() == cudaSuccess ? 0 : 4;
}

int synth_sphere_sdf(float *out, uint32_t nx, uint32_t ny, uint32_t nz, int64_t x0, int64_t y0, int64_t z0, double cx,
                     double cy, double cz, double radius, void *stream) {
    if (!out || !nx || !ny || !nz) return 1;
    sphere_kernel<<<grid_for((uint64_t)nx * ny * nz), 256, 0, (cudaStream_t)stream>>>(out, nx, ny, nz, x0, y0, z0, cx, cy,
                                                                                        cz, radius);
    return cudaGetLastError() == cudaSuccess ? 0 : 4;
}

}  // extern "C"
