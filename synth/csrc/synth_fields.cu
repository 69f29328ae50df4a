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

// ---------------------------------------------------------------- channel-flow-like field
// (mirror of synth.fields.channel_field; float32 noise, float64 profile)

__device__ __forceinline__ double exp_f64(double y) {
    const double kInvFact[21] = {1.0, 1.0, 0.5, 1.0 / 6.0, 1.0 / 24.0, 1.0 / 120.0, 1.0 / 720.0, 1.0 / 5040.0,
                                 1.0 / 40320.0, 1.0 / 362880.0, 1.0 / 3628800.0, 1.0 / 39916800.0,
                                 1.0 / 479001600.0, 1.0 / 6227020800.0, 1.0 / 87178291200.0,
                                 1.0 / 1307674368000.0, 1.0 / 20922789888000.0, 1.0 / 355687428096000.0,
                                 1.0 / 6402373705728000.0, 1.0 / 121645100408832000.0,
                                 1.0 / 2432902008176640000.0};
    const double ln2 = 0.6931471805599453;
    const double n = rint(__ddiv_rn(y, ln2));
    const double r = __dsub_rn(y, __dmul_rn(n, ln2));
    double p = kInvFact[20];
    for (int k = 19; k >= 0; k--) p = __dadd_rn(__dmul_rn(p, r), kInvFact[k]);
    return scalbn(p, (int)n);
}

__device__ __forceinline__ double tanh_pos_f64(double x) {
    const double e = exp_f64(__dmul_rn(-2.0, x));
    return __ddiv_rn(__dsub_rn(1.0, e), __dadd_rn(1.0, e));
}

__global__ void channel_profile_kernel(float *U, float *A, int64_t z0, uint32_t nz, uint32_t nz_total) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nz; i += gridDim.x * blockDim.x) {
        const double zeta = __ddiv_rn((double)(z0 + (int64_t)i), (double)(nz_total - 1));
        const double u = __dmul_rn(tanh_pos_f64(__ddiv_rn(zeta, 0.08)), tanh_pos_f64(__ddiv_rn(__dsub_rn(1.0, zeta), 0.08)));
        U[i] = __double2float_rn(u);
        A[i] = __double2float_rn(__dadd_rn(__dmul_rn(0.3, __dsub_rn(1.0, u)), 0.1));
    }
}

__device__ __forceinline__ float fade_f32(float t) {
    return __fmul_rn(__fmul_rn(__fmul_rn(t, t), t), __fadd_rn(__fmul_rn(t, __fsub_rn(__fmul_rn(t, 6.0f), 15.0f)), 10.0f));
}
__device__ __forceinline__ float lerp_f32(float a, float b, float w) { return __fadd_rn(a, __fmul_rn(w, __fsub_rn(b, a))); }

// One thread per 4x4x4 brick of the window (window origin 4-aligned): the
// brick lies inside one lattice cell of every octave (periods >= 4 and
// multiples of 4), so its 8 corner gradients are hashed once per octave.
__global__ void channel_kernel(float *out, uint32_t nx, uint32_t ny, uint32_t nz, int64_t x0, int64_t y0, int64_t z0,
                               uint64_t seed, int octaves, int64_t base_period, float gain, float scale,
                               const float *U, const float *A) {
    const uint32_t bx_n = (nx + 3) / 4, by_n = (ny + 3) / 4, bz_n = (nz + 3) / 4;
    const uint64_t nbricks = (uint64_t)bx_n * by_n * bz_n;
    for (uint64_t bi = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; bi < nbricks; bi += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t bx = (uint32_t)(bi % bx_n), by = (uint32_t)((bi / bx_n) % by_n), bz = (uint32_t)(bi / ((uint64_t)bx_n * by_n));
        const int64_t X0 = x0 + 4 * (int64_t)bx, Y0 = y0 + 4 * (int64_t)by, Z0 = z0 + 4 * (int64_t)bz;
        float acc[64];
#pragma unroll
        for (int i = 0; i < 64; i++) acc[i] = 0.0f;
        float amp = 1.0f;
        for (int o = 0; o < octaves; o++) {
            const int64_t period = base_period >> o;
            const float inv = __fdiv_rn(1.0f, (float)period);
            const int64_t cx = X0 / period, cy = Y0 / period, cz = Z0 / period;
            int g[8][3];
            for (int c = 0; c < 8; c++) {
                const uint64_t h = lattice_hash(seed, (uint64_t)o, cx + (c & 1), cy + ((c >> 1) & 1), cz + (c >> 2));
                const int *gg = kGrad[(h >> 32) % 12];
                g[c][0] = gg[0]; g[c][1] = gg[1]; g[c][2] = gg[2];
            }
            float fx[4], fy[4], fz[4], wx[4], wy[4], wz[4];
#pragma unroll
            for (int i = 0; i < 4; i++) {
                fx[i] = __fmul_rn((float)(X0 + i - cx * period), inv);
                fy[i] = __fmul_rn((float)(Y0 + i - cy * period), inv);
                fz[i] = __fmul_rn((float)(Z0 + i - cz * period), inv);
                wx[i] = fade_f32(fx[i]);
                wy[i] = fade_f32(fy[i]);
                wz[i] = fade_f32(fz[i]);
            }
#pragma unroll
            for (int k = 0; k < 4; k++)
#pragma unroll
                for (int j = 0; j < 4; j++)
#pragma unroll
                    for (int i = 0; i < 4; i++) {
                        float d[8];
#pragma unroll
                        for (int c = 0; c < 8; c++) {
                            const float dx = __fsub_rn(fx[i], (float)(c & 1)), dy = __fsub_rn(fy[j], (float)((c >> 1) & 1)),
                                        dz = __fsub_rn(fz[k], (float)(c >> 2));
                            d[c] = __fadd_rn(__fadd_rn(__fmul_rn((float)g[c][0], dx), __fmul_rn((float)g[c][1], dy)),
                                             __fmul_rn((float)g[c][2], dz));
                        }
                        const float x00 = lerp_f32(d[0], d[1], wx[i]), x10 = lerp_f32(d[2], d[3], wx[i]);
                        const float x01 = lerp_f32(d[4], d[5], wx[i]), x11 = lerp_f32(d[6], d[7], wx[i]);
                        const float val = lerp_f32(lerp_f32(x00, x10, wy[j]), lerp_f32(x01, x11, wy[j]), wz[k]);
                        acc[i + 4 * j + 16 * k] = __fadd_rn(acc[i + 4 * j + 16 * k], __fmul_rn(amp, val));
                    }
            amp = __fmul_rn(amp, gain);
        }
#pragma unroll
        for (int k = 0; k < 4; k++)
#pragma unroll
            for (int j = 0; j < 4; j++)
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    const uint32_t x = 4 * bx + i, y = 4 * by + j, z = 4 * bz + k;
                    if (x >= nx || y >= ny || z >= nz) continue;
                    const float v = __fadd_rn(U[z], __fmul_rn(A[z], __fmul_rn(acc[i + 4 * j + 16 * k], scale)));
                    out[(size_t)x + (size_t)nx * ((size_t)y + (size_t)ny * z)] = v;
                }
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

int synth_channel_field(float *out, uint32_t nx, uint32_t ny, uint32_t nz, int64_t x0, int64_t y0, int64_t z0,
                        uint64_t seed, uint32_t nz_total, int octaves, int64_t base_period, float gain, float scale,
                        float *work_profile, void *stream) {
    // work_profile: device scratch of 2*nz floats for the wall-normal profile
    if (!out || !work_profile || !nx || !ny || !nz || nz_total < 2 || octaves < 1 ||
        (base_period >> (octaves - 1)) < 4 || (x0 & 3) || (y0 & 3) || (z0 & 3))
        return 1;
    cudaStream_t st = (cudaStream_t)stream;
    channel_profile_kernel<<<(nz + 255) / 256, 256, 0, st>>>(work_profile, work_profile + nz, z0, nz, nz_total);
    const uint64_t bricks = (uint64_t)((nx + 3) / 4) * ((ny + 3) / 4) * ((nz + 3) / 4);
    channel_kernel<<<grid_for(bricks), 256, 0, st>>>(out, nx, ny, nz, x0, y0, z0, seed, octaves, base_period, gain, scale,
                                                   work_profile, work_profile + nz);
    return cudaGetLastError() == cudaSuccess ? 0 : 4;
}

}  // extern "C"
