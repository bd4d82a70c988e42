// synth.cu -- GPU generator of the seeded surrogate tumour volumes.
//
// Input synthesis only: this file holds none of the query's arithmetic and
// is built into its own library (libdbqsynth.so), separate from the query
// library.  The definition it follows (parameters, brain ellipsoid, logistic
// profile, SplitMix64 voxel noise, binary32 arithmetic, round-to-nearest-even
// to binary16) is stated in synth/__init__.py; the parameters theta, the
// noise stream keys and the brain x-ranges are computed on the host in
// binary64 and passed in, so only the per-voxel arithmetic runs here.
//
// Explicit _rn intrinsics keep the binary32 operations un-contracted, in the
// same order as the numpy generator; only expf may differ in its last bits.
#include <cstdint>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace {

__device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

template <bool kHalf>
__global__ void generate_kernel(const float* __restrict__ theta,   // [n][8]
                                const uint64_t* __restrict__ nkey, // [n]
                                const int* __restrict__ xrange,    // [nz*ny][2]
                                int nx, int ny, int nz, int64_t n, void* out)
{
    const int64_t v = (int64_t)nx * ny * nz;
    const int64_t e = blockIdx.y + (int64_t)gridDim.y * blockIdx.z;
    if (e >= n) return;
    const float* th = theta + e * 8;
    const float cx = th[0], cy = th[1], cz = th[2], R = th[3], w = th[4];
    const float ax = th[5], ay = th[6], az = th[7];
    const uint64_t key = nkey[e];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < v;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx);
        const int64_t row = i / nx;
        const int y = (int)(row % ny);
        const int z = (int)(row / ny);
        float c = 0.0f;
        if (x >= xrange[2 * row] && x <= xrange[2 * row + 1]) {
            const float dx = __fdiv_rn(__fsub_rn((float)x, cx), ax);
            const float dy = __fdiv_rn(__fsub_rn((float)y, cy), ay);
            const float dz = __fdiv_rn(__fsub_rn((float)z, cz), az);
            float r2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
            r2 = __fadd_rn(r2, __fmul_rn(dz, dz));
            const float r = __fsqrt_rn(r2);
            const float a = __fdiv_rn(__fsub_rn(r, R), w);
            c = __fdiv_rn(1.0f, __fadd_rn(1.0f, expf(a)));
            const uint64_t h = mix64(key + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull);
            const float u = __fmul_rn((float)(h >> 40), 5.9604644775390625e-8f);  // 2^-24
            const float noise = __fsub_rn(__fmul_rn(u, 0.02f), 0.01f);
            c = __fadd_rn(c, noise);
            c = fminf(fmaxf(c, 0.0f), 1.0f);
        }
        if (kHalf)
            reinterpret_cast<__half*>(out)[e * v + i] = __float2half_rn(c);
        else
            reinterpret_cast<float*>(out)[e * v + i] = c;
    }
}

}  // namespace

// Fill out[n][nz][ny][nx] (float32, or binary16 when out_f16 != 0) on `stream`.
// All pointers are device pointers.  Returns 0, or a cudaError_t value.
extern "C" int synth_generate(const float* theta, const uint64_t* nkey, const int* xrange,
                              int nx, int ny, int nz, int64_t n, int out_f16, void* out,
                              void* stream)
{
    if (n <= 0) return 0;
    if (nx <= 0 || ny <= 0 || nz <= 0 || !theta || !nkey || !xrange || !out) return 1;
    const int64_t v = (int64_t)nx * ny * nz;
    const int threads = 256;
    int64_t bx = (v + threads - 1) / threads;
    if (bx > 2048) bx = 2048;
    const int64_t gy = n < 65535 ? n : 65535;
    const int64_t gz = (n + gy - 1) / gy;
    dim3 grid((unsigned)bx, (unsigned)gy, (unsigned)gz);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (out_f16)
        generate_kernel<true><<<grid, threads, 0, s>>>(theta, nkey, xrange, nx, ny, nz, n, out);
    else
        generate_kernel<false><<<grid, threads, 0, s>>>(theta, nkey, xrange, nx, ny, nz, n, out);
    return (int)cudaGetLastError();
}
