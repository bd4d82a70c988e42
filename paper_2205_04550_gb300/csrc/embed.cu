// embed.cu -- low-dimensional embeddings of the thresholded masks for the
// L2 prefilter.
//
// Ezhov et al. (2022), Section 2.3: besides the direct loop, the paper
// queries compressed representations (downsampled volumes, autoencoder
// latents, hash codes) by the L2 distance, one per segmentation, adding
// L2_T1Gd + L2_FLAIR and taking the smallest.  Here each mask is compressed
// to the mean of every 8 x 8 x 8 block (16^3 = 4096 values at 128^3), stored
// as bfloat16 and as FP8 E4M3 with one binary32 scale per row, and the
// prefilter's survivors are re-ranked by the exact Dice loop.
//
// Values: e_b = c_b / 512 with c_b the number of set voxels of block b
// (exact in binary32).  bfloat16: round-to-nearest-even of e_b.  FP8: the
// row scale s = max_b(e_b) / 448 in binary32 (s = 1 for an empty row) and
// the code of e_b / s, rounded to nearest-even and saturated.  The squared
// row norms of the encoded vectors (sum of squares of the decoded values,
// times s^2 for FP8) are kept in binary32 for the distance epilogue.
//
// One CTA per (entry, plane).  Grids whose x-extent is a multiple of 32 keep
// each 32-voxel word inside one x-row, so byte i of a word holds the eight
// voxels of one block row: thread (word-in-row, by, bz) adds the popcounts
// of its bytes over the block's 8 x 8 rows and owns four block counts.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "kernels.h"

namespace dbq {
namespace {

constexpr int kEmbedThreads = 512;

__global__ void __launch_bounds__(kEmbedThreads)
embed_kernel(const uint32_t* __restrict__ planes, int64_t wp, int nx, int ny, int nz,
             uint16_t* __restrict__ out_bf16, uint8_t* __restrict__ out_f8,
             float* __restrict__ out_scale, float* __restrict__ out_norm_bf16,
             float* __restrict__ out_norm_f8)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int bxn = nx / 8, byn = ny / 8, bzn = nz / 8;
    const int d = bxn * byn * bzn;
    float* val = reinterpret_cast<float*>(smem_raw);     // [d] block means
    __shared__ float red[kEmbedThreads / 32];
    __shared__ float red2[kEmbedThreads / 32];
    const int64_t row = blockIdx.y * 2 + blockIdx.x;      // (entry, plane)
    const uint32_t* plane = planes + (row >> 1) * 2 * wp + (row & 1) * wp;
    const int wpr = nx / 32;                              // words per x-row
    const int tasks = wpr * byn * bzn;
    for (int t = threadIdx.x; t < tasks; t += blockDim.x) {
        const int wx = t % wpr;
        const int by = (t / wpr) % byn;
        const int bz = t / (wpr * byn);
        uint32_t c0 = 0, c1 = 0, c2 = 0, c3 = 0;
        for (int z = 8 * bz; z < 8 * bz + 8; ++z)
            for (int y = 8 * by; y < 8 * by + 8; ++y) {
                const uint32_t w = __ldg(plane + ((int64_t)z * ny + y) * wpr + wx);
                c0 += __popc(w & 0x000000ffu);
                c1 += __popc(w & 0x0000ff00u);
                c2 += __popc(w & 0x00ff0000u);
                c3 += __popc(w & 0xff000000u);
            }
        const int base = (bz * byn + by) * bxn + 4 * wx;
        val[base + 0] = (float)c0 * (1.0f / 512.0f);
        val[base + 1] = (float)c1 * (1.0f / 512.0f);
        val[base + 2] = (float)c2 * (1.0f / 512.0f);
        val[base + 3] = (float)c3 * (1.0f / 512.0f);
    }
    __syncthreads();
    // row maximum (for the FP8 scale) and bfloat16 encoding + squared norm
    float m = 0.0f, nb = 0.0f;
    uint16_t* ob = out_bf16 + row * d;
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
        const float e = val[j];
        m = fmaxf(m, e);
        const __nv_bfloat16 h = __float2bfloat16_rn(e);
        ob[j] = __bfloat16_as_ushort(h);
        const float hv = __bfloat162float(h);
        nb = __fmaf_rn(hv, hv, nb);
    }
    for (int o = 16; o > 0; o >>= 1) {
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        nb += __shfl_xor_sync(0xffffffffu, nb, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[threadIdx.x >> 5] = m;
        red2[threadIdx.x >> 5] = nb;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (int)(blockDim.x >> 5) ? red[threadIdx.x] : 0.0f;
        nb = threadIdx.x < (int)(blockDim.x >> 5) ? red2[threadIdx.x] : 0.0f;
        for (int o = 16; o > 0; o >>= 1) {
            m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
            nb += __shfl_xor_sync(0xffffffffu, nb, o);
        }
        if (threadIdx.x == 0) {
            red[0] = m;
            out_norm_bf16[row] = nb;
        }
    }
    __syncthreads();
    const float mx = red[0];
    const float s = (mx == 0.0f) ? 1.0f : __fdiv_rn(mx, 448.0f);
    __syncthreads();
    float nq = 0.0f;
    uint8_t* oq = out_f8 + row * d;
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
        const float r = __fdiv_rn(val[j], s);
        const __nv_fp8_storage_t c = __nv_cvt_float_to_fp8(r, __NV_SATFINITE, __NV_E4M3);
        oq[j] = (uint8_t)c;
        const __half_raw hr = __nv_cvt_fp8_to_halfraw(c, __NV_E4M3);
        const float qv = __half2float(__half(hr));
        nq = __fmaf_rn(qv, qv, nq);
    }
    for (int o = 16; o > 0; o >>= 1) nq += __shfl_xor_sync(0xffffffffu, nq, o);
    if ((threadIdx.x & 31) == 0) red2[threadIdx.x >> 5] = nq;
    __syncthreads();
    if (threadIdx.x < 32) {
        nq = threadIdx.x < (int)(blockDim.x >> 5) ? red2[threadIdx.x] : 0.0f;
        for (int o = 16; o > 0; o >>= 1) nq += __shfl_xor_sync(0xffffffffu, nq, o);
        if (threadIdx.x == 0) {
            out_scale[row] = s;
            out_norm_f8[row] = nq * s * s;
        }
    }
}

}  // namespace

bool embed_supported(int nx, int ny, int nz)
{
    if (nx % 32 || ny % 8 || nz % 8) return false;
    const int64_t d = (int64_t)(nx / 8) * (ny / 8) * (nz / 8);
    return d >= 1 && d * 4 <= 160 * 1024;
}

int embed_dims(int nx, int ny, int nz) { return (nx / 8) * (ny / 8) * (nz / 8); }

cudaError_t launch_embed(const uint32_t* planes, int64_t count, int64_t wp, int nx, int ny,
                         int nz, uint16_t* out_bf16, uint8_t* out_f8, float* out_scale,
                         float* out_norm_bf16, float* out_norm_f8, cudaStream_t stream)
{
    if (count <= 0) return cudaSuccess;
    const size_t smem = (size_t)embed_dims(nx, ny, nz) * sizeof(float);
    cudaError_t err = cudaFuncSetAttribute(embed_kernel,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    for (int64_t e0 = 0; e0 < count; e0 += 65535) {
        const int64_t ce = (count - e0) < 65535 ? (count - e0) : 65535;
        const int d = embed_dims(nx, ny, nz);
        embed_kernel<<<dim3(2, (unsigned)ce), kEmbedThreads, smem, stream>>>(
            planes + e0 * 2 * wp, wp, nx, ny, nz, out_bf16 + e0 * 2 * d, out_f8 + e0 * 2 * d,
            out_scale + e0 * 2, out_norm_bf16 + e0 * 2, out_norm_f8 + e0 * 2);
        err = cudaGetLastError();
        if (err != cudaSuccess) return err;
    }
    return cudaSuccess;
}

}  // namespace dbq
