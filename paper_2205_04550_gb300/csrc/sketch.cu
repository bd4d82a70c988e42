// sketch.cu -- random-projection embeddings and Hamming codes of the masks.
//
// Section 2.3 of Ezhov et al. (2022) queries compressed representations by
// L2 (autoencoder latents) and by binary codes (unsupervised hashing).
// Without trained networks, this file provides a random projection of each
// binary mask: a count sketch (one +-1 per voxel, a sparse random
// projection) of D = 4096 buckets, whose squared L2 between two masks is an
// unbiased estimate of their symmetric difference, and the sign code
// [v_j > 0] of the sketch (a sign random projection) compared by Hamming
// distance -- the popcount counterpart of the paper's hashing baseline.
// For the Hamming prefilter the code is also written as FP8 E4M3 bytes
// (1.0 for a set bit, 0 otherwise) with its popcount: for 0/1 vectors
// Hamming(a, b) = |a| + |b| - 2 a.b, a dense contraction that runs exactly on
// the tensor cores (products 0 or 1, sums of at most 4096 in binary32).
//
// Voxel x goes to bucket (h >> 32) mod D with sign (bit 31 of h ? -1 : +1),
// h = SplitMix64 output for counter x (Steele, Lea & Flood 2014).  The
// sketch is encoded like the block-mean embedding: bfloat16 (nearest-even),
// FP8 E4M3 of v / s with s = max|v| / 448 per row, squared norms of the
// decoded rows; the sign code packs 32 buckets per word.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "kernels.h"

namespace dbq {
namespace {

constexpr int kSketchThreads = 512;
constexpr int kSketchD = 4096;

__device__ __forceinline__ uint64_t splitmix64_out(uint64_t i)
{
    uint64_t z = (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ float block_reduce(float v, float* red, bool is_max)
{
    for (int o = 16; o > 0; o >>= 1) {
        const float u = __shfl_xor_sync(0xffffffffu, v, o);
        v = is_max ? fmaxf(v, u) : v + u;
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = threadIdx.x < (int)(blockDim.x >> 5) ? red[threadIdx.x] : 0.0f;
        for (int o = 16; o > 0; o >>= 1) {
            const float u = __shfl_xor_sync(0xffffffffu, v, o);
            v = is_max ? fmaxf(v, u) : v + u;
        }
        if (threadIdx.x == 0) red[0] = v;
    }
    __syncthreads();
    return red[0];
}

__global__ void __launch_bounds__(kSketchThreads)
sketch_kernel(const uint32_t* __restrict__ planes, int64_t wp, int64_t words,
              uint16_t* __restrict__ out_bf16, uint8_t* __restrict__ out_f8,
              float* __restrict__ out_scale, float* __restrict__ out_nb, float* __restrict__ out_nf,
              uint32_t* __restrict__ out_code, uint8_t* __restrict__ out_code8,
              float* __restrict__ out_cnorm)
{
    __shared__ int sk[kSketchD];
    __shared__ float red[kSketchThreads / 32];
    const int64_t row = blockIdx.y * 2 + blockIdx.x;      // (entry, plane)
    const uint32_t* plane = planes + row * wp;
    for (int j = threadIdx.x; j < kSketchD; j += blockDim.x) sk[j] = 0;
    __syncthreads();
    for (int64_t w = threadIdx.x; w < words; w += blockDim.x) {
        uint32_t word = __ldg(plane + w);
        while (word) {
            const int b = __ffs(word) - 1;
            word &= word - 1;
            const uint64_t h = splitmix64_out((uint64_t)(w * 32 + b));
            atomicAdd(&sk[(int)((h >> 32) & (kSketchD - 1))], ((h >> 31) & 1u) ? -1 : 1);
        }
    }
    __syncthreads();
    float m = 0.0f, nb = 0.0f, ones = 0.0f;
    uint16_t* ob = out_bf16 + row * kSketchD;
    uint8_t* oc8 = out_code8 + row * kSketchD;
    for (int j = threadIdx.x; j < kSketchD; j += blockDim.x) {
        const float v = (float)sk[j];
        m = fmaxf(m, fabsf(v));
        const __nv_bfloat16 hb = __float2bfloat16_rn(v);
        ob[j] = __bfloat16_as_ushort(hb);
        const float hv = __bfloat162float(hb);
        nb = __fmaf_rn(hv, hv, nb);
        // sign code: one ballot per 32 consecutive buckets, and as e4m3 0/1
        const bool pos = sk[j] > 0;
        const uint32_t bits = __ballot_sync(0xffffffffu, pos);
        if ((threadIdx.x & 31) == 0) out_code[row * (kSketchD / 32) + j / 32] = bits;
        oc8[j] = pos ? (uint8_t)0x38 : (uint8_t)0;     // 0x38 = 1.0 in E4M3
        ones += pos ? 1.0f : 0.0f;
    }
    const float mx = block_reduce(m, red, true);
    const float nbs = block_reduce(nb, red, false);
    const float pop = block_reduce(ones, red, false);     // exact: an integer <= 4096
    const float s = (mx == 0.0f) ? 1.0f : __fdiv_rn(mx, 448.0f);
    float nq = 0.0f;
    uint8_t* oq = out_f8 + row * kSketchD;
    for (int j = threadIdx.x; j < kSketchD; j += blockDim.x) {
        const float r = __fdiv_rn((float)sk[j], s);
        const __nv_fp8_storage_t c = __nv_cvt_float_to_fp8(r, __NV_SATFINITE, __NV_E4M3);
        oq[j] = (uint8_t)c;
        const __half_raw hr = __nv_cvt_fp8_to_halfraw(c, __NV_E4M3);
        const float qv = __half2float(__half(hr));
        nq = __fmaf_rn(qv, qv, nq);
    }
    const float nqs = block_reduce(nq, red, false);
    if (threadIdx.x == 0) {
        out_scale[row] = s;
        out_nb[row] = nbs;
        out_nf[row] = nqs * s * s;
        out_cnorm[row] = pop;
    }
}

}  // namespace

int sketch_dims() { return kSketchD; }

cudaError_t launch_sketch(const uint32_t* planes, int64_t count, int64_t wp, int64_t words,
                          uint16_t* out_bf16, uint8_t* out_f8, float* out_scale, float* out_nb,
                          float* out_nf, uint32_t* out_code, uint8_t* out_code8, float* out_cnorm,
                          cudaStream_t stream)
{
    for (int64_t e0 = 0; e0 < count; e0 += 65535) {
        const int64_t ce = (count - e0) < 65535 ? (count - e0) : 65535;
        sketch_kernel<<<dim3(2, (unsigned)ce), kSketchThreads, 0, stream>>>(
            planes + e0 * 2 * wp, wp, words, out_bf16 + e0 * 2 * kSketchD,
            out_f8 + e0 * 2 * kSketchD, out_scale + e0 * 2, out_nb + e0 * 2, out_nf + e0 * 2,
            out_code + e0 * 2 * (kSketchD / 32), out_code8 + e0 * 2 * kSketchD,
            out_cnorm + e0 * 2);
        const cudaError_t err = cudaGetLastError();
        if (err != cudaSuccess) return err;
    }
    return cudaSuccess;
}

}  // namespace dbq
