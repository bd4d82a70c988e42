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
// h = SplitMix64 output for counter x (Steele, Lea & Flood 2014); the
// bucket and sign of each voxel index come from a table built once.  The
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

// The bucket and sign of every voxel depend on its index only: one table of
// V entries, bucket | sign << 15, built once per grid and read (L2-resident)
// for every set voxel of every mask.
__global__ void sketch_table_kernel(int64_t v, uint16_t* __restrict__ table)
{
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < v;
         x += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t h = splitmix64_out((uint64_t)x);
        table[x] = (uint16_t)(((h >> 32) & (kSketchD - 1)) | (((h >> 31) & 1u) << 15));
    }
}

__global__ void __launch_bounds__(kSketchThreads)
sketch_kernel(const uint32_t* __restrict__ planes, int64_t wp, int64_t words,
              const uint16_t* __restrict__ table,
              uint16_t* __restrict__ out_bf16, uint8_t* __restrict__ out_f8,
              float* __restrict__ out_scale, float* __restrict__ out_nb, float* __restrict__ out_nf,
              uint32_t* __restrict__ out_code, uint8_t* __restrict__ out_code8,
              float* __restrict__ out_cnorm)
{
    __shared__ int sk[kSketchD];
    __shared__ float red[kSketchThreads / 32];
    __shared__ unsigned long long next_chunk;
    const int64_t row = blockIdx.y * 2 + blockIdx.x;      // (entry, plane)
    const uint32_t* plane = planes + row * wp;
    for (int j = threadIdx.x; j < kSketchD; j += blockDim.x) sk[j] = 0;
    if (threadIdx.x == 0) next_chunk = 0;
    __syncthreads();
    // Warps take chunks of 32 consecutive words (a lane per word) from a
    // shared counter: the set voxels sit in the tumour's few columns, so a
    // static split would leave most warps waiting at the barrier.
    constexpr int kChunks = 4;                   // chunks per grab (loads in flight)
    const int lane = threadIdx.x & 31;
    const int64_t nchunks = (words + 31) / 32;
    for (;;) {
        int64_t c0 = 0;
        if (lane == 0) c0 = atomicAdd(&next_chunk, (unsigned long long)kChunks);
        c0 = __shfl_sync(0xffffffffu, c0, 0);
        if (c0 >= nchunks) break;
        uint32_t wd[kChunks];
#pragma unroll
        for (int u = 0; u < kChunks; ++u) {
            const int64_t w = (c0 + u) * 32 + lane;
            wd[u] = (c0 + u < nchunks && w < words) ? __ldg(plane + w) : 0u;
        }
        // the warp takes the non-zero words one at a time, lane l testing
        // bit l: the table reads of one word are one coalesced 64-byte access
#pragma unroll
        for (int u = 0; u < kChunks; ++u) {
            uint32_t nz = __ballot_sync(0xffffffffu, wd[u] != 0u);
            while (nz) {
                const int j = __ffs(nz) - 1;
                nz &= nz - 1;
                const uint32_t word = __shfl_sync(0xffffffffu, wd[u], j);
                if ((word >> lane) & 1u) {
                    const uint32_t t = __ldg(table + ((c0 + u) * 32 + j) * 32 + lane);
                    atomicAdd(&sk[t & (kSketchD - 1)], (t >> 15) ? -1 : 1);
                }
            }
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

cudaError_t launch_sketch_table(int64_t v, uint16_t* table, cudaStream_t stream)
{
    if (v <= 0) return cudaSuccess;
    const int64_t want = (v + 255) / 256;
    sketch_table_kernel<<<(unsigned)(want < 4096 ? want : 4096), 256, 0, stream>>>(v, table);
    return cudaGetLastError();
}

cudaError_t launch_sketch(const uint32_t* planes, int64_t count, int64_t wp, int64_t words,
                          const uint16_t* table, uint16_t* out_bf16, uint8_t* out_f8, float* out_scale, float* out_nb,
                          float* out_nf, uint32_t* out_code, uint8_t* out_code8, float* out_cnorm,
                          cudaStream_t stream)
{
    for (int64_t e0 = 0; e0 < count; e0 += 65535) {
        const int64_t ce = (count - e0) < 65535 ? (count - e0) : 65535;
        sketch_kernel<<<dim3(2, (unsigned)ce), kSketchThreads, 0, stream>>>(
            planes + e0 * 2 * wp, wp, words, table, out_bf16 + e0 * 2 * kSketchD,
            out_f8 + e0 * 2 * kSketchD, out_scale + e0 * 2, out_nb + e0 * 2, out_nf + e0 * 2,
            out_code + e0 * 2 * (kSketchD / 32), out_code8 + e0 * 2 * kSketchD,
            out_cnorm + e0 * 2);
        const cudaError_t err = cudaGetLastError();
        if (err != cudaSuccess) return err;
    }
    return cudaSuccess;
}

}  // namespace dbq
