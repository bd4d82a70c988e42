// pack.cu -- thresholding of concentration volumes into bit planes.
//
// Section 2.3 of Ezhov et al. (2022): the simulated concentration u is
// thresholded at u_T1Gd and u_FLAIR to give the two binary segmentations
// compared with the patient's.  A voxel is in mask k when (float)u >= t_k.
// Bit b of word w of a plane is voxel 32w + b.  Each lane tests the voxels
// of one 16-byte load and the lanes sharing a word OR their bits together
// (or, for unaligned sources, a warp tests 32 voxels and ballots); the mask
// sizes |E_1|, |E_2| are popcounts of the words.
#include <cuda_fp16.h>

#include "kernels.h"

namespace dbq {
namespace {

constexpr int kPackThreads = 256;
constexpr int kPackUnroll = 8;   // loads per lane per iteration (in flight at once)

template <bool kHalf>
__device__ __forceinline__ float load_value(const void* base, int64_t i)
{
    if (kHalf) {
        const unsigned short h = __ldg(reinterpret_cast<const unsigned short*>(base) + i);
        return __half2float(__ushort_as_half(h));
    }
    return __ldg(reinterpret_cast<const float*>(base) + i);
}

// One volume: a warp-strided loop over the planes' words.  When the source
// is 16-byte aligned and V is a multiple of the voxels in 16 bytes, each lane
// loads 16 bytes (4 binary32 or 8 binary16 voxels), builds their bits for
// both thresholds, and the LPW lanes of one 32-voxel word OR their pieces
// together by shuffles; otherwise one voxel per lane and two ballots per word.
template <bool kHalf>
__device__ __forceinline__ void pack_volume(const void* __restrict__ src, int64_t v, int64_t wp,
                                            float t1, float t2, uint32_t* __restrict__ p1,
                                            uint32_t* __restrict__ p2, int64_t warp,
                                            int64_t nwarps, uint32_t& c1, uint32_t& c2)
{
    const int lane = threadIdx.x & 31;
    constexpr int VPL = kHalf ? 8 : 4;      // voxels per lane per 16-byte load
    constexpr int LPW = 32 / VPL;           // lanes per 32-bit word
    constexpr int WPL = 32 / LPW;           // words per warp-wide load
    const bool vec = (reinterpret_cast<uintptr_t>(src) & 15u) == 0 && v % VPL == 0;
    if (vec) {
        const int64_t groups = (wp + WPL - 1) / WPL;
        const uint4* s4 = reinterpret_cast<const uint4*>(src);
        for (int64_t g0 = warp * kPackUnroll; g0 < groups; g0 += nwarps * kPackUnroll) {
            uint4 raw[kPackUnroll];
#pragma unroll
            for (int u = 0; u < kPackUnroll; ++u) {
                const int64_t vox = (g0 + u) * (WPL * 32) + (int64_t)lane * VPL;
                raw[u] = (g0 + u < groups && vox < v) ? __ldcs(s4 + vox / VPL) : make_uint4(0, 0, 0, 0);
            }
#pragma unroll
            for (int u = 0; u < kPackUnroll; ++u) {
                const int64_t g = g0 + u;
                const int64_t vox = g * (WPL * 32) + (int64_t)lane * VPL;
                const uint32_t r[4] = {raw[u].x, raw[u].y, raw[u].z, raw[u].w};
                uint32_t m1 = 0, m2 = 0;
#pragma unroll
                for (int j = 0; j < VPL; ++j) {
                    float val;
                    if (kHalf)
                        val = __half2float(__ushort_as_half(
                            (unsigned short)((r[j / 2] >> (16 * (j % 2))) & 0xffffu)));
                    else
                        val = __uint_as_float(r[j]);
                    m1 |= (uint32_t)(val >= t1) << j;
                    m2 |= (uint32_t)(val >= t2) << j;
                }
                if (vox >= v) m1 = m2 = 0;
                m1 <<= VPL * (lane % LPW);
                m2 <<= VPL * (lane % LPW);
#pragma unroll
                for (int off = 1; off < LPW; off <<= 1) {
                    m1 |= __shfl_xor_sync(0xffffffffu, m1, off);
                    m2 |= __shfl_xor_sync(0xffffffffu, m2, off);
                }
                const int64_t w = g * WPL + lane / LPW;
                if (lane % LPW == 0 && g < groups && w < wp) {
                    p1[w] = m1;
                    p2[w] = m2;
                    c1 += __popc(m1);
                    c2 += __popc(m2);
                }
            }
        }
        return;
    }
    for (int64_t w0 = warp * kPackUnroll; w0 < wp; w0 += nwarps * kPackUnroll) {
        float val[kPackUnroll];
#pragma unroll
        for (int u = 0; u < kPackUnroll; ++u) {
            const int64_t x = (w0 + u) * 32 + lane;
            val[u] = (x < v) ? load_value<kHalf>(src, x) : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < kPackUnroll; ++u) {
            const int64_t w = w0 + u;
            const int64_t x = w * 32 + lane;
            const bool in = x < v;
            const uint32_t b1 = __ballot_sync(0xffffffffu, in && val[u] >= t1);
            const uint32_t b2 = __ballot_sync(0xffffffffu, in && val[u] >= t2);
            if (lane == 0 && w < wp) {
                p1[w] = b1;
                p2[w] = b2;
                c1 += __popc(b1);
                c2 += __popc(b2);
            }
        }
    }
}

template <bool kHalf>
__global__ void __launch_bounds__(kPackThreads)
pack_kernel(const void* __restrict__ vols, int64_t v, int64_t wp, float t1, float t2,
            uint32_t* __restrict__ planes, uint32_t* __restrict__ ecount, int64_t e_base)
{
    const int64_t e = e_base + blockIdx.y;
    const int64_t warp = ((int64_t)blockIdx.x * kPackThreads + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * kPackThreads) >> 5;
    const char* src = reinterpret_cast<const char*>(vols) + e * v * (kHalf ? 2 : 4);
    uint32_t* p1 = planes + e * 2 * wp;
    uint32_t c1 = 0, c2 = 0;
    pack_volume<kHalf>(src, v, wp, t1, t2, p1, p1 + wp, warp, nwarps, c1, c2);
    c1 = __reduce_add_sync(0xffffffffu, c1);
    c2 = __reduce_add_sync(0xffffffffu, c2);
    if ((threadIdx.x & 31) == 0 && (c1 | c2)) {
        atomicAdd(&ecount[2 * e], c1);
        atomicAdd(&ecount[2 * e + 1], c2);
    }
}

// One source volume per blockIdx.y, taken from a device array of pointers.
template <bool kHalf>
__global__ void __launch_bounds__(kPackThreads)
pack_ptrs_kernel(const void* const* __restrict__ srcs, int64_t v, int64_t wp, float t1, float t2,
                 uint32_t* __restrict__ planes, uint32_t* __restrict__ ecount)
{
    const int64_t e = blockIdx.y;
    const int64_t warp = ((int64_t)blockIdx.x * kPackThreads + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * kPackThreads) >> 5;
    uint32_t* p1 = planes + e * 2 * wp;
    uint32_t c1 = 0, c2 = 0;
    pack_volume<kHalf>(srcs[e], v, wp, t1, t2, p1, p1 + wp, warp, nwarps, c1, c2);
    c1 = __reduce_add_sync(0xffffffffu, c1);
    c2 = __reduce_add_sync(0xffffffffu, c2);
    if ((threadIdx.x & 31) == 0 && (c1 | c2)) {
        atomicAdd(&ecount[2 * e], c1);
        atomicAdd(&ecount[2 * e + 1], c2);
    }
}

__global__ void import_bits_kernel(const uint32_t* __restrict__ src, int64_t words, int64_t v,
                                   int64_t wp, uint32_t* __restrict__ planes,
                                   uint32_t* __restrict__ pcount)
{
    const int k = blockIdx.y;
    uint32_t c = 0;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < wp;
         w += (int64_t)gridDim.x * blockDim.x) {
        uint32_t word = 0;
        if (w < words) {
            word = src[k * words + w];
            const int64_t first = w * 32;
            if (first + 32 > v) {
                const int64_t keep = v - first;          // 0 < keep < 32 here
                word &= (keep <= 0) ? 0u : ((1u << keep) - 1u);
            }
        }
        planes[k * wp + w] = word;
        c += __popc(word);
    }
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(&pcount[k], c);
}

__global__ void to_f16_kernel(const float* __restrict__ src, int64_t n,
                              unsigned short* __restrict__ dst)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = __half_as_ushort(__float2half_rn(src[i]));
}

template <bool kSrcHalf>
__global__ void rows_to_f16_kernel(const void* __restrict__ src, int64_t v, int64_t pitch,
                                   unsigned short* __restrict__ dst, int64_t row_base)
{
    const int64_t row = row_base + blockIdx.y;
    unsigned short* d = dst + row * pitch;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < v;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (kSrcHalf)
            d[i] = reinterpret_cast<const unsigned short*>(src)[row * v + i];
        else
            d[i] = __half_as_ushort(__float2half_rn(reinterpret_cast<const float*>(src)[row * v + i]));
    }
}

// Blocks per volume: no more warps than the words of one volume need
// (kPackUnroll loads of 4 words per warp-iteration), at least 16 per volume
// when there are many volumes (each warp then loops over several
// iterations), and enough to fill the GPU (about 8 blocks per SM) when
// there are few.
int64_t pack_blocks(int64_t wp, int64_t count)
{
    const int64_t warps_needed = (wp + kPackUnroll * 4 - 1) / (kPackUnroll * 4);
    const int64_t most = (warps_needed * 32 + kPackThreads - 1) / kPackThreads;
    int64_t bx = (1216 + count - 1) / count;
    if (bx < 16) bx = 16;
    if (bx > most) bx = most;
    return bx < 1 ? 1 : bx;
}

}  // namespace

cudaError_t launch_rows_to_f16(const void* src, int src_f16, int64_t count, int64_t v,
                               int64_t pitch, uint16_t* dst, cudaStream_t stream)
{
    int64_t bx = (v + 255) / 256;
    if (bx > 1024) bx = 1024;
    if (bx < 1) bx = 1;
    unsigned short* d = reinterpret_cast<unsigned short*>(dst);
    for (int64_t r0 = 0; r0 < count; r0 += 65535) {
        const int64_t rc = (count - r0) < 65535 ? (count - r0) : 65535;
        dim3 grid((unsigned)bx, (unsigned)rc);
        if (src_f16)
            rows_to_f16_kernel<true><<<grid, 256, 0, stream>>>(src, v, pitch, d, r0);
        else
            rows_to_f16_kernel<false><<<grid, 256, 0, stream>>>(src, v, pitch, d, r0);
        const cudaError_t err = cudaGetLastError();
        if (err != cudaSuccess) return err;
    }
    return cudaSuccess;
}

cudaError_t launch_to_f16(const float* src, int64_t n, uint16_t* dst, cudaStream_t stream)
{
    if (n <= 0) return cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    to_f16_kernel<<<(unsigned)blocks, 256, 0, stream>>>(src, n,
                                                        reinterpret_cast<unsigned short*>(dst));
    return cudaGetLastError();
}

cudaError_t launch_pack(const void* vols, int src_f16, int64_t count, int64_t v, int64_t wp,
                        float t1, float t2, uint32_t* planes, uint32_t* ecount,
                        cudaStream_t stream)
{
    if (count <= 0) return cudaSuccess;
    const int64_t bx = pack_blocks(wp, count);
    for (int64_t e0 = 0; e0 < count; e0 += 65535) {
        const int64_t ce = (count - e0) < 65535 ? (count - e0) : 65535;
        dim3 grid((unsigned)bx, (unsigned)ce);
        if (src_f16)
            pack_kernel<true><<<grid, kPackThreads, 0, stream>>>(vols, v, wp, t1, t2, planes,
                                                                 ecount, e0);
        else
            pack_kernel<false><<<grid, kPackThreads, 0, stream>>>(vols, v, wp, t1, t2, planes,
                                                                  ecount, e0);
        const cudaError_t err = cudaGetLastError();
        if (err != cudaSuccess) return err;
    }
    return cudaSuccess;
}

cudaError_t launch_pack_ptrs(const void* const* srcs, int src_f16, int count, int64_t v,
                             int64_t wp, float t1, float t2, uint32_t* planes, uint32_t* ecount,
                             cudaStream_t stream)
{
    if (count <= 0) return cudaSuccess;
    const int64_t bx = pack_blocks(wp, count);
    dim3 grid((unsigned)bx, (unsigned)count);
    if (src_f16)
        pack_ptrs_kernel<true><<<grid, kPackThreads, 0, stream>>>(srcs, v, wp, t1, t2, planes, ecount);
    else
        pack_ptrs_kernel<false><<<grid, kPackThreads, 0, stream>>>(srcs, v, wp, t1, t2, planes, ecount);
    return cudaGetLastError();
}

cudaError_t launch_import_bits(const uint32_t* src, int64_t words, int64_t v, int64_t wp,
                               uint32_t* planes, uint32_t* pcount, cudaStream_t stream)
{
    int64_t bx = (wp + 255) / 256;
    if (bx > 256) bx = 256;
    if (bx < 1) bx = 1;
    import_bits_kernel<<<dim3((unsigned)bx, 2), 256, 0, stream>>>(src, words, v, wp, planes,
                                                                   pcount);
    return cudaGetLastError();
}

}  // namespace dbq
