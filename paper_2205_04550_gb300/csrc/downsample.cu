// downsample.cu -- nearest-neighbour downsampling of bit-packed masks.
//
// Section 2.3 of Ezhov et al. (2022) also queries a database downsampled to
// 64^3 and 32^3 with an order-0 (nearest-neighbour) spline, comparing it with
// the equally downsampled patient by Dice.  Nearest-neighbour sampling
// commutes with thresholding, so the downsampled masks are taken straight
// from the full-resolution bit planes: voxel (x, y, z) of the coarse grid is
// voxel (f x, f y, f z) of the fine grid (reading: stride sampling from the
// origin).  One thread per coarse 32-bit word gathers its 32 bits (when the
// coarse rows are whole words, from one source row with no per-bit index
// arithmetic); the coarse mask sizes are re-counted with popcounts.
#include "kernels.h"

namespace dbq {
namespace {

__global__ void downsample_kernel(const uint32_t* __restrict__ src, int64_t src_wp, int nx,
                                  int ny, int f, int64_t dst_words, int64_t dst_wp, int dnx,
                                  int dny, int64_t dv, uint32_t* __restrict__ dst,
                                  uint32_t* __restrict__ sizes)
{
    const int64_t row = blockIdx.y;                       // entry * 2 + plane
    const uint32_t* s = src + row * src_wp;
    uint32_t* d = dst + row * dst_wp;
    uint32_t cnt = 0;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < dst_wp;
         w += (int64_t)gridDim.x * blockDim.x) {
        uint32_t word = 0;
        if (w < dst_words && dnx % 32 == 0) {
            // the word's 32 coarse voxels are one run along x: its source bits
            // are j0, j0 + f, ..., one division per word
            const int64_t i0 = w * 32;
            const int64_t x0 = i0 % dnx, yz = i0 / dnx;
            const int64_t y = yz % dny, z = yz / dny;
            const int64_t j0 = f * x0 + (int64_t)nx * (f * y + (int64_t)ny * (f * z));
            for (int b = 0; b < 32; ++b) {
                const int64_t j = j0 + (int64_t)f * b;
                word |= ((__ldg(s + (j >> 5)) >> (j & 31)) & 1u) << b;
            }
        } else if (w < dst_words) {
            for (int b = 0; b < 32; ++b) {
                const int64_t i = w * 32 + b;             // coarse voxel
                if (i >= dv) break;
                const int64_t x = i % dnx, y = (i / dnx) % dny, z = i / ((int64_t)dnx * dny);
                const int64_t j = f * x + (int64_t)nx * (f * y + (int64_t)ny * (f * z));
                word |= ((__ldg(s + (j >> 5)) >> (j & 31)) & 1u) << b;
            }
        }
        d[w] = word;
        cnt += __popc(word);
    }
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(&sizes[row], cnt);
}

}  // namespace

cudaError_t launch_downsample(const uint32_t* src, int64_t rows, int64_t src_wp, int nx, int ny,
                              int nz, int f, int64_t dst_wp, uint32_t* dst, uint32_t* sizes,
                              cudaStream_t stream)
{
    const int dnx = nx / f, dny = ny / f, dnz = nz / f;
    const int64_t dv = (int64_t)dnx * dny * dnz;
    const int64_t dst_words = (dv + 31) / 32;
    int64_t bx = (dst_wp + 255) / 256;
    if (bx > 64) bx = 64;
    if (bx < 1) bx = 1;
    for (int64_t r0 = 0; r0 < rows; r0 += 65535) {
        const int64_t rc = (rows - r0) < 65535 ? (rows - r0) : 65535;
        downsample_kernel<<<dim3((unsigned)bx, (unsigned)rc), 256, 0, stream>>>(
            src + r0 * src_wp, src_wp, nx, ny, f, dst_words, dst_wp, dnx, dny, dv,
            dst + r0 * dst_wp, sizes + r0);
        const cudaError_t err = cudaGetLastError();
        if (err != cudaSuccess) return err;
    }
    return cudaSuccess;
}

}  // namespace dbq
