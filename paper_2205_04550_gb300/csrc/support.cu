// support.cu -- the patient's support lists for the sparse exact scan.
//
// The Dice numerator |P_k n E_k| (Section 2.3 of Ezhov et al. 2022) only
// involves voxels inside the patient's mask P_k, so a scan may skip every
// database word whose patient word is zero and still produce the exact
// counts.  This kernel lists, per plane, the 16-byte word offsets of the
// patient's non-zero 64-byte granules (four consecutive offsets per granule,
// fewer for a final partial granule), in ascending order, with a block-wide
// prefix sum; one CTA per (patient, plane).
#include "kernels.h"

namespace dbq {
namespace {

constexpr int kSupThreads = 1024;

__global__ void __launch_bounds__(kSupThreads)
support_kernel(const uint4* __restrict__ planes, int wp4, uint32_t* __restrict__ lists,
               uint32_t* __restrict__ lens)
{
    __shared__ uint32_t warp_tot[kSupThreads / 32];
    __shared__ uint32_t base_s;
    const int k = blockIdx.x;                       // plane
    const int64_t q = blockIdx.y;                   // patient
    const uint4* plane = planes + (q * 2 + k) * (int64_t)wp4;
    uint32_t* out = lists + (q * 2 + k) * (int64_t)wp4;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int granules = (wp4 + 3) / 4;
    if (tid == 0) base_s = 0;
    __syncthreads();
    for (int g0 = 0; g0 < granules; g0 += kSupThreads) {
        const int g = g0 + tid;
        uint32_t size = 0;
        if (g < granules) {
            const int first = 4 * g;
            const int cnt = (wp4 - first) < 4 ? (wp4 - first) : 4;
            bool nz = false;
            for (int r = 0; r < cnt; ++r) {
                const uint4 w = plane[first + r];
                nz |= (w.x | w.y | w.z | w.w) != 0u;
            }
            size = nz ? (uint32_t)cnt : 0u;
        }
        // exclusive prefix sum of `size` over the block
        uint32_t incl = size;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) warp_tot[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            uint32_t t = warp_tot[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t v = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += v;
            }
            warp_tot[lane] = t;        // inclusive totals per warp
        }
        __syncthreads();
        const uint32_t before = base_s + (warp ? warp_tot[warp - 1] : 0u) + incl - size;
        for (uint32_t r = 0; r < size; ++r) out[before + r] = 4u * (uint32_t)g + r;
        __syncthreads();
        if (tid == 0) base_s += warp_tot[31];
        __syncthreads();
    }
    if (tid == 0) lens[q * 2 + k] = base_s;
}

}  // namespace

cudaError_t launch_support(const uint32_t* planes, int nq, int wp4, uint32_t* lists,
                           uint32_t* lens, cudaStream_t stream)
{
    if (nq <= 0) return cudaSuccess;
    support_kernel<<<dim3(2, (unsigned)nq), kSupThreads, 0, stream>>>(
        reinterpret_cast<const uint4*>(planes), wp4, lists, lens);
    return cudaGetLastError();
}

}  // namespace dbq
