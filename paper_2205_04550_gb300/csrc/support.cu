// support.cu -- the patient's support lists for the sparse exact scan.
//
// The Dice numerator |P_k n E_k| (Section 2.3 of Ezhov et al. 2022) only
// involves voxels inside the patient's mask P_k, so a scan may skip every
// database word whose patient word is zero and still produce the exact
// counts.  This kernel lists, per plane, the 16-byte word offsets of the
// patient's non-zero 64-byte granules (four consecutive offsets per granule,
// fewer for a final partial granule), in ascending order; one CTA per
// (patient, plane).
#include "kernels.h"

namespace dbq {
namespace {

constexpr int kSupThreads = 1024;
constexpr int kSupWarps = kSupThreads / 32;
constexpr int kSupBitmapGranules = 1 << 15;   // flags kept in shared memory up to here (4 KiB)

// Is granule g (words 4 g .. 4 g + 3, fewer at the end) of the plane non-zero?
__device__ __forceinline__ bool granule_nonzero(const uint4* plane, int wp4, int g)
{
    bool nz = false;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int w = 4 * g + r;
        if (w < wp4) {
            const uint4 v = plane[w];
            nz |= (v.x | v.y | v.z | v.w) != 0u;
        }
    }
    return nz;
}

// One CTA per (patient, plane).  Warp w owns a contiguous range of granules.
// Pass 1 counts its non-zero granules reading 512 bytes per warp load (eight
// loads in flight per lane; each granule's four words OR-ed across four
// lanes) and keeps the flags in shared memory (planes of up to 2^15
// granules; larger ones are read again); the warps' counts place each warp's
// list; pass 2 takes one granule per lane, 32 at a time, and writes the four
// word offsets of each non-zero granule (fewer for a final partial granule)
// in ascending order.
__global__ void __launch_bounds__(kSupThreads)
support_kernel(const uint4* __restrict__ planes, int wp4, uint32_t* __restrict__ lists,
               uint32_t* __restrict__ lens)
{
    __shared__ uint32_t warp_cnt[kSupWarps];
    __shared__ uint32_t flags[kSupBitmapGranules / 32];
    const int k = blockIdx.x;                       // plane
    const int64_t q = blockIdx.y;                   // patient
    const uint4* plane = planes + (q * 2 + k) * (int64_t)wp4;
    uint32_t* out = lists + (q * 2 + k) * (int64_t)wp4;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int granules = (wp4 + 3) / 4;
    const bool keep = granules <= kSupBitmapGranules;
    const int per = (granules + kSupWarps - 1) / kSupWarps;
    const int per8 = (per + 31) / 32 * 32;          // ranges of whole 32-granule flag words
    const int g0 = min(granules, warp * per8);
    const int g1 = min(granules, (warp + 1) * per8);
    uint32_t cnt = 0;
    // pass 1: lane l of load u reads word 4 g0 + 32 u + l (granule g0 + 8 u + l / 4)
    const int w0 = 4 * g0, w1 = min(wp4, 4 * g1);
    for (int b = w0; b < w1; b += 32 * 8) {
        uint4 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int w = b + 32 * u + lane;
            v[u] = w < w1 ? plane[w] : make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            uint32_t nz = (v[u].x | v[u].y | v[u].z | v[u].w) != 0u ? 1u : 0u;
            nz |= __shfl_xor_sync(0xffffffffu, nz, 1);
            nz |= __shfl_xor_sync(0xffffffffu, nz, 2);
            // one bit per granule: lanes 0, 4, ..., 28 (words past w1 read as 0)
            const unsigned m = __ballot_sync(0xffffffffu, nz != 0u) & 0x11111111u;
            cnt += __popc(m);
            if (keep) {                             // granules gfirst .. gfirst + 7: a byte
                uint32_t f = 0;
#pragma unroll
                for (int i = 0; i < 8; ++i) f |= ((m >> (4 * i)) & 1u) << i;
                const int gfirst = (b + 32 * u) / 4;
                // the warp's own flag words: one writer (lane 0), no race
                if (lane == 0 && gfirst < g1) {
                    const uint32_t sh = (uint32_t)(gfirst & 31);
                    flags[gfirst >> 5] = (sh ? flags[gfirst >> 5] : 0u) | (f << sh);
                }
            }
        }
    }
    if (lane == 0) warp_cnt[warp] = cnt;
    __syncthreads();
    uint32_t base = 0, total = 0;
    for (int i = 0; i < kSupWarps; ++i) {
        const uint32_t c = warp_cnt[i];
        base += i < warp ? c : 0u;
        total += c;
    }
    // pass 2
    const int tail = wp4 & 3;                       // words of a final partial granule
    uint32_t pos = base;                            // granules listed before
    for (int g = g0; g < g1; g += 32) {
        const int mine = g + lane;
        const bool nz = mine < g1 && (keep ? ((flags[g >> 5] >> lane) & 1u) != 0u
                                           : granule_nonzero(plane, wp4, mine));
        const unsigned m = __ballot_sync(0xffffffffu, nz);
        if (nz) {
            const uint32_t at = 4u * (pos + __popc(m & ((1u << lane) - 1u)));
            const int words = (tail && mine == granules - 1) ? tail : 4;
            for (int r = 0; r < words; ++r) out[at + r] = 4u * (uint32_t)mine + r;
        }
        pos += __popc(m);
    }
    if (warp == kSupWarps - 1 && lane == 0) {
        uint32_t len = 4u * total;
        if (tail && total > 0 && granule_nonzero(plane, wp4, granules - 1)) len -= 4u - tail;
        lens[q * 2 + k] = len;
    }
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
