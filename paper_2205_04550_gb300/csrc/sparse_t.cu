// sparse_t.cu -- the sparse scan over a word-major copy of the bit planes.
//
// The intersection counts of Section 2.3 (Ezhov et al. 2022) only need the
// 16-byte words where the patient's masks are non-zero (the support lists of
// support.cu).  In the entry-major planes ([n][2][wp4], one entry's planes
// contiguous) those words are 64-byte granules in short runs inside each
// 512 KiB entry, scattered over the whole database, and HBM serves such
// reads well below its streaming rate.  A word-major copy ([2 wp4][n]: word
// w of every entry contiguous) turns the same reads into one contiguous run
// of n x 16 bytes per support word, read by whole warps 512 bytes at a time.
// The copy doubles the planes' device memory and is built on demand
// (transpose_planes_kernel) after the database changes.
//
// Counting: a CTA of kCountThreads threads owns kCountThreads consecutive
// entries (one per thread) of one patient and one of `splits` slices of that
// patient's support positions, streams those words of its entries (twelve 16-byte loads
// in flight per thread, 64 registers: four CTAs per SM; eight loads measured
// 7 % slower) and adds its partial counts into the per-entry
// counters with one atomic per entry and plane.  The fused scan
// (scan_packed.cu) then scores and ranks the entries from the counters.
#include "kernels.h"
#include "common.cuh"

namespace dbq {
namespace {

constexpr int kTransposeTile = 32;      // 32 x 32 words of 16 bytes per CTA
constexpr int kCountThreads = 256;
constexpr int kCountChunk = 2048;       // support positions cached per pass (40 KiB)

// planes [n][w4] -> planes_t [w4][n], 16-byte words; 32 x 8 threads, each
// moving four words of a 32 x 32 tile through shared memory (reads and writes
// both 512 contiguous bytes per warp).  blockIdx.x is the entry tile; the word
// tiles are blockIdx.y, blockIdx.y + gridDim.y, ...
__global__ void __launch_bounds__(256)
transpose_planes_kernel(const uint4* __restrict__ planes, int64_t n, int w4,
                        uint4* __restrict__ planes_t)
{
    __shared__ uint4 tile[kTransposeTile][kTransposeTile + 1];
    const int64_t e0 = (int64_t)blockIdx.x * kTransposeTile;
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int w0 = blockIdx.y * kTransposeTile; w0 < w4; w0 += gridDim.y * kTransposeTile) {
        __syncthreads();                       // the previous tile has been written out
#pragma unroll
        for (int r = ty; r < kTransposeTile; r += 8) {
            const int64_t e = e0 + r;
            const int w = w0 + tx;
            if (e < n && w < w4) tile[r][tx] = __ldcs(planes + e * w4 + w);
        }
        __syncthreads();
#pragma unroll
        for (int r = ty; r < kTransposeTile; r += 8) {
            const int w = w0 + r;
            const int64_t e = e0 + tx;
            if (e < n && w < w4) __stcs(planes_t + (int64_t)w * n + e, tile[tx][r]);
        }
    }
}

// Partial counts of entries [blockIdx.y * kCountThreads, +kCountThreads) of
// query blockIdx.x (the fastest grid index, so CTAs running together read the
// same entries for different patients) over support slice blockIdx.z of
// gridDim.z: positions p of the query's concatenated support (plane 1's list,
// then plane 2's), word off(p) of the entry-major layout = row off(p) of
// planes_t.  Query q's patient is patient + q * 2 wp4, its lists sup_list +
// q * 2 wp4 and lengths sup_len + 2 q; entry e's counters are
// counts[q * qstride + e * estride] (plane 1) and the same + poff (plane 2).
__global__ void __launch_bounds__(kCountThreads, 4)
sparse_t_count_kernel(const uint4* __restrict__ planes_t, int64_t n,
                      const uint4* __restrict__ patients, int wp4,
                      const uint32_t* __restrict__ sup_lists,
                      const uint32_t* __restrict__ sup_lens, uint32_t* __restrict__ counts,
                      int64_t qstride, int64_t estride, int64_t poff)
{
    __shared__ uint32_t s_off[kCountChunk];
    __shared__ uint4 s_pw[kCountChunk];
    const int q = blockIdx.x;
    const uint4* patient = patients + (int64_t)q * 2 * wp4;
    const uint32_t* sup_list = sup_lists + (int64_t)q * 2 * wp4;
    const int l1 = (int)sup_lens[2 * q], l2 = (int)sup_lens[2 * q + 1];
    const int total = l1 + l2;
    const int p0 = (int)((int64_t)total * blockIdx.z / gridDim.z);
    const int p1 = (int)((int64_t)total * (blockIdx.z + 1) / gridDim.z);
    const int64_t e = (int64_t)blockIdx.y * kCountThreads + threadIdx.x;
    const bool live = e < n;
    const uint4* col = planes_t + (live ? e : 0);
    uint32_t a1 = 0, a2 = 0;
    for (int c0 = p0; c0 < p1; c0 += kCountChunk) {
        const int cn = min(kCountChunk, p1 - c0);
        __syncthreads();                       // the previous chunk is no longer read
        for (int j = threadIdx.x; j < cn; j += kCountThreads) {
            const int p = c0 + j;
            const uint32_t o = p < l1 ? sup_list[p] : (uint32_t)wp4 + sup_list[wp4 + (p - l1)];
            s_off[j] = o;
            s_pw[j] = patient[o];
        }
        __syncthreads();
        for (int j = 0; j < cn; j += 12) {
            uint4 v[12];
#pragma unroll
            for (int u = 0; u < 12; ++u)
                v[u] = (live && j + u < cn) ? ld_stream(col + (int64_t)s_off[j + u] * n)
                                            : make_uint4(0, 0, 0, 0);
#pragma unroll
            for (int u = 0; u < 12; ++u) {
                if (j + u < cn) {
                    const uint32_t c = popc_and4(v[u], s_pw[j + u]);
                    if (c0 + j + u < l1) a1 += c;
                    else a2 += c;
                }
            }
        }
    }
    if (live) {
        uint32_t* c = counts + (int64_t)q * qstride + e * estride;
        if (a1) atomicAdd(c, a1);
        if (a2) atomicAdd(c + poff, a2);
    }
}

}  // namespace

cudaError_t launch_transpose_planes(const uint4* planes, int64_t n, int w4, uint4* planes_t,
                                    cudaStream_t stream)
{
    if (n <= 0 || w4 <= 0) return cudaSuccess;
    const int64_t tx = (n + kTransposeTile - 1) / kTransposeTile;
    const int wt = (w4 + kTransposeTile - 1) / kTransposeTile;
    const dim3 grid((unsigned)tx, (unsigned)(wt < 1024 ? wt : 1024));
    transpose_planes_kernel<<<grid, dim3(kTransposeTile, 8), 0, stream>>>(planes, n, w4,
                                                                         planes_t);
    return cudaGetLastError();
}

cudaError_t launch_sparse_t_count(const uint4* planes_t, int64_t n, int nq, const uint4* patients,
                                  int wp4, const uint32_t* sup_lists, const uint32_t* sup_lens,
                                  uint32_t* counts, int64_t qstride, int64_t estride,
                                  int64_t poff, int sms, cudaStream_t stream)
{
    if (n <= 0 || nq <= 0) return cudaSuccess;
    const int64_t by = (n + kCountThreads - 1) / kCountThreads;
    // enough CTAs for about eight per SM (two waves of four)
    int64_t splits = (8LL * sms + by * nq - 1) / (by * nq);
    if (splits < 1) splits = 1;
    if (splits > 64) splits = 64;
    const dim3 grid((unsigned)nq, (unsigned)by, (unsigned)splits);
    sparse_t_count_kernel<<<grid, kCountThreads, 0, stream>>>(planes_t, n, patients, wp4,
                                                              sup_lists, sup_lens, counts,
                                                              qstride, estride, poff);
    return cudaGetLastError();
}

}  // namespace dbq
