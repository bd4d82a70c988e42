// select.cu -- the prefilter's candidate set: for each query the c entries
// with the smallest embedding distance L = L2_T1Gd + L2_FLAIR (Section 2.3
// of Ezhov et al. 2022 takes the smallest such sum as the best match of an
// embedding query; the prefilter keeps the c smallest for exact re-ranking).
//
// One 1024-thread CTA per query.  Distances are >= 0, so their binary32 bit
// patterns order like the values.  A radix selection over the bit patterns
// finds the cut: a 4096-bin histogram of the top 12 bits locates the bin
// holding the c-th smallest; entries in lower bins are in, the boundary bin
// is refined by the next 12 bits and then the last 8; what is left in the
// boundary then has one key and is taken in index order.  Each level reads
// the query's row twice (histogram, collection); rows stay in L2 between the
// passes.  The chosen c are finally sorted by (key, index), ascending.
#include "kernels.h"

namespace dbq {
namespace {

constexpr int kThreads = 1024;
constexpr int kBins = 4096;
constexpr int kCap = 1024;            // candidates kept (c <= kCap)
constexpr int kBoundaryCap = 2048;    // boundary-bin entries sorted directly

__device__ __forceinline__ uint32_t dist_bits(const float* row, int64_t e)
{
    return __float_as_uint(__ldcg(row + e));
}

// Block-wide bitonic sort of n (power of two) (key, idx) pairs, ascending
// by key then index.
__device__ void sort_pairs(uint32_t* key, int32_t* idx, int n)
{
    for (int size = 2; size <= n; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < (n >> 1); i += blockDim.x) {
                const int lo = 2 * i - (i & (stride - 1));
                const int hi = lo + stride;
                const bool up = (lo & size) == 0;
                const bool hi_first = key[hi] < key[lo] || (key[hi] == key[lo] && idx[hi] < idx[lo]);
                if (hi_first == up) {
                    const uint32_t k = key[lo]; key[lo] = key[hi]; key[hi] = k;
                    const int32_t x = idx[lo]; idx[lo] = idx[hi]; idx[hi] = x;
                }
            }
            __syncthreads();
        }
    }
}

// Inclusive prefix sums of hist[0..kBins) in place (1024 threads, 4 bins
// each).
__device__ void prefix_bins(uint32_t* hist, uint32_t* warp_tot)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t v[4];
    uint32_t run = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        run += hist[4 * tid + j];
        v[j] = run;
    }
    uint32_t incl = run;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t t = warp_tot[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += u;
        }
        warp_tot[lane] = t;
    }
    __syncthreads();
    const uint32_t before = (warp ? warp_tot[warp - 1] : 0u) + incl - run;
#pragma unroll
    for (int j = 0; j < 4; ++j) hist[4 * tid + j] = before + v[j];
    __syncthreads();
}

__global__ void __launch_bounds__(kThreads, 1)
select_smallest_kernel(const float* __restrict__ dist, int64_t n, int c, int32_t* __restrict__ cand)
{
    __shared__ uint32_t hist[kBins];
    __shared__ uint32_t out_key[kCap];
    __shared__ int32_t out_idx[kCap];
    __shared__ uint32_t bd_key[kBoundaryCap];
    __shared__ int32_t bd_idx[kBoundaryCap];
    __shared__ uint32_t warp_tot[32];
    __shared__ int n_out, n_bd, s_bin;
    __shared__ uint32_t s_below;
    const int tid = threadIdx.x;
    const float* row = dist + (int64_t)blockIdx.x * n;

    // levels: (shift, width) = (20, 12), (8, 12), (0, 8)
    uint32_t prefix = 0;        // bits above the current level of the boundary
    int need = c;               // how many still to take from the boundary
    if (tid == 0) n_out = 0;
    int level = 0;
    for (; level < 3; ++level) {
        const int shift = level == 0 ? 20 : (level == 1 ? 8 : 0);
        const int width = level == 2 ? 8 : 12;
        const int top = shift + width;                 // bits [top, 32) must equal prefix
        for (int b = tid; b < kBins; b += kThreads) hist[b] = 0;
        __syncthreads();
        for (int64_t e = tid; e < n; e += kThreads) {
            const uint32_t u = dist_bits(row, e);
            if (top >= 32 || (u >> top) == prefix)
                atomicAdd(&hist[(u >> shift) & ((1u << width) - 1u)], 1u);
        }
        __syncthreads();
        prefix_bins(hist, warp_tot);
        // boundary bin: the first whose inclusive count reaches `need`
        for (int b = tid; b < kBins; b += kThreads) {
            const uint32_t incl = hist[b];
            const uint32_t excl = b ? hist[b - 1] : 0u;
            if (excl < (uint32_t)need && incl >= (uint32_t)need) {
                s_bin = b;
                s_below = excl;
            }
        }
        __syncthreads();
        const int bin = s_bin;
        const uint32_t below = s_below;
        const uint32_t in_bin = hist[bin] - below;
        // entries below the boundary bin are certainly in
        if (tid == 0) n_bd = 0;
        __syncthreads();
        const bool last = level == 2 || in_bin <= (uint32_t)kBoundaryCap;
        for (int64_t e = tid; e < n; e += kThreads) {
            const uint32_t u = dist_bits(row, e);
            if (top < 32 && (u >> top) != prefix) continue;
            const int b = (int)((u >> shift) & ((1u << width) - 1u));
            if (b < bin) {
                const int pos = atomicAdd(&n_out, 1);
                out_key[pos] = u;
                out_idx[pos] = (int32_t)e;
            } else if (b == bin && last && level < 2) {
                const int pos = atomicAdd(&n_bd, 1);
                bd_key[pos] = u;
                bd_idx[pos] = (int32_t)e;
            }
        }
        __syncthreads();
        need -= (int)below;
        prefix = (prefix << width) | (uint32_t)bin;
        if (last) break;
    }
    if (level < 3 && level < 2) {
        // the boundary bin fits: sort it and take the `need` smallest
        const int nb = n_bd;
        int n2 = 1;
        while (n2 < nb) n2 <<= 1;
        for (int i = nb + tid; i < n2; i += kThreads) {
            bd_key[i] = 0xffffffffu;
            bd_idx[i] = 0x7fffffff;
        }
        __syncthreads();
        sort_pairs(bd_key, bd_idx, n2);
        for (int i = tid; i < need; i += kThreads) {
            out_key[n_out + i] = bd_key[i];
            out_idx[n_out + i] = bd_idx[i];
        }
        __syncthreads();
    } else {
        // every boundary entry has the same key (`prefix`): take the `need`
        // lowest indices, scanning the row in index order
        __shared__ int s_taken;
        if (tid == 0) s_taken = 0;
        __syncthreads();
        for (int64_t e0 = 0; e0 < n; e0 += kThreads) {
            const int64_t e = e0 + tid;
            const bool hit = e < n && dist_bits(row, e) == prefix;
            const unsigned mask = __ballot_sync(0xffffffffu, hit);
            const int lane = tid & 31, warp = tid >> 5;
            if (lane == 0) warp_tot[warp] = __popc(mask);
            __syncthreads();
            int before = s_taken;
            for (int w = 0; w < warp; ++w) before += (int)warp_tot[w];
            before += __popc(mask & ((1u << lane) - 1u));
            if (hit && before < need) {
                out_key[n_out + before] = prefix;
                out_idx[n_out + before] = (int32_t)e;
            }
            __syncthreads();
            if (tid == 0) {
                int tot = 0;
                for (int w = 0; w < 32; ++w) tot += (int)warp_tot[w];
                s_taken += tot;
            }
            __syncthreads();
            if (s_taken >= need) break;
        }
    }
    // the c chosen, ascending by (key, index)
    int n2 = 1;
    while (n2 < c) n2 <<= 1;
    for (int i = c + tid; i < n2; i += kThreads) {
        out_key[i] = 0xffffffffu;
        out_idx[i] = 0x7fffffff;
    }
    __syncthreads();
    sort_pairs(out_key, out_idx, n2);
    for (int j = tid; j < c; j += kThreads) cand[(int64_t)blockIdx.x * c + j] = out_idx[j];
}

}  // namespace

cudaError_t launch_select_smallest(const float* dist, int nq, int64_t n, int c, int32_t* cand,
                                   cudaStream_t stream)
{
    if (nq < 1 || c < 1 || c > kCap || c > n || n > 0x7fffffff) return cudaErrorInvalidValue;
    select_smallest_kernel<<<nq, kThreads, 0, stream>>>(dist, n, c, cand);
    return cudaGetLastError();
}

}  // namespace dbq
