// select.cu -- the prefilter's candidate set: for each query the c entries
// with the smallest embedding distance L = L2_T1Gd + L2_FLAIR (Section 2.3
// of Ezhov et al. 2022 takes the smallest such sum as the best match of an
// embedding query; the prefilter keeps the c smallest for exact re-ranking).
//
// One 512-thread CTA per query streams its row of distances and keeps a
// running top-c with the shared-memory routines of topk.cuh; the key is the
// complement of L's bit pattern so that "better" means "closer", and ties
// go to the lower index.
#include "kernels.h"
#include "topk.cuh"

namespace dbq {
namespace {

constexpr int kSelectThreads = 512;

// Rounds of kSelectThreads distances (one coalesced load per thread); the
// append buffer is merged only when the next round might not fit, so the
// k-th best used as the offer threshold tightens quickly and most rounds
// append nothing.  Three CTAs fit on an SM (64 KiB of shared memory each).
__global__ void __launch_bounds__(kSelectThreads)
select_smallest_kernel(const float* __restrict__ dist, int64_t n, int c, int32_t* __restrict__ cand)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TopK tk;
    topk_carve(tk, smem_raw);
    const float* row = dist + (int64_t)blockIdx.x * n;
    topk_init(tk);
    const int room = kTopkCap - c;            // append slots
    for (int64_t r0 = 0; r0 < n; r0 += kSelectThreads) {
        const int64_t e = r0 + threadIdx.x;
        if (e < n) topk_offer(tk, c, distance_key(__ldcs(row + e)), e, 0, 0);
        __syncthreads();
        const int added = tk.misc[0];
        __syncthreads();   // every thread has read the count before the next round appends
        if (added > room - kSelectThreads) topk_flush(tk, c);
    }
    topk_flush(tk, c);
    for (int j = threadIdx.x; j < c; j += kSelectThreads)
        cand[(int64_t)blockIdx.x * c + j] = (int32_t)tk.idx[j];
}

}  // namespace

cudaError_t launch_select_smallest(const float* dist, int nq, int64_t n, int c, int32_t* cand,
                                   cudaStream_t stream)
{
    if (nq < 1 || c < 1 || c > 1024 || c > n || kTopkCap - c < kSelectThreads)
        return cudaErrorInvalidValue;
    const size_t smem = topk_smem_bytes();
    cudaError_t err = cudaFuncSetAttribute(select_smallest_kernel,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    select_smallest_kernel<<<nq, kSelectThreads, smem, stream>>>(dist, n, c, cand);
    return cudaGetLastError();
}

}  // namespace dbq
