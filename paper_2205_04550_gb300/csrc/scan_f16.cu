// scan_f16.cu -- the brute-force query over a half-precision database whose
// thresholds are chosen per query.
//
// Ezhov et al. (2022), Section 2.3: the simulated concentrations are
// thresholded at u_T1Gd and u_FLAIR, and every entry's two segmentations are
// compared with the patient's by Dice.  Here the database keeps binary16
// concentrations, so each query thresholds every voxel of every entry at its
// own (t1, t2) and counts |E_k| and |P_k n E_k| on the fly.
//
// Threshold test: for a threshold t in (0, 1], let th be the smallest binary16
// value >= t (computed on the host).  For every binary16 h, (float)h >= t
// holds exactly when h >= th in an ordered half comparison (NaN, -0 and
// negatives compare false, +Inf true), so one HSET2 tests two voxels.
//
// GB300 mapping (one 1024-thread CTA per SM, persistent, contiguous entry
// range per CTA, like the packed scan):
//   * An entry row holds Vp = V rounded up to 1024 halves (zero padding).
//     A warp handles one block of 1024 voxels at a time: lane i loads the
//     four 16-byte words i, i+32, i+64, i+96 of the block (coalesced), tests
//     its 32 voxels against both thresholds (16 HSET2 each) and folds the
//     masks into one 32-bit word per threshold (bit r = low half of half2
//     word r, bit 16+r = its high half).
//   * The patient's bit planes are re-ordered once per chunk into shared
//     memory in exactly that bit order (one word per lane per block), so
//     I_k += popc(mask & patient) and E_k += popc(mask).
//   * Counts are reduced per warp with redux.sync into per-entry shared
//     counters; scores, running top-k and the last-CTA merge are the shared
//     routines of topk.cuh.
#include <cuda_fp16.h>

#include "kernels.h"
#include "topk.cuh"

namespace dbq {
namespace {

constexpr int kThreads = 1024;
constexpr int kWarps = kThreads / 32;
constexpr int kGroup = 512;          // entries whose counters live in shared memory
constexpr int kMaxChunkBlocks = 512; // 1024-voxel blocks per patient chunk (128 KiB)

// Two-voxel threshold test: 0xFFFF in each half of the result whose binary16
// value is >= the threshold in the same half of `th2` (ordered compare).
__device__ __forceinline__ uint32_t ge_mask_f16x2(uint32_t h2, uint32_t th2)
{
    uint32_t m;
    asm("set.ge.u32.f16x2 %0, %1, %2;" : "=r"(m) : "r"(h2), "r"(th2));
    return m;
}

// Fold the 16 two-voxel masks of 32 voxels into one word (bit r <- low half
// of 32-bit word r, bit 16 + r <- its high half; r = 4u + q for word q of
// the u-th 16-byte load).
__device__ __forceinline__ uint32_t fold_masks(const uint4 (&v)[4], uint32_t th2)
{
    uint32_t w = 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        w |= ge_mask_f16x2(v[u].x, th2) & (0x00010001u << (4 * u + 0));
        w |= ge_mask_f16x2(v[u].y, th2) & (0x00010001u << (4 * u + 1));
        w |= ge_mask_f16x2(v[u].z, th2) & (0x00010001u << (4 * u + 2));
        w |= ge_mask_f16x2(v[u].w, th2) & (0x00010001u << (4 * u + 3));
    }
    return w;
}

// Patient bits of the 32 voxels lane `i` of a warp covers in block `b`,
// in the order of fold_masks.  `words` are the plane's words of block b.
__device__ __forceinline__ uint32_t permute_patient(const uint32_t* words, int i)
{
    uint32_t out = 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const uint32_t byte = (words[8 * u + (i >> 2)] >> (8 * (i & 3))) & 0xffu;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            out |= ((byte >> (2 * q)) & 1u) << (4 * u + q);
            out |= ((byte >> (2 * q + 1)) & 1u) << (16 + 4 * u + q);
        }
    }
    return out;
}

__global__ void __launch_bounds__(kThreads, 1)
scan_f16_kernel(const ScanF16Args a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t* pp = reinterpret_cast<uint32_t*>(smem_raw);   // [2][chunk_blocks * 32]
    TopK tk;
    uint32_t* icnt = reinterpret_cast<uint32_t*>(
        topk_carve(tk, smem_raw + (size_t)2 * a.chunk_blocks * 32 * sizeof(uint32_t)));
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int k = a.k;
    const bool want_topk = a.hits != nullptr;
    const int64_t e_begin = (int64_t)blockIdx.x * a.n / gridDim.x;
    const int64_t e_end = ((int64_t)blockIdx.x + 1) * a.n / gridDim.x;
    const uint32_t P1 = a.pcount[0];
    const uint32_t P2 = a.pcount[1];
    const uint32_t th1 = a.th1x2;
    const uint32_t th2 = a.th2x2;
    const int row4 = a.blocks * 128;     // uint4 per entry row

    topk_init(tk);
    int loaded_chunk = -1;
    const int cb_max = a.chunk_blocks;

    for (int64_t g0 = e_begin; g0 < e_end; g0 += kGroup) {
        const int gn = (int)((e_end - g0) < kGroup ? (e_end - g0) : kGroup);
        for (int i = tid; i < 4 * kGroup; i += kThreads) icnt[i] = 0u;
        for (int c = 0; c < a.nchunks; ++c) {
            const int b0 = c * cb_max;
            const int cb = (a.blocks - b0) < cb_max ? (a.blocks - b0) : cb_max;
            if (loaded_chunk != c) {
                __syncthreads();
                for (int t = tid; t < cb * 32; t += kThreads) {
                    const int b = t >> 5, i = t & 31;
                    pp[t] = permute_patient(a.patient + (int64_t)(b0 + b) * 32, i);
                    pp[cb_max * 32 + t] =
                        permute_patient(a.patient + a.wp + (int64_t)(b0 + b) * 32, i);
                }
                loaded_chunk = c;
            }
            __syncthreads();
            for (int i0 = 0; i0 < gn; ++i0) {
                const uint4* row = a.vols + (g0 + i0) * (int64_t)row4 + (int64_t)b0 * 128;
                uint32_t ci1 = 0, ci2 = 0, ce1 = 0, ce2 = 0;
                for (int b = warp; b < cb; b += 2 * kWarps) {
                    uint4 v0[4], v1[4];
                    const bool second = b + kWarps < cb;
#pragma unroll
                    for (int u = 0; u < 4; ++u) v0[u] = ld_stream(row + b * 128 + lane + 32 * u);
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        v1[u] = second ? ld_stream(row + (b + kWarps) * 128 + lane + 32 * u)
                                       : make_uint4(0, 0, 0, 0);
                    {
                        const uint32_t m1 = fold_masks(v0, th1);
                        const uint32_t m2 = fold_masks(v0, th2);
                        ce1 += __popc(m1);
                        ce2 += __popc(m2);
                        ci1 += __popc(m1 & pp[b * 32 + lane]);
                        ci2 += __popc(m2 & pp[cb_max * 32 + b * 32 + lane]);
                    }
                    if (second) {
                        const int bb = b + kWarps;
                        const uint32_t m1 = fold_masks(v1, th1);
                        const uint32_t m2 = fold_masks(v1, th2);
                        ce1 += __popc(m1);
                        ce2 += __popc(m2);
                        ci1 += __popc(m1 & pp[bb * 32 + lane]);
                        ci2 += __popc(m2 & pp[cb_max * 32 + bb * 32 + lane]);
                    }
                }
                ci1 = __reduce_add_sync(0xffffffffu, ci1);
                ci2 = __reduce_add_sync(0xffffffffu, ci2);
                ce1 = __reduce_add_sync(0xffffffffu, ce1);
                ce2 = __reduce_add_sync(0xffffffffu, ce2);
                if (lane == 0) {
                    if (ci1) atomicAdd(&icnt[4 * i0 + 0], ci1);
                    if (ci2) atomicAdd(&icnt[4 * i0 + 1], ci2);
                    if (ce1) atomicAdd(&icnt[4 * i0 + 2], ce1);
                    if (ce2) atomicAdd(&icnt[4 * i0 + 3], ce2);
                }
            }
        }
        __syncthreads();
        for (int i = tid; i < gn; i += kThreads) {
            const int64_t e = g0 + i;
            const uint32_t I1 = icnt[4 * i], I2 = icnt[4 * i + 1];
            const uint32_t E1 = icnt[4 * i + 2], E2 = icnt[4 * i + 3];
            if (a.counts_out)
                reinterpret_cast<uint4*>(a.counts_out)[e] = make_uint4(I1, I2, E1, E2);
            if (want_topk)
                topk_offer_counts(tk, k, I1, I2, E1, E2, P1, P2, e);
        }
        if (want_topk) topk_flush(tk, k);
        else __syncthreads();
    }
    if (!want_topk) return;
    if (!topk_publish(tk, k, a.cand, a.ticket)) return;
    topk_merge_published(tk, k, a.cand, (int64_t)gridDim.x * k);
    for (int j = tid; j < k; j += kThreads) {
        Hit h;
        h.index = tk.idx[j];
        h.score = key_score(tk.key[j]);
        h.i1 = (uint32_t)(tk.pay0[j] & 0xffffffffu);
        h.i2 = (uint32_t)(tk.pay0[j] >> 32);
        h.e1 = (uint32_t)(tk.pay1[j] & 0xffffffffu);
        h.e2 = (uint32_t)(tk.pay1[j] >> 32);
        h.p1 = P1;
        h.p2 = P2;
        a.hits[j] = h;
    }
}

}  // namespace

void scan_f16_chunking(int blocks, int* chunk_blocks, int* nchunks)
{
    int nc = (blocks + kMaxChunkBlocks - 1) / kMaxChunkBlocks;
    if (nc < 1) nc = 1;
    int cb = (blocks + nc - 1) / nc;
    if (cb < 1) cb = 1;
    *chunk_blocks = cb;
    *nchunks = (blocks + cb - 1) / cb;
}

size_t scan_f16_smem(int chunk_blocks)
{
    return (size_t)2 * chunk_blocks * 32 * sizeof(uint32_t) + topk_smem_bytes() +
           (size_t)kGroup * 4 * sizeof(uint32_t);
}

uint16_t f16_threshold_bits(float t)
{
    // smallest non-negative binary16 pattern whose value is >= t; the values
    // of patterns 0 .. 0x7C00 increase with the pattern
    uint32_t lo = 0, hi = 0x7C00;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) / 2;
        const float v = __half2float(__ushort_as_half((unsigned short)mid));
        if (v >= t) hi = mid;
        else lo = mid + 1;
    }
    return (uint16_t)lo;
}

cudaError_t launch_scan_f16(const ScanF16Args& a, int grid, cudaStream_t stream)
{
    const size_t smem = scan_f16_smem(a.chunk_blocks);
    cudaError_t err = cudaFuncSetAttribute(scan_f16_kernel,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    scan_f16_kernel<<<grid, kThreads, smem, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace dbq
