// gemm_tc.cu -- L2 prefilter distances on the 5th-generation tensor cores.
//
// For every (query q, entry e) and each segmentation k the squared L2
// distance of the embeddings is |q_k|^2 + |e_k|^2 - 2 q_k . e_k; the
// prefilter's distance is L = d_1 + d_2 with d_k the (non-squared) distance,
// following the paper's L2_T1Gd + L2_FLAIR combination (Section 2.3).  The
// dot products are a dense contraction (Q queries x N entries x D dims per
// segmentation), so they run as a tcgen05 GEMM with fp32 accumulation in
// tensor memory.  The same kernel gives the Hamming distance of binary codes
// stored as E4M3 0/1 bytes: with the popcounts as norms, |q| + |e| - 2 q.e
// summed over the two segmentations is exact (integer products and sums
// below 2^24 in binary32), so no square root is taken.
//
//   * one CTA per SM, clusters of two CTAs on neighbouring SMs that run one
//     2-SM MMA together (tcgen05 cta_group::2, M = 256 entries: 128 in each
//     CTA's TMEM), persistent over 256-entry tiles;
//   * warp 0 of each CTA (one thread) issues TMA loads of 128-byte-swizzled
//     K-slices of its 128 entry rows and of half of the 256 query rows into
//     a 6-stage shared-memory ring; both CTAs' loads complete on the leader
//     CTA's full barrier, so each SM fills only half of the query tile (the
//     MMA reads the other half from the peer's shared memory);
//   * warp 1 of each CTA allocates 512 TMEM columns as a pair; one thread of
//     the leader issues tcgen05.mma.cta_group::2 (N = 256 queries, K = 16
//     bf16 or 32 fp8 per instruction): columns [0, 256) accumulate
//     q_1 . e_1, [256, 512) q_2 . e_2; its commits free each stage in both
//     CTAs and, per segmentation, tell both epilogues that the columns are
//     complete;
//   * warps 2-17 read the accumulators with tcgen05.ld (a warp may only touch
//     its 32-lane quarter, warp % 4; four warps share a quarter and take 64
//     query columns each), form L in binary32 and store L[q][e] coalesced.
//     Each segmentation's columns are handed back as soon as they are read,
//     so the epilogue of one tile runs under the MMAs of the next.  The square
//     roots use the SFU's sqrt.approx.f32 (relative error about 2^-23): the
//     correctly rounded square root with its special-case path doubled the
//     launch time, and the error is far inside the tolerance of the binary32
//     accumulation.
// Every mbarrier wait is bounded (iteration count and %globaltimer); on a
// timeout the CTA records an error code in `status`, stops issuing work,
// waits (bounded) for the copies and MMAs it has in flight, frees its TMEM
// and returns.
#include <cuda.h>

#include "kernels.h"
#include "tcgen05.cuh"

namespace dbq {
namespace {

constexpr int kBM = 128;          // entries per CTA (TMEM lanes); 256 per CTA pair
constexpr int kBN = 256;          // queries per launch (MMA N)
constexpr int kStages = 6;
constexpr int kTileABytes = kBM * 128;   // 128 rows x 128 bytes (one swizzle atom wide)
constexpr int kTileBBytes = kBN * 128;
constexpr int kStageBytes = kTileABytes + kTileBBytes / 2;   // per CTA: its A rows, half of B
constexpr int kEpiWarps = 16;            // four per TMEM lane quarter, 64 columns each
constexpr int kEpiCols = kBN / (kEpiWarps / 4);
constexpr int kThreads = 64 + 32 * kEpiWarps;   // warp 0 TMA, warp 1 MMA, warps 2-17 epilogue
constexpr int kCluster = 2;                               // the CTA pair of one MMA

// TMA load into this CTA's shared memory whose completion is signalled on an
// mbarrier of either CTA of the pair (a shared::cluster address).
__device__ __forceinline__ void tma_load_2d_pair(uint32_t dst, const CUtensorMap* map,
                                                 uint32_t bar_cluster, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar_cluster), "r"(x), "r"(y)
        : "memory");
}

// The shared::cluster address of this CTA's shared variable `saddr` in CTA
// `rank` of the cluster.
__device__ __forceinline__ uint32_t map_to_rank(uint32_t saddr, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
    return r;
}

__device__ __forceinline__ void mbar_arrive_cluster(uint32_t bar_cluster)
{
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar_cluster)
                 : "memory");
}

__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release;\n barrier.cluster.wait.acquire;" ::: "memory");
}

// One MMA of the CTA pair: D (M = 256 rows, 128 in each CTA's TMEM) +=
// A (each CTA's 128 rows at `adesc` in its own shared memory) x B^T (N = 256
// columns, 128 from each CTA's shared memory at `bdesc`).
template <bool kFp8>
__device__ __forceinline__ void umma_pair(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accumulate)
{
    if (kFp8) {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    } else {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    }
}

// Arrives on the mbarrier at this offset in both CTAs of the pair once the
// pair MMAs issued so far by this thread have completed.
__device__ __forceinline__ void umma_commit_pair(uint32_t bar)
{
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
        " [%0], %1;" ::"r"(bar), "h"((uint16_t)3)
        : "memory");
}

__device__ __forceinline__ float sqrt_approx(float x)
{
    float y;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Instruction descriptor: fp32 accumulator, A/B K-major, M = 256 (the CTA
// pair), N = 256; operand format bf16 (kind::f16) or E4M3 (kind::f8f6f4).
template <bool kFp8>
__host__ __device__ constexpr uint32_t instr_desc()
{
    return (1u << 4)                                   // D format: f32
           | ((kFp8 ? 0u : 1u) << 7)                   // A format: e4m3 / bf16
           | ((kFp8 ? 0u : 1u) << 10)                  // B format
           | ((uint32_t)(kBN >> 3) << 17)              // N / 8
           | ((uint32_t)((kCluster * kBM) >> 4) << 24);   // M / 16
}

template <bool kFp8, bool kHam>
__global__ void __cluster_dims__(kCluster, 1, 1) __launch_bounds__(kThreads, 1)
prefilter_gemm_kernel(const __grid_constant__ CUtensorMap tm_e,
                      const __grid_constant__ CUtensorMap tm_q, GemmArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte alignment for the swizzle atoms
    unsigned char* base = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char* ring = base;                                   // kStages x kStageBytes
    uint64_t* bars = reinterpret_cast<uint64_t*>(ring + kStages * kStageBytes);
    // bars: full[kStages], empty[kStages], seg_full[2], seg_free[2], drain
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kStages + 5);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    float* qnorm = reinterpret_cast<float*>(tmem_slot + 4);       // [2][kBN]
    float* qscale = qnorm + 2 * kBN;                               // [2][kBN]

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int ktiles = a.dims / (kFp8 ? 128 : 64);                 // K-slices per segmentation
    const int rank = (int)cluster_rank();
    const bool leader = rank == 0;
    const int pair0 = blockIdx.x / kCluster, npairs_grid = gridDim.x / kCluster;
    const int npairs = (int)((a.n + kCluster * kBM - 1) / (kCluster * kBM));

    const uint32_t full0 = smem_u32(bars);
    const uint32_t empty0 = smem_u32(bars + kStages);
    // seg_full[k]: the MMAs of segmentation k of the current tile are done
    // (both CTAs); seg_free[k] (the leader's): both CTAs' epilogues have read
    // TMEM columns [k*256, k*256+256)
    const uint32_t seg_full0 = smem_u32(bars + 2 * kStages);
    const uint32_t seg_free0 = smem_u32(bars + 2 * kStages + 2);
    const uint32_t drain = smem_u32(bars + 2 * kStages + 4);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(full0 + 8 * s, 1);             // the leader's producer, plus bytes
            mbar_init(empty0 + 8 * s, 1);            // the leader's MMA commit
        }
        for (int k = 0; k < 2; ++k) {
            mbar_init(seg_full0 + 8 * k, 1);
            mbar_init(seg_free0 + 8 * k, kCluster * 32 * kEpiWarps);
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int i = threadIdx.x; i < 2 * kBN; i += blockDim.x) {
        const int q = i % kBN, k = i / kBN;
        qnorm[i] = q < a.nq ? a.qnorm[2 * q + k] : 0.0f;
        qscale[i] = (kFp8 && !kHam && q < a.nq) ? a.qscale[2 * q + k] : 1.0f;
    }
    if (warp == 1) {
        // one warp of each CTA of the pair allocates together
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                         smem_u32(tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    // the peer's barriers must be initialised before either CTA signals them
    cluster_sync();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    // the leader's barriers as seen from this CTA
    const uint32_t full0_lead = map_to_rank(full0, 0);
    const uint32_t seg_free0_lead = map_to_rank(seg_free0, 0);

    uint32_t issued = 0;     // producer: stage loads issued

    if (warp == 0) {
        if (lane == 0) {
            uint32_t it = 0;
            bool ok = true;
            for (int pair = pair0; pair < npairs && ok; pair += npairs_grid) {
                // this CTA's 128 entries of the pair's 256 (past the last
                // entry the TMA reads zeros)
                const int row0 = pair * (kCluster * kBM) + rank * kBM;
                for (int seg = 0; seg < 2 && ok; ++seg) {
                    for (int kt = 0; kt < ktiles; ++kt, ++it) {
                        const int s = it % kStages;
                        const uint32_t ph = ((it / kStages) & 1) ^ 1;
                        if (!mbar_wait(empty0 + 8 * s, ph, abort_flag)) { ok = false; break; }
                        const uint32_t sa = smem_u32(ring + s * kStageBytes);
                        const uint32_t sb = sa + kTileABytes;
                        // the leader's full barrier counts both CTAs' bytes
                        if (leader) mbar_arrive_expect_tx(full0 + 8 * s, kCluster * kStageBytes);
                        const int x = seg * a.dims + kt * (kFp8 ? 128 : 64);
                        tma_load_2d_pair(sa, &tm_e, full0_lead + 8 * s, x, row0);
                        tma_load_2d_pair(sb, &tm_q, full0_lead + 8 * s, x, rank * (kBN / 2));
                        ++issued;
                    }
                }
            }
            if (!ok) {
                a.status[0] = 1;
                *abort_flag = 1;
            }
        }
    } else if (warp == 1) {
        if (lane == 0 && leader) {
            constexpr uint32_t idesc = instr_desc<kFp8>();
            uint32_t it = 0, tiles_done = 0;
            bool ok = true;
            for (int pair = pair0; pair < npairs && ok; pair += npairs_grid, ++tiles_done) {
                for (int seg = 0; seg < 2 && ok; ++seg) {
                    // both CTAs have read the previous tile's columns of this
                    // segmentation
                    if (!mbar_wait(seg_free0 + 8 * seg, (tiles_done & 1) ^ 1, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d_tmem = tmem + seg * kBN;
                    for (int kt = 0; kt < ktiles; ++kt, ++it) {
                        const int s = it % kStages;
                        if (!mbar_wait(full0 + 8 * s, (it / kStages) & 1, abort_flag)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t sa = smem_u32(ring + s * kStageBytes);
                        const uint32_t sb = sa + kTileABytes;
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            // K step of 32 bytes inside the 128-byte swizzle atom
                            umma_pair<kFp8>(d_tmem, sw128_desc(sa + 32 * kk),
                                            sw128_desc(sb + 32 * kk), idesc,
                                            (kt > 0 || kk > 0) ? 1u : 0u);
                        }
                        // frees the stage in both CTAs when these MMAs finish
                        umma_commit_pair(empty0 + 8 * s);
                    }
                    if (ok) umma_commit_pair(seg_full0 + 8 * seg);
                }
            }
            if (!ok) {
                a.status[0] = 2;
                *abort_flag = 1;
            }
            // every MMA issued by this thread has completed once `drain` fires;
            // TMEM is released only after that (or after the time limit)
            umma_commit_pair(drain);
            if (!mbar_wait(drain, 0, nullptr)) a.status[0] = 3;
        }
    } else {
        // epilogue warps 2..17: TMEM lane quarter = warp % 4, 64 columns by
        // warp.  Each CTA holds its own 128 rows of the pair's accumulator.
        // The first segmentation's distances are taken into registers as
        // soon as its MMAs finish (the second's run meanwhile), which frees
        // its columns for the next tile; the second's are combined and stored
        // while the next tile's first segmentation is being accumulated.
        const int quarter = warp & 3;
        const int c_begin = ((warp - 2) / 4) * kEpiCols;
        const int row = quarter * 32 + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16) + c_begin;
        uint32_t tiles_done = 0;
        for (int pair = pair0; pair < npairs; pair += npairs_grid, ++tiles_done) {
            const int64_t e = (int64_t)pair * (kCluster * kBM) + rank * kBM + row;
            const bool valid = e < a.n;
            float en0 = 0.f, en1 = 0.f, es0 = 1.f, es1 = 1.f;
            if (valid) {
                en0 = a.enorm[2 * e];
                en1 = a.enorm[2 * e + 1];
                if (kFp8 && !kHam) {
                    es0 = a.escale[2 * e];
                    es1 = a.escale[2 * e + 1];
                }
            }
            if (!mbar_wait(seg_full0, tiles_done & 1, abort_flag)) {
                a.status[0] = 4;
                *abort_flag = 1;
                break;
            }
            tc_fence_after();
            float d0[kEpiCols];
#pragma unroll
            for (int cc = 0; cc < kEpiCols / 16; ++cc) {
                uint32_t r[16];
                tmem_ld16(lane_base + 16 * cc, r);
                tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int q = c_begin + 16 * cc + j;
                    float dot = __uint_as_float(r[j]);
                    if (kHam) {
                        // 0/1 codes: |q| + |e| - 2 q.e, exact in binary32
                        d0[16 * cc + j] = qnorm[q] + en0 - 2.0f * dot;
                        continue;
                    }
                    if (kFp8) dot = dot * (qscale[q] * es0);
                    d0[16 * cc + j] = sqrt_approx(fmaxf(qnorm[q] + en0 - 2.0f * dot, 0.0f));
                }
            }
            tc_fence_before();
            mbar_arrive_cluster(seg_free0_lead);
            if (!mbar_wait(seg_full0 + 8, tiles_done & 1, abort_flag)) {
                a.status[0] = 4;
                *abort_flag = 1;
                break;
            }
            tc_fence_after();
#pragma unroll
            for (int cc = 0; cc < kEpiCols / 16; ++cc) {
                uint32_t r[16];
                tmem_ld16(lane_base + kBN + 16 * cc, r);
                tmem_wait_ld();
                if (valid) {
                    const int c = c_begin + 16 * cc;
                    float* out = a.dist + (int64_t)c * a.n + e;
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int q = c + j;
                        if (q < a.nq) {
                            float dot = __uint_as_float(r[j]);
                            if (kHam) {
                                out[(int64_t)j * a.n] =
                                    d0[16 * cc + j] + (qnorm[kBN + q] + en1 - 2.0f * dot);
                                continue;
                            }
                            if (kFp8) dot = dot * (qscale[kBN + q] * es1);
                            const float s1 = fmaxf(qnorm[kBN + q] + en1 - 2.0f * dot, 0.0f);
                            out[(int64_t)j * a.n] = d0[16 * cc + j] + sqrt_approx(s1);
                        }
                    }
                }
            }
            tc_fence_before();
            mbar_arrive_cluster(seg_free0_lead + 8);
        }
    }

    __syncthreads();
    if (warp == 0 && lane == 0 && leader && *abort_flag) {
        // let the loads already issued land before shared memory is released:
        // the last fill of stage s completed phase (count_s - 1)
        for (int s = 0; s < kStages; ++s) {
            const uint32_t count_s = (issued + kStages - 1 - s) / kStages;
            if (count_s == 0) continue;
            mbar_wait(full0 + 8 * s, (count_s - 1) & 1, nullptr);
        }
    }
    __syncthreads();
    // the leader's MMAs (which read the peer's shared memory and write its
    // TMEM) have completed before either CTA releases anything
    cluster_sync();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, 512;" ::"r"(tmem)
                     : "memory");
    }
    cluster_sync();
}

bool make_map(CUtensorMap* m, const void* base, bool fp8, int64_t rows, int64_t cols, int box_rows)
{
    EncodeTiledFn enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)cols * (fp8 ? 1 : 2)};
    const cuuint32_t box[2] = {(cuuint32_t)(fp8 ? 128 : 64), (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return enc(m, fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
               const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

EncodeTiledFn tensor_map_encoder()
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

size_t gemm_smem_bytes()
{
    return 1024 + (size_t)kStages * kStageBytes + (2 * kStages + 5) * 8 + 16 + 4 * kBN * 4;
}

int gemm_max_queries() { return kBN; }

template <bool kFp8, bool kHam>
cudaError_t launch_kind(const CUtensorMap& tm_e, const CUtensorMap& tm_q, const GemmArgs& a,
                        int grid, size_t smem, cudaStream_t stream)
{
    cudaError_t err = cudaFuncSetAttribute(prefilter_gemm_kernel<kFp8, kHam>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    prefilter_gemm_kernel<kFp8, kHam><<<grid, kThreads, smem, stream>>>(tm_e, tm_q, a);
    return cudaGetLastError();
}

cudaError_t launch_prefilter_gemm(const GemmArgs& a, int kind, int grid, cudaStream_t stream)
{
    const bool fp8 = kind != kGemmBf16;
    if (kind < kGemmBf16 || kind > kGemmHamming) return cudaErrorInvalidValue;
    if (a.nq < 1 || a.nq > kBN || a.n < 1 || a.dims % (fp8 ? 128 : 64) != 0)
        return cudaErrorInvalidValue;
    CUtensorMap tm_e, tm_q;
    const void* eb = fp8 ? (const void*)a.e_f8 : (const void*)a.e_bf16;
    const void* qb = fp8 ? (const void*)a.q_f8 : (const void*)a.q_bf16;
    if (!make_map(&tm_e, eb, fp8, a.n, 2 * (int64_t)a.dims, kBM) ||
        !make_map(&tm_q, qb, fp8, a.nq, 2 * (int64_t)a.dims, kBN / kCluster))
        return cudaErrorInvalidValue;
    const size_t smem = gemm_smem_bytes();
    const int ntiles = (int)((a.n + kBM - 1) / kBM);
    const int npairs = (ntiles + kCluster - 1) / kCluster;
    grid = grid / kCluster;                       // clusters, one CTA per SM
    if (grid > npairs) grid = npairs;
    if (grid < 1) grid = 1;
    grid *= kCluster;
    if (kind == kGemmHamming) return launch_kind<true, true>(tm_e, tm_q, a, grid, smem, stream);
    if (kind == kGemmFp8) return launch_kind<true, false>(tm_e, tm_q, a, grid, smem, stream);
    return launch_kind<false, false>(tm_e, tm_q, a, grid, smem, stream);
}

}  // namespace dbq
