// tc_scan.cu -- the exact loop of Section 2.3 (Ezhov et al. 2022) for many
// patients against one bit-packed database at once, on the tensor cores.
//
// For Q patients and N entries the intersections I_k(q, e) = |P_k(q) n E_k(e)|
// are dot products of 0/1 vectors over the V voxels: one dense contraction
// [Q x V] . [V x N] per segmentation.  The masks are stored as bits, which
// the tensor cores cannot read, so converter warps expand each K-slice of 128
// voxels of the patients' rows and of 256 entry rows into E4M3 bytes (2.0 for
// a set bit, 0 otherwise) in the 128-byte-swizzled K-major layout of tcgen05
// shared-memory operands, and one thread issues tcgen05.mma (kind::f8f6f4,
// M = 128 patient rows -- the rows past Q are zero --, N = 256 entries,
// K = 32 per instruction) with binary32 accumulators in tensor memory.  An
// MMA instruction costs about the same for any N, so the entries, not the
// few patients, take the N side.  Every product is 0 or 4 and every partial
// sum 4 times an integer no larger than V <= 2^24, so the accumulators hold
// 4 x the exact counts (2.0 is 0x40: one bit per byte, which saves a
// multiply per output word over 1.0 = 0x38).
//
//   * work units are (256-entry tile, segmentation), round-robin over one
//     persistent CTA per SM; each unit writes its own component of the
//     counts, so no unit waits for another;
//   * warps 6-17 (converters): thread t < 256 copies with cp.async the 16
//     bytes (128 voxels) of entry row t of every K-slice, thread 256 + r
//     those of patient row r < Q, four slices ahead, expands them into a
//     4-stage ring of operand tiles and makes the stores visible to the
//     tensor core (fence.proxy.async); one lane per warp then arrives on the
//     stage's full barrier (the warp's stores ordered before it by
//     __syncwarp), and one lane per warp waits for a stage to be free.  The
//     patient rows past Q are cleared once at the start;
//   * warp 0 (one thread): per K-slice four MMAs into the unit's 256
//     accumulator columns in one of two TMEM buffers, so the epilogue of a
//     unit overlaps the next unit's MMAs; its commits free the stage and, at
//     the end of a unit, hand the buffer to the epilogue;
//   * warps 2-5 (epilogue, one TMEM lane quarter each, lane = patient row):
//     tcgen05.ld the counts of 16 entries at a time and store them into
//     counts[q][e];
//   * warp 1 allocates and frees the 512 TMEM columns.
// The expanded operands pass through shared memory twice (converter stores,
// tensor-core reads): about 24 bytes of shared-memory traffic per byte of
// bits, which bounds this design near 8 bytes of bits per cycle per SM.
// The mask sizes, binary64 scores and each patient's top-k follow in
// tc_select_kernel.  Every mbarrier wait is bounded; on a timeout the CTA
// records an error code in `status`, stops, drains its MMAs and copies and
// frees its TMEM.
#include "kernels.h"
#include "tcgen05.cuh"
#include "topk.cuh"

namespace dbq {
namespace {

constexpr int kTcQ = 128;                    // query rows of the MMA (M), zero-padded
constexpr int kTcE = 256;                    // entries per tile (MMA N)
constexpr int kTcMaxN = 128;                 // queries per launch
constexpr int kTcStages = 4;                 // operand stages, 48 KiB each
constexpr int kTcAhead = 4;                  // K-slices in flight per converter thread
constexpr int kTcConv = kTcE + kTcQ;         // converter threads: 256 entry rows + 128 query rows
constexpr int kTcConvWarps = kTcConv / 32;
constexpr int kTcConv0 = 192;                // first converter thread (warps 0-5: MMA, TMEM, epilogue)
constexpr int kTcThreads = kTcConv0 + kTcConv;
constexpr int kTcSliceWords = 4;             // 128 voxels per K-slice and row
constexpr int kTcABytes = kTcQ * 128;        // query operand of a stage
constexpr int kTcBBytes = kTcE * 128;        // entry operand of a stage
constexpr int kTcStageBytes = kTcABytes + kTcBBytes;

__host__ __device__ constexpr size_t ring_bytes() { return (size_t)kTcAhead * kTcConv * 16; }

// 1 KiB of alignment slack, the stages, the cp.async ring, the mbarriers
// (full and empty per stage, two accumulator pairs, the drain), TMEM slot and
// abort flag.
size_t smem_bytes()
{
    return 1024 + (size_t)kTcStages * kTcStageBytes + ring_bytes() + (2 * kTcStages + 5) * 8 + 16;
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, bool valid)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
                 "r"(valid ? 16 : 0)
                 : "memory");
}

__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;" ::: "memory");
}

template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c,
                                             uint32_t d)
{
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c),
                 "r"(d)
                 : "memory");
}

__device__ __forceinline__ void umma_f8(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                        uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrives on the mbarrier once the MMAs issued so far by this thread are done.
__device__ __forceinline__ void umma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     bar)
                 : "memory");
}

// Four mask bits (x < 16) -> four E4M3 bytes, 2.0 (0x40) where a bit is set:
// x * 0x204081 places bit j of x at bit 8j (the four shifted copies do not
// overlap, so nothing carries); shifted by 6 more, at bit 8j + 6.
__device__ __forceinline__ uint32_t expand4(uint32_t x)
{
    return (x * (0x00204081u << 6)) & 0x40404040u;
}

// 128 mask bits (four words, voxel 32i + b = bit b of word i) -> one
// 128-byte operand row: 16-byte chunk c (voxels 16c .. 16c + 15) goes to
// chunk position c ^ (row mod 8) of the row, the 128-byte swizzle.
__device__ __forceinline__ void expand_row(uint32_t row_base, int row, const uint4& bits)
{
    const uint32_t w[4] = {bits.x, bits.y, bits.z, bits.w};
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const uint32_t h = w[c >> 1] >> ((c & 1) * 16);
        st_shared_v4(row_base + (uint32_t)(((c ^ (row & 7)) & 7) << 4), expand4(h & 0xFu),
                     expand4((h >> 4) & 0xFu), expand4((h >> 8) & 0xFu),
                     expand4((h >> 12) & 0xFu));
    }
}

// Byte offset of row `row` in a K-major 128-byte-swizzled column: 8-row
// groups of 1024 bytes, 128 bytes per row.
__device__ __forceinline__ uint32_t row_offset(int row)
{
    return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128);
}

__global__ void __launch_bounds__(kTcThreads, 1) tc_scan_kernel(const TcScanArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char* stages = base;                                  // kTcStages x (A | B)
    unsigned char* ring = stages + (size_t)kTcStages * kTcStageBytes;   // [ahead][kTcConv] x 16 B
    uint64_t* bars = reinterpret_cast<uint64_t*>(ring + ring_bytes());
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kTcStages + 5);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t ntiles = (a.n + kTcE - 1) / kTcE;
    const int64_t nunits = ntiles * 2;                             // (tile, plane)
    const int64_t my_units = nunits > blockIdx.x ? (nunits - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int64_t nk = (a.wp + kTcSliceWords - 1) / kTcSliceWords;
    const int64_t total = my_units * nk;

    const uint32_t full0 = smem_u32(bars);
    const uint32_t empty0 = smem_u32(bars + kTcStages);
    const uint32_t acc_full0 = smem_u32(bars + 2 * kTcStages);
    const uint32_t acc_free0 = smem_u32(bars + 2 * kTcStages + 2);
    const uint32_t drain = smem_u32(bars + 2 * kTcStages + 4);

    // the query rows past nq stay zero in every stage: cleared once here
    for (int i = threadIdx.x; i < kTcStages * (kTcABytes / 16); i += blockDim.x) {
        const int st = i / (kTcABytes / 16), off = i % (kTcABytes / 16);
        const int row = ((off * 16) / 1024) * 8 + ((off * 16) % 1024) / 128;   // row of this 16 B
        if (row >= a.nq)
            *reinterpret_cast<uint4*>(stages + (size_t)st * kTcStageBytes + off * 16) =
                make_uint4(0, 0, 0, 0);
    }
    fence_proxy_async();
    if (threadIdx.x == 0) {
        for (int s = 0; s < kTcStages; ++s) {
            mbar_init(full0 + 8 * s, kTcConvWarps);
            mbar_init(empty0 + 8 * s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(acc_full0 + 8 * b, 1);
            mbar_init(acc_free0 + 8 * b, 128);
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                         smem_u32(tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // D f32, A and B E4M3, K-major, N = 256 entries, M = 128 query rows
            const uint32_t idesc =
                (1u << 4) | ((uint32_t)(kTcE >> 3) << 17) | ((uint32_t)(kTcQ >> 4) << 24);
            int s = 0;
            uint32_t phase = 0;
            bool ok = true;
            const uint64_t desc0 = sw128_desc(smem_u32(stages));
            const uint64_t b_off = (uint64_t)(kTcABytes >> 4);
            uint64_t sdesc = desc0;
            for (int64_t u = 0; u < my_units && ok; ++u) {
                const int buf = (int)(u & 1);
                if (!mbar_wait(acc_free0 + 8 * buf, (uint32_t)(((u >> 1) & 1) ^ 1), abort_flag)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d_tmem = tmem + (uint32_t)(buf * kTcE);
                for (int64_t kc = 0; kc < nk; ++kc) {
                    if (!mbar_wait(full0 + 8 * s, phase, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        umma_f8(d_tmem, sdesc + (uint64_t)(2 * kk), sdesc + b_off + (uint64_t)(2 * kk),
                                idesc, (kc > 0 || kk > 0) ? 1u : 0u);
                    umma_commit(empty0 + 8 * s);
                    sdesc += kTcStageBytes >> 4;
                    if (++s == kTcStages) {
                        s = 0;
                        phase ^= 1u;
                        sdesc = desc0;
                    }
                }
                if (ok) umma_commit(acc_full0 + 8 * buf);
            }
            if (!ok) {
                a.status[0] = 2;
                *abort_flag = 1;
            }
            umma_commit(drain);
            if (!mbar_wait(drain, 0, nullptr)) a.status[0] = 3;
        }
    } else if (warp >= 2 && warp < 6) {
        // lane = query row; columns = the unit's 256 entries
        const int quarter = warp & 3;
        const int q = quarter * 32 + lane;
        uint32_t* cnt = reinterpret_cast<uint32_t*>(a.counts);
        for (int64_t u = 0; u < my_units; ++u) {
            const int buf = (int)(u & 1);
            if (!mbar_wait(acc_full0 + 8 * buf, (uint32_t)((u >> 1) & 1), abort_flag)) {
                a.status[0] = 4;
                *abort_flag = 1;
                break;
            }
            tc_fence_after();
            const int64_t unit = blockIdx.x + u * gridDim.x;
            const int64_t e0 = (unit >> 1) * kTcE;
            const int plane = (int)(unit & 1);
            const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(buf * kTcE);
            for (int c0 = 0; c0 < kTcE; c0 += 16) {
                uint32_t r[16];
                tmem_ld16(lane_base + c0, r);
                tmem_wait_ld();
                if (q < a.nq) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int64_t e = e0 + c0 + j;
                        if (e < a.n)   // 4 x the count, exact
                            cnt[((int64_t)q * a.n + e) * 2 + plane] =
                                (uint32_t)(__uint_as_float(r[j]) * 0.25f);
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(acc_free0 + 8 * buf);
        }
    } else if (warp >= kTcConv0 / 32) {
        // converters: thread ct < 256 expands entry row ct of the tile, thread
        // 256 + r query row r (r < nq)
        const int ct = threadIdx.x - kTcConv0;
        const bool is_b = ct < kTcE;
        const int row = is_b ? ct : ct - kTcE;
        const bool active = is_b || row < a.nq;
        int64_t i_u = 0, i_kc = 0;
        int i_slot = 0;
        const uint32_t* src_row = nullptr;
        bool row_ok = false;
        auto row_start = [&]() {
            const int64_t unit = blockIdx.x + i_u * gridDim.x;
            const int plane = (int)(unit & 1);
            if (is_b) {
                const int64_t e = (unit >> 1) * kTcE + row;
                row_ok = e < a.n;
                src_row = a.planes + (e * 2 + plane) * a.wp;
            } else {
                row_ok = true;
                src_row = a.qplanes + ((int64_t)row * 2 + plane) * a.wp;
            }
        };
        if (active) row_start();
        const uint32_t ring0 = smem_u32(ring) + (uint32_t)(ct * 16);
        auto issue = [&]() {
            if (active && i_u < my_units) {
                const int64_t w = i_kc * kTcSliceWords;
                const bool v = row_ok && w < a.wp;
                cp_async16(ring0 + (uint32_t)(i_slot * kTcConv * 16), v ? src_row + w : a.planes, v);
                if (++i_kc == nk) {
                    i_kc = 0;
                    ++i_u;
                    if (i_u < my_units) row_start();
                }
            }
            cp_async_commit();
            if (++i_slot == kTcAhead) i_slot = 0;
        };
        for (int d = 0; d < kTcAhead; ++d) issue();
        int c_slot = 0, s = 0;
        uint32_t phase = 0;
        const uint32_t dst = (is_b ? (uint32_t)kTcABytes : 0u) + row_offset(row);
        const uint32_t stage0 = smem_u32(stages);
        for (int64_t it = 0; it < total; ++it) {
            cp_async_wait<kTcAhead - 1>();
            uint4 bits = make_uint4(0, 0, 0, 0);
            if (active) bits = *reinterpret_cast<const uint4*>(ring + ct * 16 + c_slot * kTcConv * 16);
            if (++c_slot == kTcAhead) c_slot = 0;
            int ok = 1;
            if (lane == 0) ok = mbar_wait(empty0 + 8 * s, phase ^ 1u, abort_flag);
            ok = __shfl_sync(0xffffffffu, ok, 0);
            __syncwarp();
            if (!ok) {
                if (lane == 0) {
                    a.status[0] = 1;
                    *abort_flag = 1;
                }
                break;
            }
            if (active) expand_row(stage0 + (uint32_t)(s * kTcStageBytes) + dst, row, bits);
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) mbar_arrive(full0 + 8 * s);
            if (++s == kTcStages) {
                s = 0;
                phase ^= 1u;
            }
            issue();
        }
        cp_async_wait<0>();
    }

    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem)
                     : "memory");
    }
}

// Scores and top-k of one patient (one CTA per patient) from its counts:
// the same binary64 Dice scores, keys and order as the fused scans.
__global__ void __launch_bounds__(1024, 1)
tc_select_kernel(const QueryTask* __restrict__ tasks, int task0, const uint2* __restrict__ counts,
                 int64_t n)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TopK tk;
    topk_carve(tk, smem_raw);
    const QueryTask& t = tasks[task0 + blockIdx.x];
    const int k = t.k;
    const uint32_t P1 = t.pcount[0], P2 = t.pcount[1];
    const uint2* ecount2 = reinterpret_cast<const uint2*>(t.ecount);
    const uint2* row = counts + (int64_t)blockIdx.x * n;
    topk_init(tk);
    for (int64_t b0 = 0; b0 < n; b0 += blockDim.x) {
        const int64_t e = b0 + threadIdx.x;
        if (e < n) {
            const uint2 I = row[e];
            const uint2 E = ecount2[e];
            topk_offer(tk, k, score_key(score_rn(I.x, I.y, E.x, E.y, P1, P2)), e,
                       (uint64_t)I.x | ((uint64_t)I.y << 32),
                       (uint64_t)E.x | ((uint64_t)E.y << 32));
        }
        __syncthreads();
        // room for another round of offers
        if (tk.misc[0] > kTopkCap - k - (int)blockDim.x) topk_flush(tk, k);
    }
    topk_flush(tk, k);
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        Hit h;
        h.index = tk.idx[j];
        h.score = key_score(tk.key[j]);
        h.i1 = (uint32_t)(tk.pay0[j] & 0xffffffffu);
        h.i2 = (uint32_t)(tk.pay0[j] >> 32);
        h.e1 = (uint32_t)(tk.pay1[j] & 0xffffffffu);
        h.e2 = (uint32_t)(tk.pay1[j] >> 32);
        h.p1 = P1;
        h.p2 = P2;
        t.hits[j] = h;
    }
}

}  // namespace

int tc_scan_max_queries() { return kTcMaxN; }

cudaError_t launch_tc_scan(const TcScanArgs& a, int grid, cudaStream_t stream)
{
    if (a.nq < 1 || a.nq > kTcMaxN || a.n < 1 || a.wp < 4 || a.wp % 4 != 0 ||
        (reinterpret_cast<uintptr_t>(a.planes) & 15) || (reinterpret_cast<uintptr_t>(a.qplanes) & 15))
        return cudaErrorInvalidValue;
    const size_t smem = smem_bytes();
    cudaError_t err = cudaFuncSetAttribute(tc_scan_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
    if (err != cudaSuccess) return err;
    const int64_t nunits = (a.n + kTcE - 1) / kTcE * 2;
    if (grid > nunits) grid = (int)nunits;
    if (grid < 1) grid = 1;
    tc_scan_kernel<<<grid, kTcThreads, smem, stream>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_tc_select(const QueryTask* tasks, int task0, int nq, const uint2* counts,
                             int64_t n, cudaStream_t stream)
{
    if (nq < 1 || n < 1) return cudaErrorInvalidValue;
    const size_t smem = topk_smem_bytes();
    cudaError_t err = cudaFuncSetAttribute(tc_select_kernel,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    tc_select_kernel<<<nq, 1024, smem, stream>>>(tasks, task0, counts, n);
    return cudaGetLastError();
}

}  // namespace dbq
