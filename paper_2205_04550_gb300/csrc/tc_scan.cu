// tc_scan.cu -- the exact loop of Section 2.3 (Ezhov et al. 2022) for many
// patients against one bit-packed database at once, on the tensor cores.
//
// For Q patients and N entries the intersections I_k(q, e) = |P_k(q) n E_k(e)|
// are dot products of 0/1 vectors over the V voxels: one dense contraction
// [Q x V] . [V x N] per segmentation.  The masks are stored as bits, which
// the tensor cores cannot read, so converter warps expand each K-slice of 256
// voxels of the patients' rows and of 240 entry rows into 4-bit E2M1 values
// (1.0 for a set bit, 0 otherwise; two voxels per byte) in the
// 128-byte-swizzled K-major layout of tcgen05 shared-memory operands, and one
// thread issues block-scaled tcgen05.mma (kind::mxf4, every UE8M0 scale 1.0;
// M = 128 patient rows -- the rows past Q are zero --, N = 240 entries,
// K = 64 per instruction) with binary32 accumulators in tensor memory.  An
// MMA instruction costs about the same for any N, so the entries, not the
// few patients, take the N side.  Every product is 0 or 1 and every partial
// sum an integer no larger than V <= 2^24, so the accumulators hold the
// exact counts.
//
// Voxel order inside a K-slice: a dot product does not depend on the order
// of its terms as long as both operands use the same one, so the expansion
// takes whatever order is cheapest: 16-byte chunk c of a row holds the 32
// voxels of bit word c, its 32-bit word j holds bits j, j + 4, ..., j + 28 of
// that word, one per nibble ((u >> j) & 0x11111111, shifted to the 1.0 code
// 0x2).  That is two integer instructions per 8 voxels.
//
//   * work units are (240-entry tile, segmentation), round-robin over one
//     persistent CTA per SM; each unit writes its own component of the
//     counts, so no unit waits for another;
//   * warps 6-17 (converters): thread t < 240 expands entry row t of the
//     tile, thread 240 + r patient row r < Q; each keeps the 32 bytes of bits
//     of the next three K-slices in registers (loads issued three slices
//     ahead), expands one slice into a 4-stage ring of operand tiles and makes
//     the stores visible to the tensor core (fence.proxy.async); one lane per
//     warp then arrives on the stage's full barrier, and one lane per warp
//     waits for a stage to be free.  The patient rows past Q are cleared once;
//   * warp 0 (one thread): per K-slice four MMAs into the unit's 240
//     accumulator columns in one of two TMEM buffers (columns 0 and 256), so
//     the epilogue of a unit overlaps the next unit's MMAs; its commits free
//     the stage and, at the end of a unit, hand the buffer to the epilogue;
//   * warps 2-5 (epilogue, one TMEM lane quarter each, lane = patient row):
//     fill the scale columns (240-255 for A, 496-511 for B) with UE8M0 1.0
//     once, then tcgen05.ld the counts of 16 entries at a time and store them
//     as 64-byte rows of counts[plane][q][e];
//   * warp 1 allocates and frees the 512 TMEM columns.
// Per 256-voxel slice the expanded operands (46 KB) pass through shared
// memory twice (converter stores, tensor-core reads), about 1.5 bytes per
// entry bit in each direction; that traffic, not the FP4 tensor rate, is the
// kernel's bound.  The mask sizes, binary64 scores and each patient's top-k
// follow in tc_select_kernel.  Every mbarrier wait is bounded; on a timeout
// the CTA records an error code in `status`, stops, drains its MMAs and frees
// its TMEM.
#include "kernels.h"
#include "tcgen05.cuh"
#include "topk.cuh"

namespace dbq {
namespace {

constexpr int kTcQ = 128;                    // query rows of the MMA (M), zero-padded
constexpr int kTcE = 240;                    // entries per tile (MMA N)
constexpr int kTcMaxN = 128;                 // queries per launch
constexpr int kTcStages = 4;                 // operand stages, 46 KiB each
constexpr int kTcConv = 384;                 // converter threads: 240 entry + 128 query rows + 16 idle
constexpr int kTcConvWarps = kTcConv / 32;
constexpr int kTcConv0 = 192;                // first converter thread (warps 0-5: MMA, TMEM, epilogue)
constexpr int kTcThreads = kTcConv0 + kTcConv;
constexpr int kTcSliceWords = 8;             // 256 voxels per K-slice and row
constexpr int kTcABytes = kTcQ * 128;        // query operand of a stage
constexpr int kTcBBytes = kTcE * 128;        // entry operand of a stage
constexpr int kTcStageBytes = kTcABytes + kTcBBytes;
constexpr uint32_t kTcBufCols = 256;         // TMEM columns between the two accumulators
constexpr uint32_t kTcScaleA = 240;          // TMEM columns of the unit scales
constexpr uint32_t kTcScaleB = 496;
constexpr uint32_t kUnitScales = 0x7F7F7F7Fu;   // four UE8M0 bytes of 2^0

static_assert(kTcE % 16 == 0 && kTcE <= 256, "MMA N");
static_assert(kTcScaleA >= kTcE && kTcScaleA + 16 <= kTcBufCols, "scale columns");
static_assert(kTcScaleB >= kTcBufCols + kTcE && kTcScaleB + 16 <= 512, "scale columns");
static_assert(kTcABytes % 1024 == 0 && kTcStageBytes % 1024 == 0, "swizzle atoms");

// 1 KiB of alignment slack, the stages, the mbarriers (full and empty per
// stage, two accumulator pairs, the drain, the test stall), TMEM slot and
// abort flag.
size_t smem_bytes()
{
    return 1024 + (size_t)kTcStages * kTcStageBytes + (2 * kTcStages + 6) * 8 + 16;
}

__device__ __forceinline__ uint4 ldg_stream(const uint32_t* p)
{
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
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

__device__ __forceinline__ void st_global_v4(uint32_t* p, uint32_t a, uint32_t b, uint32_t c,
                                             uint32_t d)
{
    asm volatile("st.global.v4.b32 [%0], {%1, %2, %3, %4};" ::"l"(p), "r"(a), "r"(b), "r"(c),
                 "r"(d)
                 : "memory");
}

__device__ __forceinline__ void umma_f4(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                        uint32_t idesc, uint32_t sfa, uint32_t sfb,
                                        uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %6, 0;\n"
        " tcgen05.mma.cta_group::1.kind::mxf4.block_scale.scale_vec::2X [%0], %1, %2, %3, [%4], "
        "[%5], p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(sfa), "r"(sfb), "r"(accumulate)
        : "memory");
}

// Arrives on the mbarrier once the MMAs issued so far by this thread are done.
__device__ __forceinline__ void umma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     bar)
                 : "memory");
}

// 256 mask bits (eight words, voxel 32i + b = bit b of word i) -> one
// 128-byte operand row of E2M1 nibbles: chunk c (the 32 voxels of word c)
// goes to chunk position c ^ (row mod 8) of the row, the 128-byte swizzle.
__device__ __forceinline__ void expand_row(uint32_t row_base, int row, const uint4& lo,
                                           const uint4& hi)
{
    const uint32_t w[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const uint32_t u = w[c];
        st_shared_v4(row_base + (uint32_t)(((c ^ (row & 7)) & 7) << 4), (u << 1) & 0x22222222u,
                     u & 0x22222222u, (u >> 1) & 0x22222222u, (u >> 2) & 0x22222222u);
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
    uint64_t* bars = reinterpret_cast<uint64_t*>(stages + (size_t)kTcStages * kTcStageBytes);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kTcStages + 6);
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
    const uint32_t stall = smem_u32(bars + 2 * kTcStages + 5);    // nothing ever arrives here

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
        mbar_init(stall, 1);
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
    if (warp >= 2 && warp < 6) {
        // unit scales for both operands, every lane of this warp's quarter
        const uint32_t lanes = tmem + ((uint32_t)((warp & 3) * 32) << 16);
        asm volatile(
            "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1, %1, "
            "%1, %1, %1, %1, %1, %1, %1};" ::"r"(lanes + kTcScaleA),
            "r"(kUnitScales)
            : "memory");
        asm volatile(
            "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1, %1, "
            "%1, %1, %1, %1, %1, %1, %1};" ::"r"(lanes + kTcScaleB),
            "r"(kUnitScales)
            : "memory");
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    if (warp == 0) {
        if (lane == 0) {
            // block-scaled descriptor: A and B E2M1 (MXF4 format 1), K-major,
            // UE8M0 scales, N = 240 entries, M = 128 query rows, K = 64
            const uint32_t idesc = (1u << 7) | (1u << 10) | ((uint32_t)(kTcE >> 3) << 17) |
                                   (1u << 23) | ((uint32_t)(kTcQ >> 4) << 24);
            int s = 0;
            uint32_t phase = 0;
            bool ok = true;
            if (a.stall_ns && !mbar_wait_for(stall, 0, abort_flag, a.stall_ns)) {
                a.status[0] = 5;           // the test stall ran out, as it must
                ok = false;
            }
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
                const uint32_t d_tmem = tmem + (uint32_t)buf * kTcBufCols;
                for (int64_t kc = 0; kc < nk; ++kc) {
                    if (!mbar_wait(full0 + 8 * s, phase, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)   // 64 voxels = 32 bytes per row each
                        umma_f4(d_tmem, sdesc + (uint64_t)(2 * kk), sdesc + b_off + (uint64_t)(2 * kk),
                                idesc, tmem + kTcScaleA, tmem + kTcScaleB,
                                (kc > 0 || kk > 0) ? 1u : 0u);
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
                if (a.status[0] == 0) a.status[0] = 2;
                *abort_flag = 1;
            }
            umma_commit(drain);
            if (!mbar_wait(drain, 0, nullptr)) a.status[0] = 3;
        }
    } else if (warp >= 2 && warp < 6) {
        // lane = query row; columns = the unit's 240 entries
        const int quarter = warp & 3;
        const int q = quarter * 32 + lane;
        for (int64_t u = 0; u < my_units; ++u) {
            const int buf = (int)(u & 1);
            if (!mbar_wait(acc_full0 + 8 * buf, (uint32_t)((u >> 1) & 1), abort_flag)) {
                if (a.status[0] == 0) a.status[0] = 4;
                *abort_flag = 1;
                break;
            }
            tc_fence_after();
            const int64_t unit = blockIdx.x + u * gridDim.x;
            const int64_t e0 = (unit >> 1) * kTcE;
            const int plane = (int)(unit & 1);
            const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)buf * kTcBufCols;
            for (int c0 = 0; c0 < kTcE; c0 += 16) {
                uint32_t r[16];
                tmem_ld16(lane_base + c0, r);
                tmem_wait_ld();
                if (q < a.nq) {
                    uint32_t* row = a.counts + ((int64_t)plane * a.nq + q) * a.stride;
                    uint32_t v[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) v[j] = (uint32_t)__uint_as_float(r[j]);   // exact
                    const int64_t e = e0 + c0;
                    if (e + 16 <= a.n) {
#pragma unroll
                        for (int j = 0; j < 16; j += 4)
                            st_global_v4(row + e + j, v[j], v[j + 1], v[j + 2], v[j + 3]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (e + j < a.n) row[e + j] = v[j];
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(acc_free0 + 8 * buf);
        }
    } else if (warp >= kTcConv0 / 32) {
        // converters: thread ct < 240 expands entry row ct of the tile, thread
        // 240 + r query row r (r < nq); threads past 367 only take part in the
        // warps' barrier arrivals
        const int ct = threadIdx.x - kTcConv0;
        const bool is_b = ct < kTcE;
        const int row = is_b ? ct : ct - kTcE;
        const bool active = is_b || row < a.nq;
        int64_t i_u = 0, i_kc = 0;
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
        if (active && my_units > 0) row_start();
        // the bits of the next K-slice of this thread's row (zeros past the
        // row's end, for a missing entry and for inactive threads)
        auto load_next = [&](uint4& lo, uint4& hi) {
            lo = make_uint4(0, 0, 0, 0);
            hi = lo;
            if (active && i_u < my_units) {
                const int64_t w = i_kc * kTcSliceWords;
                if (row_ok) {
                    if (w < a.wp) lo = ldg_stream(src_row + w);
                    if (w + 4 < a.wp) hi = ldg_stream(src_row + w + 4);
                }
                if (++i_kc == nk) {
                    i_kc = 0;
                    ++i_u;
                    if (i_u < my_units) row_start();
                }
            }
        };
        int s = 0;
        uint32_t phase = 0;
        const uint32_t dst = (is_b ? (uint32_t)kTcABytes : 0u) + row_offset(active ? row : 0);
        const uint32_t stage0 = smem_u32(stages);
        // expand one K-slice into the next stage; false after an abort
        auto step = [&](const uint4& lo, const uint4& hi) -> bool {
            int ok = 1;
            if (lane == 0) ok = mbar_wait(empty0 + 8 * s, phase ^ 1u, abort_flag);
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) {
                if (lane == 0) {
                    if (a.status[0] == 0) a.status[0] = 1;
                    *abort_flag = 1;
                }
                return false;
            }
            if (active) expand_row(stage0 + (uint32_t)(s * kTcStageBytes) + dst, row, lo, hi);
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) mbar_arrive(full0 + 8 * s);
            if (++s == kTcStages) {
                s = 0;
                phase ^= 1u;
            }
            return true;
        };
        uint4 p0l, p0h, p1l, p1h, p2l, p2h;
        load_next(p0l, p0h);
        load_next(p1l, p1h);
        load_next(p2l, p2h);
        for (int64_t it = 0; it < total; it += 3) {
            if (!step(p0l, p0h)) break;
            load_next(p0l, p0h);
            if (it + 1 >= total) break;
            if (!step(p1l, p1h)) break;
            load_next(p1l, p1h);
            if (it + 2 >= total) break;
            if (!step(p2l, p2h)) break;
            load_next(p2l, p2h);
        }
    }

    tc_fence_before();
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
tc_select_kernel(const QueryTask* __restrict__ tasks, int task0, int nq,
                 const uint32_t* __restrict__ counts, int64_t n, int64_t stride)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TopK tk;
    topk_carve(tk, smem_raw);
    const QueryTask& t = tasks[task0 + blockIdx.x];
    const int k = t.k;
    const uint32_t P1 = t.pcount[0], P2 = t.pcount[1];
    const uint2* ecount2 = reinterpret_cast<const uint2*>(t.ecount);
    const uint32_t* row1 = counts + (int64_t)blockIdx.x * stride;
    const uint32_t* row2 = counts + ((int64_t)nq + blockIdx.x) * stride;
    topk_init(tk);
    for (int64_t b0 = 0; b0 < n; b0 += blockDim.x) {
        const int64_t e = b0 + threadIdx.x;
        if (e < n) {
            const uint32_t I1 = row1[e], I2 = row2[e];
            const uint2 E = ecount2[e];
            topk_offer(tk, k, score_key(score_rn(I1, I2, E.x, E.y, P1, P2)), e,
                       (uint64_t)I1 | ((uint64_t)I2 << 32),
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

int64_t tc_counts_stride(int64_t n) { return (n + 3) / 4 * 4; }

cudaError_t launch_tc_scan(const TcScanArgs& a, int grid, cudaStream_t stream)
{
    if (a.nq < 1 || a.nq > kTcMaxN || a.n < 1 || a.wp < 4 || a.wp % 4 != 0 ||
        a.stride < a.n || a.stride % 4 != 0 ||
        (reinterpret_cast<uintptr_t>(a.planes) & 15) || (reinterpret_cast<uintptr_t>(a.qplanes) & 15) ||
        (reinterpret_cast<uintptr_t>(a.counts) & 15))
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

cudaError_t launch_tc_select(const QueryTask* tasks, int task0, int nq, const uint32_t* counts,
                             int64_t n, int64_t stride, cudaStream_t stream)
{
    if (nq < 1 || n < 1 || stride < n) return cudaErrorInvalidValue;
    const size_t smem = topk_smem_bytes();
    cudaError_t err = cudaFuncSetAttribute(tc_select_kernel,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    tc_select_kernel<<<nq, 1024, smem, stream>>>(tasks, task0, nq, counts, n, stride);
    return cudaGetLastError();
}

}  // namespace dbq
