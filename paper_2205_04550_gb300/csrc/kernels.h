// kernels.h -- host-side launchers of the libdbq kernels (internal).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace dbq {

// Threshold volumes into bit planes (Section 2.3 thresholding) and count the
// mask sizes.  vols: [count][v] float32 (src_f16 = 0) or binary16 bits
// (src_f16 = 1), device.  planes: [count][2][wp] words, ecount: [count][2];
// ecount must be zeroed by the caller.  Words past ceil(v/32) are written 0.
cudaError_t launch_pack(const void* vols, int src_f16, int64_t count, int64_t v, int64_t wp,
                        float t1, float t2, uint32_t* planes, uint32_t* ecount,
                        cudaStream_t stream);

// launch_pack for `count` (<= 65535) volumes whose device addresses are in
// the device array srcs[count].
cudaError_t launch_pack_ptrs(const void* const* srcs, int src_f16, int count, int64_t v,
                             int64_t wp, float t1, float t2, uint32_t* planes, uint32_t* ecount,
                             cudaStream_t stream);

// Round float32 to binary16, nearest-even (storage conversion of the
// half-precision database).
cudaError_t launch_to_f16(const float* src, int64_t n, uint16_t* dst, cudaStream_t stream);

// Copy caller bit planes [2][words] into padded planes [2][wp], clearing bits
// past voxel v-1, and count them into pcount[2] (zeroed by the caller).
cudaError_t launch_import_bits(const uint32_t* src, int64_t words, int64_t v, int64_t wp,
                               uint32_t* planes, uint32_t* pcount, cudaStream_t stream);

// Support lists of nq patients' planes [nq][2][wp4 uint4] -> lists
// [nq][2][wp4] (16-byte word offsets of non-zero 64-byte granules) and
// lens [nq][2].
cudaError_t launch_support(const uint32_t* planes, int nq, int wp4, uint32_t* lists,
                           uint32_t* lens, cudaStream_t stream);

// Arguments of the fused exact packed scan.
struct ScanPackedArgs {
    const uint4* planes;      // [n][2][wp4] database bit planes
    const uint32_t* ecount;   // [n][2] |E_1|, |E_2|
    const uint4* patient;     // [2][wp4] patient bit planes
    const uint32_t* pcount;   // [2] |P_1|, |P_2|
    int64_t n;                // entries
    int wp4;                  // uint4 per plane (padded)
    int chunk4;               // uint4 per plane per patient chunk held in shared memory
    int nchunks;              // ceil(wp4 / chunk4)
    int k;                    // results wanted (1..1024)
    Cand* cand;               // scratch [gridDim.x][k]
    unsigned int* ticket;     // scratch counter, 0 between launches
    Hit* hits;                // [k] output (device), may be null when counts_out is set
    uint32_t* counts_out;     // [n][4] per-entry (I1, I2, E1, E2), or null
    const uint32_t* sup_list; // [2][wp4] patient support lists, or null for the dense scan
    const uint32_t* sup_len;  // [2]
    Cand* group_lists;        // [ceil(grid / 8)][k]: two-level merge; null = one-level
    unsigned int* tickets;    // [1 + ceil(grid / 8)] counters of the two-level merge
    const uint32_t* counts_in = nullptr;   // [n][2] intersection counts already computed (the
                                 // word-major sparse scan), or null: the scan counts them
};

// Grid size (CTAs) the scan uses on this device, and its shared memory bytes.
int scan_packed_grid(int device);
size_t scan_packed_smem(int chunk4);
void scan_packed_chunking(int wp4, int* chunk4, int* nchunks);

cudaError_t launch_scan_packed(const ScanPackedArgs& a, int grid, cudaStream_t stream);

// Word-major copy of the planes: planes [n][w4] -> planes_t [w4][n] (16-byte
// words; w4 = 2 wp4), and the sparse counts over it for nq patients
// (patients [nq][2][wp4], support lists [nq][2][wp4] and lengths [nq][2],
// device): the intersections of entry e with patient q are added to
// counts[q qstride + e estride] (plane 1) and to that + poff (plane 2), which
// the caller zeroes beforehand.
cudaError_t launch_transpose_planes(const uint4* planes, int64_t n, int w4, uint4* planes_t,
                                    cudaStream_t stream);
cudaError_t launch_sparse_t_count(const uint4* planes_t, int64_t n, int nq, const uint4* patients,
                                  int wp4, const uint32_t* sup_lists, const uint32_t* sup_lens,
                                  uint32_t* counts, int64_t qstride, int64_t estride,
                                  int64_t poff, int sms, cudaStream_t stream);

// Arguments of the fused half-precision scan (per-query thresholds).
struct ScanF16Args {
    const uint4* vols;        // [n][blocks * 128] binary16 rows, 1024 voxels per block
    const uint32_t* patient;  // [2][wp] patient bit planes, wp = blocks * 32 words
    const uint32_t* pcount;   // [2] |P_1|, |P_2|
    int64_t n;                // entries
    int blocks;               // 1024-voxel blocks per entry row
    int wp;                   // words per patient plane (= blocks * 32)
    int chunk_blocks;         // blocks per patient chunk held in shared memory
    int nchunks;              // ceil(blocks / chunk_blocks)
    int k;                    // results wanted (1..1024)
    uint32_t th1x2, th2x2;    // smallest binary16 >= t_k, in both halves
    Cand* cand;               // scratch [gridDim.x][k]
    unsigned int* ticket;     // scratch counter, 0 between launches
    Hit* hits;                // [k] output, or null when only counts_out is wanted
    uint32_t* counts_out;     // [n][4] per-entry (I1, I2, E1, E2), or null
};

void scan_f16_chunking(int blocks, int* chunk_blocks, int* nchunks);
size_t scan_f16_smem(int chunk_blocks);
// Smallest binary16 bit pattern whose value is >= t (0 < t <= 1).
uint16_t f16_threshold_bits(float t);
cudaError_t launch_scan_f16(const ScanF16Args& a, int grid, cudaStream_t stream);

// Copy `count` rows of `v` binary16 values (or float32 values rounded to
// nearest-even) into rows of `pitch` halves; the padding is left untouched.
cudaError_t launch_rows_to_f16(const void* src, int src_f16, int64_t count, int64_t v,
                               int64_t pitch, uint16_t* dst, cudaStream_t stream);

// ---- embedding prefilter (a6-a8)

// Embeddings need nx % 32 == 0 and ny, nz multiples of 8.
bool embed_supported(int nx, int ny, int nz);
int embed_dims(int nx, int ny, int nz);   // (nx/8)(ny/8)(nz/8) per segmentation
// planes [count][2][wp] -> bf16 [count][2][d], e4m3 [count][2][d], scale,
// squared norms of the decoded bf16 / fp8 rows [count][2].
cudaError_t launch_embed(const uint32_t* planes, int64_t count, int64_t wp, int nx, int ny,
                         int nz, uint16_t* out_bf16, uint8_t* out_f8, float* out_scale,
                         float* out_norm_bf16, float* out_norm_f8, cudaStream_t stream);

// Count-sketch embeddings (sketch.cu): D = sketch_dims() buckets per
// segmentation, the same encodings as launch_embed, plus the sign code
// [count][2][D/32] (bit j of a row = bucket j > 0), the same code as E4M3
// 0/1 bytes [count][2][D] and its popcount per row [count][2] (binary32).
// Any grid; `words` meaningful words of each wp-word plane.
int sketch_dims();
// table [V]: bucket | sign << 15 of every voxel index (built once per grid).
cudaError_t launch_sketch_table(int64_t v, uint16_t* table, cudaStream_t stream);
cudaError_t launch_sketch(const uint32_t* planes, int64_t count, int64_t wp, int64_t words,
                          const uint16_t* table, uint16_t* out_bf16, uint8_t* out_f8, float* out_scale, float* out_nb,
                          float* out_nf, uint32_t* out_code, uint8_t* out_code8, float* out_cnorm,
                          cudaStream_t stream);
// Reaction-diffusion forward model (rd.cu).
struct RdSim {
    float a;        // dt * D_w
    float b;        // dt * rho
    int32_t steps;  // explicit steps of the simulation in this slot (0: slot idle)
    int32_t sx, sy, sz;   // seed voxel
    int32_t start;  // launch index of the slot's step 0
};
struct RdStepArgs {
    const RdSim* sims;               // [count]
    const float* hx;                 // [V] face coefficient to the +x neighbour
    const float* hy;
    const float* hz;
    const float* hym;                // [V] face coefficient to the -y neighbour
    const unsigned int* tile_any;    // [rd_tiles] 1 if the tile holds a domain voxel
    float* buf0;                     // [slots][V] u at even steps of each slot
    float* buf1;                     // [slots][V] u at odd steps
    unsigned long long* updates;     // voxel updates computed (or NULL)
    int nx, ny, nz;
};
int rd_tiles(int nx, int ny, int nz);
cudaError_t launch_rd_faces(const float* m, int nx, int ny, int nz, float* hx, float* hy,
                            float* hz, float* hym, unsigned int* tile_any, cudaStream_t stream);
// One launch: every slot with start <= launch < start + steps advances by one
// step (its local step launch - start).
cudaError_t launch_rd_step(const RdStepArgs& g, int slots, int launch, cudaStream_t stream);

struct GemmArgs {
    const uint16_t* e_bf16;   // [n][2*dims] entry embeddings (bf16 bits)
    const uint8_t* e_f8;      // [n][2*dims] entry embeddings (e4m3 codes)
    const float* enorm;       // [n][2] squared norms of the encoding used
    const float* escale;      // [n][2] e4m3 row scales (fp8 only)
    const uint16_t* q_bf16;   // [nq][2*dims]
    const uint8_t* q_f8;      // [nq][2*dims]
    const float* qnorm;       // [nq][2]
    const float* qscale;      // [nq][2]
    int64_t n;
    int nq;                   // <= gemm_max_queries()
    int dims;                 // per segmentation, multiple of 64 (bf16) / 128 (fp8)
    float* dist;              // [nq][n] L = d_1 + d_2
    int* status;              // device int, 0 = ok, else the role that timed out
};
size_t gemm_smem_bytes();
int gemm_max_queries();
// kind: kGemmBf16 / kGemmFp8 -- L = d_1 + d_2 of the L2 distances of the
// encoded embeddings; kGemmHamming -- E4M3 0/1 codes with their popcounts as
// norms, dist = sum over both segmentations of |q| + |e| - 2 q.e (exact).
enum GemmKind { kGemmBf16 = 0, kGemmFp8 = 1, kGemmHamming = 2 };
cudaError_t launch_prefilter_gemm(const GemmArgs& a, int kind, int grid, cudaStream_t stream);

// The c smallest distances per query (ties to the lower index), ascending:
// dist [nq][n] -> cand [nq][c] entry indices.  c <= 1024, c <= n.
cudaError_t launch_select_smallest(const float* dist, int nq, int64_t n, int c, int32_t* cand,
                                   cudaStream_t stream);

// Exact re-ranking: for each query q, the packed scan restricted to the
// entries cand[q][0..c) -> top-k hits [nq][k].  patient planes [nq][2][wp],
// pcount [nq][2]; scratch: cand lists [nq][slices][k] and tickets [nq]
// (zero between launches).
struct RerankArgs {
    const uint4* planes;        // database [n][2][wp4]
    const uint32_t* ecount;     // [n][2]
    int64_t n;
    int wp4, chunk4, nchunks;
    const uint4* patients;      // [nq][2][wp4]
    const uint32_t* pcounts;    // [nq][2]
    const int32_t* cand;        // [nq][c]
    int nq, c, k, slices;
    Cand* scratch;              // [nq][slices][k]
    unsigned int* tickets;      // [nq]
    Hit* hits;                  // [nq][k]
    const uint32_t* sup_lists;  // [nq][2][wp4] support lists, or null (dense)
    const uint32_t* sup_lens;   // [nq][2]
    unsigned int* sched;        // sparse only: item counter, zero between launches (nq <= 512),
                                // or null for the round-robin order
};
cudaError_t launch_rerank(const RerankArgs& a, cudaStream_t stream);

// The same hits for a dense batch, each distinct candidate entry read once
// (rerank_dedupe.cu): the pairs sorted by entry, slice counts against the
// patients' slices in shared memory, their sums, a top-k per query.
// sup_lists must be null; nq <= kRerankDedupeMaxQ, c <= 1024.
constexpr int kRerankDedupeMaxQ = 256;
struct RerankDedupeWork {
    uint32_t* hist;             // [n], zero between launches (the launch leaves it zero)
    uint2* tiles;               // [rerank_dedupe_tiles(n)]
    uint32_t* start;            // [n + 1]
    int32_t* uniq;              // [n]
    uint32_t* ubeg;             // [n + 1]
    uint32_t* nuniq;            // [1]
    uint16_t* qof;              // [nq * c]
    uint32_t* posof;            // [nq * c]
    uint16_t* partial;          // [2 * rerank_dedupe_slices(wp4)][rerank_dedupe_pstride(nq * c)]
    int64_t partial_elems;
    uint32_t* cnt;              // [2][nq * c]
};
int rerank_dedupe_slices(int wp4);
int64_t rerank_dedupe_pstride(int64_t npairs);
int64_t rerank_dedupe_tiles(int64_t n);
cudaError_t launch_rerank_dedupe(const RerankArgs& a, const RerankDedupeWork& w,
                                 cudaStream_t stream);

// ---- many exact queries in one persistent launch
struct QueryTask {
    const uint4* planes;        // database planes [n][2][wp4]
    const uint32_t* ecount;     // [n][2]
    int64_t n;
    int wp4, chunk4, nchunks;
    int k;                      // hits wanted (<= 1024)
    int slices;                 // work items of this query
    const uint4* patient;       // [2][wp4]
    const uint32_t* pcount;     // [2]
    const uint32_t* sup_list;   // [2][wp4] support lists, or null (dense)
    const uint32_t* sup_len;    // [2]
    Cand* scratch;              // [slices][k]
    unsigned int* ticket;       // zero between launches
    Hit* hits;                  // [k]
};
size_t scan_tasks_smem(bool sparse);

// ---- many exact queries against one database on the tensor cores
struct TcScanArgs {
    const uint32_t* planes;     // database [n][2][wp] bit planes (16-byte aligned)
    int64_t n;
    int64_t wp;                 // words per plane, a multiple of 4
    const uint32_t* qplanes;    // patients [nq][2][wp] bit planes (16-byte aligned)
    int nq;                     // 1 .. tc_scan_max_queries()
    uint32_t* counts;           // out: [2][nq][stride] I_k of (patient, entry), 16-byte aligned
    int64_t stride;             // tc_counts_stride(n)
    int* status;                // device word: nonzero after a timed-out wait
    unsigned long long stall_ns;  // test only: 0, or first wait this long on a barrier
                                  // nothing arrives at (the timeout path; status 5)
};
int tc_scan_max_queries();
int64_t tc_scan_min_words();     // words per plane the contraction needs at least
int64_t tc_counts_stride(int64_t n);
// Exact only while V <= 2^24 (the binary32 accumulators count voxels).
cudaError_t launch_tc_scan(const TcScanArgs& a, int grid, cudaStream_t stream);
// Scores and top-k of patients tasks[task0 .. task0 + nq) from counts
// [2][nq][stride] (mask sizes, k and the hit output taken from each task).
cudaError_t launch_tc_select(const QueryTask* tasks, int task0, int nq, const uint32_t* counts,
                             int64_t n, int64_t stride, cudaStream_t stream);
// items[i] = (task, slice), every slice of the ntasks tasks once; next_item
// is a device counter (cleared here); any_sparse: some task has support
// lists, and the items are then re-ordered in place, costliest first.
cudaError_t launch_scan_tasks(const QueryTask* tasks, int ntasks, int2* items, int nitems,
                              unsigned int* next_item, int grid, bool any_sparse,
                              cudaStream_t stream);

// Nearest-neighbour downsampling of `rows` bit planes (rows = entries * 2)
// of an nx x ny x nz grid by factor f: dst [rows][dst_wp], sizes [rows]
// (mask sizes of the coarse planes; zeroed by the caller).
cudaError_t launch_downsample(const uint32_t* src, int64_t rows, int64_t src_wp, int nx, int ny,
                              int nz, int f, int64_t dst_wp, uint32_t* dst, uint32_t* sizes,
                              cudaStream_t stream);

// Set the calling thread's db_last_error() message; returns `code`.
int record_error(int code, const char* msg);

}  // namespace dbq
