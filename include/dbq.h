/*
 * dbq.h -- C ABI of the GB300 tumour-database query library (libdbq.so).
 *
 * The library implements the database query of Ezhov et al., "A for-loop is
 * all you need" (2022): every simulated tumour concentration volume of a
 * database is thresholded at u_T1Gd and u_FLAIR (Section 2.3, "Query to a
 * database of synthetic tumors"), each entry's two segmentations are compared
 * with the patient's two segmentations by the Dice coefficient (same
 * section), the two Dice values are combined by addition (reported as their
 * mean, which orders entries identically), and the best match -- the
 * arg-max -- and the top-k entries are returned together with their model
 * parameters theta (Section 3, "Data").  The brute-force loop over the whole
 * database is the paper's "baseline for-loop search" (Section 2.3).
 *
 * Definitions used by every call:
 *   voxel order   volumes are [nz][ny][nx], x fastest: i = x + nx*(y + ny*z).
 *   mask          m_k(i) = [ (float)c(i) >= t_k ],  k = 1 (T1Gd), 2 (FLAIR).
 *   bit planes    plane k of a volume is an array of uint32 words; bit b of
 *                 word w is voxel 32*w + b.  Bits past the last voxel are 0.
 *   counts        I_k = |P_k n E_k|, E_k = |E_k|, P_k = |P_k| (patient).
 *   Dice          D_k = 2 I_k / (P_k + E_k) in IEEE binary64, round to
 *                 nearest;  D_k = 1 when P_k + E_k = 0 (both masks empty).
 *   score         S = (D_1 + D_2) * 0.5 in binary64.
 *   order         entries are ranked by (S descending, index ascending):
 *                 of two equal scores the lower database index ranks first.
 *
 * Conventions:
 *   * Every call returns a dbq_status; on failure db_last_error() returns a
 *     thread-local message and no output has been written -- except that a
 *     failure of the device itself (DBQ_ECUDA, DBQ_ETIMEOUT) can leave
 *     partial results in device-memory outputs that kernels write directly.
 *   * "host or device" pointers are classified with cudaPointerGetAttributes;
 *     host memory may be pageable or pinned.  A pinned (page-locked), 16-byte
 *     aligned host patient is read in place by the packing kernel over the
 *     host link; other host patients are first copied to device staging.
 *   * `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *     whose outputs are host memory return only after their work is complete.
 *     The *_async calls only enqueue work on `stream`.
 *   * A handle is thread-safe (an internal mutex serialises calls), but all
 *     work of one handle shares one query workspace in device memory, so
 *     asynchronous calls on one handle must not overlap on the GPU: issue them
 *     on one stream, or synchronise between streams.
 *   * The library owns all database device memory and frees it in
 *     db_destroy(); the caller owns every buffer it passes in.
 */
#ifndef DBQ_H
#define DBQ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dbq_db dbq_db;

/* Status codes. */
enum dbq_status {
    DBQ_OK = 0,
    DBQ_EINVAL = -1,   /* bad argument: null pointer, bad size, bad threshold  */
    DBQ_ENOMEM = -2,   /* device or host allocation failed                     */
    DBQ_ESTATE = -3,   /* call not valid in the handle's state (e.g. unbuilt)  */
    DBQ_ECUDA = -4,    /* a CUDA runtime call or a kernel launch failed         */
    DBQ_ETIMEOUT = -5, /* a bounded device wait of a tensor-core kernel gave up  */
    DBQ_ERANGE = -6    /* k or an index outside [0, N]                          */
};

/* Element kinds of volumes passed in. */
enum dbq_kind {
    DBQ_F32 = 0,   /* float32 concentrations [V]                               */
    DBQ_F16 = 1,   /* IEEE binary16 concentrations [V] (uint16 bit patterns)   */
    DBQ_BITS = 2   /* two bit planes [2][ceil(V/32)] uint32 (patients only)    */
};

/* Database storage. */
enum dbq_storage {
    DBQ_STORE_BITS = 0, /* masks thresholded at build time, 1 bit per voxel per
                           threshold; queries use the build thresholds       */
    DBQ_STORE_F16 = 1   /* binary16 concentrations; each query thresholds the
                           database at its own (t1, t2)                      */
};

/* db_create flags. */
#define DBQ_FLAG_EMBED 1u  /* also build the prefilter embeddings (see db_query_batch) */
#define DBQ_FLAG_SKETCH 2u /* build count-sketch embeddings and sign codes instead  */

/* Options of db_set_option. */
enum dbq_option {
    DBQ_OPT_SPARSE = 1,  /* 1: exact scans of a bit-packed database read only the
                            words where the patient's mask is non-zero (exact
                            counts, fewer bytes); 2: the same from a word-major
                            copy of the planes (faster, twice the planes' memory);
                            0 (default): read every word */
    DBQ_OPT_RERANK = 2   /* re-ranking of db_query_batch's embedding modes on a
                            dense bit-packed database: 2 reads each distinct
                            candidate entry of a batch once, 1 reads every
                            (query, candidate) pair's entry, 0 (default) takes
                            2 for batches of 32 queries or more, else 1 */
};

/* Query modes of db_query_batch. */
enum dbq_mode {
    DBQ_MODE_EXACT = 0,       /* the brute-force loop over every entry           */
    DBQ_MODE_EMBED_BF16 = 1,  /* bfloat16 embedding prefilter + exact re-ranking  */
    DBQ_MODE_EMBED_FP8 = 2,   /* FP8 E4M3 embedding prefilter + exact re-ranking  */
    DBQ_MODE_HASH = 3         /* Hamming prefilter on sign codes + re-ranking     */
};

/* One ranked result.  p1/p2 are the patient's mask sizes. */
typedef struct dbq_hit {
    int64_t index;     /* database entry                                      */
    double score;      /* (Dice_T1Gd + Dice_FLAIR) / 2                         */
    uint32_t i1, i2;   /* |P_1 n E_1|, |P_2 n E_2|                              */
    uint32_t e1, e2;   /* |E_1|, |E_2| of the entry                             */
    uint32_t p1, p2;   /* |P_1|, |P_2| of the patient                           */
} dbq_hit;

/*
 * db_create -- make an empty database of `capacity` entries on the current
 * CUDA device.
 *   nx, ny, nz   grid of every volume (each >= 1; V = nx*ny*nz < 2^31).
 *   capacity     number of entries N (>= 1); all are allocated up front:
 *                BITS storage 2*ceil4(ceil(V/32))*4 bytes per entry,
 *                F16 storage 2*V bytes per entry.
 *   storage      DBQ_STORE_BITS or DBQ_STORE_F16.
 *   t1, t2       BITS storage: the T1Gd and FLAIR thresholds the masks are
 *                built with (Section 2.3 uses 0.6 and 0.2); each must be a
 *                finite number in (0, 1].  F16 storage: ignored.
 *   n_params     doubles of theta kept per entry (0..64), returned with hits.
 *   flags        0, or DBQ_FLAG_EMBED: BITS storage only, nx a multiple of 32
 *                and ny, nz multiples of 8; db_build_masks() then also builds
 *                the prefilter embeddings (2 x (nx/8)(ny/8)(nz/8) values per
 *                entry, bfloat16 and FP8 E4M3 with per-row scales).
 *                Or DBQ_FLAG_SKETCH: BITS storage, any grid; the embedding of
 *                each mask is instead a count sketch, a random projection of
 *                the mask onto D = 4096 values per segmentation: voxel x adds
 *                s(x) = +-1 to bucket b(x), where h = SplitMix64 (Steele, Lea &
 *                Flood 2014) of counter x, b(x) = (h >> 32) mod D and s(x) =
 *                -1 iff bit 31 of h is set.  |sk(A) - sk(B)|^2 is an unbiased
 *                estimate of |A xor B|.  The sketch is encoded like the block
 *                means (bf16, FP8 with scale max|v|/448), and its sign code
 *                (bit j = [v_j > 0], 32 buckets per word) is kept for
 *                DBQ_MODE_HASH, also as one E4M3 byte per bucket (1.0 or 0)
 *                with its popcount, the operands of the exact tensor-core
 *                Hamming distance.  Device memory per entry: 2 x 4096 x
 *                (2 + 1 + 1) bytes + 1 KiB of bits + 24 bytes, plus a 2 x V
 *                byte bucket table per database.  The two flags exclude each
 *                other.
 * Returns DBQ_OK and *out, or DBQ_EINVAL / DBQ_ENOMEM / DBQ_ECUDA.
 */
int db_create(dbq_db** out, int nx, int ny, int nz, int64_t capacity, int storage,
              float t1, float t2, int n_params, uint32_t flags);

/*
 * db_load_volumes -- put entries [first, first+count) into the database.
 *   vols     [count][V] DBQ_F32 or DBQ_F16 volumes, host or device memory.
 *            BITS storage thresholds them at (t1, t2) into bit planes and
 *            the per-entry mask sizes |E_1|, |E_2| (the build step of the
 *            thresholding in Section 2.3); no concentration is kept.
 *            F16 storage keeps binary16 values (float32 input is rounded to
 *            nearest-even).
 *   params   host [count][n_params] doubles (theta), or NULL (zeros).
 * Entries may be loaded in any order and reloaded.  Loading clears the built
 * state; call db_build_masks() again before querying.
 */
int db_load_volumes(dbq_db* db, int64_t first, int64_t count, const void* vols, int kind,
                    const double* params, void* stream);

/*
 * db_build_masks -- finish the build: check that every entry in
 * [0, capacity) has been loaded and make the database queryable.  The masks
 * themselves are written as volumes are loaded.  With DBQ_FLAG_EMBED this
 * call computes each mask's embedding: the mean of every 8 x 8 x 8 block
 * (the low-dimensional representations queried by L2 in Section 2.3),
 * encoded as bfloat16 (round to nearest-even) and as FP8 E4M3 of e / s with
 * s = max(e) / 448 per row (binary32), plus the rows' squared norms.
 * Returns DBQ_ESTATE if an entry is missing.
 */
int db_build_masks(dbq_db* db, void* stream);

/*
 * db_query -- the brute-force query: score the patient against every entry
 * and return the k best under the order above.
 *   patient  host or device; kind DBQ_F32 / DBQ_F16 volume [V] (thresholded
 *            here at (t1, t2)), or DBQ_BITS planes [2][ceil(V/32)] (bits
 *            past voxel V-1 are ignored).
 *   t1, t2   BITS storage: must equal the build thresholds, or be NaN to
 *            mean "the build thresholds".  F16 storage: the thresholds
 *            applied to the database and to a volume patient, in (0, 1].
 *   k        1 <= k <= min(N, 1024); DBQ_ERANGE otherwise.
 *   hits     host [k], written in rank order.
 *   params   host [k][n_params] theta of the hits, or NULL.
 * Returns after the results are in host memory.
 */
int db_query(dbq_db* db, const void* patient, int kind, float t1, float t2, int k,
             dbq_hit* hits, double* params, void* stream);

/*
 * db_query_async -- as db_query, but the patient must be device memory and
 * the k hits are written to device memory `hits_dev` [k]; the work is only
 * enqueued on `stream` (no host synchronisation, no host copies), so the
 * call can be captured in a CUDA graph.
 */
int db_query_async(dbq_db* db, const void* patient_dev, int kind, float t1, float t2,
                   int k, dbq_hit* hits_dev, void* stream);

/*
 * db_prepare_patient / db_query_prepared -- the two steps of db_query_async
 * issued separately: the first thresholds (or imports) a device-memory
 * patient into the handle's workspace (the patient's segmentations, Section
 * 2.3), the second runs the scan, scoring and top-k selection against that
 * prepared patient and writes `k` hits to device memory.  Both only enqueue
 * work on `stream`.  db_query_prepared returns DBQ_ESTATE if no patient has
 * been prepared since the handle was created.
 */
int db_prepare_patient(dbq_db* db, const void* patient_dev, int kind, float t1, float t2,
                       void* stream);
int db_query_prepared(dbq_db* db, int k, dbq_hit* hits_dev, void* stream);

/*
 * db_scan_counts -- the per-entry counts of one patient, for every entry:
 * counts [N][4] = (I_1, I_2, E_1, E_2), host or device memory, plus the
 * patient's (P_1, P_2) in pcount [2] (host or device).  Same patient and
 * threshold rules as db_query.  Returns after the counts are written.
 */
int db_scan_counts(dbq_db* db, const void* patient, int kind, float t1, float t2,
                   uint32_t* counts, uint32_t* pcount, void* stream);

/*
 * db_get_masks -- copy the packed planes of entries [first, first+count) to
 * `planes` [count][2][words] (host or device) and their mask sizes to
 * `sizes` [count][2] (host or device, or NULL).  BITS storage only.
 * `words` = ceil(V/32); see db_info().
 */
int db_get_masks(dbq_db* db, int64_t first, int64_t count, uint32_t* planes,
                 uint32_t* sizes, void* stream);

/*
 * db_info -- sizes of a handle: out[0] = N, out[1] = V, out[2] = words per
 * plane ceil(V/32), out[3] = padded words per plane, out[4] = storage,
 * out[5] = built (0/1), out[6] = n_params, out[7] = device bytes held.
 */
int db_info(const dbq_db* db, int64_t out[8]);

/*
 * db_query_batch -- `nq` queries, each against the database
 * dbs[db_of_query[q]], returning k hits per query.
 *   patients      [nq] pointers (host or device), each a volume of `kind`
 *                 (DBQ_F32 / DBQ_F16) or DBQ_BITS planes for its database.
 *   t1, t2        [nq] per-query thresholds, or NULL (NaN: the build
 *                 thresholds of a bit-packed database).
 *   mode          DBQ_MODE_EXACT: the full loop per query (any storage).
 *                 DBQ_MODE_EMBED_BF16 / _FP8: for databases built with
 *                 DBQ_FLAG_EMBED, the L2 prefilter over the embeddings
 *                 (L = L2_T1Gd + L2_FLAIR of the non-squared distances,
 *                 Section 2.3; a tensor-core GEMM with fp32 accumulation)
 *                 keeps the `n_candidates` closest entries per query (ties to
 *                 the lower index), which are re-ranked by the exact Dice
 *                 loop; the hits are exact for the entries they name.
 *                 DBQ_MODE_HASH: for databases built with DBQ_FLAG_SKETCH,
 *                 the same with the Hamming distance between the sign codes
 *                 (summed over both segmentations; the binary-code queries of
 *                 Section 2.3) as the prefilter distance.
 *   n_candidates  1 <= k <= n_candidates <= min(N, 1024) (embedding modes).
 *   hits          host [nq][k]; params host [nq][k][n_params] or NULL.
 * Queries are processed in groups of up to 256 per database.  Returns after
 * the results are in host memory.
 */
int db_query_batch(dbq_db* const* dbs, const int* db_of_query, int nq,
                   const void* const* patients, int kind, const float* t1, const float* t2,
                   int k, int mode, int n_candidates, dbq_hit* hits, double* params,
                   void* stream);

/*
 * Query plans: many exact queries against several bit-packed databases (of
 * any resolutions) in one persistent launch.  A plan owns the device
 * workspace for up to `max_queries` queries of k hits each; db_plan_query
 * only enqueues work (no host synchronisation, no allocation), so it can be
 * captured into a CUDA graph and replayed.
 *
 * db_plan_create  dbs[ndb] must live on one device, be bit-packed and
 *                 built, and outlive the plan.  1 <= k <= 1024.
 * db_plan_set     DBQ_PLAN_ITEMS_PER_SM: work items (query slices) per SM
 *                 of one launch (default 4; chosen by the autotuner).
 *                 DBQ_PLAN_TC_MIN_QUERIES: a database queried by at least
 *                 this many queries in one call, with V <= 2^24 voxels and
 *                 at least 32 words per plane, is scanned for all of them at once
 *                 as a contraction on the tensor cores (the intersections
 *                 of Section 2.3 as 0/1 dot products over the voxels, exact
 *                 in binary32; up to 128 queries per pass), then scored and
 *                 ranked per query -- the same hits as the CUDA-core loop.
 *                 A contraction reads every word, whatever the database's
 *                 DBQ_OPT_SPARSE setting (which then only selects the
 *                 CUDA-core loop's variant below the threshold).
 *                 Default 16; 0 keeps every query on the CUDA-core loop.
 * db_plan_query   patients_dev[nq] device pointers (kind DBQ_F32 / DBQ_F16
 *                 volumes or DBQ_BITS planes of the query's database),
 *                 t1/t2 per query or NULL (NaN = build thresholds; others
 *                 must equal them), hits_dev [nq][k] device output.  Each
 *                 query honours its database's DBQ_OPT_SPARSE setting.  The
 *                 plan's host-side tables are rewritten by each call: a call
 *                 outside stream capture waits until the previous call's
 *                 tables have been copied to the device.
 * db_plan_status  synchronises `stream` and reports whether a bounded wait
 *                 of the tensor-core path has timed out since the last call
 *                 (DBQ_ETIMEOUT, and the affected hits are not valid) or
 *                 not (DBQ_OK); clears the condition.  Not capturable.
 * db_plan_destroy frees the plan (NULL accepted).
 */
typedef struct dbq_plan dbq_plan;
enum dbq_plan_param {
    DBQ_PLAN_ITEMS_PER_SM = 1,
    DBQ_PLAN_TC_MIN_QUERIES = 2,
    DBQ_PLAN_TEST_STALL_NS = 3   /* test hook, default 0: with value > 0, each
                                    tensor-core launch first waits up to that
                                    many ns on a barrier that nothing arrives
                                    at, gives up, and takes its timeout path
                                    (no hits are valid; db_plan_status then
                                    returns DBQ_ETIMEOUT).  At most 2e9. */
};
int db_plan_create(dbq_plan** out, dbq_db* const* dbs, int ndb, int max_queries, int k);
int db_plan_set(dbq_plan* plan, int param, int64_t value);
/* db_plan_set_for -- DBQ_PLAN_TC_MIN_QUERIES for database dbs[db_index] of
 * the plan alone (the crossover between the two paths depends on the
 * database's resolution and size); -1 returns it to the plan-wide value.
 * DBQ_ERANGE for an index outside the plan. */
int db_plan_set_for(dbq_plan* plan, int db_index, int param, int64_t value);
int db_plan_query(dbq_plan* plan, const int* db_of_query, int nq, const void* const* patients_dev,
                  int kind, const float* t1, const float* t2, dbq_hit* hits_dev, void* stream);
int db_plan_status(dbq_plan* plan, void* stream);
int db_plan_destroy(dbq_plan* plan);

/*
 * db_prefilter -- the prefilter step of db_query_batch alone, for
 * measurement and checking: distances dist [nq][N] (host or device, or
 * NULL) and the n_candidates closest entries per query, ascending, cand
 * [nq][n_candidates] int32 (host or device, or NULL).  nq <= 256; bit-packed
 * databases built with DBQ_FLAG_EMBED or DBQ_FLAG_SKETCH only.  In
 * DBQ_MODE_HASH the distances are the Hamming distances (exact integers).
 */
int db_prefilter(dbq_db* db, int nq, const void* const* patients, int kind, int mode,
                 int n_candidates, float* dist, int32_t* cand, void* stream);

/*
 * db_set_option -- set a per-handle option (enum dbq_option).
 * DBQ_OPT_SPARSE: |P_k n E_k| only involves the voxels of the patient's
 * masks (the Dice numerator, Section 2.3), so with value 1 every exact scan
 * and every re-ranking of a bit-packed database lists the patient's non-zero
 * 64-byte granules first and reads only those words of each entry.  Results
 * are identical; the bytes read per entry shrink to the patient's support.
 * Ignored by half-precision databases (their mask sizes are computed at
 * query time from every voxel).  Value 2 does the same for the
 * single-patient scans (db_query, db_query_async, db_query_prepared,
 * db_scan_counts) over a word-major copy of the planes ([2 wp][n] 16-byte
 * words: each support word of every entry is one contiguous run), which
 * the library allocates here (DBQ_ENOMEM if the device lacks room: N x 2 x
 * words-per-plane x 4 bytes plus N x 8) and builds in db_build_masks (or
 * here, if the database is already built).  Plans use
 * the copy too, for a database's queries that do not go to the tensor-core
 * contraction: the counts of all of them over the copy, then the
 * contraction's per-query selection.  The other paths treat 2 as 1.
 * DBQ_EINVAL for 2 on half-precision storage or for any value outside 0..2.
 * DBQ_OPT_RERANK: how db_query_batch re-ranks the prefilter's candidates
 * when DBQ_OPT_SPARSE is 0.  The queries of a batch share candidates, so
 * with 2 the candidate pairs are sorted by entry and every distinct entry
 * is read once, slice by slice, against the slices of all the queries that
 * picked it (held in shared memory); with 1 each query reads its own
 * candidates; 0 (default) takes 2 for a group of 32 queries or more of one
 * database, else 1.  The hits are the same.  A sparse database always
 * re-ranks per query, reading only the patient's support.  DBQ_EINVAL
 * outside 0..2.
 */
int db_set_option(dbq_db* db, int option, int64_t value);

/*
 * db_last_support -- with DBQ_OPT_SPARSE, the lengths (in 16-byte words) of
 * the support lists of the last patient prepared by a single-patient call:
 * out[0] plane 1, out[1] plane 2.  Bytes read per entry by the sparse scan =
 * 16 * (out[0] + out[1]).  DBQ_ESTATE without such a patient.
 */
int db_last_support(dbq_db* db, int64_t out[2]);

/*
 * db_stage_times -- GPU milliseconds of the stages of the handle's last
 * embedding-mode db_query_batch group: ms[0] patient thresholding, ms[1]
 * query embeddings, ms[2] distances (tensor-core GEMM, or Hamming in
 * DBQ_MODE_HASH), ms[3] candidate selection,
 * ms[4] exact re-ranking.  n <= 5 values are written; DBQ_ESTATE if no such
 * batch has run.
 */
int db_stage_times(dbq_db* db, float* ms, int n);

/*
 * db_get_embeddings -- copy the embeddings of entries [first, first+count):
 * bf16 [count][2][d] (uint16 bit patterns), e4m3 [count][2][d] codes, scale
 * [count][2], norm_bf16 and norm_fp8 [count][2] (squared norms of the
 * decoded rows).  Any output may be NULL; host or device memory.
 */
int db_get_embeddings(dbq_db* db, int64_t first, int64_t count, uint16_t* bf16, uint8_t* e4m3,
                      float* scale, float* norm_bf16, float* norm_fp8, void* stream);

/*
 * db_get_codes -- copy the sign codes of entries [first, first+count) to
 * `codes` [count][2][128] uint32 (host or device).  Databases built with
 * DBQ_FLAG_SKETCH only (DBQ_ESTATE otherwise).
 */
int db_get_codes(dbq_db* db, int64_t first, int64_t count, uint32_t* codes, void* stream);

/*
 * db_create_downsampled -- a bit-packed database made from `src` by
 * nearest-neighbour downsampling by `factor` (Section 2.3's queries on a
 * database downsampled to 64^3 or 32^3 with an order-0 spline): voxel
 * (x, y, z) of the coarse grid is voxel (f x, f y, f z) of the source.  The
 * new handle is built, shares nothing with `src` afterwards, keeps the same
 * thresholds and theta, and takes patients at the SOURCE resolution in
 * db_query / db_query_async / db_prepare_patient / db_scan_counts,
 * downsampling them the same way.  src must be bit-packed and built, its
 * grid divisible by factor (2..16).  Batches and plans do not accept such a
 * handle (DBQ_ESTATE).
 */
int db_create_downsampled(dbq_db** out, dbq_db* src, int factor);

/*
 * db_scan_packed_noalloc -- the bit-packed exact query for callers that
 * cannot allocate device memory (a memory pool that owns the whole GPU, a
 * request path that must not synchronise on an allocation, a plug-in host
 * that forbids device allocations).  The paper has no counterpart: it is an
 * interface variant of db_query_prepared, not a step of the method.
 *   planes          device [n][2][stride_words] bit planes (layout above;
 *                   bits past the last voxel 0), 16-byte aligned.
 *   sizes           device [n][2] mask sizes |E_1|, |E_2|, 8-byte aligned.
 *   stride_words    words per plane in `planes` and `patient_planes`; a
 *                   multiple of 4 that covers ceil(V/32).
 *   patient_planes  device [2][stride_words] patient planes, 16-byte aligned.
 *   patient_sizes   device [2] |P_1|, |P_2|.
 *   k               1 <= k <= min(n, 64); DBQ_ERANGE otherwise.
 *   hits            device [k] output, 8-byte aligned.
 * Only enqueues work on `stream`; allocates nothing.  Its scratch is one
 * fixed array of 512.25 KiB in device memory that every GPU loading the
 * library keeps until exit, shared by all calls: calls that overlap on the
 * GPU race.  Each call made outside stream capture looks up the array's
 * device address and caches it per device (so a device reset between calls
 * is harmless); a call made during capture uses the cached address, so make
 * the first call on a device before any capture (DBQ_ESTATE otherwise).
 * Devices with more than 256 SMs are rejected.
 */
int db_scan_packed_noalloc(const uint32_t* planes, const uint32_t* sizes, int64_t n,
                           int64_t stride_words, const uint32_t* patient_planes,
                           const uint32_t* patient_sizes, int k, dbq_hit* hits, void* stream);

/* db_destroy -- free everything the handle owns.  NULL is accepted. */
int db_destroy(dbq_db* db);

/* Last error message of the calling thread ("" if none). */
const char* db_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* DBQ_H */
