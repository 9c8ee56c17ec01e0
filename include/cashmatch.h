/*
 * cashmatch — cascade-hashing feature matching over MBR-scheduled image blocks,
 * for NVIDIA B300 (sm_103a).  C ABI.
 *
 * Method: "Efficient Feature Matching for UAV Images based on Compact GPU Data
 * Scheduling" (arXiv 2505.22089).  Cascade hashing, Sec. 2.3.1 steps (1)-(4):
 * hash lookup in L tables of 2^m buckets, remapping to n-bit codes, Hamming
 * ranking to the top K, Euclidean rerank and ratio test.  Schedule blocks by
 * matrix band reduction, Sec. 2.2 steps (1)-(5) with the GPS ordering of
 * Algorithm 2.  Block-row load / match / free, Sec. 2.3.2 and Algorithm 1.
 *
 * Conventions for every call:
 *  - Return value: CM_OK or an error code; nothing is thrown across the ABI.
 *    cm_last_error() returns a message for the calling thread's last error.
 *  - "device" pointers are CUDA global-memory addresses on the current device;
 *    "host" pointers are CPU addresses (pinned memory gives overlapped copies).
 *  - Streams are cudaStream_t values passed as cm_stream (NULL = legacy
 *    default stream).  Calls documented "async" only enqueue work: inputs must
 *    stay valid and outputs must not be read until the stream is synchronised.
 *  - Ownership: the caller owns every buffer it passes.  The library owns the
 *    handles it returns and frees them in the matching cm_*_destroy / cm_free_*.
 *    The library never calls cudaMalloc: all device storage of an index comes
 *    from the caller's arena.
 *  - Descriptors are uint8 [rows][128], row-major, 128 bytes per row.  An
 *    image holds at most 65,535 descriptors.
 */
#ifndef CASHMATCH_H
#define CASHMATCH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* cm_stream;

typedef enum {
    CM_OK = 0,
    CM_ERR_INVALID = 1,  /* bad argument: NULL, out-of-range id, i == j, N > 65535, bad params */
    CM_ERR_BUDGET = 2,   /* arena / HBM budget too small for what was asked */
    CM_ERR_CUDA = 3,     /* a CUDA runtime call failed (message has the CUDA error) */
    CM_ERR_TIMEOUT = 4,  /* a bounded device wait gave up; results of that launch are invalid */
    CM_ERR_NOMEM = 5,    /* host allocation failed */
    CM_ERR_STATE = 6     /* call not valid in the object's current state (e.g. image not resident) */
} cm_status;

/* How the top-K candidates are re-scored by Euclidean distance (step (4)). */
typedef enum {
    CM_RERANK_FP32 = 0,  /* CUDA cores, FP32 arithmetic (exact: all partial sums are integers < 2^24) */
    CM_RERANK_BF16 = 1,  /* tensor cores (tcgen05, kind::f16), BF16 inputs, FP32 accumulate (exact for uint8) */
    CM_RERANK_FP8 = 2,   /* tensor cores, FP8 e4m3 with a per-descriptor scale, FP32 accumulate; the top 2
                            are re-scored exactly in FP32 */
    CM_RERANK_INT = 3    /* CUDA cores, 4-way byte SIMD integer arithmetic (exact) */
} cm_rerank;

/* Thread mapping of the match kernel (both compute the same result). */
typedef enum {
    CM_ALGO_AUTO = 0,    /* library choice: CM_ALGO_BUCKET */
    CM_ALGO_TILE = 1,    /* one lane per query; a CTA keeps a tile of queries' top-K in shared memory and
                            sweeps the tables with the queries sorted by bucket */
    CM_ALGO_WARP = 2,    /* one warp per query; top-K kept across the warp with ballots and shuffles */
    CM_ALGO_TC = 3,      /* a CTA per pair; each bucket's queries x database points block of Hamming
                            distances on the tensor cores (code bits as E4M3 +-1: dot = 128 - 2 h, exact);
                            then a separate rerank launch.  K in {4, 8, 16} */
    CM_ALGO_BUCKET = 4   /* bucket-major (the AUTO choice): a CTA per pair sweeps the tables; a warp takes 32
                            queries of one bucket and streams that bucket's database run through shared memory
                            (bulk copies), every lane reading the same candidate; lists kept in the plan */
} cm_algo;

/* How the projections onto the hyperplanes are computed (both decide the same
 * sign bits up to projections within FP32 rounding of zero). */
typedef enum {
    CM_PROJ_TC = 0,      /* tensor cores: x in BF16 (exact), W as a sum of three BF16 parts, FP32 accumulate */
    CM_PROJ_FFMA = 1     /* CUDA cores: FP32 fused multiply-add */
} cm_projection;

/* Where descriptor pointers given to the library live. */
typedef enum {
    CM_MEM_HOST = 0,          /* host memory: the library copies it into the arena (H2D) */
    CM_MEM_DEVICE = 1,        /* device memory: the library copies it into the arena (D2D) */
    CM_MEM_DEVICE_INPLACE = 2 /* device memory used in place; the caller keeps it alive and unchanged */
} cm_mem;

/* Cascade-hashing parameters.  Paper defaults (Sec. 2.3.1): L = 6, m = 8,
 * n = 128, K = 8; ratio threshold t_r = ratio_num / ratio_den (0.8 = 4/5 in
 * SiftGPU, 0.5 chosen in Sec. 3.2).  The ratio test dis(q1) < t_r dis(q2) is
 * decided exactly. */
typedef struct cm_params {
    int32_t L;           /* hash tables, 1..8 */
    int32_t m;           /* bits per bucket key, 0..8 (2^m buckets per table) */
    int32_t n_bits;      /* fine code bits; must be 128 */
    int32_t K;           /* Hamming top-K kept for the rerank: 2, 4, 8 or 16 */
    int32_t ratio_num;   /* t_r numerator, >= 0 */
    int32_t ratio_den;   /* t_r denominator, >= 1; num/den <= 4 */
    uint64_t seed;       /* seed of the projection weights (splitmix64 + Box-Muller, see cm_make_weights) */
    int32_t rerank;      /* cm_rerank */
    int32_t query_tile;  /* queries per work item of the match kernel, multiple of 64; 0 = default (2048, less
                            for K = 16 so the tile kernel's shared memory fits) */
    int32_t algo;        /* cm_algo */
    int32_t projection;  /* cm_projection */
} cm_params;

typedef struct { int32_t i, j; } cm_pair;  /* query image i, database image j (i != j) */

typedef struct cm_index cm_index;
typedef struct cm_schedule cm_schedule;
typedef struct cm_match_plan cm_match_plan;
typedef struct cm_sequence cm_sequence;

/* Outputs of a match launch: per query row, device pointers, any may be NULL
 * except best_j.  Rows of pair k start at row_off(k) = sum of N_i over the
 * pairs before k in the plan's pair list. */
typedef struct cm_match_out {
    int32_t* best_j;     /* index in image j of the accepted nearest neighbour, or -1 */
    uint32_t* d1sq;      /* squared distance to q1 (UINT32_MAX if fewer than 1 candidate) */
    uint32_t* d2sq;      /* squared distance to q2 (UINT32_MAX if fewer than 2 candidates) */
    int32_t* topk;       /* [rows][K] Hamming top-K in rank order, -1 padded (diagnostic) */
    uint32_t* stats;     /* [4] accumulated counters: 0 FP64 re-checks, 1 matches, 2 FP8 top-2 swaps, 3 reserved */
} cm_match_out;

/* One row of a schedule (Sec. 2.3.2: load the row's new block, match, free the first block). */
typedef struct cm_schedule_row {
    int32_t iteration;      /* MBR iteration (Sec. 2.2 step (5)) */
    int32_t n_load;         /* images to make resident before the row */
    const int32_t* load;
    int32_t n_free;         /* images released after the row */
    const int32_t* free_ids;
    int64_t n_pairs;        /* pairs matched in this row, as indices into the caller's pair list */
    const int64_t* pairs;
} cm_schedule_row;

/* ---- library ------------------------------------------------------------ */
const char* cm_version(void);
/* Message of the calling thread's last failed call ("" if none).  Valid until the next call on the thread. */
const char* cm_last_error(void);
/* Fills paper defaults: L=6, m=8, n_bits=128, K=8, t_r=4/5, rerank=FP32. */
cm_status cm_params_default(cm_params* p);
/* Checks a parameter set; CM_ERR_INVALID with a message if unsupported. */
cm_status cm_params_check(const cm_params* p);

/* Projection weights W[128][P] (host, row-major, P = L*m + n_bits): random
 * hyperplanes through the centred origin (Sec. 2.3.1 "LSH ... random hashing
 * functions").  Columns t*m .. t*m+m-1 give the bucket key of table t (bit b =
 * column t*m+b), columns L*m .. P-1 the fine code.  W is drawn from one
 * splitmix64 stream seeded with p->seed: each pair of outputs (r1, r2) gives
 * u1 = ((r1>>11)+1) 2^-53, u2 = (r2>>11) 2^-53 and the Box-Muller pair
 * sqrt(-2 ln u1) (cos, sin)(2 pi u2), filled row-major and rounded to float. */
cm_status cm_make_weights(const cm_params* p, float* W_host);

/* Arena bytes one resident image of n descriptors occupies (layout of the
 * index: descriptors, keys, codes, bucket-sorted codes and indices, offsets,
 * norms, and the tensor-core copy for BF16/FP8 reranks). */
cm_status cm_image_bytes(const cm_params* p, int32_t n_desc, uint64_t* bytes);
/* Arena bytes for an index holding every image of n_desc resident (descriptors
 * in place when inplace != 0), plus its fixed tables. */
cm_status cm_index_bytes(const cm_params* p, int32_t n_images, const int32_t* n_desc, int32_t inplace,
                         uint64_t* bytes);

/* ---- schedule blocks (Sec. 2.2; Algorithm 1, CascadeHashingMatching; Algorithm 2) */
/* Symmetrises the pair graph, orders it by GPS, cuts the order into chunks of
 * at most max_images_per_block images (Size_blk), and forms block rows: the
 * window of consecutive chunks whose resident bytes (cm_image_bytes) fit
 * hbm_budget.  Each row takes the unprocessed pairs whose lower chunk is the
 * row's first chunk and whose other image lies in the window; the rest wait
 * for the next MBR iteration, which re-orders the remaining graph.  Repeats
 * until every pair is placed.  Host only, synchronous.
 * Errors: CM_ERR_INVALID (id out of range, i == j), CM_ERR_BUDGET (a pair's two
 * images exceed the budget). */
cm_status cm_schedule_blocks(const cm_pair* pairs, int64_t n_pairs, int32_t n_images, const int32_t* n_desc,
                             const cm_params* p, uint64_t hbm_budget, int32_t max_images_per_block,
                             cm_schedule** out);
/* A schedule from the caller's own rows, for strategies other than the MBR
 * blocks (one pair at a time, load/free lists, graph partitions); it runs
 * through cm_run_schedule like a block schedule.  The rows are copied and
 * checked by replaying residency: a row loads only non-resident images and
 * frees only resident ones; both images of each of its pairs are resident
 * during the row; every index 0..n_pairs-1 of `pairs` appears in exactly one
 * row.  Errors: CM_ERR_INVALID with the first violation in cm_last_error(). */
cm_status cm_schedule_from_rows(int32_t n_rows, const cm_schedule_row* rows, const cm_pair* pairs, int64_t n_pairs,
                                int32_t n_images, cm_schedule** out);
int32_t cm_schedule_num_rows(const cm_schedule* s);
int32_t cm_schedule_num_iterations(const cm_schedule* s);
/* View of row r; pointers stay valid until cm_free_schedule. */
cm_status cm_schedule_get_row(const cm_schedule* s, int32_t r, cm_schedule_row* row);
void cm_free_schedule(cm_schedule* s);
/* GPS ordering (Algorithm 2) of the undirected graph on n nodes with the given
 * edges (int32 pairs).  Writes the non-isolated nodes in their new order to
 * order[] (capacity n) and their count to *n_order. */
cm_status cm_gps_order(int32_t n, int64_t n_edges, const int32_t* edges, int32_t* order, int32_t* n_order);

/* ---- index (Sec. 2.3.2 step (1): load, hash, build lookup tables) -------- */
/* Creates an empty index over n_images images of the given sizes, using the
 * caller's device arena for all its device storage.  Nothing resident yet. */
cm_status cm_index_create(const cm_params* p, int32_t n_images, const int32_t* n_desc, void* d_arena,
                          uint64_t arena_bytes, cm_index** out);
/* Centring mean from exact column sums: mu = sums / n_total (host values;
 * the upload is enqueued on stream). */
cm_status cm_index_set_mean(cm_index* ix, const uint64_t* col_sums_host, uint64_t n_total, cm_stream stream);
/* Centring mean from the exact column sums of n_rows device descriptor rows
 * (async, on stream). */
cm_status cm_index_mean_device(cm_index* ix, const uint8_t* d_desc, uint64_t n_rows, cm_stream stream);
/* Centring mean of the whole index from host rows (the a2 statistics of an
 * end-to-end run whose descriptors start in host memory): desc_host[i] points
 * at image i's n_desc[i] rows (NULL allowed for an empty image).  The rows
 * are copied through staging blocks taken from the free part of the arena
 * (up to 2 x 64 MiB) and summed exactly in uint64 on the GPU (k_colsum_rows),
 * then mu = sums / N.  Pinned host memory makes the copies asynchronous.
 * Async on stream; the rows must stay valid until the stream is synchronised.
 * Errors: CM_ERR_INVALID (NULL rows of a non-empty image, no rows at all),
 * CM_ERR_BUDGET (not even 1 MiB of the arena free), CM_ERR_CUDA. */
cm_status cm_index_mean_host(cm_index* ix, const uint8_t* const* desc_host, cm_stream stream);
/* Exact column sums and row count behind the current centring mean, copied to
 * host (waits for stream).  Valid after cm_build_index, cm_index_mean_device,
 * cm_index_mean_host, cm_index_rehash or cm_index_set_mean. */
cm_status cm_index_col_sums(cm_index* ix, uint64_t* sums_host, uint64_t* n_total, cm_stream stream);
/* Makes images resident (async): copies their descriptors into the arena
 * (unless CM_MEM_DEVICE_INPLACE), computes keys and codes and builds the per
 * table buckets.  desc[k] points at image ids[k]'s rows.  The mean must be set.
 * Errors: CM_ERR_STATE (already resident / mean unset), CM_ERR_BUDGET (arena full). */
cm_status cm_index_load(cm_index* ix, int32_t count, const int32_t* ids, const uint8_t* const* desc,
                        int32_t mem, cm_stream stream);
/* Waits for stream and reports whether a bounded device wait of the index's
 * kernels gave up since the last check (CM_ERR_TIMEOUT; the results of that
 * work are invalid).  Clears the flag. */
cm_status cm_index_check(cm_index* ix, cm_stream stream);
/* Recomputes centring statistics from the resident descriptors, then keys,
 * codes and buckets of every resident image (async; a whole hashing pass). */
cm_status cm_index_rehash(cm_index* ix, cm_stream stream);
/* Exact uint64 column sums of the listed resident images' descriptors into
 * d_sums (device, 128 entries; zeroed first), asynchronous on stream.  With
 * cm_index_set_mean_device and cm_index_hash this splits cm_index_rehash so
 * the sums can be reduced across processes in between: each process of a
 * sharded job sums the images it owns, an all-reduce of the 128 integers
 * (exact in any order) gives every process the global sums.  Errors:
 * CM_ERR_INVALID (ids, NULL), CM_ERR_STATE (an image not resident). */
cm_status cm_index_col_sums_of(cm_index* ix, int32_t count, const int32_t* ids, uint64_t* d_sums, cm_stream stream);
/* Centring mean mu = sums / n_total from 128 exact column sums in device
 * memory (async, on stream).  The index keeps a copy of the sums. */
cm_status cm_index_set_mean_device(cm_index* ix, const uint64_t* d_sums, uint64_t n_total, cm_stream stream);
/* Keys, codes and buckets of every resident image under the current mean
 * (async; cm_index_rehash without recomputing the mean).  CM_ERR_STATE when
 * no mean is set or nothing is resident. */
cm_status cm_index_hash(cm_index* ix, cm_stream stream);
/* Releases resident images (Sec. 2.3.2 step (3)) and refreshes the device
 * tables on stream.  Every call on an index must use the same stream: work
 * already enqueued that reads an evicted image then precedes any later load
 * that reuses its arena space. */
cm_status cm_index_evict(cm_index* ix, int32_t count, const int32_t* ids, cm_stream stream);
/* Builds an index with every image resident: create + mean over all given
 * descriptors + load.  desc = all images' rows concatenated in image order. */
cm_status cm_build_index(const cm_params* p, int32_t n_images, const int32_t* n_desc, const uint8_t* desc,
                         int32_t mem, void* d_arena, uint64_t arena_bytes, cm_stream stream, cm_index** out);
/* Device pointers of a resident image's index data (diagnostics / tests):
 * keys u64[n] (byte t = key of table t), codes 4 x u32 [n], sorted codes
 * [L][n] (16 B), sorted local indices u16 [L][n], offsets u32 [L][2^m+1]. */
cm_status cm_index_image_view(const cm_index* ix, int32_t image, const void** keys, const void** codes,
                              const void** sorted_codes, const void** sorted_idx, const void** offsets);
void cm_index_destroy(cm_index* ix);
/* The same as cm_index_destroy (the name the problem statement's interface uses). */
void cm_free_index(cm_index* ix);

/* ---- matching (Sec. 2.3.1 steps (1)-(4), one launch per block) ------------ */
/* Arena bytes a plan of n_pairs pairs and `rows` query rows (the largest
 * query image having max_query_rows) takes from its index: the pair table and
 * work counter; for the BF16 / FP8 reranks and the CM_ALGO_TC scan the top-K
 * hand-over between the scan and the rerank launch (index and squared norm of
 * each kept candidate, 6 K bytes per row; FP8 adds its scale, 10 K); for
 * CM_ALGO_TC also per-table top-K lists of 160 concurrent pairs
 * (160 * max_query_rows * L * K * 4 bytes). */
cm_status cm_plan_bytes(const cm_params* p, int64_t n_pairs, int64_t rows, int32_t max_query_rows, uint64_t* bytes);
/* Plans a batch of pairs (host list): validates ids and residency and uploads
 * the work table into the index arena (async, on stream).  The plan keeps the
 * index's parameters of that moment (K, work-item size, thread mapping).  A plan can be run
 * many times and captured in a CUDA graph; it must not outlive the residency
 * of its images. */
cm_status cm_match_plan_create(cm_index* ix, const cm_pair* pairs, int64_t n_pairs, cm_stream stream,
                               cm_match_plan** out);
/* Total query rows of the plan (sum of N_i) — the size of each output array. */
int64_t cm_match_plan_rows(const cm_match_plan* pl);
/* One persistent fused launch over every pair of the plan (async): bucket
 * lookup, Hamming ranking, top-K, rerank and ratio test.  With the BF16 / FP8
 * reranks the rerank and ratio test run in a second, tensor-core launch that
 * reads the first one's top-K lists. */
cm_status cm_match_plan_run(cm_match_plan* pl, const cm_match_out* out, cm_stream stream);
/* cm_match_plan_run that also records scan_done (a cudaEvent_t created by the
 * caller, or NULL) on the stream right after the lookup / Hamming / top-K
 * launch, before the rerank launch of the BF16 / FP8 / TC-scan forms (after
 * the single launch of the fused forms).  Events around the call then time
 * the two launches apart.  The event stays owned by the caller; errors as for
 * cm_match_plan_run, plus CM_ERR_CUDA when the record fails. */
cm_status cm_match_plan_run_marked(cm_match_plan* pl, const cm_match_out* out, void* scan_done, cm_stream stream);
/* Compaction of the plan's decisions into per-pair match lists, the initial
 * matches handed to outlier removal (Algorithm 1).  From d_best_j (a
 * cm_match_plan_run output) writes, all device memory: d_counts [n_pairs]
 * matches per pair; d_offsets [n_pairs] exclusive prefix of the counts;
 * d_total (optional) the sum; d_matches (optional) the matches, entry
 * query << 16 | database index, pair k's at d_offsets[k] in query order.
 * Entries past `capacity` are dropped (counts stay exact).  Async. */
cm_status cm_match_plan_compact(cm_match_plan* pl, const int32_t* d_best_j, uint32_t* d_counts, uint64_t* d_offsets,
                                uint64_t* d_total, uint32_t* d_matches, uint64_t capacity, cm_stream stream);
/* Two-way (mutual) consistency of a run's decisions, a matching variant next
 * to the one-directional ratio test of Sec. 2.3.1 step (4): for each pair (I, J)
 * of the plan whose reverse (J, I) is also in the plan, a match q -> j is kept
 * only if (J, I) matched j back to q; pairs without a reverse keep their
 * decisions.  d_best_in: a cm_match_plan_run best_j output; d_best_out: a
 * distinct device array of the same rows.  Async. */
cm_status cm_match_plan_mutual(cm_match_plan* pl, const int32_t* d_best_in, int32_t* d_best_out, cm_stream stream);
/* Device workspace of cm_match_plan_sao for this plan. */
cm_status cm_match_plan_sao_bytes(const cm_match_plan* pl, uint64_t* bytes);
/* The SAO local constraint (see cm_sao_filter: same neighbours, orders,
 * scores and decisions, bit for bit) on the GPU for every pair of the plan:
 * each pair's initial matches are the queries with d_best_in >= 0, in query
 * order; a match whose score exceeds max_score gets -1 in d_best_out, so the
 * compaction that follows hands only kept matches to verification.
 *  - d_best_in: a cm_match_plan_run best_j; d_best_out may be the same array.
 *  - d_kp: device float [rows][2] keypoints of all images concatenated;
 *    d_kp_off: device int64 [n_images + 1] first row of each image there.
 *  - k_nn: 1..16; max_score >= 0.
 *  - d_score (optional): device float per plan row, the match's score (0 for
 *    rows without a match).
 *  - d_work / work_bytes: cm_match_plan_sao_bytes, 256-byte aligned.
 * Asynchronous on `stream`.  Errors: CM_ERR_INVALID, CM_ERR_STATE (index
 * destroyed), CM_ERR_BUDGET (workspace), CM_ERR_CUDA. */
cm_status cm_match_plan_sao(cm_match_plan* pl, const int32_t* d_best_in, int32_t* d_best_out, const float* d_kp,
                            const int64_t* d_kp_off, int32_t k_nn, float max_score, float* d_score, void* d_work,
                            uint64_t work_bytes, cm_stream stream);
void cm_match_plan_destroy(cm_match_plan* pl);
/* Device workspace (bytes) cm_match_pairs needs for this pair list: the pair
 * table, the work counter and, for the BF16 / FP8 reranks, the top-K
 * hand-over (as cm_plan_bytes).  Host only; the images need not be resident
 * yet.  CM_ERR_INVALID for an image id out of range. */
cm_status cm_match_pairs_workspace_bytes(const cm_index* ix, const cm_pair* pairs, int64_t n_pairs, uint64_t* bytes);
/* Device workspace (bytes) that matching block row `block` of schedule s with
 * cm_match_pairs takes (the row's pairs as the schedule holds them; the
 * schedule keeps a copy of the pair list it was made from), or the largest
 * over all rows when block = -1.  Host only.  Errors: CM_ERR_INVALID (block
 * out of range, a pair naming an image the index does not have). */
cm_status cm_index_workspace_bytes(const cm_index* ix, const cm_schedule* s, int32_t block, uint64_t* bytes);
/* Matches a batch of pairs of resident images (Sec. 2.3.1 steps (1)-(4) for
 * each query of image i against image j) in one fused launch (two for the
 * BF16 / FP8 reranks), without taking anything from the index arena:
 *  - pairs: host list; every image must be resident (CM_ERR_STATE otherwise).
 *  - d_workspace / ws_bytes: caller-owned device memory, 256-byte aligned, at
 *    least cm_match_pairs_workspace_bytes (CM_ERR_BUDGET otherwise).  It must
 *    not be reused until the stream has run past this call.
 *  - d_best_j (required when any query exists), d_d1sq, d_d2sq (optional):
 *    caller-owned device outputs, one entry per query row, pair k's rows
 *    starting at the sum of N_i over the pairs before it (as cm_match_out).
 * Asynchronous on `stream`: the call returns once the work is enqueued; the
 * inputs must stay valid and resident until the stream is synchronised.
 * Errors: CM_ERR_INVALID (ids, i == j, NULL, misaligned workspace),
 * CM_ERR_STATE, CM_ERR_BUDGET, CM_ERR_CUDA. */
cm_status cm_match_pairs(cm_index* ix, const cm_pair* pairs, int64_t n_pairs, void* d_workspace, uint64_t ws_bytes,
                         int32_t* d_best_j, uint32_t* d_d1sq, uint32_t* d_d2sq, cm_stream stream);

/* ---- captured block sequence (CUDA graph) -------------------------------- */
/* Compaction outputs of one plan inside a sequence (see cm_match_plan_compact);
 * counts == NULL means no compaction for that plan. */
typedef struct cm_compact_out {
    uint32_t* counts;    /* device [n_pairs] */
    uint64_t* offsets;   /* device [n_pairs] */
    uint64_t* total;     /* device [1], optional */
    uint32_t* matches;   /* device [capacity], optional */
    uint64_t capacity;
} cm_compact_out;
/* Captures, without running it, the device work of a block sequence whose
 * images are resident as one CUDA graph (stream capture on `stream`, which
 * must not be the legacy default stream): if rehash != 0 a cm_index_rehash
 * (centring statistics, keys, codes, buckets: Sec. 2.3.1 steps (1)-(2)), then
 * for each plan k in order its fused match launch into outs[k] and, when
 * compacts != NULL and compacts[k].counts != NULL, its compaction.  Buffers
 * named in outs / compacts are baked into the graph and must outlive it.
 * Errors: CM_ERR_INVALID (arguments, default stream), CM_ERR_STATE (a plan of
 * another index or detached), CM_ERR_CUDA (capture or instantiation failed;
 * the stream is left out of capture mode). */
cm_status cm_sequence_create(cm_index* ix, int32_t rehash, int32_t n_plans, cm_match_plan* const* plans,
                             const cm_match_out* outs, const cm_compact_out* compacts, cm_stream stream,
                             cm_sequence** out);
/* Replays the captured graph on stream (async; one graph launch).
 * CM_ERR_STATE when the index changed since capture (an image loaded or
 * evicted, a plan destroyed) or was destroyed: the graph's tables would be stale. */
cm_status cm_sequence_launch(cm_sequence* q, cm_stream stream);
/* Kernel nodes of the captured graph (launch accounting). */
int32_t cm_sequence_kernels(const cm_sequence* q);
void cm_sequence_destroy(cm_sequence* q);

/* ---- block-row pipeline (Sec. 2.3.2, Algorithm 1) ------------------------ */
/* Geometric verification callback.  Called on a library worker thread for
 * each pair of a block row whose matches have reached host memory, while the
 * GPU already works on the following rows (the GPU/CPU overlap of Sec. 2.3.2).
 * pair_id indexes the caller's pair list; matches[k] = query << 16 | database
 * index, in query order, valid during the call only.  Several workers call it
 * at once for different pairs: it must be thread-safe.  A non-zero return
 * stops the pipeline (cm_run_schedule returns CM_ERR_STATE). */
typedef int32_t (*cm_verify_fn)(void* user, int32_t row, int64_t pair_id, const cm_pair* pair, int64_t n_matches,
                                const uint32_t* matches);

typedef struct cm_pipeline_stats {
    int32_t rows;            /* block rows run */
    int32_t workers;         /* verification threads */
    int64_t pairs;           /* pairs matched */
    int64_t queries;         /* query rows matched (sum of N_i over pairs) */
    int64_t matches;         /* initial matches handed to verification */
    int64_t kernels;         /* kernel launches enqueued */
    uint64_t h2d_bytes;      /* descriptor bytes copied host to device */
    uint64_t d2h_bytes;      /* result bytes device to host: per row the offsets and the match lists */
    double wall_ms;          /* host wall time of the whole call */
    double gpu_ms;           /* sum over rows of the device time from the row's first copy to its last write */
    double verify_ms;        /* time spent inside the callback, summed over workers */
    double stall_ms;         /* host time spent waiting for a result buffer still held by verification */
    double tail_ms;          /* wall time after the last row's device work completed */
    int64_t prefetched_rows; /* rows whose new images were copied during the previous row */
} cm_pipeline_stats;

/* Arena bytes for an index that runs schedule s (made from pairs[n_pairs])
 * with cm_run_schedule: the fixed tables, the largest set of images resident
 * at once (a row's loads count before the row, its frees after it), a margin
 * for fragmentation of the arena's first-fit placement (1/8 of that set plus
 * its largest image), and the largest row's plan (cm_plan_bytes). */
cm_status cm_schedule_arena_bytes(const cm_schedule* s, const cm_params* p, int32_t n_images, const int32_t* n_desc,
                                  const cm_pair* pairs, int64_t n_pairs, uint64_t* bytes);
/* Device workspace of cm_run_schedule for this schedule (bytes). */
cm_status cm_pipeline_workspace_bytes(const cm_index* ix, const cm_schedule* s, const cm_pair* pairs, int64_t n_pairs,
                                      uint64_t* bytes);
/* Runs a schedule row by row (Algorithm 1): for row r, on `stream`, make the
 * row's new images resident from host memory (H2D, hashing, buckets), match
 * all its pairs in one fused launch, compact the decisions into per-pair match
 * lists written straight into mapped pinned host memory, then release the
 * row's freed images; worker threads verify row r while the GPU runs rows
 * r+1, r+2 (two result buffers).  Returns when every row is verified.
 *  - ix: an index whose centring mean is set (cm_index_set_mean) and on which
 *    no image of the schedule is resident; images still resident at the end
 *    are released.
 *  - s / pairs / n_pairs: a schedule from cm_schedule_blocks and the pair list
 *    it was made from.
 *  - desc_host[i]: host rows of image i (pinned memory gives async copies).
 *  - d_work / work_bytes: device workspace, at least cm_pipeline_workspace_bytes.
 *  - verify (may be NULL: matches are only counted), user: the callback.
 *  - n_workers: verification threads, 1..256.
 *  - stats (optional): filled on return.
 * Blocks the calling thread.  Errors: those of the calls it makes,
 * CM_ERR_STATE if a callback stops the pipeline, CM_ERR_TIMEOUT if a bounded
 * device wait gave up. */
cm_status cm_run_schedule(cm_index* ix, const cm_schedule* s, const cm_pair* pairs, int64_t n_pairs,
                          const uint8_t* const* desc_host, void* d_work, uint64_t work_bytes, cm_verify_fn verify,
                          void* user, int32_t n_workers, cm_stream stream, cm_pipeline_stats* stats);

/* Options of cm_run_schedule_ex (all zero: as cm_run_schedule).  sao_k > 0 runs the SAO local constraint
 * on the GPU for every row, right after the match launch
 * (cm_match_plan_sao), so verification receives only the kept matches;
 * d_kp / d_kp_off are as in cm_match_plan_sao and must cover every image. */
typedef struct cm_pipeline_opts {
    int32_t sao_k;             /* 0: off; 1..16 */
    float sao_max_score;
    const float* d_kp;         /* device float [rows][2], all images concatenated */
    const int64_t* d_kp_off;   /* device int64 [n_images + 1] */
    int32_t centre;            /* 1: the run computes the centring mean itself from desc_host (exact column
                                  sums on the GPU): the first row's images are copied into their slots and
                                  summed there, every other image's rows pass once through a staging block
                                  of the workspace; the index needs no mean beforehand */
} cm_pipeline_opts;
/* cm_pipeline_workspace_bytes for a run with these options (NULL: none). */
cm_status cm_pipeline_workspace_bytes_ex(const cm_index* ix, const cm_schedule* s, const cm_pair* pairs,
                                         int64_t n_pairs, const cm_pipeline_opts* opts, uint64_t* bytes);
/* cm_run_schedule with options (NULL: the same as cm_run_schedule). */
cm_status cm_run_schedule_ex(cm_index* ix, const cm_schedule* s, const cm_pair* pairs, int64_t n_pairs,
                             const uint8_t* const* desc_host, void* d_work, uint64_t work_bytes, cm_verify_fn verify,
                             void* user, int32_t n_workers, const cm_pipeline_opts* opts, cm_stream stream,
                             cm_pipeline_stats* stats);

/* RANSAC fit of a 2-D affine map u = A [x y 1]^T from the query image's
 * keypoints to the database image's over one pair's matches (the global
 * geometric constraint of Sec. 2.3.2; an affine map is exact for the planar
 * scenes seen by near-nadir views).  kp_i / kp_j: host float [n][2] pixel
 * positions of the two images' descriptors; matches: as in cm_verify_fn.
 * Minimal samples of 3 matches drawn by splitmix64 from seed; at most
 * max_iters samples, fewer once a sample with the best inlier share makes a
 * better one unlikely (p = 0.999); a match is an inlier when its residual is
 * <= thresh_px; the best model is refit by least squares on its inliers and
 * the inliers recounted.  Outputs (any may be NULL): A[6] row-major 2x3,
 * inlier_mask[n_matches] (0/1), *n_inliers (0 when fewer than 3 matches or no
 * non-degenerate sample).  Host only, thread-safe. */
cm_status cm_verify_affine(const float* kp_i, const float* kp_j, int64_t n_matches, const uint32_t* matches,
                           float thresh_px, int32_t max_iters, uint64_t seed, float* A, uint8_t* inlier_mask,
                           int64_t* n_inliers);
/* Spatial-angular-order local geometric constraint (Sec. 2.3.3, Fig. 4): a
 * dissimilarity score per initial match of one pair, computed before RANSAC
 * so that the global fit sees fewer outliers.  For match m = (p_m, q_m): its
 * k_nn nearest other matches around p_m in the query image and, found
 * independently, around q_m in the database image (squared Euclidean
 * distance, ties by match index; the Euclidean k-NN set that the Delaunay
 * graph of the matched keypoints yields); each list in angular order around
 * its centre (from the horizontal axis, [0, 2*pi), a zero vector at angle 0,
 * ties by match index); Score = d_ced / N with d_ced the cyclic unit-cost
 * edit distance of the two label sequences and N = min(k_nn, n_matches - 1)
 * (Score 0 when N = 0), in float.  A match is kept when Score <= max_score.
 *  - kp_i / kp_j: host float [n][2] keypoints of the query / database image.
 *  - matches: n_matches entries query << 16 | database index (as in cm_verify_fn).
 *  - k_nn: 1..32 (8 is the usual choice); max_score >= 0 (0.875 keeps a match
 *    unless its two orders need one edit per neighbour at k_nn = 8).
 *  - score[n_matches], keep[n_matches] (0/1), *n_kept: outputs, any may be NULL.
 * Host only, thread-safe, deterministic.  CM_ERR_INVALID on a bad argument. */
cm_status cm_sao_filter(const float* kp_i, const float* kp_j, int64_t n_matches, const uint32_t* matches,
                        int32_t k_nn, float max_score, float* score, uint8_t* keep, int64_t* n_kept);

/* A ready-made cm_verify_fn running cm_verify_affine; user = cm_affine_verifier*.
 * With sao_k > 0 the pair's matches first pass cm_sao_filter(sao_k,
 * sao_max_score) and RANSAC fits the kept ones (the local-then-global
 * outlier removal of Sec. 2.3.3). */
typedef struct cm_affine_verifier {
    const float* const* keypoints;  /* per image: host float [n][2] */
    float thresh_px;
    int32_t max_iters;
    uint64_t seed;                  /* pair k uses seed ^ k */
    int64_t* inliers;               /* [n_pairs of the caller's list]: inlier count written per pair */
    int32_t sao_k;                  /* 0: no local constraint; 1..32: its k */
    float sao_max_score;
    int64_t* sao_kept;              /* optional [n_pairs]: matches kept by the local constraint per pair */
} cm_affine_verifier;
int32_t cm_affine_verify_cb(void* user, int32_t row, int64_t pair_id, const cm_pair* pair, int64_t n_matches,
                            const uint32_t* matches);

/* ---- VLAD image encoding (Sec. 2.1, the retrieval front end) ------------- */
/* Device workspace of cm_vlad_encode for n_images images of n_rows rows in all. */
cm_status cm_vlad_workspace_bytes(int32_t n_images, int64_t n_rows, uint64_t* bytes);
/* VLAD vector of every image, against a codebook on the descriptors' integer
 * grid (e.g. k-means centroids rounded to integers; the paper trains the
 * codebook with Lloyd's k-means, outside this call):
 *  1. each descriptor goes to its nearest codeword by exact squared Euclidean
 *     distance (ties to the smaller codeword index) - a 128 x C x 128 BF16
 *     tensor-core contraction per tile of 128 descriptors, exact on integers;
 *  2. per codeword c, r_c = sum over the image's descriptors assigned to c of
 *     (x - c), exact integers, concatenated codeword-major (C x 128);
 *  3. signed square root of every component, then L2 normalisation of the
 *     vector (FP64 sum of squares); an all-zero vector stays zero.
 *  - desc: device uint8 [n_rows][128], all images' rows concatenated.
 *  - img_off: host int64 [n_images + 1], img_off[0] = 0, ascending; image i
 *    owns rows img_off[i] .. img_off[i+1]-1 (an empty image gives zeros).
 *  - codebook: device uint8 [n_codewords][128], 1 <= n_codewords <= 256.
 *  - d_work / work_bytes: device workspace of cm_vlad_workspace_bytes, 256-byte aligned.
 *  - assign (optional): device uint16 [n_rows], the codeword of each row.
 *  - vlad: device float [n_images][n_codewords * 128].
 * Asynchronous on `stream`; cm_workspace_status(d_work, stream) waits for it and
 * reports CM_ERR_TIMEOUT if a bounded device wait gave up.  Errors:
 * CM_ERR_INVALID (bad argument), CM_ERR_BUDGET (workspace too small), CM_ERR_CUDA. */
cm_status cm_vlad_encode(const uint8_t* desc, const int64_t* img_off, int32_t n_images, const uint8_t* codebook,
                         int32_t n_codewords, void* d_work, uint64_t work_bytes, uint16_t* assign, float* vlad,
                         cm_stream stream);
/* Synchronises `stream` and reads the device status of the last call that used
 * the workspace d_work (cm_vlad_encode, cm_nn_pairs): CM_ERR_TIMEOUT if a
 * bounded device wait gave up, CM_ERR_STATE if a device-side bounds check
 * failed, else CM_OK. */
cm_status cm_workspace_status(const void* d_work, cm_stream stream);

/* Diagnostic: runs the bounded-wait path every kernel uses, on the device,
 * without a fault.  One CTA holds tensor memory, waits on an mbarrier that
 * nothing completes, gives up after `polls` (1..2^24) polls, records the
 * timeout and frees its tensor memory.  Returns CM_ERR_TIMEOUT (the status a
 * launch whose wait ran out reports); the context stays usable.  Blocks until
 * done.  CM_ERR_INVALID for polls out of range. */
cm_status cm_selftest_wait(int32_t polls, cm_stream stream);

/* Diagnostic: measured throughput of the integer operations the Hamming scan
 * is made of, per clock per SM (the ALU roofline of the lookup kernel).  One
 * CTA of 1024 threads per SM runs `iters` steps of 8 independent chains per
 * thread and times them with the SM's clock64 counter (median over the
 * CTAs).  kind: CM_PROBE_POPC (population counts), CM_PROBE_LOP3 (3-input
 * logic ops), CM_PROBE_HAM4 (128-bit Hamming distances as 4 XOR + 4 POPC +
 * adds), CM_PROBE_HAM3 (the same distances through a carry-save sum with 3
 * POPC).  d_work: device scratch of >= SMs * (8 + 4096) bytes.  Blocks until
 * done.  Errors: CM_ERR_INVALID, CM_ERR_BUDGET, CM_ERR_CUDA. */
enum { CM_PROBE_POPC = 0, CM_PROBE_LOP3 = 1, CM_PROBE_HAM4 = 2, CM_PROBE_HAM3 = 3 };
cm_status cm_probe_int(int32_t kind, int32_t iters, void* d_work, uint64_t work_bytes, cm_stream stream,
                       double* per_clock_per_sm);

/* ---- exhaustive nearest neighbours (quality ceiling) --------------------- */
/* Device workspace of cm_nn_pairs for these images and pairs (it holds a BF16
 * operand copy of every database image the pairs name: 72 KB per 256 rows,
 * -2y and the base-256 digits of |y|^2 in the tensor-core tile layout). */
cm_status cm_nn_workspace_bytes(const int64_t* img_off, int32_t n_images, const cm_pair* pairs, int64_t n_pairs,
                                uint64_t* bytes);
/* Exhaustive nearest neighbours with the exact ratio test for each pair: for
 * every query x of image i, q1 and q2 = the two smallest (d^2, j) over ALL
 * rows y of image j (d^2 exact squared Euclidean distance on the uint8 rows,
 * ties to the smaller j), and best_j = j1 when den^2 d1^2 < num^2 d2^2 (no
 * match with fewer than 2 rows in j).  These are the matches cascade hashing
 * gives with every database point a candidate (Sec. 2.3.1 with K = N_J): the
 * ceiling its recall is measured against.  d^2 = |x|^2 + t with
 * t = |y|^2 - 2 x.y from one BF16 tensor-core product (|y|^2 enters as an
 * extra K block of digits), exact on integers.
 *  - desc: device uint8 [rows][128], all images concatenated; img_off: host
 *    int64 [n_images + 1], img_off[0] = 0, ascending, <= 65535 rows per image.
 *  - pairs: host, n_pairs entries; output rows: pair k owns rows
 *    row_off[k] .. row_off[k] + n_i - 1, row_off the prefix sum of the query
 *    counts (the layout of a match plan).
 *  - best_j (required), d1sq, d2sq (optional): device outputs per row;
 *    0xFFFFFFFF where q1 / q2 do not exist.
 *  - d_work / work_bytes: cm_nn_workspace_bytes, 256-byte aligned.
 * Asynchronous on `stream`; cm_workspace_status reports device-side failures.
 * Errors: CM_ERR_INVALID, CM_ERR_BUDGET (workspace), CM_ERR_CUDA. */
cm_status cm_nn_pairs(const uint8_t* desc, const int64_t* img_off, int32_t n_images, const cm_pair* pairs,
                      int64_t n_pairs, int32_t ratio_num, int32_t ratio_den, void* d_work, uint64_t work_bytes,
                      int32_t* best_j, uint32_t* d1sq, uint32_t* d2sq, cm_stream stream);

/* ---- autotuning of the match launch -------------------------------------- */
typedef struct cm_tune_result {
    int32_t query_tile;  /* chosen queries per work item */
    int32_t algo;        /* chosen cm_algo (TILE or WARP) */
    int32_t K;           /* chosen K (the index's K unless K candidates were given) */
    int32_t trials;      /* configurations timed */
    float ms;            /* mean time of one match launch over the sample with the choice */
    float agreement;     /* share of the sample's queries whose decision equals the largest K's */
} cm_tune_result;
/* Times the match launch on a sample of resident pairs under each work-item
 * size (256 .. 4096 queries, where the tile kernel's shared memory fits) and
 * thread mapping (tile; warp-per-query for the CUDA-core reranks), checks that
 * all of them decide every query identically (CM_ERR_STATE otherwise), and
 * keeps the fastest.  With n_K > 0 it then times each K of K_candidates and
 * keeps the fastest K whose decisions agree with the largest candidate's on at
 * least min_agreement of the sample's queries (K changes the method's result:
 * Sec. 2.3.1 step (3)).  The choice is written to *out and becomes the index's
 * parameters for plans made afterwards; plans that exist keep theirs.
 * Synchronous (waits for stream); scratch comes from the index arena. */
cm_status cm_autotune(cm_index* ix, const cm_pair* pairs, int64_t n_pairs, const int32_t* K_candidates, int32_t n_K,
                      float min_agreement, cm_stream stream, cm_tune_result* out);

/* ---- matching without any device allocation ------------------------------ */
/* The paper has no counterpart: this entry point serves callers that may not
 * allocate GPU memory (code running inside another framework's memory budget,
 * plug-ins of a host process that owns the device, real-time paths where an
 * allocation could block or fail).  It matches one pair, image i (queries)
 * against image j: hashing of both images into bucket keys and binary codes,
 * their bucket tables, the Hamming top-K lookup, the exact rerank and the
 * ratio test, all on the GPU.  Its only scratch is a file-scope device array
 * of 5 MiB that every GPU which loads this library holds until the process
 * exits; the call allocates nothing, on the device or through a library.
 *  - d_desc_i / d_desc_j: device uint8 [n][128] descriptor rows, at most 8,192
 *    per image (CM_ERR_BUDGET beyond, with a message); read in place.  An
 *    empty database image (n_j = 0) gives no matches.
 *  - col_sums_host / n_total: the exact column sums and row count that define
 *    the centring mean (e.g. from cm_index_col_sums), host memory, read
 *    before the call returns.
 *  - d_best_j (required), d_d1sq, d_d2sq (optional): device outputs of n_i
 *    rows, as in cm_match_out.
 *  - p->rerank: CM_RERANK_FP32 or CM_RERANK_INT; p->projection: CM_PROJ_FFMA
 *    only (the tensor-core projection needs a status word the call could not
 *    report); p->algo: CM_ALGO_TILE or CM_ALGO_WARP as asked, CM_ALGO_AUTO the
 *    tile mapping when its shared memory fits, else the warp mapping;
 *    CM_ALGO_TC is rejected.  Other values give CM_ERR_INVALID.
 * Async on stream: the per-call tables reach the array through set-up
 * kernels that take them as kernel arguments, so the host does not wait.
 * The first call on a device (and the first after a new CUDA context, e.g.
 * after cudaDeviceReset) looks up the array's device address with
 * cudaGetSymbolAddress; make that first call before any stream capture.
 * All calls share the one array and it keeps the last call's contents (the
 * call clears what must start at zero), so calls that overlap on the GPU
 * (other streams or host threads) race: serialise them. */
cm_status cm_match_pair_noalloc(const cm_params* p, const uint8_t* d_desc_i, int32_t n_i, const uint8_t* d_desc_j,
                                int32_t n_j, const uint64_t* col_sums_host, uint64_t n_total, int32_t* d_best_j,
                                uint32_t* d_d1sq, uint32_t* d_d2sq, cm_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* CASHMATCH_H */
