// Internal types shared by the host library and the kernels (not part of the ABI).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/cashmatch.h"

namespace cm {

// The FP32 band of the ratio test for t_r = num / den (cm_ratio.cuh): a query
// passes when d1 < lo d2 and fails when d1 > hi d2, with lo = (t_r - 1e-3)^2
// (-1 when t_r <= 1e-3) and hi = (t_r + 1e-3)^2.  Computed once per launch on
// the host, so the kernels read both from their parameters.
struct RatioBand {
    float lo, hi;
};
inline RatioBand ratio_band(int num, int den) {
    const float tr = (float)num / (float)den;
    return {tr > 1e-3f ? (tr - 1e-3f) * (tr - 1e-3f) : -1.f, (tr + 1e-3f) * (tr + 1e-3f)};
}

constexpr int kDim = 128;          // descriptor length (SIFT)
constexpr int kMaxL = 8;
constexpr int kMaxM = 8;
constexpr int kMaxP = 192;         // L*m + 128 <= 192
constexpr int kHashTile = 64;      // descriptors per hash tile
constexpr int kHashThreads = 256;
constexpr int kMatchThreads = 1024;
constexpr int kDefaultQueryTile = 2048;  // queries per work item
constexpr size_t kMatchSmemLimit = 214 * 1024;  // dynamic shared memory of the tile kernel (static extra)
constexpr int kWqThreads = 256;          // warp-per-query matcher: 8 warps per CTA
constexpr int kBmThreads = 512;          // bucket-major matcher: 16 warps per CTA, 2 CTAs per SM
constexpr int kWqBlocksPerSM = 3;
constexpr uint32_t kEmpty = 0xFFFFFFFFu;

// One resident image, as the kernels see it.  All pointers are into the arena
// (desc may point at caller memory when loaded in place).
struct DevImage {
    const uint8_t* desc;   // [n][128]
    uint64_t* key;         // [n]   byte t = bucket key of table t
    uint4* code;           // [n]   128-bit fine code
    uint4* scode;          // [L][n] codes sorted by bucket, per table
    uint16_t* sidx;        // [L][n] local indices sorted by bucket (ascending inside a bucket)
    uint32_t* off;         // [L][B+1] bucket offsets
    uint32_t* hist;        // [L][B] bucket counts (zero between hashing passes)
    uint8_t* brank;        // [L][256] rank of each bucket by run length (ties by bucket id)
    uint32_t* norm;        // [n]   squared norm of the raw descriptor (tensor-core forms)
    void* xq;              // [n] rows of the tensor-core rerank copy: BF16 [128] (256 B) or E4M3 [128] (128 B)
    float* xscale;         // [n]   FP8 row scale (max / 448)
    int32_t n;
    int32_t pad;
};

// One pair of a match plan.
struct DevPair {
    int32_t i, j;          // query image, database image
    int64_t row_off;       // first output row of this pair
    int32_t item0;         // first work item of this pair
    int32_t nitems;        // work items (query tiles) of this pair
    int32_t rev;           // index of the pair (j, i) in the same plan, -1 if absent
    int32_t ni;            // rows of image i (the pair's queries)
};

struct HashLaunch {
    const DevImage* imgs;
    const int32_t* batch;      // image ids of the batch
    const int32_t* tile_pref;  // [n_batch+1] prefix of 64-row tiles per image
    const int32_t* tile_pref128;  // [n_batch+1] prefix of 128-row tiles per image (tensor-core kernel)
    int32_t n_batch;
    int32_t n_tiles;
    int32_t n_tiles128;
    const float* bias;         // [P_pad] mu . W (tensor-core kernel)
    int* err;                  // set to 1 when a bounded device wait gives up
    const float* W;            // [128][P_pad]
    const float* mu;           // [128]
    int32_t L, m, P_pad;
    int32_t rerank;
};

struct MatchLaunch {
    const DevImage* imgs;
    const DevPair* pairs;
    int32_t n_pairs;
    int32_t n_items;
    int32_t S;                 // queries per work item
    int32_t L, m, K;
    int32_t ratio_num, ratio_den;
    float ratio_lo, ratio_hi;  // FP32 band of the ratio test (ratio_band)
    int32_t rerank;
    int32_t algo;              // CM_ALGO_TILE, CM_ALGO_WARP, CM_ALGO_BUCKET or CM_ALGO_TC
    unsigned* counter;         // work counter (zeroed before each launch)
    int* err;                  // set to 1 when a bounded device wait gives up
    // tensor-core forms, scan -> rerank hand-over, [rows][K] in rank order:
    uint16_t* topk16;          // database indices (0xFFFF empty)
    uint32_t* hnorm;           // their squared norms
    float* hscale;             // their FP8 row scales (FP8 form)
    uint32_t* lists;           // tensor-core Hamming scan: per-CTA [max_ni][L][K] per-table top-K keys
    int32_t max_ni;            // largest query image of the launch
    uint32_t* klists;          // bucket-major matcher: [rows][K] running top-K keys (Hamming << 16 | index)
    const int32_t* order;      // bucket-major matcher: the pairs in the order its CTAs take them
    cm_match_out out;
};

// Kernel launchers (cm_kernels.cu).  Return cudaGetLastError().
cudaError_t launch_colsum_rows(const uint8_t* desc, uint64_t n_rows, unsigned long long* sums, cudaStream_t s);
cudaError_t launch_colsum_images(const HashLaunch& h, unsigned long long* sums, cudaStream_t s);
cudaError_t launch_mean(const unsigned long long* sums, const unsigned long long* n_total_dev, uint64_t n_total,
                        float* mu, cudaStream_t s);
cudaError_t launch_count_rows(const HashLaunch& h, unsigned long long* n_total, cudaStream_t s);
cudaError_t launch_hash(const HashLaunch& h, int sm_count, cudaStream_t s);       // CUDA-core FP32 projection
cudaError_t launch_hash_tc(const HashLaunch& h, int sm_count, cudaStream_t s);    // tensor-core projection (cm_hash_tc.cu)
cudaError_t launch_bias(const float* W, const float* mu, int P_pad, float* bias, cudaStream_t s);
cudaError_t launch_bucket(const HashLaunch& h, cudaStream_t s);
cudaError_t launch_match(const MatchLaunch& m, int sm_count, cudaStream_t s);      // lane per query (cm_match.cu)
cudaError_t launch_match_wq(const MatchLaunch& m, int sm_count, cudaStream_t s);   // warp per query (cm_match_wq.cu)
size_t match_smem_bytes(int S, int K);
cudaError_t launch_match_bm(const MatchLaunch& m, int sm_count, cudaStream_t s);   // bucket-major (cm_match_bm.cu)
size_t match_bm_smem_bytes();
cudaError_t launch_compact(const DevPair* pairs, int n_pairs, const DevImage* imgs, const int32_t* best,
                           uint32_t* counts, unsigned long long* offsets, unsigned long long* total, uint32_t* out,
                           unsigned long long capacity, cudaStream_t s);                 // cm_compact.cu
cudaError_t launch_mutual(const DevPair* pairs, int n_pairs, const DevImage* imgs, const int32_t* best_in,
                          int32_t* best_out, cudaStream_t s);                                // cm_compact.cu
int hash_npg(int P_pad);
// Tensor-core rerank (cm_rerank_tc.cu): row copies written after hashing, and
// the rerank of a plan's top-K lists.
cudaError_t launch_xcopy(const HashLaunch& h, cudaStream_t s);
cudaError_t launch_rerank_tc(const MatchLaunch& m, int sm_count, cudaStream_t s);
// Tensor-core Hamming scan (cm_scan_tc.cu) and the CUDA-core rerank of a hand-over (cm_rerank_cc.cu).
cudaError_t launch_scan_tc(const MatchLaunch& m, int grid, cudaStream_t s);
cudaError_t launch_rerank_cc(const MatchLaunch& m, int sm_count, cudaStream_t s);

}  // namespace cm
