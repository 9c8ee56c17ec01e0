// Host-side internals shared by the C-ABI translation units (not part of the ABI).
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <set>
#include <vector>

#include "cm_internal.h"

namespace cm {

// Records a failure for cm_last_error() and returns st (cm_api.cpp).
cm_status host_fail(cm_status st, const char* fmt, ...);

#define CM_CUDA(call)                                                                                    \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess)                                                                           \
            return ::cm::host_fail(CM_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

inline static int proj_count(const cm_params* p) { return p->L * p->m + p->n_bits; }
inline static int proj_pad(const cm_params* p) { return (proj_count(p) + 15) / 16 * 16; }

// Default work-item size: kDefaultQueryTile, shrunk until the tile kernel's
// shared memory (top-K lists and hit buffers of the tile) fits.
inline int query_tile(const cm_params* p) {
    if (p->query_tile) return p->query_tile;
    int S = kDefaultQueryTile;
    while (S > 64 && match_smem_bytes(S, p->K) > kMatchSmemLimit) S -= 64;
    return S;
}

constexpr uint64_t kAlign = 256;
inline uint64_t align_up(uint64_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct SlotLayout {
    uint64_t desc, key, code, scode, sidx, off, hist, brank, norm, xq, xscale, total;
};

inline bool tc_rerank(const cm_params* p) { return p->rerank == CM_RERANK_BF16 || p->rerank == CM_RERANK_FP8; }

inline SlotLayout slot_layout(const cm_params* p, int64_t n, bool inplace) {
    const int64_t B = 1ll << p->m;
    SlotLayout s{};
    uint64_t o = 0;
    auto take = [&](uint64_t bytes) { uint64_t at = o; o = align_up(o + bytes); return at; };
    s.desc = inplace ? 0 : take((uint64_t)n * kDim);
    s.key = take((uint64_t)n * 8);
    s.code = take((uint64_t)n * 16);
    s.scode = take((uint64_t)p->L * n * 16);
    s.sidx = take((uint64_t)p->L * n * 2);
    s.off = take((uint64_t)p->L * (B + 1) * 4);
    s.hist = take((uint64_t)p->L * B * 4);
    s.brank = take((uint64_t)p->L * 256);
    s.norm = take((uint64_t)n * 4);
    s.xq = 0;
    s.xscale = 0;
    if (p->rerank == CM_RERANK_BF16) s.xq = take((uint64_t)n * 256);   // rows start on 256-byte boundaries
    if (p->rerank == CM_RERANK_FP8) {
        s.xq = take((uint64_t)n * 128);
        s.xscale = take((uint64_t)n * 4);
    }
    s.total = o;
    return s;
}

// Fixed tables at the start of the arena.
struct FixedLayout {
    uint64_t imgs, W, mu, sums, ntot, batch, tiles, rbatch, rtiles, tiles128, rtiles128, bias, err, total;
};

inline FixedLayout fixed_layout(const cm_params* p, int n_images) {
    FixedLayout f{};
    uint64_t o = 0;
    auto take = [&](uint64_t bytes) { uint64_t at = o; o = align_up(o + bytes); return at; };
    f.imgs = take((uint64_t)n_images * sizeof(DevImage));
    f.W = take((uint64_t)kDim * proj_pad(p) * 4);
    f.mu = take(kDim * 4);
    f.sums = take(kDim * 8);
    f.ntot = take(8);
    f.batch = take((uint64_t)n_images * 4);
    f.tiles = take((uint64_t)(n_images + 1) * 4);
    f.rbatch = take((uint64_t)n_images * 4);
    f.rtiles = take((uint64_t)(n_images + 1) * 4);
    f.tiles128 = take((uint64_t)(n_images + 1) * 4);
    f.rtiles128 = take((uint64_t)(n_images + 1) * 4);
    f.bias = take((uint64_t)kMaxP * 4);
    f.err = take(4);
    f.total = o;
    return f;
}

// First-fit allocator over [begin, end) of the arena (host bookkeeping only).
class ArenaAlloc {
   public:
    void init(uint64_t begin, uint64_t end) {
        free_.clear();
        if (end > begin) free_[begin] = end - begin;
    }
    bool alloc(uint64_t bytes, uint64_t* at) {
        bytes = align_up(bytes ? bytes : kAlign);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *at = it->first;
                const uint64_t rest = it->second - bytes, base = it->first + bytes;
                free_.erase(it);
                if (rest) free_[base] = rest;
                used_[*at] = bytes;
                return true;
            }
        }
        return false;
    }
    void release(uint64_t at) {
        auto u = used_.find(at);
        if (u == used_.end()) return;
        uint64_t base = at, size = u->second;
        used_.erase(u);
        auto next = free_.lower_bound(base);
        if (next != free_.end() && base + size == next->first) {
            size += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == base) {
                prev->second += size;
                return;
            }
        }
        free_[base] = size;
    }

   private:
    std::map<uint64_t, uint64_t> free_, used_;
};

// Pinned host buffers for table uploads; a buffer is reused once the copy that
// read it has completed on its stream.
class Staging {
   public:
    ~Staging() {
        for (auto& b : bufs_) {
            cudaEventDestroy(b.ev);
            cudaFreeHost(b.p);
        }
    }
    cudaError_t upload(void* dst, const void* src, size_t bytes, cudaStream_t s) {
        if (!bytes) return cudaSuccess;
        Buf* use = nullptr;
        for (auto& b : bufs_) {
            if (b.cap >= bytes && (!b.pending || cudaEventQuery(b.ev) == cudaSuccess)) {
                use = &b;
                break;
            }
        }
        if (!use) {
            Buf b{};
            b.cap = std::max<size_t>(bytes, 1 << 16);
            cudaError_t e = cudaHostAlloc(&b.p, b.cap, cudaHostAllocDefault);
            if (e != cudaSuccess) return e;
            e = cudaEventCreateWithFlags(&b.ev, cudaEventDisableTiming);
            if (e != cudaSuccess) return e;
            bufs_.push_back(b);
            use = &bufs_.back();
        }
        memcpy(use->p, src, bytes);
        cudaError_t e = cudaMemcpyAsync(dst, use->p, bytes, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return e;
        e = cudaEventRecord(use->ev, s);
        use->pending = true;
        return e;
    }

   private:
    struct Buf {
        void* p;
        size_t cap;
        cudaEvent_t ev;
        bool pending;
    };
    std::vector<Buf> bufs_;
};

}  // namespace cm

using namespace cm;

struct cm_match_plan;
struct cm_sequence;
void cm_sequence_detach(cm_sequence* q);   // the index is going away (cm_pipeline.cpp)

struct cm_index {
    cm_params p{};
    std::set<cm_match_plan*> plans;    // live plans (detached when the index is destroyed)
    std::set<cm_sequence*> seqs;       // live captured sequences (detached likewise)
    uint64_t generation = 0;           // bumped by load, evict and plan destruction
    int P = 0, P_pad = 0, B = 0, sms = 148;
    int n_images = 0;
    std::vector<int32_t> n_desc;
    uint8_t* arena = nullptr;
    uint64_t arena_bytes = 0;
    FixedLayout fx{};
    ArenaAlloc alloc;
    std::vector<DevImage> h_imgs;
    std::vector<uint64_t> slot_at;     // arena offset of each image's slot (valid if resident)
    std::vector<char> resident;
    std::vector<char> pending;         // slot placed and descriptors on their way, not yet published
    uint64_t plan_reserve_at = 0;      // arena block reserved by cm_run_schedule for its rows' plans
    uint64_t plan_reserve_bytes = 0;   // 0: none
    bool plan_reserve_busy = false;    // a live plan occupies it
    bool mean_set = false;
    bool sums_on_host = false;         // the mean came from cm_index_set_mean
    uint64_t host_sums[kDim] = {};
    uint64_t n_total = 0;              // rows behind the current mean
    Staging staging;
    // cm_run_schedule's two host result buffers (pinned; the match lists are
    // mapped), kept between calls: page-locking them costs more than a row
    struct PinnedResult {
        uint64_t* offsets = nullptr;
        size_t n_offsets = 0;
        uint32_t* matches = nullptr;
        uint32_t* d_matches = nullptr;
        size_t n_matches = 0;
    } pinned[2];

    ~cm_index() {
        for (auto& b : pinned) {
            if (b.offsets) cudaFreeHost(b.offsets);
            if (b.matches) cudaFreeHost(b.matches);
        }
    }

    template <class T>
    T* at(uint64_t off) const { return reinterpret_cast<T*>(arena + off); }

    HashLaunch hash_launch(bool resident_set, int n_batch, int n_tiles, int n_tiles128) const {
        HashLaunch h{};
        h.imgs = at<DevImage>(fx.imgs);
        h.batch = at<int32_t>(resident_set ? fx.rbatch : fx.batch);
        h.tile_pref = at<int32_t>(resident_set ? fx.rtiles : fx.tiles);
        h.tile_pref128 = at<int32_t>(resident_set ? fx.rtiles128 : fx.tiles128);
        h.n_batch = n_batch;
        h.n_tiles = n_tiles;
        h.n_tiles128 = n_tiles128;
        h.bias = at<float>(fx.bias);
        h.err = at<int>(fx.err);
        h.W = at<float>(fx.W);
        h.mu = at<float>(fx.mu);
        h.L = p.L;
        h.m = p.m;
        h.P_pad = P_pad;
        h.rerank = p.rerank;
        return h;
    }
};

// Early loading for the pipeline: index_prefetch places the slots of images
// (all or none; *placed = false when the arena has no room now) and copies
// their descriptors from host memory on copy_stream; index_publish later makes
// them resident and hashes them on the main stream, which must first wait for
// the copies; index_cancel_prefetch returns placed slots that were never
// published.
namespace cm {
cm_status index_prefetch(cm_index* ix, int32_t count, const int32_t* ids, const uint8_t* const* desc,
                         cudaStream_t copy_stream, bool* placed);
// centre_first: before hashing, add the batch's column sums to the index's
// sums and set the mean over all images from them (the pipeline's own
// centring pass, which summed every other image's host rows first).
cm_status index_publish(cm_index* ix, int32_t count, const int32_t* ids, cudaStream_t s, bool centre_first = false);
cm_status index_stream_sums(cm_index* ix, int32_t count, const int32_t* ids, const uint8_t* const* desc_host,
                            uint8_t* stage, uint64_t stage_bytes, cudaStream_t s, uint64_t* rows);
cm_status index_mean_from_sums(cm_index* ix, uint64_t n_total, cudaStream_t s);
void index_cancel_prefetch(cm_index* ix, int32_t count, const int32_t* ids);
// Device workspace of cm_match_plan_sao for a plan of n_pairs pairs and rows query rows.
uint64_t sao_work_bytes(int64_t n_pairs, int64_t rows);
// The pair list a schedule was made from (cm_sched.cpp); valid while the schedule lives.
const cm_pair* schedule_pairs(const cm_schedule* s, int64_t* n);
}  // namespace cm

// Arena bytes of a plan: its pair table, the work counter and:
//   - for the bucket-major matcher, the order in which its CTAs take the
//     pairs (largest n_i * n_j first) and every query row's running top-K
//     keys, [rows][K] u32;
//   - for the tensor-core reranks, the [rows][K] top-K hand-over from scan to
//     rerank (index u16, squared norm u32 and, for FP8, scale f32 of every
//     kept candidate);
//   - for the tensor-core Hamming scan, per-CTA scratch for per-table top-K
//     lists: [kMaxScanCtas][max query rows][L][K] u32.
constexpr int kMaxScanCtas = 160;   // >= the SM count; the scan's grid is capped to it
// AUTO takes the bucket-major matcher for plans with at least this many pairs
// (it runs one pair per CTA: two CTAs per SM on 148 SMs); smaller plans take
// the tile form, whose work items are tiles of queries.
constexpr int64_t kBucketMinPairs = 256;
struct HandOver {
    uint64_t order, idx, norm, scale, lists, klists, total;
};
inline bool needs_hand_over(const cm_params* p) { return tc_rerank(p) || p->algo == CM_ALGO_TC; }
// The matcher a plan's launch uses: the tensor-core scan, the warp-per-query
// form, the tile form, or the bucket-major form (AUTO: by the plan's size).
inline int resolved_algo(const cm_params* p, int64_t n_pairs) {
    if (p->algo == CM_ALGO_TC || p->algo == CM_ALGO_WARP || p->algo == CM_ALGO_TILE) return p->algo;
    if (p->algo == CM_ALGO_BUCKET) return CM_ALGO_BUCKET;
    return n_pairs >= kBucketMinPairs ? CM_ALGO_BUCKET : CM_ALGO_TILE;
}
inline HandOver hand_over(const cm_params* p, int64_t n_pairs, int64_t rows, int32_t max_ni) {
    HandOver h{};
    const uint64_t e = (uint64_t)rows * (uint64_t)p->K;
    const bool bucket = resolved_algo(p, n_pairs) == CM_ALGO_BUCKET;
    uint64_t o = 0;
    h.order = o;
    if (bucket) o += align_up((uint64_t)n_pairs * 4);
    if (needs_hand_over(p)) {
        h.idx = o;
        h.norm = h.idx + align_up(e * 2);
        h.scale = h.norm + align_up(e * 4);
        h.lists = h.scale + (p->rerank == CM_RERANK_FP8 ? align_up(e * 4) : 0);
        o = h.lists;
        if (p->algo == CM_ALGO_TC)
            o += align_up((uint64_t)kMaxScanCtas * (uint64_t)max_ni * (uint64_t)p->L * (uint64_t)p->K * 4);
    }
    h.klists = o;
    if (bucket) o += align_up(e * 4);
    h.total = o;
    return h;
}
inline uint64_t plan_bytes(const cm_params* p, int64_t n_pairs, int64_t rows, int32_t max_ni) {
    return align_up((uint64_t)n_pairs * sizeof(DevPair)) + kAlign + hand_over(p, n_pairs, rows, max_ni).total;
}
// The bucket-major matcher's pair order: descending n_i * n_j (the work of a
// pair grows with it), ties by position, so the last pairs dealt are small.
namespace cm {
std::vector<int32_t> pair_order(const std::vector<DevPair>& tab, const std::vector<int32_t>& n_desc);
}  // namespace cm

struct cm_match_plan {
    cm_index* ix = nullptr;
    cm_params p{};           // the index's parameters when the plan was made (K, query tile, algo)
    int32_t S = 0;           // queries per work item
    uint64_t table_at = 0;   // arena offset: [n_pairs] DevPair, the work counter, the top-K hand-over
    int64_t n_pairs = 0;
    int64_t rows = 0;
    int32_t n_items = 0;
    int32_t max_ni = 0;      // largest query image of the plan
    bool reserved = false;   // placed in the index's reserved plan block
    uint8_t* ext = nullptr;  // caller's workspace holding the table instead of the arena (cm_match_pairs)
    // device address of the plan's table (then the work counter and the hand-over)
    uint8_t* base() const { return ext ? ext : ix->arena + table_at; }
};


