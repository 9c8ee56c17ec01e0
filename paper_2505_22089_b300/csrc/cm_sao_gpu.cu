// The SAO local constraint (Sec. 2.3.3, Fig. 4) on the GPU, over every pair
// of a match plan at once: the same scores and decisions as cm_sao_filter on
// the host, computed where the initial matches already are.
//
// The plan's decisions are first compacted into per-pair match lists in the
// workspace (query order, as the verifier receives them).  Then one CTA per
// pair walks its list in chunks of 256 matches, one thread per match:
//   - nearest neighbours, in the query image and then in the database image:
//     the pair's matched keypoints stream through shared memory in tiles of
//     1,024 and each thread keeps the T = k + 4 smallest FP32 squared
//     distances (by distance, then index); those T are re-scored exactly in
//     FP64 and sorted by (d^2, index).  The FP32 pre-selection is exact:
//     every point left out has an FP32 distance at least that of the T-th,
//     hence an exact one above d_T / (1 + 1e-6); when the k-th exact distance
//     is not below that bound, the thread scans all points in FP64 instead;
//   - angular order by half-plane and the sign of an exact cross product,
//     the cyclic edit distance of the two label sequences, the score and the
//     decision, with the same roundings as the host (no fused multiply-adds).
// A rejected match's decision becomes -1 in the output, so the usual
// compaction afterwards hands only the kept matches to verification.
#include <cuda_runtime.h>

#include <cstdint>

#include "cm_host.h"

namespace cm {

namespace {

constexpr int kSaoThreads = 256;
constexpr int kSaoTile = 1024;
constexpr int kSaoMaxK = 16;

// One space (query or database image) of a pair's match list: entry e has its
// keypoint at kp[2 * idx(e)], idx = the query (high 16 bits) or database (low
// 16 bits) index of list word e.
struct Space {
    const float* kp;
    int shift;   // 16: query index, 0: database index
    __device__ __forceinline__ float2 at(const uint32_t* list, int e) const {
        const int i = (int)((list[e] >> shift) & 0xFFFFu);
        return make_float2(kp[2 * i], kp[2 * i + 1]);
    }
};

__device__ __forceinline__ double d2_exact(double ax, double ay, double bx, double by) {
    const double dx = __dsub_rn(bx, ax), dy = __dsub_rn(by, ay);
    return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
}

// true when ray a comes before ray b (angle from the +x axis in [0, 2 pi), a
// zero vector at angle 0, ties by label)
__device__ __forceinline__ bool ray_less(double ax, double ay, int al, double bx, double by, int bl) {
    const int ha = (ay < 0 || (ay == 0 && ax < 0)) ? 1 : 0;
    const int hb = (by < 0 || (by == 0 && bx < 0)) ? 1 : 0;
    if (ha != hb) return ha < hb;
    const bool za = ay == 0 && ax >= 0, zb = by == 0 && bx >= 0;
    if (za || zb) return za && zb ? al < bl : za;
    const double cr = __dsub_rn(__dmul_rn(ax, by), __dmul_rn(ay, bx));
    if (cr != 0) return cr > 0;
    return al < bl;
}

// Exact k nearest list entries of entry m in one space, by (d^2, entry), then
// their labels in angular order around m.  Returns the neighbour count.
template <int T>
__device__ int neighbours(const uint32_t* list, int n, int m, bool active, Space sp, int k, float* tx, float* ty,
                          int32_t* labels) {
    const int tid = threadIdx.x;
    float2 me = make_float2(0.f, 0.f);
    if (active) me = sp.at(list, m);
    // FP32 pre-selection of T candidates, kept as (float bits << 32 | entry), ascending
    uint64_t s[T];
#pragma unroll
    for (int t = 0; t < T; ++t) s[t] = ~0ull;
    for (int t0 = 0; t0 < n; t0 += kSaoTile) {
        __syncthreads();
        for (int u = tid; u < kSaoTile && t0 + u < n; u += kSaoThreads) {
            const float2 p = sp.at(list, t0 + u);
            tx[u] = p.x;
            ty[u] = p.y;
        }
        __syncthreads();
        if (!active) continue;
        const int lim = min(kSaoTile, n - t0);
        for (int u = 0; u < lim; ++u) {
            const float dx = tx[u] - me.x, dy = ty[u] - me.y;
            const float d = dx * dx + dy * dy;
            const uint64_t key = ((uint64_t)__float_as_uint(d) << 32) | (uint32_t)(t0 + u);
            if (key < s[T - 1] && t0 + u != m) {
#pragma unroll
                for (int i = T - 1; i > 0; --i) s[i] = max(s[i - 1], min(s[i], key));
                s[0] = min(s[0], key);
            }
        }
    }
    if (!active) return 0;
    const int want = min(k, n - 1);
    if (want <= 0) return 0;
    const int have = min(T, n - 1);
    // exact FP64 distances of the candidates, sorted by (d^2, entry)
    double dd[T];
    int ee[T];
    const double mx = me.x, my = me.y;
    for (int c = 0; c < have; ++c) {
        const int e = (int)(s[c] & 0xFFFFFFFFu);
        const float2 p = sp.at(list, e);
        const double d = d2_exact(mx, my, p.x, p.y);
        int pos = c;
        while (pos > 0 && (d < dd[pos - 1] || (d == dd[pos - 1] && e < ee[pos - 1]))) {
            dd[pos] = dd[pos - 1];
            ee[pos] = ee[pos - 1];
            --pos;
        }
        dd[pos] = d;
        ee[pos] = e;
    }
    if (have < n - 1) {
        // a point outside the candidates has an exact distance above this bound
        const double bound = (double)__uint_as_float((uint32_t)(s[T - 1] >> 32)) / (1.0 + 1e-6);
        if (!(dd[want - 1] < bound)) {
            // not decided by the pre-selection: every point in FP64
            for (int c = 0; c < want; ++c) {
                dd[c] = __longlong_as_double(0x7FF0000000000000ll);
                ee[c] = 0x7FFFFFFF;
            }
            for (int e = 0; e < n; ++e) {
                if (e == m) continue;
                const float2 p = sp.at(list, e);
                const double d = d2_exact(mx, my, p.x, p.y);
                if (!(d < dd[want - 1] || (d == dd[want - 1] && e < ee[want - 1]))) continue;
                int pos = want - 1;
                while (pos > 0 && (d < dd[pos - 1] || (d == dd[pos - 1] && e < ee[pos - 1]))) {
                    dd[pos] = dd[pos - 1];
                    ee[pos] = ee[pos - 1];
                    --pos;
                }
                dd[pos] = d;
                ee[pos] = e;
            }
        }
    }
    // angular order of the want nearest around m
    double rx[kSaoMaxK], ry[kSaoMaxK];
    for (int c = 0; c < want; ++c) {
        const float2 p = sp.at(list, ee[c]);
        const double x = __dsub_rn((double)p.x, mx), y = __dsub_rn((double)p.y, my);
        int pos = c;
        while (pos > 0 && ray_less(x, y, ee[c], rx[pos - 1], ry[pos - 1], labels[pos - 1])) {
            rx[pos] = rx[pos - 1];
            ry[pos] = ry[pos - 1];
            labels[pos] = labels[pos - 1];
            --pos;
        }
        rx[pos] = x;
        ry[pos] = y;
        labels[pos] = ee[c];
    }
    return want;
}

// Unit-cost edit distance, or a value above cap once a whole DP row exceeds it.
__device__ int levenshtein(const int32_t* a, int na, const int32_t* b, int nb, int cap) {
    int row[kSaoMaxK + 1];
    for (int j = 0; j <= nb; ++j) row[j] = j;
    for (int i = 1; i <= na; ++i) {
        int diag = row[0];
        row[0] = i;
        int lo = i;
        for (int j = 1; j <= nb; ++j) {
            const int up = row[j];
            const int v = min(min(up + 1, row[j - 1] + 1), diag + (a[i - 1] == b[j - 1] ? 0 : 1));
            row[j] = v;
            diag = up;
            lo = min(lo, v);
        }
        if (lo > cap) return lo;
    }
    return row[nb];
}

// Cyclic edit distance: rotations of a only (an alignment of two rotations can
// be re-cut where b starts), the rotation starting with b's first label first.
__device__ int cyclic_edit_distance(const int32_t* a, int na, const int32_t* b, int nb) {
    if (na == 0 || nb == 0) return max(na, nb);
    int r0 = 0;
    for (int t = 0; t < na; ++t)
        if (a[t] == b[0]) r0 = t;
    if (na == nb) {
        int t = 0;
        while (t < na && a[(r0 + t) % na] == b[t]) ++t;
        if (t == na) return 0;
    }
    int32_t rot[kSaoMaxK];
    int best = na + nb;
    for (int step = 0; step < na && best > 0; ++step) {
        const int r = (r0 + step) % na;
        for (int t = 0; t < na; ++t) rot[t] = a[(r + t) % na];
        best = min(best, levenshtein(rot, na, b, nb, best - 1));
    }
    return best;
}

template <int T>
__global__ void __launch_bounds__(kSaoThreads) k_sao_pairs(const DevPair* __restrict__ pairs,
                                                           const unsigned long long* __restrict__ offsets,
                                                           const uint32_t* __restrict__ matches,
                                                           const float* __restrict__ kp,
                                                           const int64_t* __restrict__ kp_off, int k, float max_score,
                                                           int32_t* __restrict__ best_out, float* __restrict__ score) {
    __shared__ float tx[kSaoTile], ty[kSaoTile];
    const DevPair P = pairs[blockIdx.x];
    const unsigned long long o0 = offsets[blockIdx.x];
    const int n = (int)(offsets[blockIdx.x + 1] - o0);
    const uint32_t* list = matches + o0;
    const Space sp{kp + 2 * kp_off[P.i], 16}, sq{kp + 2 * kp_off[P.j], 0};
    for (int c0 = 0; c0 < n; c0 += kSaoThreads) {
        const int m = c0 + (int)threadIdx.x;
        const bool active = m < n;
        int32_t la[kSaoMaxK], lb[kSaoMaxK];
        const int na = neighbours<T>(list, n, m, active, sp, k, tx, ty, la);
        const int nb = neighbours<T>(list, n, m, active, sq, k, tx, ty, lb);
        if (!active) continue;
        const float s = na ? (float)cyclic_edit_distance(la, na, lb, nb) / (float)na : 0.f;
        const int64_t row = P.row_off + (int64_t)(list[m] >> 16);
        if (!(s <= max_score)) best_out[row] = -1;
        if (score) score[row] = s;
    }
}

struct SaoWork {
    uint64_t counts, offsets, matches, total;
};

SaoWork sao_layout(int64_t n_pairs, int64_t rows) {
    SaoWork w{};
    w.counts = 0;
    w.offsets = align_up(4 * (uint64_t)n_pairs);
    w.matches = align_up(w.offsets + 8 * (uint64_t)(n_pairs + 1));
    w.total = align_up(w.matches + 4 * (uint64_t)std::max<int64_t>(rows, 1));
    return w;
}

}  // namespace

uint64_t sao_work_bytes(int64_t n_pairs, int64_t rows) { return sao_layout(n_pairs, rows).total; }

}  // namespace cm

using namespace cm;

extern "C" cm_status cm_match_plan_sao_bytes(const cm_match_plan* pl, uint64_t* bytes) {
    if (!pl || !bytes) return host_fail(CM_ERR_INVALID, "cm_match_plan_sao_bytes: bad argument");
    *bytes = sao_layout(pl->n_pairs, pl->rows).total;
    return CM_OK;
}

extern "C" cm_status cm_match_plan_sao(cm_match_plan* pl, const int32_t* d_best_in, int32_t* d_best_out,
                                       const float* d_kp, const int64_t* d_kp_off, int32_t k_nn, float max_score,
                                       float* d_score, void* d_work, uint64_t work_bytes, cm_stream stream) {
    if (!pl || !d_best_in || !d_best_out || !d_kp || !d_kp_off || !d_work || k_nn < 1 || k_nn > kSaoMaxK ||
        !(max_score >= 0.f))
        return host_fail(CM_ERR_INVALID, "cm_match_plan_sao: bad argument (1 <= k_nn <= 16)");
    if (!pl->ix) return host_fail(CM_ERR_STATE, "cm_match_plan_sao: the plan's index was destroyed");
    const SaoWork w = sao_layout(pl->n_pairs, pl->rows);
    if (work_bytes < w.total || (reinterpret_cast<uintptr_t>(d_work) & (kAlign - 1)))
        return host_fail(CM_ERR_BUDGET, "cm_match_plan_sao: workspace smaller than cm_match_plan_sao_bytes");
    if (pl->n_pairs == 0) return CM_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cm_index* ix = pl->ix;
    unsigned char* base = static_cast<unsigned char*>(d_work);
    const DevPair* dp = reinterpret_cast<const DevPair*>(ix->arena + pl->table_at);
    auto* offsets = reinterpret_cast<unsigned long long*>(base + w.offsets);
    auto* matches = reinterpret_cast<uint32_t*>(base + w.matches);
    if (d_best_out != d_best_in)
        CM_CUDA(cudaMemcpyAsync(d_best_out, d_best_in, 4 * (size_t)pl->rows, cudaMemcpyDeviceToDevice, s));
    if (d_score) CM_CUDA(cudaMemsetAsync(d_score, 0, 4 * (size_t)pl->rows, s));
    CM_CUDA(launch_compact(dp, (int)pl->n_pairs, ix->at<DevImage>(ix->fx.imgs), d_best_in,
                           reinterpret_cast<uint32_t*>(base + w.counts), offsets, offsets + pl->n_pairs, matches,
                           (unsigned long long)std::max<int64_t>(pl->rows, 1), s));
    if (k_nn + 4 <= 12)
        k_sao_pairs<12><<<(unsigned)pl->n_pairs, kSaoThreads, 0, s>>>(dp, offsets, matches, d_kp, d_kp_off, k_nn,
                                                                       max_score, d_best_out, d_score);
    else
        k_sao_pairs<20><<<(unsigned)pl->n_pairs, kSaoThreads, 0, s>>>(dp, offsets, matches, d_kp, d_kp_off, k_nn,
                                                                       max_score, d_best_out, d_score);
    CM_CUDA(cudaGetLastError());
    return CM_OK;
}
