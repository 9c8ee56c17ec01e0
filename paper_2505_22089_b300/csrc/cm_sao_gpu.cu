// The SAO local constraint (Sec. 2.3.3, Fig. 4) on the GPU, over every pair
// of a match plan at once: the same scores and decisions as cm_sao_filter on
// the host, computed where the initial matches already are.
//
// The plan's decisions are first compacted into per-pair match lists in the
// workspace (query order, as the verifier receives them).  Then one CTA per
// pair:
//   - builds, for the query image and for the database image, a uniform grid
//     over the pair's matched keypoints (about two per cell, shaped like the
//     bounding box; a counting sort into workspace memory);
//   - walks its list in chunks of 256 matches, one thread per match: a ring
//     by ring grid search for the k + 4 nearest in FP32 (cells skipped, and
//     the search stopped, by FP32 bounds widened for FP32 rounding), those
//     re-scored in FP64 and ordered by (d^2, entry); when the k-th exact
//     distance does not clear the FP32 screen by its error margin, the same
//     search runs in FP64 alone.  Then the angular order: FP32 comparisons
//     where their outcome is certain, the host's FP64 comparison otherwise;
//     the cyclic edit distance, the score and the decision.  Every decision
//     is the host's: FP64 arithmetic without fused multiply-adds
//     (cm_sao_common.cuh) wherever FP32 cannot be certain.
// A rejected match's decision becomes -1 in the output, so the usual
// compaction afterwards hands only the kept matches to verification.
#include <cuda_runtime.h>

#include <cstdint>

#include "cm_host.h"
#include "cm_sao_common.cuh"

namespace cm {

namespace {

constexpr int kSaoThreads = 256;
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

// A grid over one space of a pair's match list, in the pair's workspace.
struct Grid {
    double x0, y0, csx, csy, slack;
    float fx0, fy0, fcsx, fcsy, fslack;   // the same in FP32, the slack wide enough for FP32 rounding
    int gx, gy;
    int32_t* start;   // [gx * gy + 1] first sorted entry of each cell
    float2* pts;      // [n] keypoints in cell order
    int32_t* ids;     // [n] their list entries
};

__device__ __forceinline__ int cell_coord(double v, double cs, int g) {
    const int c = (int)(v / cs);
    return c < 0 ? 0 : (c >= g ? g - 1 : c);
}

// Builds the grid of one space (all threads of the CTA take part).
__device__ void build_grid(const uint32_t* list, int n, Space sp, Grid& G, int32_t* fill, double* red) {
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    float lo_x = __uint_as_float(0x7F800000u), lo_y = lo_x, hi_x = -lo_x, hi_y = -lo_x;
    for (int e = tid; e < n; e += kSaoThreads) {
        const float2 p = sp.at(list, e);
        lo_x = fminf(lo_x, p.x);
        lo_y = fminf(lo_y, p.y);
        hi_x = fmaxf(hi_x, p.x);
        hi_y = fmaxf(hi_y, p.y);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo_x = fminf(lo_x, __shfl_xor_sync(0xFFFFFFFFu, lo_x, o));
        lo_y = fminf(lo_y, __shfl_xor_sync(0xFFFFFFFFu, lo_y, o));
        hi_x = fmaxf(hi_x, __shfl_xor_sync(0xFFFFFFFFu, hi_x, o));
        hi_y = fmaxf(hi_y, __shfl_xor_sync(0xFFFFFFFFu, hi_y, o));
    }
    __syncthreads();   // red may still be read from the previous build
    if (lane == 0) {
        red[4 * w + 0] = lo_x;
        red[4 * w + 1] = lo_y;
        red[4 * w + 2] = hi_x;
        red[4 * w + 3] = hi_y;
    }
    __syncthreads();
    if (tid == 0) {
        double x0 = red[0], y0 = red[1], x1 = red[2], y1 = red[3];
        for (int k = 1; k < kSaoThreads / 32; ++k) {
            x0 = fmin(x0, red[4 * k]);
            y0 = fmin(y0, red[4 * k + 1]);
            x1 = fmax(x1, red[4 * k + 2]);
            y1 = fmax(y1, red[4 * k + 3]);
        }
        const double wd = x1 - x0, hd = y1 - y0;
        const double cells = fmax(1.0, floor((double)n / 2.0));
        int gx, gy;
        if (wd > 0 && hd > 0) {
            gx = (int)fmin(fmax(round(sqrt(cells * wd / hd)), 1.0), cells);
            gy = (int)fmin(fmax(round(cells / gx), 1.0), cells);
        } else {
            gx = wd > 0 ? (int)cells : 1;
            gy = hd > 0 ? (int)cells : 1;
        }
        G.x0 = x0;
        G.y0 = y0;
        G.gx = gx;
        G.gy = gy;
        G.csx = wd > 0 ? wd / gx : 1.0;
        G.csy = hd > 0 ? hd / gy : 1.0;
        G.slack = 1e-9 * (wd + hd + fabs(x0) + fabs(y0) + 1.0);
        G.fx0 = (float)x0;
        G.fy0 = (float)y0;
        G.fcsx = (float)G.csx;
        G.fcsy = (float)G.csy;
        G.fslack = (float)(1e-5 * (wd + hd + fabs(x0) + fabs(y0) + 1.0));
    }
    __syncthreads();
    const int nc = G.gx * G.gy;
    for (int c = tid; c < nc; c += kSaoThreads) fill[c] = 0;
    __syncthreads();
    for (int e = tid; e < n; e += kSaoThreads) {
        const float2 p = sp.at(list, e);
        const int c = cell_coord((double)p.x - G.x0, G.csx, G.gx) + G.gx * cell_coord((double)p.y - G.y0, G.csy, G.gy);
        atomicAdd(&fill[c], 1);
    }
    __syncthreads();
    // exclusive prefix of the counts into start (chunks of the CTA), then fill restarts at 0
    __shared__ int s_part[kSaoThreads];
    __shared__ int s_carry;
    if (tid == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < nc; base += kSaoThreads) {
        const int c = base + tid;
        const int v = c < nc ? fill[c] : 0;
        s_part[tid] = v;
        __syncthreads();
        for (int o = 1; o < kSaoThreads; o <<= 1) {
            const int add = tid >= o ? s_part[tid - o] : 0;
            __syncthreads();
            s_part[tid] += add;
            __syncthreads();
        }
        if (c < nc) {
            G.start[c] = s_carry + s_part[tid] - v;
            fill[c] = 0;
        }
        __syncthreads();
        if (tid == kSaoThreads - 1) s_carry += s_part[tid];
        __syncthreads();
    }
    if (tid == 0) G.start[nc] = n;
    __syncthreads();
    for (int e = tid; e < n; e += kSaoThreads) {
        const float2 p = sp.at(list, e);
        const int c = cell_coord((double)p.x - G.x0, G.csx, G.gx) + G.gx * cell_coord((double)p.y - G.y0, G.csy, G.gy);
        const int pos = G.start[c] + atomicAdd(&fill[c], 1);
        G.pts[pos] = p;
        G.ids[pos] = e;
    }
    __syncthreads();
}

// Exact k nearest list entries of entry m by (d^2 in FP64, entry), searched
// ring by ring; writes them ascending to dd / ee.
__device__ void knn_exact(int m, double px, double py, const Grid& G, int want, double* dd, int* ee) {
    const int cx = cell_coord(px - G.x0, G.csx, G.gx), cy = cell_coord(py - G.y0, G.csy, G.gy);
    int cnt = 0;
    for (int r = 0;; ++r) {
        const int xa = cx - r, xb = cx + r, ya = cy - r, yb = cy + r;
        for (int yy = max(ya, 0); yy <= min(yb, G.gy - 1); ++yy) {
            const bool edge_row = yy == ya || yy == yb;
            const double gy0 = G.y0 + yy * G.csy - G.slack - py, gy1 = py - (G.y0 + (yy + 1) * G.csy + G.slack);
            const double ry = gy0 > 0 ? gy0 : (gy1 > 0 ? gy1 : 0.0);
            for (int xx = max(xa, 0); xx <= min(xb, G.gx - 1); ++xx) {
                if (!edge_row && xx != xa && xx != xb) continue;   // the ring only
                if (cnt == want) {   // a cell that cannot hold a point closer than the k-th
                    const double gx0 = G.x0 + xx * G.csx - G.slack - px, gx1 = px - (G.x0 + (xx + 1) * G.csx + G.slack);
                    const double rx = gx0 > 0 ? gx0 : (gx1 > 0 ? gx1 : 0.0);
                    if (sao::add(sao::mul(rx, rx), sao::mul(ry, ry)) > dd[cnt - 1]) continue;
                }
                const int c = yy * G.gx + xx;
                for (int t = G.start[c]; t < G.start[c + 1]; ++t) {
                    const int e = G.ids[t];
                    if (e == m) continue;
                    const float2 p = G.pts[t];
                    const double d = sao::d2(px, py, p.x, p.y);
                    if (cnt == want && !(d < dd[cnt - 1] || (d == dd[cnt - 1] && e < ee[cnt - 1]))) continue;
                    int pos = cnt < want ? cnt++ : cnt - 1;
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
        if (xa <= 0 && ya <= 0 && xb >= G.gx - 1 && yb >= G.gy - 1) break;
        if (cnt == want) {   // distance from p to the nearest cell outside the visited block
            double lb = __longlong_as_double(0x7FF0000000000000ll);
            if (xa > 0) lb = fmin(lb, px - (G.x0 + xa * G.csx));
            if (xb < G.gx - 1) lb = fmin(lb, G.x0 + (xb + 1) * G.csx - px);
            if (ya > 0) lb = fmin(lb, py - (G.y0 + ya * G.csy));
            if (yb < G.gy - 1) lb = fmin(lb, G.y0 + (yb + 1) * G.csy - py);
            lb -= G.slack;
            if (lb > 0 && dd[cnt - 1] < sao::mul(lb, lb)) break;
        }
    }
}

// The same set from an FP32 search of T = want + 4 candidates, re-scored in
// FP64 and sorted by (d^2, entry).  A point left out either has an FP32
// distance (relative error below 1e-6) at least the T-th candidate's d_T, or
// lies in a cell whose FP32 lower bound, widened by a slack for FP32
// rounding, exceeds d_T (1 + 4e-6).  So when the want-th exact distance is
// below d_T / (1 + 1e-6), no point left out can rank among the first want and
// the set is exact.  Returns false when that test fails (knn_exact decides).
__device__ bool knn_fast(const uint32_t* list, Space sp, int m, int n, float pxf, float pyf, const Grid& G, int want,
                         double* dd, int* ee) {
    const int T = min(want + 4, n - 1);
    const float grow = 1.f + 4e-6f;
    float df[kSaoMaxK + 4];
    int ef[kSaoMaxK + 4];
    int cnt = 0;
    const int cx = cell_coord((double)pxf - G.x0, G.csx, G.gx), cy = cell_coord((double)pyf - G.y0, G.csy, G.gy);
    for (int r = 0;; ++r) {
        const int xa = cx - r, xb = cx + r, ya = cy - r, yb = cy + r;
        for (int yy = max(ya, 0); yy <= min(yb, G.gy - 1); ++yy) {
            const bool edge_row = yy == ya || yy == yb;
            const float gy0 = G.fy0 + yy * G.fcsy - G.fslack - pyf, gy1 = pyf - (G.fy0 + (yy + 1) * G.fcsy + G.fslack);
            const float ry = gy0 > 0 ? gy0 : (gy1 > 0 ? gy1 : 0.f);
            for (int xx = max(xa, 0); xx <= min(xb, G.gx - 1); ++xx) {
                if (!edge_row && xx != xa && xx != xb) continue;
                if (cnt == T) {
                    const float gx0 = G.fx0 + xx * G.fcsx - G.fslack - pxf, gx1 = pxf - (G.fx0 + (xx + 1) * G.fcsx + G.fslack);
                    const float rx = gx0 > 0 ? gx0 : (gx1 > 0 ? gx1 : 0.f);
                    if (rx * rx + ry * ry > df[T - 1] * grow) continue;
                }
                const int c = yy * G.gx + xx;
                for (int t = G.start[c]; t < G.start[c + 1]; ++t) {
                    const int e = G.ids[t];
                    if (e == m) continue;
                    const float2 p = G.pts[t];
                    const float dx = p.x - pxf, dy = p.y - pyf;
                    const float d = dx * dx + dy * dy;
                    if (cnt == T && !(d < df[T - 1] || (d == df[T - 1] && e < ef[T - 1]))) continue;
                    int pos = cnt < T ? cnt++ : T - 1;
                    while (pos > 0 && (d < df[pos - 1] || (d == df[pos - 1] && e < ef[pos - 1]))) {
                        df[pos] = df[pos - 1];
                        ef[pos] = ef[pos - 1];
                        --pos;
                    }
                    df[pos] = d;
                    ef[pos] = e;
                }
            }
        }
        if (xa <= 0 && ya <= 0 && xb >= G.gx - 1 && yb >= G.gy - 1) break;
        if (cnt == T) {
            float lb = __uint_as_float(0x7F800000u);
            if (xa > 0) lb = fminf(lb, pxf - (G.fx0 + xa * G.fcsx));
            if (xb < G.gx - 1) lb = fminf(lb, G.fx0 + (xb + 1) * G.fcsx - pxf);
            if (ya > 0) lb = fminf(lb, pyf - (G.fy0 + ya * G.fcsy));
            if (yb < G.gy - 1) lb = fminf(lb, G.fy0 + (yb + 1) * G.fcsy - pyf);
            lb -= G.fslack;
            if (lb > 0 && df[T - 1] * grow < lb * lb) break;
        }
    }
    // exact re-score of the candidates, keeping the first want by (d^2, entry)
    const double px = pxf, py = pyf;
    int kept = 0;
    for (int c = 0; c < cnt; ++c) {
        const int e = ef[c];
        const float2 p = sp.at(list, e);
        const double d = sao::d2(px, py, p.x, p.y);
        if (kept == want && !(d < dd[want - 1] || (d == dd[want - 1] && e < ee[want - 1]))) continue;
        int pos = kept < want ? kept++ : want - 1;
        while (pos > 0 && (d < dd[pos - 1] || (d == dd[pos - 1] && e < ee[pos - 1]))) {
            dd[pos] = dd[pos - 1];
            ee[pos] = ee[pos - 1];
            --pos;
        }
        dd[pos] = d;
        ee[pos] = e;
    }
    if (cnt < n - 1) {
        const double bound = (double)df[T - 1] / (1.0 + 1e-6);
        if (!(dd[want - 1] < bound)) return false;
    }
    return true;
}

// Exact k nearest list entries of entry m, then their labels in angular
// order around m.  Returns the neighbour count.
__device__ int neighbours(const uint32_t* list, int n, int m, Space sp, const Grid& G, int k, int32_t* labels) {
    const int want = min(k, n - 1);
    if (want <= 0) return 0;
    const float2 me = sp.at(list, m);
    double dd[kSaoMaxK];
    int ee[kSaoMaxK];
    if (!knn_fast(list, sp, m, n, me.x, me.y, G, want, dd, ee)) knn_exact(m, me.x, me.y, G, want, dd, ee);
    // angular order of the want nearest around m.  Rays are compared in FP32
    // where that is certain: the half-plane tests use only signs and zeros of
    // the coordinate differences, which FP32 subtraction keeps, and a cross
    // product whose FP32 value exceeds 1e-6 of its terms' magnitudes has the
    // sign of the exact one; otherwise the host's FP64 comparison decides.
    const double px = me.x, py = me.y;
    float xs[kSaoMaxK], ys[kSaoMaxK];
    for (int c = 0; c < want; ++c) {
        const float2 p = sp.at(list, ee[c]);
        const float x = p.x - me.x, y = p.y - me.y;
        const int e = ee[c];
        int pos = c;
        while (pos > 0) {
            const float bx = xs[pos - 1], by = ys[pos - 1];
            const int bl = labels[pos - 1];
            bool less;
            const int ha = (y < 0 || (y == 0 && x < 0)) ? 1 : 0, hb = (by < 0 || (by == 0 && bx < 0)) ? 1 : 0;
            const bool za = y == 0 && x >= 0, zb = by == 0 && bx >= 0;
            if (ha != hb) {
                less = ha < hb;
            } else if (za || zb) {
                less = za && zb ? e < bl : za;
            } else {
                const float t1 = x * by, t2 = y * bx, cr = t1 - t2;
                if (fabsf(cr) > 1e-6f * (fabsf(t1) + fabsf(t2))) {
                    less = cr > 0;
                } else {   // too close to call in FP32: the host's FP64 comparison
                    const float2 q = sp.at(list, bl);
                    less = sao::ray_less(sao::sub((double)p.x, px), sao::sub((double)p.y, py), e,
                                         sao::sub((double)q.x, px), sao::sub((double)q.y, py), bl);
                }
            }
            if (!less) break;
            xs[pos] = xs[pos - 1];
            ys[pos] = ys[pos - 1];
            labels[pos] = labels[pos - 1];
            --pos;
        }
        xs[pos] = x;
        ys[pos] = y;
        labels[pos] = e;
    }
    return want;
}

__global__ void __launch_bounds__(kSaoThreads) k_sao_pairs(const DevPair* __restrict__ pairs,
                                                           const unsigned long long* __restrict__ offsets,
                                                           const uint32_t* __restrict__ matches,
                                                           const float* __restrict__ kp,
                                                           const int64_t* __restrict__ kp_off, int k, float max_score,
                                                           int32_t* __restrict__ best_out, float* __restrict__ score,
                                                           float2* __restrict__ gpts, int32_t* __restrict__ gids,
                                                           int32_t* __restrict__ gcells, int64_t rows) {
    __shared__ Grid grid[2];
    __shared__ double red[4 * (kSaoThreads / 32)];
    const DevPair P = pairs[blockIdx.x];
    const unsigned long long o0 = offsets[blockIdx.x];
    const int n = (int)(offsets[blockIdx.x + 1] - o0);
    if (n == 0) return;
    const uint32_t* list = matches + o0;
    const Space sp[2] = {{kp + 2 * kp_off[P.i], 16}, {kp + 2 * kp_off[P.j], 0}};
    // workspace of this pair: entries [o0, o0 + n) per space, and for the cells
    // (at most n / 2 + 1 starts and counts) slots [o0 + pair, o0 + pair + n + 1)
    for (int g = 0; g < 2; ++g) {
        const int64_t cbase = (int64_t)o0 + blockIdx.x;
        if (threadIdx.x == 0) {
            grid[g].pts = gpts + g * rows + o0;
            grid[g].ids = gids + g * rows + o0;
            grid[g].start = gcells + g * 2 * (rows + gridDim.x) + cbase;
        }
        __syncthreads();
        build_grid(list, n, sp[g], grid[g], gcells + (g * 2 + 1) * (rows + gridDim.x) + cbase, red);
    }
    for (int c0 = 0; c0 < n; c0 += kSaoThreads) {
        const int m = c0 + (int)threadIdx.x;
        if (m >= n) continue;
        int32_t la[kSaoMaxK], lb[kSaoMaxK];
        const int na = neighbours(list, n, m, sp[0], grid[0], k, la);
        const int nb = neighbours(list, n, m, sp[1], grid[1], k, lb);
        const float s = na ? (float)sao::cyclic_edit_distance(la, na, lb, nb) / (float)na : 0.f;
        const int64_t row = P.row_off + (int64_t)(list[m] >> 16);
        if (!(s <= max_score)) best_out[row] = -1;
        if (score) score[row] = s;
    }
}

// Workspace: compaction (counts, offsets, match lists), then per space the
// grid's sorted keypoints and entries [rows] and its cell starts and counts
// [rows + pairs] each.
struct SaoWork {
    uint64_t counts, offsets, matches, pts, ids, cells, total;
};

SaoWork sao_layout(int64_t n_pairs, int64_t rows) {
    SaoWork w{};
    const uint64_t r = (uint64_t)std::max<int64_t>(rows, 1);
    w.counts = 0;
    w.offsets = align_up(4 * (uint64_t)n_pairs);
    w.matches = align_up(w.offsets + 8 * (uint64_t)(n_pairs + 1));
    w.pts = align_up(w.matches + 4 * r);
    w.ids = align_up(w.pts + 2 * 8 * r);
    w.cells = align_up(w.ids + 2 * 4 * r);
    w.total = align_up(w.cells + 4 * 4 * (r + (uint64_t)n_pairs));
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
    const DevPair* dp = reinterpret_cast<const DevPair*>(pl->base());
    auto* offsets = reinterpret_cast<unsigned long long*>(base + w.offsets);
    auto* matches = reinterpret_cast<uint32_t*>(base + w.matches);
    if (d_best_out != d_best_in)
        CM_CUDA(cudaMemcpyAsync(d_best_out, d_best_in, 4 * (size_t)pl->rows, cudaMemcpyDeviceToDevice, s));
    if (d_score) CM_CUDA(cudaMemsetAsync(d_score, 0, 4 * (size_t)pl->rows, s));
    CM_CUDA(launch_compact(dp, (int)pl->n_pairs, ix->at<DevImage>(ix->fx.imgs), d_best_in,
                           reinterpret_cast<uint32_t*>(base + w.counts), offsets, offsets + pl->n_pairs, matches,
                           (unsigned long long)std::max<int64_t>(pl->rows, 1), s));
    const int64_t r = std::max<int64_t>(pl->rows, 1);
    k_sao_pairs<<<(unsigned)pl->n_pairs, kSaoThreads, 0, s>>>(
        dp, offsets, matches, d_kp, d_kp_off, k_nn, max_score, d_best_out, d_score,
        reinterpret_cast<float2*>(base + w.pts), reinterpret_cast<int32_t*>(base + w.ids),
        reinterpret_cast<int32_t*>(base + w.cells), r);
    CM_CUDA(cudaGetLastError());
    return CM_OK;
}
