// Spatial-angular-order (SAO) local geometric constraint of Sec. 2.3.3
// (Fig. 4), run on the host ahead of the RANSAC global constraint.
//
// For match m = (p_m, q_m): the k nearest other matched keypoints of p_m in
// the query image and, independently, of q_m in the database image (squared
// Euclidean distance, ties by match index), each list put in angular order
// around its centre (angle from the horizontal axis in [0, 2*pi), a zero
// vector at angle 0, ties by match index); the score is the cyclic edit
// distance of the two label sequences over the neighbour count N.
//
// Host design: nearest neighbours come from a uniform grid over each image's
// matched keypoints (about two points per cell) searched ring by ring until
// the k-th candidate is closer than any unvisited cell; that returns exactly
// the Euclidean k-NN set, which is also what a best-first search of the
// Delaunay graph returns.  Angular order uses half-planes and the sign of a
// cross product, no trigonometry.  The cyclic edit distance rotates one
// sequence only: any alignment of two rotated sequences can be re-cut where
// the second sequence starts, giving an alignment of the same cost between a
// rotation of the first and the second as given.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "cm_host.h"
#include "cm_sao_common.cuh"

namespace {

constexpr int kMaxSaoK = cm::sao::kMaxK;

struct Nb {
    double d2;
    int32_t id;
    bool operator<(const Nb& o) const { return d2 < o.d2 || (d2 == o.d2 && id < o.id); }
};

// Exact k nearest neighbours of a point among the others, by (squared
// distance, index), from a grid whose cells exactly tile the bounding box.
// Coordinates are copied in cell order so that a cell's points are adjacent.
class Grid {
public:
    Grid(const std::vector<double>& x, const std::vector<double>& y, double per_cell = 2.0) {
        const int64_t n = (int64_t)x.size();
        n_ = n;
        if (n == 0) return;
        double x1 = x[0], y1 = y[0];
        x0_ = x[0];
        y0_ = y[0];
        for (int64_t i = 1; i < n; ++i) {
            x0_ = std::min(x0_, x[i]);
            y0_ = std::min(y0_, y[i]);
            x1 = std::max(x1, x[i]);
            y1 = std::max(y1, y[i]);
        }
        // about per_cell points per cell, the cell grid shaped like the bounding box
        const double w = x1 - x0_, h = y1 - y0_;
        const double cells = std::max(1.0, std::floor((double)n / per_cell));
        if (w > 0 && h > 0) {
            gx_ = (int)std::clamp(std::round(std::sqrt(cells * w / h)), 1.0, cells);
            gy_ = (int)std::clamp(std::round(cells / gx_), 1.0, cells);
        } else {
            gx_ = w > 0 ? (int)cells : 1;
            gy_ = h > 0 ? (int)cells : 1;
        }
        csx_ = w > 0 ? w / gx_ : 1.0;
        csy_ = h > 0 ? h / gy_ : 1.0;
        std::vector<int32_t> cell(n);
        start_.assign((size_t)gx_ * gy_ + 1, 0);
        for (int64_t i = 0; i < n; ++i) {
            const int cx = cell_coord(x[i] - x0_, csx_, gx_), cy = cell_coord(y[i] - y0_, csy_, gy_);
            cell[i] = cy * gx_ + cx;
            ++start_[cell[i] + 1];
        }
        for (size_t c = 1; c < start_.size(); ++c) start_[c] += start_[c - 1];
        sx_.resize(n);
        sy_.resize(n);
        sid_.resize(n);
        home_.resize(n);
        std::vector<int32_t> fill(start_.begin(), start_.end() - 1);
        for (int64_t i = 0; i < n; ++i) {
            const int32_t t = fill[cell[i]]++;
            sx_[t] = x[i];
            sy_[t] = y[i];
            sid_[t] = (int32_t)i;
            home_[i] = cell[i];
        }
        slack_ = 1e-9 * (w + h + std::fabs(x0_) + std::fabs(y0_) + 1.0);
    }

    // k nearest of point (px, py) = point m; nearest first; returns min(k, n - 1).
    int query(int64_t m, double px, double py, int k, Nb* out) const {
        const int want = (int)std::min<int64_t>(k, n_ - 1);
        if (want <= 0) return 0;
        const int cx = home_[m] % gx_, cy = home_[m] / gx_;
        int cnt = 0;   // out[0..cnt) ascending
        for (int r = 0;; ++r) {
            const int xa = cx - r, xb = cx + r, ya = cy - r, yb = cy + r;
            for (int yy = std::max(ya, 0); yy <= std::min(yb, gy_ - 1); ++yy) {
                const bool edge_row = yy == ya || yy == yb;
                // vertical gap from p to this row of cells (a lower bound for its points)
                const double gy0 = y0_ + yy * csy_ - slack_ - py, gy1 = py - (y0_ + (yy + 1) * csy_ + slack_);
                const double ry = gy0 > 0 ? gy0 : (gy1 > 0 ? gy1 : 0.0);
                auto visit = [&](int xx) {
                    if (cnt == want) {   // skip a cell that cannot hold a point closer than the k-th
                        const double gx0 = x0_ + xx * csx_ - slack_ - px, gx1 = px - (x0_ + (xx + 1) * csx_ + slack_);
                        const double rx = gx0 > 0 ? gx0 : (gx1 > 0 ? gx1 : 0.0);
                        if (rx * rx + ry * ry > out[cnt - 1].d2) return;
                    }
                    const int c = yy * gx_ + xx;
                    for (int32_t t = start_[c]; t < start_[c + 1]; ++t) {
                        const int32_t id = sid_[t];
                        if (id == m) continue;
                        const Nb cand{cm::sao::d2(px, py, sx_[t], sy_[t]), id};
                        if (cnt == want && !(cand < out[cnt - 1])) continue;
                        int pos = cnt < want ? cnt++ : cnt - 1;
                        while (pos > 0 && cand < out[pos - 1]) {
                            out[pos] = out[pos - 1];
                            --pos;
                        }
                        out[pos] = cand;
                    }
                };
                if (edge_row) {
                    for (int xx = std::max(xa, 0); xx <= std::min(xb, gx_ - 1); ++xx) visit(xx);
                } else {   // the ring's two side cells of this row
                    if (xa >= 0) visit(xa);
                    if (xb < gx_) visit(xb);
                }
            }
            const bool all = xa <= 0 && ya <= 0 && xb >= gx_ - 1 && yb >= gy_ - 1;
            if (all) break;
            if (cnt == want) {
                // distance from p to the nearest cell outside the visited block
                double lb = INFINITY;
                if (xa > 0) lb = std::min(lb, px - (x0_ + xa * csx_));
                if (xb < gx_ - 1) lb = std::min(lb, x0_ + (xb + 1) * csx_ - px);
                if (ya > 0) lb = std::min(lb, py - (y0_ + ya * csy_));
                if (yb < gy_ - 1) lb = std::min(lb, y0_ + (yb + 1) * csy_ - py);
                lb -= slack_;   // a coordinate on a cell edge may have been rounded into the next cell
                if (lb > 0 && out[cnt - 1].d2 < lb * lb) break;
            }
        }
        return cnt;
    }

private:
    static int cell_coord(double v, double cs, int g) {
        const int c = (int)(v / cs);
        return c < 0 ? 0 : (c >= g ? g - 1 : c);
    }

    int64_t n_ = 0;
    double x0_ = 0, y0_ = 0, csx_ = 1, csy_ = 1, slack_ = 0;
    int gx_ = 1, gy_ = 1;
    std::vector<int32_t> start_;
    std::vector<double> sx_, sy_;
    std::vector<int32_t> sid_, home_;
};

struct Ray {
    double dx, dy;
    int32_t id;
};

bool ray_less(const Ray& a, const Ray& b) { return cm::sao::ray_less(a.dx, a.dy, a.id, b.dx, b.dy, b.id); }

// Neighbour labels of centre m in angular order.
int ordered(const Grid& g, const std::vector<double>& x, const std::vector<double>& y, int64_t m, int k,
            int32_t* labels) {
    Nb nb[kMaxSaoK];
    const int cnt = g.query(m, x[m], y[m], k, nb);
    Ray r[kMaxSaoK];
    for (int t = 0; t < cnt; ++t) r[t] = {cm::sao::sub(x[nb[t].id], x[m]), cm::sao::sub(y[nb[t].id], y[m]), nb[t].id};
    std::sort(r, r + cnt, ray_less);
    for (int t = 0; t < cnt; ++t) labels[t] = r[t].id;
    return cnt;
}

}  // namespace

extern "C" cm_status cm_sao_filter(const float* kp_i, const float* kp_j, int64_t n_matches, const uint32_t* matches,
                                   int32_t k_nn, float max_score, float* score, uint8_t* keep, int64_t* n_kept) {
    if (n_matches < 0 || n_matches > (int64_t)INT32_MAX || (n_matches && (!kp_i || !kp_j || !matches)) ||
        k_nn < 1 || k_nn > kMaxSaoK || !(max_score >= 0.f))
        return cm::host_fail(CM_ERR_INVALID, "cm_sao_filter: bad argument");
    const size_t n = (size_t)n_matches;
    std::vector<double> px(n), py(n), qx(n), qy(n);
    for (size_t m = 0; m < n; ++m) {
        const uint32_t q = matches[m] >> 16, j = matches[m] & 0xFFFFu;
        px[m] = kp_i[2 * (size_t)q];
        py[m] = kp_i[2 * (size_t)q + 1];
        qx[m] = kp_j[2 * (size_t)j];
        qy[m] = kp_j[2 * (size_t)j + 1];
    }
    const Grid gp(px, py), gq(qx, qy);
    int64_t kept = 0;
    for (size_t m = 0; m < n; ++m) {
        int32_t a[kMaxSaoK], b[kMaxSaoK];
        const int na = ordered(gp, px, py, (int64_t)m, k_nn, a);
        const int nb = ordered(gq, qx, qy, (int64_t)m, k_nn, b);
        const float s = na ? (float)cm::sao::cyclic_edit_distance(a, na, b, nb) / (float)na : 0.f;
        const bool k = s <= max_score;
        if (score) score[m] = s;
        if (keep) keep[m] = k;
        kept += k;
    }
    if (n_kept) *n_kept = kept;
    return CM_OK;
}
