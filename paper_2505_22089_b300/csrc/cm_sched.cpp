// Schedule blocks by matrix band reduction (Sec. 2.2 steps (1)-(5)) with the
// Gibbs-Poole-Stockmeyer ordering of Algorithm 2.  Host C++.
//
// Readings where the paper is silent (the same ones the test oracle states):
//  - each connected component is ordered on its own, components by smallest
//    node id; isolated nodes leave the matrix (step (4));
//  - minimum-degree ties go to the smallest id; a level structure is the BFS
//    layering, its depth the index of its last level;
//  - combined levels: nodes whose two candidate levels (lev_u, depth - lev_v)
//    agree take it; the others, in id order, take the candidate level holding
//    fewer nodes at that moment (ties to lev_u);
//  - numbering level by level; level 0 by (degree, id), later levels by (the
//    smallest number of a neighbour in the previous level, degree, id);
//  - chunks of at most Size_blk images, closed early when they would pass half
//    the budget; a block row is the window of consecutive chunks that fits the
//    budget and takes the edges whose lower chunk is its first chunk; edges
//    outside every window wait for the next iteration; an iteration that
//    places nothing falls back to one row per edge.
#include <algorithm>
#include <climits>
#include <cstdarg>
#include <cstdio>
#include <map>
#include <set>
#include <string>
#include <memory>
#include <vector>

#include "cm_internal.h"

namespace {

struct Graph {
    int n = 0;
    std::vector<std::vector<int>> adj;   // sorted, de-duplicated neighbours
    explicit Graph(int n_) : n(n_), adj(n_) {}
    void finish() {
        for (auto& a : adj) {
            std::sort(a.begin(), a.end());
            a.erase(std::unique(a.begin(), a.end()), a.end());
        }
    }
    int deg(int v) const { return (int)adj[v].size(); }
};

// BFS layering from root inside the component marked comp_id; lev[v] = level or -1.
int layering(const Graph& g, int root, const std::vector<int>& comp, int comp_id, std::vector<int>& lev,
             std::vector<int>& last_level) {
    std::vector<int> frontier{root}, next;
    for (int v : frontier) lev[v] = 0;
    int depth = 0;
    last_level = frontier;
    for (;;) {
        next.clear();
        for (int x : frontier)
            for (int y : g.adj[x])
                if (comp[y] == comp_id && lev[y] < 0) {
                    lev[y] = depth + 1;
                    next.push_back(y);
                }
        if (next.empty()) break;
        ++depth;
        frontier.swap(next);
        last_level = frontier;
    }
    return depth;
}

void order_component(const Graph& g, const std::vector<int>& nodes, const std::vector<int>& comp, int comp_id,
                     std::vector<int>& out) {
    if (nodes.size() == 1) {
        out.push_back(nodes[0]);
        return;
    }
    auto by_deg_id = [&](int a, int b) { return g.deg(a) != g.deg(b) ? g.deg(a) < g.deg(b) : a < b; };
    // Algorithm 2, PseudoPeripheralNodeSelection
    std::vector<int> lev_u(g.n, -1), lev_v(g.n, -1), last_u, last_v;
    int u = *std::min_element(nodes.begin(), nodes.end(), by_deg_id);
    int depth_u = layering(g, u, comp, comp_id, lev_u, last_u);
    int v = -1, depth_v = -1;
    for (;;) {
        v = *std::min_element(last_u.begin(), last_u.end(), by_deg_id);
        for (int x : nodes) lev_v[x] = -1;
        depth_v = layering(g, v, comp, comp_id, lev_v, last_v);
        if (depth_v > depth_u) {
            u = v;
            depth_u = depth_v;
            lev_u.swap(lev_v);
            last_u.swap(last_v);
        } else {
            break;
        }
    }
    // Algorithm 2, GpsOrdering: combined level structure
    const int k = depth_u;
    std::vector<int> size(k + 1, 0), level(g.n, -1);
    std::vector<int> sorted_nodes(nodes);
    std::sort(sorted_nodes.begin(), sorted_nodes.end());
    std::vector<int> undecided;
    for (int w : sorted_nodes) {
        const int i = lev_u[w], j = k - lev_v[w];
        if (i == j) {
            level[w] = i;
            ++size[i];
        } else {
            undecided.push_back(w);
        }
    }
    for (int w : undecided) {
        const int i = lev_u[w], j = k - lev_v[w];
        const int c = size[i] <= size[j] ? i : j;
        level[w] = c;
        ++size[c];
    }
    std::vector<std::vector<int>> by_level(k + 1);
    for (int w : sorted_nodes) by_level[level[w]].push_back(w);
    std::vector<int> number(g.n, -1);
    std::vector<long long> first(g.n, LLONG_MAX);   // smallest number of a neighbour in the previous level
    int next_number = (int)out.size();
    for (int l = 0; l <= k; ++l) {
        auto& members = by_level[l];
        if (l == 0) {
            std::sort(members.begin(), members.end(), by_deg_id);
        } else {
            for (int w : members) {
                long long best = LLONG_MAX;
                for (int y : g.adj[w])
                    if (number[y] >= 0 && level[y] == l - 1) best = std::min<long long>(best, number[y]);
                first[w] = best;
            }
            std::sort(members.begin(), members.end(), [&](int a, int b) {
                if (first[a] != first[b]) return first[a] < first[b];
                return by_deg_id(a, b);
            });
        }
        for (int w : members) {
            number[w] = next_number++;
            out.push_back(w);
        }
    }
}

std::vector<int> gps(int n, const std::vector<std::pair<int, int>>& edges) {
    Graph g(n);
    for (auto& e : edges)
        if (e.first != e.second) {
            g.adj[e.first].push_back(e.second);
            g.adj[e.second].push_back(e.first);
        }
    g.finish();
    std::vector<int> comp(n, -1), out;
    int cid = 0;
    for (int s = 0; s < n; ++s) {
        if (comp[s] >= 0 || g.adj[s].empty()) continue;
        std::vector<int> nodes, stack{s};
        comp[s] = cid;
        while (!stack.empty()) {
            int x = stack.back();
            stack.pop_back();
            nodes.push_back(x);
            for (int y : g.adj[x])
                if (comp[y] < 0) {
                    comp[y] = cid;
                    stack.push_back(y);
                }
        }
        order_component(g, nodes, comp, cid, out);
        ++cid;
    }
    return out;
}

thread_local std::string t_msg;

}  // namespace

struct cm_schedule {
    struct Row {
        int32_t iteration;
        std::vector<int32_t> load, free_ids;
        std::vector<int64_t> pairs;
    };
    std::vector<Row> rows;
    int32_t iterations = 0;
    std::vector<cm_pair> pairs;   // the caller's pair list the rows index (cm_index_workspace_bytes)
};

namespace cm {
const cm_pair* schedule_pairs(const cm_schedule* s, int64_t* n) {
    *n = (int64_t)s->pairs.size();
    return s->pairs.data();
}
}  // namespace cm

// Error text is routed through cm_last_error by a small shim in cm_api.cpp.
extern "C" cm_status cm_internal_fail(cm_status st, const char* msg);

static cm_status sfail(cm_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return cm_internal_fail(st, buf);
}

extern "C" cm_status cm_gps_order(int32_t n, int64_t n_edges, const int32_t* edges, int32_t* order,
                                  int32_t* n_order) {
    if (n < 0 || n_edges < 0 || (n_edges && !edges) || !order || !n_order)
        return sfail(CM_ERR_INVALID, "cm_gps_order: bad argument");
    std::vector<std::pair<int, int>> e((size_t)n_edges);
    for (int64_t k = 0; k < n_edges; ++k) {
        const int a = edges[2 * k], b = edges[2 * k + 1];
        if (a < 0 || b < 0 || a >= n || b >= n) return sfail(CM_ERR_INVALID, "cm_gps_order: edge %lld out of range", (long long)k);
        e[k] = {a, b};
    }
    std::vector<int> o = gps(n, e);
    std::copy(o.begin(), o.end(), order);
    *n_order = (int32_t)o.size();
    return CM_OK;
}

extern "C" cm_status cm_schedule_blocks(const cm_pair* pairs, int64_t n_pairs, int32_t n_images,
                                        const int32_t* n_desc, const cm_params* p, uint64_t budget,
                                        int32_t max_images_per_block, cm_schedule** out) {
    if (!out || n_pairs < 0 || (n_pairs && !pairs) || n_images < 1 || !n_desc || max_images_per_block < 1)
        return sfail(CM_ERR_INVALID, "cm_schedule_blocks: bad argument");
    std::vector<uint64_t> nbytes(n_images);
    for (int i = 0; i < n_images; ++i) {
        cm_status st = cm_image_bytes(p, n_desc[i], &nbytes[i]);
        if (st != CM_OK) return st;
    }
    // step (1): symmetric adjacency; an edge carries every input pair on it.  The
    // pairs sorted by edge (min, max, then pair id): edge e owns pair ids
    // epair[ebeg[e] .. ebeg[e+1]), edges in (min, max) order.
    std::vector<std::pair<uint64_t, int64_t>> keyed((size_t)n_pairs);
    for (int64_t k = 0; k < n_pairs; ++k) {
        const int a = pairs[k].i, b = pairs[k].j;
        if (a < 0 || b < 0 || a >= n_images || b >= n_images)
            return sfail(CM_ERR_INVALID, "schedule: pair %lld has an image id out of range", (long long)k);
        if (a == b) return sfail(CM_ERR_INVALID, "schedule: pair %lld matches image %d with itself", (long long)k, a);
        if (nbytes[a] + nbytes[b] > budget)
            return sfail(CM_ERR_BUDGET, "schedule: pair %lld (%d,%d) needs %llu bytes, budget %llu", (long long)k, a, b,
                         (unsigned long long)(nbytes[a] + nbytes[b]), (unsigned long long)budget);
        keyed[(size_t)k] = {((uint64_t)std::min(a, b) << 32) | (uint64_t)std::max(a, b), k};
    }
    std::sort(keyed.begin(), keyed.end());
    std::vector<std::pair<int, int>> edge;   // (min, max) per edge
    std::vector<int64_t> ebeg, epair((size_t)n_pairs);
    for (size_t q = 0; q < keyed.size(); ++q) {
        if (q == 0 || keyed[q].first != keyed[q - 1].first) {
            edge.push_back({(int)(keyed[q].first >> 32), (int)(keyed[q].first & 0xFFFFFFFFu)});
            ebeg.push_back((int64_t)q);
        }
        epair[q] = keyed[q].second;
    }
    ebeg.push_back((int64_t)keyed.size());
    const int n_edges = (int)edge.size();
    cm_schedule* s = new (std::nothrow) cm_schedule();
    if (!s) return sfail(CM_ERR_NOMEM, "schedule: host allocation");
    s->pairs.assign(pairs, pairs + n_pairs);
    std::vector<char> alive((size_t)n_edges, 1);   // not yet placed in a row
    int n_remaining = n_edges;
    auto edge_pair_ids = [&](int e, std::vector<int64_t>& dst) {
        dst.insert(dst.end(), epair.begin() + ebeg[e], epair.begin() + ebeg[e + 1]);
    };
    int it = 0;
    while (n_remaining > 0) {
        // step (2): GPS permutation of the remaining graph
        std::vector<std::pair<int, int>> E;
        E.reserve((size_t)n_remaining);
        for (int e = 0; e < n_edges; ++e)
            if (alive[e]) E.push_back(edge[e]);
        const std::vector<int> order = gps(n_images, E);
        // step (3): chunks and block rows
        std::vector<std::vector<int>> chunks;
        std::vector<int> cur;
        uint64_t cur_bytes = 0;
        for (int w : order) {
            const uint64_t b = nbytes[w];
            if (!cur.empty() && ((int)cur.size() >= max_images_per_block || cur_bytes + b > budget / 2)) {
                chunks.push_back(cur);
                cur.clear();
                cur_bytes = 0;
            }
            cur.push_back(w);
            cur_bytes += b;
        }
        if (!cur.empty()) chunks.push_back(cur);
        const int nc = (int)chunks.size();
        std::vector<int> chunk_of(n_images, -1);
        std::vector<uint64_t> chunk_bytes(nc, 0);
        for (int c = 0; c < nc; ++c)
            for (int w : chunks[c]) {
                chunk_of[w] = c;
                chunk_bytes[c] += nbytes[w];
            }
        // edges by their lower chunk: (upper chunk, edge id), in edge order
        std::vector<std::vector<std::pair<int, int>>> by_lower(nc);
        for (int e = 0; e < n_edges; ++e)
            if (alive[e]) {
                const int ca = chunk_of[edge[e].first], cb = chunk_of[edge[e].second];
                by_lower[std::min(ca, cb)].push_back({std::max(ca, cb), e});
            }
        std::vector<int> resident;
        std::vector<char> is_res(n_images, 0);
        int64_t placed = 0;
        for (int r = 0; r < nc; ++r) {
            int hi = r;
            uint64_t tot = chunk_bytes[r];
            while (hi + 1 < nc && tot + chunk_bytes[hi + 1] <= budget) {
                ++hi;
                tot += chunk_bytes[hi];
            }
            cm_schedule::Row row;
            row.iteration = it;
            for (int c = r; c <= hi; ++c)
                for (int w : chunks[c])
                    if (!is_res[w]) {
                        row.load.push_back(w);
                        resident.push_back(w);
                        is_res[w] = 1;
                    }
            for (auto& ce : by_lower[r])
                if (ce.first <= hi) {
                    edge_pair_ids(ce.second, row.pairs);
                    alive[ce.second] = 0;
                    --n_remaining;
                    ++placed;
                }
            std::sort(row.pairs.begin(), row.pairs.end());
            // step (4) / Sec. 2.3.2 step (3): free the first block; everything after the last row
            std::vector<int> freed = (r == nc - 1) ? resident : chunks[r];
            for (int w : freed) is_res[w] = 0;
            std::vector<int> keep;
            for (int w : resident)
                if (is_res[w]) keep.push_back(w);
            resident.swap(keep);
            row.free_ids.assign(freed.begin(), freed.end());
            s->rows.push_back(std::move(row));
        }
        if (placed == 0) {
            for (int e = 0; e < n_edges; ++e) {
                if (!alive[e]) continue;
                cm_schedule::Row row;
                row.iteration = it;
                row.load = {edge[e].first, edge[e].second};
                row.free_ids = {edge[e].first, edge[e].second};
                edge_pair_ids(e, row.pairs);
                std::sort(row.pairs.begin(), row.pairs.end());
                s->rows.push_back(std::move(row));
                alive[e] = 0;
            }
            n_remaining = 0;
        }
        ++it;
    }
    s->iterations = it;
    *out = s;
    return CM_OK;
}

// A schedule from the caller's rows (another strategy than the MBR blocks),
// checked by replaying its residency: a row may load only images that are
// not resident and free only resident ones, both images of each of its pairs
// must be resident while it runs, and every pair index appears in exactly one
// row.  Images still resident after the last row are allowed (cm_run_schedule
// releases them).
extern "C" cm_status cm_schedule_from_rows(int32_t n_rows, const cm_schedule_row* rows, const cm_pair* pairs,
                                           int64_t n_pairs, int32_t n_images, cm_schedule** out) {
    if (!out || n_rows < 0 || (n_rows && !rows) || n_pairs < 0 || (n_pairs && !pairs) || n_images < 0)
        return sfail(CM_ERR_INVALID, "schedule_from_rows: bad argument");
    *out = nullptr;
    std::vector<char> res((size_t)n_images, 0), seen((size_t)n_pairs, 0);
    auto s = std::make_unique<cm_schedule>();
    s->rows.resize((size_t)n_rows);
    s->pairs.assign(pairs, pairs + n_pairs);
    int32_t iters = 0;
    for (int32_t r = 0; r < n_rows; ++r) {
        const cm_schedule_row& R = rows[r];
        if (R.n_load < 0 || R.n_free < 0 || R.n_pairs < 0 || (R.n_load && !R.load) || (R.n_free && !R.free_ids) ||
            (R.n_pairs && !R.pairs))
            return sfail(CM_ERR_INVALID, "schedule_from_rows: row %d is malformed", r);
        for (int k = 0; k < R.n_load; ++k) {
            const int32_t i = R.load[k];
            if (i < 0 || i >= n_images) return sfail(CM_ERR_INVALID, "schedule_from_rows: row %d loads image %d", r, i);
            if (res[i]) return sfail(CM_ERR_INVALID, "schedule_from_rows: row %d loads resident image %d", r, i);
            res[i] = 1;
        }
        for (int64_t k = 0; k < R.n_pairs; ++k) {
            const int64_t id = R.pairs[k];
            if (id < 0 || id >= n_pairs || seen[id])
                return sfail(CM_ERR_INVALID, "schedule_from_rows: row %d: pair %lld out of range or repeated", r,
                             (long long)id);
            seen[id] = 1;
            const cm_pair pr = pairs[id];
            if (pr.i < 0 || pr.j < 0 || pr.i >= n_images || pr.j >= n_images || pr.i == pr.j)
                return sfail(CM_ERR_INVALID, "schedule_from_rows: pair %lld is invalid", (long long)id);
            if (!res[pr.i] || !res[pr.j])
                return sfail(CM_ERR_INVALID, "schedule_from_rows: row %d matches pair %lld without its images resident",
                             r, (long long)id);
        }
        for (int k = 0; k < R.n_free; ++k) {
            const int32_t i = R.free_ids[k];
            if (i < 0 || i >= n_images || !res[i])
                return sfail(CM_ERR_INVALID, "schedule_from_rows: row %d frees image %d that is not resident", r, i);
            res[i] = 0;
        }
        auto& D = s->rows[r];
        D.iteration = R.iteration;
        D.load.assign(R.load, R.load + R.n_load);
        D.free_ids.assign(R.free_ids, R.free_ids + R.n_free);
        D.pairs.assign(R.pairs, R.pairs + R.n_pairs);
        iters = std::max(iters, R.iteration + 1);
    }
    for (int64_t k = 0; k < n_pairs; ++k)
        if (!seen[k]) return sfail(CM_ERR_INVALID, "schedule_from_rows: pair %lld is in no row", (long long)k);
    s->iterations = iters;
    *out = s.release();
    return CM_OK;
}

extern "C" int32_t cm_schedule_num_rows(const cm_schedule* s) { return s ? (int32_t)s->rows.size() : -1; }
extern "C" int32_t cm_schedule_num_iterations(const cm_schedule* s) { return s ? s->iterations : -1; }

extern "C" cm_status cm_schedule_get_row(const cm_schedule* s, int32_t r, cm_schedule_row* row) {
    if (!s || !row || r < 0 || r >= (int32_t)s->rows.size()) return sfail(CM_ERR_INVALID, "schedule_get_row: bad row");
    const auto& R = s->rows[r];
    row->iteration = R.iteration;
    row->n_load = (int32_t)R.load.size();
    row->load = R.load.data();
    row->n_free = (int32_t)R.free_ids.size();
    row->free_ids = R.free_ids.data();
    row->n_pairs = (int64_t)R.pairs.size();
    row->pairs = R.pairs.data();
    return CM_OK;
}

extern "C" void cm_free_schedule(cm_schedule* s) { delete s; }
