// Block-row pipeline (Sec. 2.3.2, Algorithm 1), the captured device-resident
// block sequence (one CUDA graph), and the host-side geometric verification
// (affine RANSAC) that consumes the initial matches.
//
// Pipeline, per block row r of a schedule, all device work on one stream:
//   load the row's new images (H2D, hash, buckets) -> one fused match launch
//   over the row's pairs -> compaction, whose scatter writes the per-pair match
//   lists straight into mapped pinned host memory (only the matches cross the
//   bus) -> release the row's freed images (host bookkeeping; stream order
//   keeps a later load from overwriting data still being read).
// Two host result buffers alternate between rows.  Worker threads wait on the
// row's completion event, then verify its pairs while the stream runs ahead.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <string>
#include <algorithm>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "cm_host.h"

#define fail ::cm::host_fail

// ---------------------------------------------------------------------------
// captured sequence
// ---------------------------------------------------------------------------
struct cm_sequence {
    cm_index* ix = nullptr;
    uint64_t generation = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int32_t kernels = 0;
};

void cm_sequence_detach(cm_sequence* q) { q->ix = nullptr; }

extern "C" cm_status cm_sequence_create(cm_index* ix, int32_t rehash, int32_t n_plans, cm_match_plan* const* plans,
                                        const cm_match_out* outs, const cm_compact_out* compacts, cm_stream stream,
                                        cm_sequence** out) {
    if (!ix || !out || n_plans < 0 || (n_plans && (!plans || !outs)))
        return fail(CM_ERR_INVALID, "cm_sequence_create: bad argument");
    if (!stream) return fail(CM_ERR_INVALID, "cm_sequence_create: capture needs a stream other than the legacy default");
    for (int k = 0; k < n_plans; ++k) {
        if (!plans[k] || plans[k]->ix != ix)
            return fail(CM_ERR_STATE, "cm_sequence_create: plan %d is NULL, detached or of another index", k);
        if (!outs[k].best_j && plans[k]->rows) return fail(CM_ERR_INVALID, "cm_sequence_create: outs[%d].best_j NULL", k);
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    std::unique_ptr<cm_sequence> q(new (std::nothrow) cm_sequence());
    if (!q) return fail(CM_ERR_NOMEM, "cm_sequence_create: host allocation");
    CM_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    cm_status st = CM_OK;
    if (rehash) st = cm_index_rehash(ix, stream);
    for (int k = 0; k < n_plans && st == CM_OK; ++k) {
        st = cm_match_plan_run(plans[k], &outs[k], stream);
        if (st == CM_OK && compacts && compacts[k].counts)
            st = cm_match_plan_compact(plans[k], outs[k].best_j, compacts[k].counts, compacts[k].offsets,
                                       compacts[k].total, compacts[k].matches, compacts[k].capacity, stream);
    }
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(s, &g);  // always leave capture mode
    if (st != CM_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (ce != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail(CM_ERR_CUDA, "cm_sequence_create: capture failed: %s", cudaGetErrorString(ce));
    }
    q->graph = g;
    size_t n_nodes = 0;
    CM_CUDA(cudaGraphGetNodes(g, nullptr, &n_nodes));
    std::vector<cudaGraphNode_t> nodes(n_nodes);
    if (n_nodes) CM_CUDA(cudaGraphGetNodes(g, nodes.data(), &n_nodes));
    for (auto n : nodes) {
        cudaGraphNodeType t;
        CM_CUDA(cudaGraphNodeGetType(n, &t));
        q->kernels += t == cudaGraphNodeTypeKernel;
    }
    const cudaError_t ie = cudaGraphInstantiate(&q->exec, g, 0);
    if (ie != cudaSuccess) {
        cudaGraphDestroy(g);
        q->graph = nullptr;
        return fail(CM_ERR_CUDA, "cm_sequence_create: instantiation failed: %s", cudaGetErrorString(ie));
    }
    q->ix = ix;
    q->generation = ix->generation;
    ix->seqs.insert(q.get());
    *out = q.release();
    return CM_OK;
}

extern "C" cm_status cm_sequence_launch(cm_sequence* q, cm_stream stream) {
    if (!q) return fail(CM_ERR_INVALID, "cm_sequence_launch: NULL");
    if (!q->ix) return fail(CM_ERR_STATE, "cm_sequence_launch: the index was destroyed");
    if (q->ix->generation != q->generation)
        return fail(CM_ERR_STATE, "cm_sequence_launch: residency or plans changed since capture; capture again");
    CM_CUDA(cudaGraphLaunch(q->exec, reinterpret_cast<cudaStream_t>(stream)));
    return CM_OK;
}

extern "C" int32_t cm_sequence_kernels(const cm_sequence* q) { return q ? q->kernels : -1; }

extern "C" void cm_sequence_destroy(cm_sequence* q) {
    if (!q) return;
    if (q->ix) q->ix->seqs.erase(q);
    if (q->exec) cudaGraphExecDestroy(q->exec);
    if (q->graph) cudaGraphDestroy(q->graph);
    delete q;
}

// ---------------------------------------------------------------------------
// affine RANSAC (host)
// ---------------------------------------------------------------------------
namespace {

uint64_t mix64(uint64_t z) {  // splitmix64 finaliser
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Solves the 3x3 system M a = r (Cramer's rule); false when |det| is tiny
// against the entries' scale (a near-collinear sample).
bool solve3(const double M[3][3], const double r[3], double a[3]) {
    const double det = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
                       M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                       M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
    double scale = 0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) scale = std::max(scale, std::fabs(M[i][j]));
    if (!(std::fabs(det) > 1e-9 * scale * scale * scale)) return false;
    for (int c = 0; c < 3; ++c) {
        double T[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) T[i][j] = j == c ? r[i] : M[i][j];
        a[c] = (T[0][0] * (T[1][1] * T[2][2] - T[1][2] * T[2][1]) - T[0][1] * (T[1][0] * T[2][2] - T[1][2] * T[2][0]) +
                T[0][2] * (T[1][0] * T[2][1] - T[1][1] * T[2][0])) / det;
    }
    return true;
}

struct Corr {
    double x, y, u, v;
};

int64_t count_inliers(const std::vector<Corr>& c, const double A[6], double t2, uint8_t* mask) {
    int64_t n = 0;
    for (size_t k = 0; k < c.size(); ++k) {
        const double du = A[0] * c[k].x + A[1] * c[k].y + A[2] - c[k].u;
        const double dv = A[3] * c[k].x + A[4] * c[k].y + A[5] - c[k].v;
        const bool in = du * du + dv * dv <= t2;
        if (mask) mask[k] = in;
        n += in;
    }
    return n;
}

// Least-squares affine map over the correspondences flagged in mask.
bool refit(const std::vector<Corr>& c, const uint8_t* mask, double A[6]) {
    double M[3][3] = {}, ru[3] = {}, rv[3] = {};
    for (size_t k = 0; k < c.size(); ++k) {
        if (!mask[k]) continue;
        const double p[3] = {c[k].x, c[k].y, 1.0};
        for (int i = 0; i < 3; ++i) {
            for (int j = 0; j < 3; ++j) M[i][j] += p[i] * p[j];
            ru[i] += p[i] * c[k].u;
            rv[i] += p[i] * c[k].v;
        }
    }
    double a[3], b[3];
    if (!solve3(M, ru, a) || !solve3(M, rv, b)) return false;
    for (int i = 0; i < 3; ++i) {
        A[i] = a[i];
        A[3 + i] = b[i];
    }
    return true;
}

}  // namespace

extern "C" cm_status cm_verify_affine(const float* kp_i, const float* kp_j, int64_t n_matches, const uint32_t* matches,
                                      float thresh_px, int32_t max_iters, uint64_t seed, float* A_out,
                                      uint8_t* inlier_mask, int64_t* n_inliers) {
    if (n_matches < 0 || (n_matches && (!kp_i || !kp_j || !matches)) || !(thresh_px > 0.f) || max_iters < 1)
        return fail(CM_ERR_INVALID, "cm_verify_affine: bad argument");
    std::vector<Corr> c((size_t)n_matches);
    for (int64_t k = 0; k < n_matches; ++k) {
        const uint32_t q = matches[k] >> 16, j = matches[k] & 0xFFFFu;
        c[k] = {kp_i[2 * q], kp_i[2 * q + 1], kp_j[2 * j], kp_j[2 * j + 1]};
    }
    const double t2 = (double)thresh_px * thresh_px;
    double best[6] = {0, 0, 0, 0, 0, 0};
    int64_t best_n = 0;
    if (n_matches >= 3) {
        int64_t need = max_iters;
        for (int64_t it = 0; it < need && it < max_iters; ++it) {
            int64_t s[3];
            uint64_t r = seed * 0x2545F4914F6CDD1Dull + (uint64_t)it;
            for (int d = 0; d < 3; ++d) {  // three distinct indices
                for (;;) {
                    r = mix64(r);
                    s[d] = (int64_t)(r % (uint64_t)n_matches);
                    bool dup = false;
                    for (int e = 0; e < d; ++e) dup |= s[e] == s[d];
                    if (!dup) break;
                }
            }
            double M[3][3], ru[3], rv[3], a[3], b[3];
            for (int d = 0; d < 3; ++d) {
                M[d][0] = c[s[d]].x;
                M[d][1] = c[s[d]].y;
                M[d][2] = 1.0;
                ru[d] = c[s[d]].u;
                rv[d] = c[s[d]].v;
            }
            if (!solve3(M, ru, a) || !solve3(M, rv, b)) continue;
            const double A[6] = {a[0], a[1], a[2], b[0], b[1], b[2]};
            const int64_t n = count_inliers(c, A, t2, nullptr);
            if (n > best_n) {
                best_n = n;
                std::copy(A, A + 6, best);
                // samples needed for p = 0.999 of drawing an all-inlier triple at this share
                const double w = (double)n / (double)n_matches, w3 = w * w * w;
                if (w3 >= 1.0) need = it + 1;
                else if (w3 > 0.0) need = std::min<int64_t>(max_iters, (int64_t)std::ceil(std::log(1e-3) / std::log1p(-w3)));
            }
        }
        if (best_n >= 3) {
            std::vector<uint8_t> mask((size_t)n_matches);
            count_inliers(c, best, t2, mask.data());
            double R[6];
            if (refit(c, mask.data(), R)) {
                const int64_t n = count_inliers(c, R, t2, nullptr);
                if (n >= best_n) {
                    best_n = n;
                    std::copy(R, R + 6, best);
                }
            }
        }
    }
    if (inlier_mask) {
        if (best_n) count_inliers(c, best, t2, inlier_mask);
        else std::fill(inlier_mask, inlier_mask + n_matches, (uint8_t)0);
    }
    if (A_out)
        for (int i = 0; i < 6; ++i) A_out[i] = (float)best[i];
    if (n_inliers) *n_inliers = best_n;
    return CM_OK;
}

extern "C" int32_t cm_affine_verify_cb(void* user, int32_t, int64_t pair_id, const cm_pair* pair, int64_t n_matches,
                                       const uint32_t* matches) {
    auto* v = static_cast<cm_affine_verifier*>(user);
    const float *ki = v->keypoints[pair->i], *kj = v->keypoints[pair->j];
    std::vector<uint32_t> kept;
    if (v->sao_k > 0) {   // local constraint first, RANSAC on the survivors
        std::vector<uint8_t> keep((size_t)n_matches);
        int64_t nk = 0;
        if (cm_sao_filter(ki, kj, n_matches, matches, v->sao_k, v->sao_max_score, nullptr, keep.data(), &nk) != CM_OK)
            return 1;
        kept.reserve((size_t)nk);
        for (int64_t m = 0; m < n_matches; ++m)
            if (keep[m]) kept.push_back(matches[m]);
        if (v->sao_kept) v->sao_kept[pair_id] = nk;
        matches = kept.data();
        n_matches = nk;
    }
    int64_t n = 0;
    if (cm_verify_affine(ki, kj, n_matches, matches, v->thresh_px, v->max_iters, v->seed ^ (uint64_t)pair_id, nullptr,
                         nullptr, &n) != CM_OK)
        return 1;
    if (v->inliers) v->inliers[pair_id] = n;
    return 0;
}

// ---------------------------------------------------------------------------
// block-row pipeline
// ---------------------------------------------------------------------------
namespace {

struct WorkLayout {
    uint64_t best_j, counts, offsets, sao, sao_bytes, stage, stage_bytes, total;
};
constexpr uint64_t kCentreStage = 64ull << 20;   // staging block of the pipeline's own centring pass

// Workspace of the largest row: best_j per query, counts and offsets (+ total)
// per pair, and, with the GPU SAO constraint, its compaction scratch.
WorkLayout work_layout(int64_t max_rows, int64_t max_pairs, bool sao, bool centre) {
    WorkLayout w{};
    uint64_t o = 0;
    auto take = [&](uint64_t bytes) { uint64_t at = o; o = align_up(o + bytes); return at; };
    w.best_j = take((uint64_t)std::max<int64_t>(max_rows, 1) * 4);
    w.counts = take((uint64_t)std::max<int64_t>(max_pairs, 1) * 4);
    w.offsets = take((uint64_t)(max_pairs + 1) * 8);  // the total sits right after the offsets
    w.sao_bytes = sao ? sao_work_bytes(max_pairs, max_rows) : 0;
    w.sao = take(w.sao_bytes);
    w.stage_bytes = centre ? kCentreStage : 0;
    w.stage = take(w.stage_bytes);
    w.total = o;
    return w;
}

bool sao_on(const cm_pipeline_opts* o) { return o && o->sao_k > 0; }
bool centre_on(const cm_pipeline_opts* o) { return o && o->centre; }

cm_status row_sizes(const cm_index* ix, const cm_schedule* s, const cm_pair* pairs, int64_t n_pairs, int64_t* max_rows,
                    int64_t* max_pairs, uint64_t* max_plan = nullptr) {
    const int32_t R = cm_schedule_num_rows(s);
    *max_rows = *max_pairs = 0;
    if (max_plan) *max_plan = 0;
    for (int32_t r = 0; r < R; ++r) {
        cm_schedule_row row{};
        cm_status st = cm_schedule_get_row(s, r, &row);
        if (st != CM_OK) return st;
        int64_t q = 0;
        int32_t max_ni = 0;
        for (int64_t k = 0; k < row.n_pairs; ++k) {
            const int64_t id = row.pairs[k];
            if (id < 0 || id >= n_pairs) return fail(CM_ERR_INVALID, "pipeline: schedule names pair %lld of %lld",
                                                     (long long)id, (long long)n_pairs);
            const int i = pairs[id].i;
            if (i < 0 || i >= ix->n_images) return fail(CM_ERR_INVALID, "pipeline: pair %lld has a bad image id", (long long)id);
            q += ix->n_desc[i];
            max_ni = std::max(max_ni, ix->n_desc[i]);
        }
        *max_rows = std::max(*max_rows, q);
        *max_pairs = std::max<int64_t>(*max_pairs, row.n_pairs);
        if (max_plan && row.n_pairs) *max_plan = std::max(*max_plan, plan_bytes(&ix->p, row.n_pairs, q, max_ni));
    }
    return CM_OK;
}

using Clock = std::chrono::steady_clock;
double ms_since(Clock::time_point t0) { return std::chrono::duration<double, std::milli>(Clock::now() - t0).count(); }

constexpr int kBufs = 2;  // host result buffers (rows in flight between GPU and verification)

struct HostBuf {
    uint64_t* offsets = nullptr;  // pinned [max_pairs + 1]
    uint32_t* matches = nullptr;  // mapped pinned [max_rows]
    uint32_t* d_matches = nullptr;
    bool busy = false;
};

struct RowJob {
    int32_t row = 0;
    int b = 0;
    int64_t n = 0;                // pairs still to be claimed up to n (cut short on abort)
    const int64_t* ids = nullptr;
    cudaEvent_t done = nullptr;
    int64_t next = 0, finished = 0;
    bool synced = false, popped = false;
};

struct Pipe {
    std::mutex mu;
    std::condition_variable cv_job, cv_buf;
    std::deque<RowJob*> queue;
    HostBuf buf[kBufs];
    bool stop = false;
    bool abort = false;
    int64_t matches = 0;
    double verify_ms = 0;
    const cm_pair* pairs = nullptr;
    cm_verify_fn verify = nullptr;
    void* user = nullptr;
    std::string err;

    // All members are guarded by mu.  A row's buffer is released exactly once:
    // when the row is popped with every claimed pair finished, or by the last
    // pair to finish after the pop.
    void release(RowJob* j) {
        buf[j->b].busy = false;
        cv_buf.notify_all();
    }

    void set_abort(const std::string& why) {
        if (!abort) err = why;
        abort = true;
        cv_buf.notify_all();
    }

    void worker() {
        double my_ms = 0;
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
            cv_job.wait(lk, [&] { return stop || !queue.empty(); });
            if (queue.empty()) break;  // stop requested and nothing left
            RowJob* j = queue.front();
            if (!j->synced) {
                lk.unlock();
                const cudaError_t e = cudaEventSynchronize(j->done);
                lk.lock();
                if (e != cudaSuccess) set_abort(std::string("pipeline: row completion: ") + cudaGetErrorString(e));
                if (!j->synced) {
                    j->synced = true;
                    if (e == cudaSuccess) matches += (int64_t)buf[j->b].offsets[j->n];
                }
                continue;
            }
            if (abort) j->n = j->next;  // claimed pairs finish, the rest are skipped
            if (j->next == j->n) {
                queue.pop_front();
                j->popped = true;
                if (j->finished == j->n) release(j);
                continue;
            }
            const int64_t k = j->next++;
            const HostBuf& hb = buf[j->b];
            lk.unlock();
            int32_t rc = 0;
            if (verify) {
                const auto t0 = Clock::now();
                const int64_t id = j->ids[k];
                const uint64_t o0 = hb.offsets[k], o1 = hb.offsets[k + 1];
                rc = verify(user, j->row, id, &pairs[id], (int64_t)(o1 - o0), hb.matches + o0);
                my_ms += ms_since(t0);
            }
            lk.lock();
            if (rc) set_abort("pipeline: the verification callback returned " + std::to_string(rc));
            if (++j->finished == j->n && j->popped) release(j);
        }
        verify_ms += my_ms;
    }
};

}  // namespace

extern "C" cm_status cm_schedule_arena_bytes(const cm_schedule* s, const cm_params* p, int32_t n_images,
                                             const int32_t* n_desc, const cm_pair* pairs, int64_t n_pairs,
                                             uint64_t* bytes) {
    cm_status st = cm_params_check(p);
    if (st != CM_OK) return st;
    if (!s || !bytes || n_images < 0 || (n_images && !n_desc) || n_pairs < 0 || (n_pairs && !pairs))
        return fail(CM_ERR_INVALID, "cm_schedule_arena_bytes: bad argument");
    std::vector<char> res(n_images, 0);
    uint64_t cur = 0, peak = 0, largest = 0, plan = 0;
    const int32_t R = cm_schedule_num_rows(s);
    // bytes each row loads: cm_run_schedule places row r+1's loads while row r
    // is still resident, to copy them during row r
    std::vector<uint64_t> load_bytes(R + 1, 0);
    for (int32_t r = 0; r < R; ++r) {
        cm_schedule_row row{};
        if ((st = cm_schedule_get_row(s, r, &row)) != CM_OK) return st;
        for (int k = 0; k < row.n_load; ++k) {
            const int i = row.load[k];
            if (i < 0 || i >= n_images) return fail(CM_ERR_INVALID, "cm_schedule_arena_bytes: image %d", i);
            load_bytes[r] += align_up(slot_layout(p, n_desc[i], false).total);
        }
    }
    for (int32_t r = 0; r < R; ++r) {
        cm_schedule_row row{};
        if ((st = cm_schedule_get_row(s, r, &row)) != CM_OK) return st;
        for (int k = 0; k < row.n_load; ++k) {
            const int i = row.load[k];
            const uint64_t b = align_up(slot_layout(p, n_desc[i], false).total);
            if (!res[i]) cur += b;
            res[i] = 1;
            largest = std::max(largest, b);
        }
        peak = std::max(peak, cur + load_bytes[r + 1]);
        int64_t rows = 0;
        int32_t max_ni = 0;
        for (int64_t k = 0; k < row.n_pairs; ++k) {
            const int64_t id = row.pairs[k];
            if (id < 0 || id >= n_pairs || pairs[id].i < 0 || pairs[id].i >= n_images)
                return fail(CM_ERR_INVALID, "cm_schedule_arena_bytes: pair %lld", (long long)id);
            rows += n_desc[pairs[id].i];
            max_ni = std::max(max_ni, n_desc[pairs[id].i]);
        }
        plan = std::max(plan, plan_bytes(p, row.n_pairs, rows, max_ni));
        for (int k = 0; k < row.n_free; ++k) {
            const int i = row.free_ids[k];
            if (i >= 0 && i < n_images && res[i]) {
                cur -= align_up(slot_layout(p, n_desc[i], false).total);
                res[i] = 0;
            }
        }
    }
    // first-fit placement of unequal slots can fragment: 1/8 of the peak plus the largest slot of margin
    *bytes = fixed_layout(p, n_images).total + peak + peak / 8 + largest + plan + 64 * kAlign;
    return CM_OK;
}

extern "C" cm_status cm_pipeline_workspace_bytes_ex(const cm_index* ix, const cm_schedule* s, const cm_pair* pairs,
                                                    int64_t n_pairs, const cm_pipeline_opts* opts, uint64_t* bytes) {
    if (!ix || !s || !bytes || n_pairs < 0 || (n_pairs && !pairs))
        return fail(CM_ERR_INVALID, "cm_pipeline_workspace_bytes: bad argument");
    int64_t mr = 0, mp = 0;
    cm_status st = row_sizes(ix, s, pairs, n_pairs, &mr, &mp);
    if (st != CM_OK) return st;
    *bytes = work_layout(mr, mp, sao_on(opts), centre_on(opts)).total;
    return CM_OK;
}

extern "C" cm_status cm_pipeline_workspace_bytes(const cm_index* ix, const cm_schedule* s, const cm_pair* pairs,
                                                 int64_t n_pairs, uint64_t* bytes) {
    return cm_pipeline_workspace_bytes_ex(ix, s, pairs, n_pairs, nullptr, bytes);
}

extern "C" cm_status cm_run_schedule(cm_index* ix, const cm_schedule* s, const cm_pair* pairs, int64_t n_pairs,
                                     const uint8_t* const* desc_host, void* d_work, uint64_t work_bytes,
                                     cm_verify_fn verify, void* user, int32_t n_workers, cm_stream stream,
                                     cm_pipeline_stats* stats) {
    return cm_run_schedule_ex(ix, s, pairs, n_pairs, desc_host, d_work, work_bytes, verify, user, n_workers, nullptr,
                              stream, stats);
}

extern "C" cm_status cm_run_schedule_ex(cm_index* ix, const cm_schedule* s, const cm_pair* pairs, int64_t n_pairs,
                                        const uint8_t* const* desc_host, void* d_work, uint64_t work_bytes,
                                        cm_verify_fn verify, void* user, int32_t n_workers,
                                        const cm_pipeline_opts* opts, cm_stream stream, cm_pipeline_stats* stats) {
    const auto t_start = Clock::now();
    if (!ix || !s || !desc_host || !d_work || n_pairs < 0 || (n_pairs && !pairs) || n_workers < 1 || n_workers > 256)
        return fail(CM_ERR_INVALID, "cm_run_schedule: bad argument");
    if (sao_on(opts) && (opts->sao_k > 16 || !opts->d_kp || !opts->d_kp_off || !(opts->sao_max_score >= 0.f)))
        return fail(CM_ERR_INVALID, "cm_run_schedule: bad SAO options (1 <= sao_k <= 16, keypoints on the device)");
    if (!ix->mean_set && !centre_on(opts)) return fail(CM_ERR_STATE, "cm_run_schedule: centring mean not set");
    if (centre_on(opts))
        for (int i = 0; i < ix->n_images; ++i)
            if (ix->resident[i] || ix->pending[i])
                return fail(CM_ERR_STATE, "cm_run_schedule: centring from host rows needs an index with nothing resident");
    int64_t max_rows = 0, max_pairs = 0;
    uint64_t max_plan = 0;
    cm_status st = row_sizes(ix, s, pairs, n_pairs, &max_rows, &max_pairs, &max_plan);
    if (st != CM_OK) return st;
    const WorkLayout wl = work_layout(max_rows, max_pairs, sao_on(opts), centre_on(opts));
    if (work_bytes < wl.total)
        return fail(CM_ERR_BUDGET, "cm_run_schedule: workspace %llu bytes, %llu needed", (unsigned long long)work_bytes,
                    (unsigned long long)wl.total);
    uint8_t* work = static_cast<uint8_t*>(d_work);
    int32_t* d_best = reinterpret_cast<int32_t*>(work + wl.best_j);
    uint32_t* d_counts = reinterpret_cast<uint32_t*>(work + wl.counts);
    uint64_t* d_offsets = reinterpret_cast<uint64_t*>(work + wl.offsets);
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    const int32_t R = cm_schedule_num_rows(s);

    cm_pipeline_stats S{};
    S.workers = n_workers;
    Pipe P;
    P.pairs = pairs;
    P.verify = verify;
    P.user = user;
    std::vector<cudaEvent_t> ev_start(R, nullptr), ev_done(R, nullptr), ev_copied(R, nullptr);
    // row r's loads were placed and copied early: 1 during row r-1, 2 (row 0) by the centring pass
    std::vector<char> prefetched(R, 0);
    cudaStream_t cpy = nullptr;           // copies of the next row's descriptors
    cudaEvent_t ev_origin = nullptr;
    std::vector<std::unique_ptr<RowJob>> jobs;
    std::vector<int32_t> loaded_by_us;
    std::vector<std::thread> threads;

    // Everything acquired below is released at `done`, whatever happened.
    auto cleanup = [&]() {
        {
            std::lock_guard<std::mutex> lk(P.mu);
            P.stop = true;
        }
        P.cv_job.notify_all();
        for (auto& t : threads) t.join();
        cudaStreamSynchronize(cs);
        if (cpy) cudaStreamSynchronize(cpy);
        for (int32_t r = 0; r < R; ++r)   // slots placed for a row that never ran
            if (prefetched[r]) {
                cm_schedule_row row{};
                if (cm_schedule_get_row(s, r, &row) == CM_OK) index_cancel_prefetch(ix, row.n_load, row.load);
                prefetched[r] = 0;
            }
        if (ix->plan_reserve_bytes) {   // the rows' plans are gone: give the reserved block back
            ix->alloc.release(ix->plan_reserve_at);
            ix->plan_reserve_bytes = 0;
            ix->plan_reserve_busy = false;
        }
        for (auto e : ev_start) if (e) cudaEventDestroy(e);
        for (auto e : ev_done) if (e) cudaEventDestroy(e);
        for (auto e : ev_copied) if (e) cudaEventDestroy(e);
        if (ev_origin) cudaEventDestroy(ev_origin);
        if (cpy) cudaStreamDestroy(cpy);
    };
    auto bail = [&](cm_status code) {
        std::string msg = cm_last_error();
        {
            std::lock_guard<std::mutex> lk(P.mu);
            P.set_abort(msg);
        }
        cleanup();
        if (!loaded_by_us.empty())  // best effort: leave the index as it was found
            cm_index_evict(ix, (int32_t)loaded_by_us.size(), loaded_by_us.data(), stream);
        host_fail(code, "%s", msg.c_str());
        return code;
    };

    static_assert(kBufs == 2, "one cached pinned buffer per result buffer");
    for (int k = 0; k < kBufs; ++k) {   // the index's cached buffers, grown when this schedule needs more
        auto& c = ix->pinned[k];
        const size_t no = (size_t)(max_pairs + 1), nm = (size_t)std::max<int64_t>(max_rows, 1);
        bool ok = true;
        if (c.n_offsets < no) {
            if (c.offsets) cudaFreeHost(c.offsets);
            c.offsets = nullptr;
            c.n_offsets = 0;
            ok = cudaHostAlloc(reinterpret_cast<void**>(&c.offsets), no * 8, cudaHostAllocDefault) == cudaSuccess;
            if (ok) c.n_offsets = no;
        }
        if (ok && c.n_matches < nm) {
            if (c.matches) cudaFreeHost(c.matches);
            c.matches = c.d_matches = nullptr;
            c.n_matches = 0;
            ok = cudaHostAlloc(reinterpret_cast<void**>(&c.matches), nm * 4, cudaHostAllocMapped) == cudaSuccess &&
                 cudaHostGetDevicePointer(reinterpret_cast<void**>(&c.d_matches), c.matches, 0) == cudaSuccess;
            if (ok) c.n_matches = nm;
        }
        if (!ok) {
            fail(CM_ERR_NOMEM, "cm_run_schedule: pinned result buffers (%lld matches)", (long long)max_rows);
            return bail(CM_ERR_NOMEM);
        }
        P.buf[k].offsets = c.offsets;
        P.buf[k].matches = c.matches;
        P.buf[k].d_matches = c.d_matches;
    }
    for (int32_t r = 0; r < R; ++r)
        if (cudaEventCreate(&ev_start[r]) != cudaSuccess || cudaEventCreate(&ev_done[r]) != cudaSuccess ||
            cudaEventCreateWithFlags(&ev_copied[r], cudaEventDisableTiming) != cudaSuccess) {
            fail(CM_ERR_CUDA, "cm_run_schedule: event creation");
            return bail(CM_ERR_CUDA);
        }
    if (cudaStreamCreateWithFlags(&cpy, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev_origin, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(ev_origin, cs) != cudaSuccess) {
        fail(CM_ERR_CUDA, "cm_run_schedule: copy stream");
        return bail(CM_ERR_CUDA);
    }
    // Places row r+1's loads and copies their descriptors on the copy stream
    // while row r runs.  The copy waits for everything enqueued before row r
    // (ev_done[r-1]): the space it writes was freed by earlier rows, whose
    // readers all precede that event; row r's own images and plan are still
    // placed, so the new slots cannot overlap them.  No room, or an image that
    // row r frees and row r+1 loads again: row r+1 loads in order as usual.
    auto prefetch_next = [&](int32_t r) -> cm_status {
        if (r + 1 >= R) return CM_OK;
        cm_schedule_row next{};
        cm_status st2 = cm_schedule_get_row(s, r + 1, &next);
        if (st2 != CM_OK || !next.n_load) return st2;
        for (int k = 0; k < next.n_load; ++k) {   // an image row r frees and row r+1 loads again: load in order
            const int i = next.load[k];
            if (i < 0 || i >= ix->n_images || ix->resident[i] || ix->pending[i]) return CM_OK;
        }
        if (cudaStreamWaitEvent(cpy, r == 0 ? ev_origin : ev_done[r - 1], 0) != cudaSuccess)
            return fail(CM_ERR_CUDA, "cm_run_schedule: copy stream wait");
        std::vector<const uint8_t*> src(next.n_load);
        for (int k = 0; k < next.n_load; ++k) src[k] = desc_host[next.load[k]];
        bool placed = false;
        if ((st2 = index_prefetch(ix, next.n_load, next.load, src.data(), cpy, &placed)) != CM_OK) return st2;
        if (placed) {
            if (cudaEventRecord(ev_copied[r + 1], cpy) != cudaSuccess)
                return fail(CM_ERR_CUDA, "cm_run_schedule: event record");
            prefetched[r + 1] = 1;
        }
        return CM_OK;
    };
    // One block of the arena serves every row's plan in turn, placed before any
    // image of the run: plans then never fragment the space the images use.
    // No room: each plan is placed on its own as usual.
    if (max_plan && !ix->plan_reserve_bytes && ix->alloc.alloc(max_plan, &ix->plan_reserve_at)) {
        ix->plan_reserve_bytes = max_plan;
        ix->plan_reserve_busy = false;
    }
    // The run's own centring pass: row 0's images go straight into their slots
    // (summed there when they are published), every other image's rows pass
    // once through the workspace's staging block; each image is read from the
    // host once before its first hashing.
    if (centre_on(opts)) {
        bool kept0 = false;
        cm_schedule_row row0{};
        if (R > 0 && (st = cm_schedule_get_row(s, 0, &row0)) != CM_OK) return bail(st);
        std::vector<char> in0(ix->n_images, 0);
        if (R > 0 && row0.n_load) {
            std::vector<const uint8_t*> src(row0.n_load);
            for (int k = 0; k < row0.n_load; ++k) src[k] = desc_host[row0.load[k]];
            if ((st = index_prefetch(ix, row0.n_load, row0.load, src.data(), cs, &kept0)) != CM_OK) return bail(st);
            if (kept0) {
                prefetched[0] = 2;
                for (int k = 0; k < row0.n_load; ++k) in0[row0.load[k]] = 1;
            }
        }
        std::vector<int32_t> rest;
        for (int i = 0; i < ix->n_images; ++i)
            if (!in0[i]) rest.push_back(i);
        uint64_t rows_streamed = 0;
        if (cudaMemsetAsync(ix->arena + ix->fx.sums, 0, kDim * 8, cs) != cudaSuccess) {
            fail(CM_ERR_CUDA, "cm_run_schedule: clearing the sums");
            return bail(CM_ERR_CUDA);
        }
        if ((st = index_stream_sums(ix, (int32_t)rest.size(), rest.data(), desc_host, work + wl.stage, wl.stage_bytes,
                                    cs, &rows_streamed)) != CM_OK)
            return bail(st);
        S.h2d_bytes += rows_streamed * kDim;
        S.kernels += (int64_t)((rows_streamed * kDim + wl.stage_bytes - 1) / wl.stage_bytes);
        if (!kept0) {   // nothing kept: the mean is complete already
            uint64_t total = 0;
            for (int i = 0; i < ix->n_images; ++i) total += (uint64_t)ix->n_desc[i];
            if ((st = index_mean_from_sums(ix, total, cs)) != CM_OK) return bail(st);
            S.kernels += 1;
        } else {
            S.kernels += 2;   // the kept images' column sums and the mean, at publication
        }
    }
    for (int w = 0; w < n_workers; ++w) threads.emplace_back([&P] { P.worker(); });
    // hashing: (bias +) projection + buckets (+ the rerank row copies); matching: scan (+ tensor-core rerank)
    const int hash_kernels = (ix->p.projection == CM_PROJ_TC ? 3 : 2) + (tc_rerank(&ix->p) ? 1 : 0);
    const int match_kernels = needs_hand_over(&ix->p) ? 2 : 1;

    for (int32_t r = 0; r < R; ++r) {
        cm_schedule_row row{};
        if ((st = cm_schedule_get_row(s, r, &row)) != CM_OK) return bail(st);
        const int b = r % kBufs;
        {
            const auto t0 = Clock::now();
            std::unique_lock<std::mutex> lk(P.mu);
            P.cv_buf.wait(lk, [&] { return !P.buf[b].busy || P.abort; });
            if (P.abort) break;
            P.buf[b].busy = true;
            S.stall_ms += ms_since(t0);
        }
        if (cudaEventRecord(ev_start[r], cs) != cudaSuccess) {
            fail(CM_ERR_CUDA, "cm_run_schedule: event record");
            return bail(CM_ERR_CUDA);
        }
        // (1) the row's new images: copy, hash, buckets
        if (row.n_load) {
            std::vector<const uint8_t*> src(row.n_load);
            for (int k = 0; k < row.n_load; ++k) {
                src[k] = desc_host[row.load[k]];
                S.h2d_bytes += (uint64_t)ix->n_desc[row.load[k]] * kDim;
            }
            if (prefetched[r] == 2) {   // copied by the centring pass: sum, set the mean, hash
                if ((st = index_publish(ix, row.n_load, row.load, cs, true)) != CM_OK) return bail(st);
                prefetched[r] = 0;
            } else if (prefetched[r]) {   // copied during the previous row: make resident and hash
                S.prefetched_rows++;
                if (cudaStreamWaitEvent(cs, ev_copied[r], 0) != cudaSuccess) {
                    fail(CM_ERR_CUDA, "cm_run_schedule: stream wait");
                    return bail(CM_ERR_CUDA);
                }
                if ((st = index_publish(ix, row.n_load, row.load, cs)) != CM_OK) return bail(st);
                prefetched[r] = 0;
            } else if ((st = cm_index_load(ix, row.n_load, row.load, src.data(), CM_MEM_HOST, stream)) != CM_OK) {
                return bail(st);
            }
            loaded_by_us.insert(loaded_by_us.end(), row.load, row.load + row.n_load);
            S.kernels += hash_kernels;
        }
        // (2) one fused launch over the row's pairs, (3) compaction into host memory
        std::vector<cm_pair> rp((size_t)row.n_pairs);
        for (int64_t k = 0; k < row.n_pairs; ++k) rp[k] = pairs[row.pairs[k]];
        if (row.n_pairs) {
            cm_match_plan* pl = nullptr;
            if ((st = cm_match_plan_create(ix, rp.data(), row.n_pairs, stream, &pl)) != CM_OK) return bail(st);
            cm_match_out mo{};
            mo.best_j = d_best;
            st = cm_match_plan_run(pl, &mo, stream);
            if (st == CM_OK && sao_on(opts)) {   // local constraint on the GPU: rejected matches leave best_j
                st = cm_match_plan_sao(pl, d_best, d_best, opts->d_kp, opts->d_kp_off, opts->sao_k,
                                       opts->sao_max_score, nullptr, work + wl.sao, wl.sao_bytes, stream);
                S.kernels += 4;
            }
            if (st == CM_OK)
                st = cm_match_plan_compact(pl, d_best, d_counts, d_offsets, d_offsets + row.n_pairs, P.buf[b].d_matches,
                                           (uint64_t)pl->rows, stream);
            S.queries += pl->rows;
            S.kernels += (pl->n_items ? match_kernels : 0) + 3;
            if (st == CM_OK) st = prefetch_next(r);   // while this row's plan still holds its space
            cm_match_plan_destroy(pl);  // its table is reused only by work ordered after this row
            if (st != CM_OK) return bail(st);
            if (cudaMemcpyAsync(P.buf[b].offsets, d_offsets, (size_t)(row.n_pairs + 1) * 8, cudaMemcpyDeviceToHost,
                                cs) != cudaSuccess) {
                fail(CM_ERR_CUDA, "cm_run_schedule: offsets copy");
                return bail(CM_ERR_CUDA);
            }
            S.d2h_bytes += (uint64_t)(row.n_pairs + 1) * 8;
        } else {
            P.buf[b].offsets[0] = 0;
            if ((st = prefetch_next(r)) != CM_OK) return bail(st);
        }
        if (cudaEventRecord(ev_done[r], cs) != cudaSuccess) {
            fail(CM_ERR_CUDA, "cm_run_schedule: event record");
            return bail(CM_ERR_CUDA);
        }
        // (4) release the row's freed images (Sec. 2.3.2 step (3))
        if (row.n_free) {
            if ((st = cm_index_evict(ix, row.n_free, row.free_ids, stream)) != CM_OK) return bail(st);
            for (int k = 0; k < row.n_free; ++k)
                loaded_by_us.erase(std::remove(loaded_by_us.begin(), loaded_by_us.end(), row.free_ids[k]),
                                   loaded_by_us.end());
        }
        auto job = std::make_unique<RowJob>();
        job->row = r;
        job->b = b;
        job->n = row.n_pairs;
        job->ids = row.pairs;
        job->done = ev_done[r];
        {
            std::lock_guard<std::mutex> lk(P.mu);
            P.queue.push_back(job.get());
        }
        P.cv_job.notify_all();
        jobs.push_back(std::move(job));
        S.rows++;
        S.pairs += row.n_pairs;
    }
    if (!loaded_by_us.empty()) {
        if ((st = cm_index_evict(ix, (int32_t)loaded_by_us.size(), loaded_by_us.data(), stream)) != CM_OK)
            return bail(st);
    }
    if (S.rows) {
        const cudaError_t e = cudaEventSynchronize(ev_done[S.rows - 1]);
        if (e != cudaSuccess) {
            fail(CM_ERR_CUDA, "cm_run_schedule: %s", cudaGetErrorString(e));
            return bail(CM_ERR_CUDA);
        }
    }
    const auto t_gpu_done = Clock::now();
    {
        std::lock_guard<std::mutex> lk(P.mu);
        P.stop = true;
    }
    P.cv_job.notify_all();
    for (auto& t : threads) t.join();
    threads.clear();
    S.tail_ms = ms_since(t_gpu_done);
    for (int32_t r = 0; r < S.rows; ++r) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ev_start[r], ev_done[r]) == cudaSuccess) S.gpu_ms += ms;
    }
    bool aborted;
    std::string perr;
    {
        std::lock_guard<std::mutex> lk(P.mu);
        S.matches = P.matches;
        S.verify_ms = P.verify_ms;
        aborted = P.abort;
        perr = P.err;
    }
    S.d2h_bytes += (uint64_t)S.matches * 4;
    cleanup();
    S.wall_ms = ms_since(t_start);
    if (stats) *stats = S;
    if (aborted) return fail(CM_ERR_STATE, "%s", perr.c_str());
    return cm_index_check(ix, stream);
}
