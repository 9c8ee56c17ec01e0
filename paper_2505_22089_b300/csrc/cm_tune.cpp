// Autotuner of the match launch: picks the thread mapping (bucket-major, tile
// or warp-per-query) and, for the tile forms, the work-item size (queries per
// CTA work item) by timing them on
// a sample of pairs, and optionally the Hamming top-K size K under a floor on
// decision agreement with the largest K tried.
//
// Tile size and thread mapping change only how the same result is computed:
// every configuration's decisions are compared with the first one's and must
// be identical.  K changes the method's result (Sec. 2.3.1 step (3) keeps K
// candidates), so it is chosen only when the caller asks and states the
// agreement it requires.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "cm_host.h"

#define fail ::cm::host_fail

namespace {

struct Timing {
    float ms = 0.f;
    cm_status st = CM_OK;
};

// Runs one plan of the sample under the index's current parameters: one
// untimed run, then `reps` timed runs; copies the decisions to host.
Timing time_config(cm_index* ix, const cm_pair* pairs, int64_t n_pairs, int32_t* d_best, std::vector<int32_t>& host,
                   cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, int reps) {
    Timing t;
    cm_match_plan* pl = nullptr;
    t.st = cm_match_plan_create(ix, pairs, n_pairs, reinterpret_cast<cm_stream>(s), &pl);
    if (t.st != CM_OK) return t;
    cm_match_out mo{};
    mo.best_j = d_best;
    t.st = cm_match_plan_run(pl, &mo, reinterpret_cast<cm_stream>(s));
    if (t.st == CM_OK && cudaEventRecord(e0, s) != cudaSuccess) t.st = fail(CM_ERR_CUDA, "autotune: event record");
    for (int r = 0; r < reps && t.st == CM_OK; ++r) t.st = cm_match_plan_run(pl, &mo, reinterpret_cast<cm_stream>(s));
    if (t.st == CM_OK && cudaEventRecord(e1, s) != cudaSuccess) t.st = fail(CM_ERR_CUDA, "autotune: event record");
    if (t.st == CM_OK) {
        host.resize((size_t)pl->rows);
        if (cudaMemcpyAsync(host.data(), d_best, host.size() * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess || cudaEventElapsedTime(&t.ms, e0, e1) != cudaSuccess)
            t.st = fail(CM_ERR_CUDA, "autotune: timing");
        t.ms /= (float)reps;
    }
    cm_match_plan_destroy(pl);
    if (t.st == CM_OK) t.st = cm_index_check(ix, reinterpret_cast<cm_stream>(s));
    return t;
}

}  // namespace

extern "C" cm_status cm_autotune(cm_index* ix, const cm_pair* pairs, int64_t n_pairs, const int32_t* K_candidates,
                                 int32_t n_K, float min_agreement, cm_stream stream, cm_tune_result* out) {
    if (!ix || !pairs || n_pairs < 1 || !out || n_K < 0 || (n_K && !K_candidates))
        return fail(CM_ERR_INVALID, "cm_autotune: bad argument");
    if (n_K && !(min_agreement >= 0.f && min_agreement <= 1.f))
        return fail(CM_ERR_INVALID, "cm_autotune: min_agreement must be in [0, 1]");
    int64_t rows = 0;
    for (int64_t k = 0; k < n_pairs; ++k) {
        const int i = pairs[k].i;
        if (i < 0 || i >= ix->n_images) return fail(CM_ERR_INVALID, "cm_autotune: pair %lld", (long long)k);
        rows += ix->n_desc[i];
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const cm_params saved = ix->p;
    uint64_t scratch_at = 0;
    if (!ix->alloc.alloc((uint64_t)std::max<int64_t>(rows, 1) * 4, &scratch_at))
        return fail(CM_ERR_BUDGET, "cm_autotune: arena full (%lld decision rows)", (long long)rows);
    int32_t* d_best = ix->at<int32_t>(scratch_at);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cm_status st = CM_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        st = fail(CM_ERR_CUDA, "cm_autotune: event creation");

    cm_tune_result r{};
    std::vector<int32_t> ref, cur;
    const bool tcr = tc_rerank(&ix->p);
    const int tiles[] = {256, 512, 1024, 2048, 4096};
    float best_ms = -1.f;
    for (int a = 0; a < 3 && st == CM_OK; ++a) {
        const int algo = a == 0 ? CM_ALGO_BUCKET : (a == 1 ? CM_ALGO_TILE : CM_ALGO_WARP);
        if (algo == CM_ALGO_WARP && tcr) continue;   // the tensor-core forms need a tile or bucket scan
        for (int S : tiles) {
            if (algo == CM_ALGO_BUCKET && S != tiles[0]) continue;   // no work-item size: one trial
            if (algo == CM_ALGO_TILE && match_smem_bytes(S, ix->p.K) > kMatchSmemLimit) continue;
            ix->p = saved;
            ix->p.query_tile = S;
            ix->p.algo = algo;
            const Timing t = time_config(ix, pairs, n_pairs, d_best, cur, s, e0, e1, 3);
            if ((st = t.st) != CM_OK) break;
            ++r.trials;
            if (ref.empty()) ref = cur;
            else if (cur != ref) {
                st = fail(CM_ERR_STATE, "cm_autotune: query tile %d / algo %d changed the decisions", S, algo);
                break;
            }
            if (best_ms < 0.f || t.ms < best_ms) {
                best_ms = t.ms;
                r.query_tile = algo == CM_ALGO_BUCKET ? 0 : S;
                r.algo = algo;
            }
        }
    }
    r.K = saved.K;
    r.ms = best_ms;
    r.agreement = 1.f;
    if (st == CM_OK && n_K) {
        // K: the fastest candidate whose decisions agree with the largest candidate's often enough
        std::vector<int32_t> Ks(K_candidates, K_candidates + n_K);
        std::sort(Ks.begin(), Ks.end());
        std::vector<float> ms(Ks.size());
        std::vector<std::vector<int32_t>> dec(Ks.size());
        for (size_t q = 0; q < Ks.size() && st == CM_OK; ++q) {
            ix->p = saved;
            ix->p.K = Ks[q];
            ix->p.query_tile = r.query_tile;
            ix->p.algo = r.algo;
            if ((st = cm_params_check(&ix->p)) != CM_OK) break;
            if (r.algo == CM_ALGO_TILE && match_smem_bytes(r.query_tile, Ks[q]) > kMatchSmemLimit)
                ix->p.query_tile = 0;   // the default tile that fits this K
            const Timing t = time_config(ix, pairs, n_pairs, d_best, dec[q], s, e0, e1, 3);
            if ((st = t.st) != CM_OK) break;
            ++r.trials;
            ms[q] = t.ms;
        }
        if (st == CM_OK) {
            const std::vector<int32_t>& top = dec.back();
            int chosen = (int)Ks.size() - 1;
            float chosen_agree = 1.f;
            for (size_t q = 0; q < Ks.size(); ++q) {
                int64_t same = 0;
                for (size_t e = 0; e < top.size(); ++e) same += dec[q][e] == top[e];
                const float agree = top.empty() ? 1.f : (float)((double)same / (double)top.size());
                if (agree >= min_agreement && ms[q] < ms[chosen]) {
                    chosen = (int)q;
                    chosen_agree = agree;
                }
            }
            r.K = Ks[chosen];
            r.ms = ms[chosen];
            r.agreement = chosen_agree;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    ix->alloc.release(scratch_at);
    ix->p = saved;
    if (st != CM_OK) return st;
    // the chosen configuration applies to plans made from now on
    ix->p.query_tile = r.query_tile;
    ix->p.algo = r.algo;
    ix->p.K = r.K;
    if (r.algo == CM_ALGO_TILE && match_smem_bytes(r.query_tile, r.K) > kMatchSmemLimit) ix->p.query_tile = 0;
    *out = r;
    return CM_OK;
}
