// Exhaustive nearest neighbours of every query over all of the database
// image, for a list of pairs, with the exact ratio test: the matches cascade
// hashing would give with every database point a candidate (Sec. 2.3.1 with
// K = N_J), i.e. the quality ceiling against which the lookup's recall is
// measured.
//
// k_nn_exhaustive: a work item is a tile of 128 queries of one pair.  The
// tile is staged once as the A operand; the database image is walked in
// chunks of up to 256 rows, each staged as the B operand and multiplied on
// the tensor cores (128 x N x 128, BF16, FP32 accumulate: every partial sum
// of x.y is an integer below 2^24, so exact).  The 4 warps read their lanes
// back and keep, per query, the smallest (d^2, j) and the second smallest
// d^2, with d^2 = |x|^2 + |y|^2 - 2 x.y exact as an FP32 integer; the last
// chunk is followed by the exact integer ratio test.  Two CTAs per SM overlap one's
// staging with the other's MMA and epilogue.
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "cm_host.h"
#include "cm_stage.cuh"
#include "cm_tc.cuh"

namespace cm {

namespace {

constexpr int kNnThreads = 128;
constexpr int kNnRows = 128;      // queries per work item (M)
constexpr int kNnChunk = 256;     // database rows per MMA (N)
constexpr int kNnPolls = 1 << 24;

struct NnPair {
    int32_t i, j;
    int64_t row_off;   // first output row
    int32_t item0;     // first work item
    int32_t pad;
};

__global__ void __launch_bounds__(kNnThreads, 2)
k_nn_exhaustive(const uint8_t* __restrict__ desc, const int64_t* __restrict__ img_off, const NnPair* __restrict__ pairs,
                int n_pairs, int n_items, int ratio_num, int ratio_den, int32_t* __restrict__ best_j,
                uint32_t* __restrict__ d1sq, uint32_t* __restrict__ d2sq, int* err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* At = smem;                                    // 128 x 256 B
    unsigned char* Bt = At + kNnRows * 256;                      // 256 x 256 B
    float* nb = reinterpret_cast<float*>(Bt + kNnChunk * 256);   // [256] |y|^2 (+inf past the image)
    uint64_t* mbar = reinterpret_cast<uint64_t*>(nb + kNnChunk);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
    const int tid = threadIdx.x, warp = tid >> 5;
    const float kInf = __uint_as_float(0x7F800000u);

    if (tid == 0) tc::mbar_init(mbar, 1);
    if (warp == 0) tc::tmem_alloc(tslot, kNnChunk);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * warp) << 16);
    uint32_t parity = 0;
    bool failed = false;

    for (int item = blockIdx.x; item < n_items && !failed; item += gridDim.x) {
        int lo = 0, hi = n_pairs;   // last pair with item0 <= item
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (pairs[mid].item0 <= item) lo = mid; else hi = mid;
        }
        const NnPair P = pairs[lo];
        const int64_t oi = img_off[P.i], oj = img_off[P.j];
        const int ni = (int)(img_off[P.i + 1] - oi), nj = (int)(img_off[P.j + 1] - oj);
        const int q = (item - P.item0) * kNnRows + tid;
        const bool qv = q < ni;
        uint4 v[8];
        stage::load_row(desc + (size_t)(oi + (qv ? q : 0)) * kDim, qv, v);
        const float nq = (float)stage::store_row(v, At, tid, kNnRows);
        float e1 = kInf, e2 = kInf;
        int j1 = -1;

        for (int c0 = 0; c0 < nj; c0 += kNnChunk) {
            const int nc = min(kNnChunk, nj - c0);
            const int N = (nc + 15) / 16 * 16;
            for (int r = tid; r < N; r += kNnThreads) {
                const bool have = r < nc;
                stage::load_row(desc + (size_t)(oj + c0 + (have ? r : 0)) * kDim, have, v);
                const uint32_t nn = stage::store_row(v, Bt, r, N);
                nb[r] = have ? (float)nn : kInf;
            }
            tc::fence_proxy_async();
            __syncthreads();
            if (tid == 0) {
                tc::fence_after();
                stage::mma_128xN(tmem, At, Bt, N);
                tc::commit(mbar);
            }
            const bool ok = tc::mbar_wait(mbar, parity, kNnPolls);
            parity ^= 1u;
            if (__syncthreads_or(!ok)) {
                // the accumulator never completed: report, give the MMA a last bounded wait, stop
                if (tid == 0) atomicExch(err, 1);
                tc::mbar_wait(mbar, parity ^ 1u, kNnPolls);
                failed = true;
                break;
            }
            tc::fence_after();
            // q1 keeps its index, q2 only its value (the outputs need no j2);
            // columns in ascending j, so a tie keeps the smaller j as q1
            for (int cc = 0; cc < N; cc += 16) {
                uint32_t acc[16];
                tc::tmem_ld16(lane_base + cc, acc);
                tc::tmem_wait_ld();
                const int jb = c0 + cc;
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    // exact: |x|^2 + |y|^2 < 2^24 and the result is a squared distance
                    const float d = fmaf(-2.f, __uint_as_float(acc[u]), nq + nb[cc + u]);
                    j1 = d < e1 ? jb + u : j1;
                    e2 = fminf(e2, fmaxf(e1, d));
                    e1 = fminf(e1, d);
                }
            }
            tc::fence_before();
            __syncthreads();   // TMEM and the B tile are reused by the next chunk
        }
        if (!failed && qv) {
            const int64_t row = P.row_off + q;
            const bool has2 = nj >= 2;   // e2 is finite exactly when J has two rows
            const uint32_t u1 = j1 >= 0 ? (uint32_t)e1 : 0xFFFFFFFFu, u2 = has2 ? (uint32_t)e2 : 0xFFFFFFFFu;
            const bool pass = has2 && (int64_t)ratio_den * ratio_den * u1 < (int64_t)ratio_num * ratio_num * u2;
            best_j[row] = pass ? j1 : -1;
            if (d1sq) d1sq[row] = u1;
            if (d2sq) d2sq[row] = u2;
        }
        __syncthreads();   // the A tile is restaged by the next item
    }
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kNnChunk);
}

// Workspace: error flag (fixed place), image offsets, pair records.
struct NnWork {
    uint64_t err, off, pairs, total;
};

NnWork nn_layout(int32_t n_images, int64_t n_pairs) {
    NnWork w{};
    w.err = 0;
    w.off = align_up(4);
    w.pairs = align_up(w.off + 8 * (uint64_t)(n_images + 1));
    w.total = align_up(w.pairs + sizeof(NnPair) * (uint64_t)n_pairs);
    return w;
}

}  // namespace

}  // namespace cm

using namespace cm;

extern "C" cm_status cm_nn_workspace_bytes(int32_t n_images, int64_t n_pairs, uint64_t* bytes) {
    if (n_images < 0 || n_pairs < 0 || !bytes) return host_fail(CM_ERR_INVALID, "cm_nn_workspace_bytes: bad argument");
    *bytes = nn_layout(n_images, n_pairs).total;
    return CM_OK;
}

extern "C" cm_status cm_nn_pairs(const uint8_t* desc, const int64_t* img_off, int32_t n_images, const cm_pair* pairs,
                                 int64_t n_pairs, int32_t ratio_num, int32_t ratio_den, void* d_work,
                                 uint64_t work_bytes, int32_t* best_j, uint32_t* d1sq, uint32_t* d2sq,
                                 cm_stream stream) {
    if (n_images < 0 || !img_off || n_pairs < 0 || (n_pairs && (!pairs || !best_j)) || !d_work || ratio_num < 1 ||
        ratio_den <= ratio_num || ratio_den > 1024)
        return host_fail(CM_ERR_INVALID, "cm_nn_pairs: bad argument");
    if (img_off[0] != 0) return host_fail(CM_ERR_INVALID, "cm_nn_pairs: img_off[0] must be 0");
    for (int32_t i = 0; i < n_images; ++i)
        if (img_off[i + 1] < img_off[i] || img_off[i + 1] - img_off[i] > 65535)
            return host_fail(CM_ERR_INVALID, "cm_nn_pairs: img_off not ascending or an image above 65535 rows");
    const NnWork w = nn_layout(n_images, n_pairs);
    if (work_bytes < w.total || (reinterpret_cast<uintptr_t>(d_work) & (kAlign - 1)))
        return host_fail(CM_ERR_BUDGET, "cm_nn_pairs: workspace smaller than cm_nn_workspace_bytes or not 256-byte aligned");
    std::vector<NnPair> rec((size_t)n_pairs);
    int64_t rows = 0, items = 0;
    for (int64_t k = 0; k < n_pairs; ++k) {
        const cm_pair pr = pairs[k];
        if (pr.i < 0 || pr.j < 0 || pr.i >= n_images || pr.j >= n_images)
            return host_fail(CM_ERR_INVALID, "cm_nn_pairs: pair %lld names an image out of range", (long long)k);
        const int64_t ni = img_off[pr.i + 1] - img_off[pr.i];
        rec[k] = {pr.i, pr.j, rows, (int32_t)items, 0};
        rows += ni;
        items += (ni + kNnRows - 1) / kNnRows;
        if (items > INT32_MAX) return host_fail(CM_ERR_INVALID, "cm_nn_pairs: too many work items");
    }
    if (rows > 0 && !desc) return host_fail(CM_ERR_INVALID, "cm_nn_pairs: desc is NULL");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned char* base = static_cast<unsigned char*>(d_work);
    int* err = reinterpret_cast<int*>(base + w.err);
    CM_CUDA(cudaMemsetAsync(err, 0, 4, s));
    if (items == 0) return CM_OK;
    CM_CUDA(cudaMemcpyAsync(base + w.off, img_off, 8 * (size_t)(n_images + 1), cudaMemcpyHostToDevice, s));
    CM_CUDA(cudaMemcpyAsync(base + w.pairs, rec.data(), sizeof(NnPair) * rec.size(), cudaMemcpyHostToDevice, s));
    int dev = 0, sms = 148;
    CM_CUDA(cudaGetDevice(&dev));
    CM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // two CTAs per SM at most: their TMEM (2 x 256 columns) always fits
    size_t smem = (size_t)kNnRows * 256 + (size_t)kNnChunk * 256 + kNnChunk * 4 + 64;
    smem = std::max(smem, (size_t)(228 * 1024) / 3 + 1024);
    CM_CUDA(cudaFuncSetAttribute(k_nn_exhaustive, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int grid = (int)std::min<int64_t>(items, 2 * (int64_t)sms);
    k_nn_exhaustive<<<grid, kNnThreads, smem, s>>>(desc, reinterpret_cast<const int64_t*>(base + w.off),
                                                   reinterpret_cast<const NnPair*>(base + w.pairs), (int)n_pairs,
                                                   (int)items, ratio_num, ratio_den, best_j, d1sq, d2sq, err);
    CM_CUDA(cudaGetLastError());
    return CM_OK;
}
