// cm_match_pair_noalloc: one image pair matched with no device allocation.
//
// For callers that may not allocate GPU memory themselves or through a
// framework allocator: code running inside another framework's memory
// budget, plug-ins loaded into a host process that owns the device, or
// real-time paths where an allocation could block or fail.  All scratch -
// projection weights, centring mean, both images' keys, codes and bucket
// tables, the work counter - lives in one file-scope device array of
// kNoAllocBytes that every GPU which loads this library keeps until the
// process exits.  The caller passes only its inputs and outputs.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "cm_internal.h"

extern "C" cm_status cm_internal_fail(cm_status st, const char* msg);

namespace {

using namespace cm;

constexpr int kNoAllocMaxDesc = 8192;              // descriptors per image
constexpr size_t kNoAllocBytes = size_t(5) << 20;  // 5 MiB of device scratch
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_setup_mu;
unsigned char* g_scratch_ptr[kMaxDevices] = {};    // device address of the array, per device
float g_w_host[kDim * kMaxP];                      // host staging of the weights (under g_setup_mu)

constexpr uint64_t kA = 256;
inline uint64_t up(uint64_t v) { return (v + kA - 1) / kA * kA; }

struct Layout {
    uint64_t W, mu, imgs, batch, tiles, pair, counter;
    uint64_t key[2], code[2], scode[2], sidx[2], off[2], hist[2], brank[2], norm[2];
    uint64_t total;
};

Layout layout(const cm_params* p, const int n[2]) {
    Layout g{};
    uint64_t o = 0;
    auto take = [&](uint64_t bytes) { const uint64_t at = o; o = up(o + bytes); return at; };
    const int P_pad = (p->L * p->m + p->n_bits + 15) / 16 * 16;
    const uint64_t B = 1ull << p->m;
    g.W = take((uint64_t)kDim * P_pad * 4);
    g.mu = take(kDim * 4);
    g.imgs = take(2 * sizeof(DevImage));
    g.batch = take(2 * 4);
    g.tiles = take(3 * 4);
    g.pair = take(sizeof(DevPair));
    g.counter = take(4);
    for (int k = 0; k < 2; ++k) {
        g.key[k] = take((uint64_t)n[k] * 8);
        g.code[k] = take((uint64_t)n[k] * 16);
        g.scode[k] = take((uint64_t)p->L * n[k] * 16);
        g.sidx[k] = take((uint64_t)p->L * n[k] * 2);
        g.off[k] = take((uint64_t)p->L * (B + 1) * 4);
        g.hist[k] = take((uint64_t)p->L * B * 4);
        g.brank[k] = take((uint64_t)p->L * 256);
        g.norm[k] = take((uint64_t)n[k] * 4);
    }
    g.total = o;
    return g;
}

cm_status fail(cm_status st, const char* msg) { return cm_internal_fail(st, msg); }

}  // namespace

extern "C" cm_status cm_match_pair_noalloc(const cm_params* p, const uint8_t* d_desc_i, int32_t n_i,
                                           const uint8_t* d_desc_j, int32_t n_j, const uint64_t* col_sums_host,
                                           uint64_t n_total, int32_t* d_best_j, uint32_t* d_d1sq, uint32_t* d_d2sq,
                                           cm_stream stream) {
    cm_status st = cm_params_check(p);
    if (st != CM_OK) return st;
    if (p->rerank != CM_RERANK_FP32 && p->rerank != CM_RERANK_INT)
        return fail(CM_ERR_INVALID, "cm_match_pair_noalloc: only the FP32 and INT reranks are available");
    if (n_i < 0 || n_j < 0 || n_i > kNoAllocMaxDesc || n_j > kNoAllocMaxDesc)
        return fail(CM_ERR_BUDGET, "cm_match_pair_noalloc: images are limited to 8192 descriptors each");
    if ((n_i && !d_desc_i) || (n_j && !d_desc_j) || !col_sums_host || !n_total || (n_i && !d_best_j))
        return fail(CM_ERR_INVALID, "cm_match_pair_noalloc: bad argument");
    const int n[2] = {n_i, n_j};
    const Layout g = layout(p, n);
    if (g.total > kNoAllocBytes)
        return fail(CM_ERR_BUDGET, "cm_match_pair_noalloc: parameters need more than the 5 MiB scratch");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

    // set-up, once per device: the device address of the scratch array
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fail(CM_ERR_CUDA, "cm_match_pair_noalloc: no current device");
    unsigned char* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mu);
        if (!g_scratch_ptr[dev]) {
            void* ptr = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess || !ptr) return fail(CM_ERR_CUDA, "cm_match_pair_noalloc: cudaGetSymbolAddress failed");
            g_scratch_ptr[dev] = static_cast<unsigned char*>(ptr);
        }
        base = g_scratch_ptr[dev];
    }
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);

    // small tables are copied from host memory of this call (pageable copies
    // are staged by the driver before cudaMemcpyAsync returns)
    const int P = p->L * p->m + p->n_bits, P_pad = (P + 15) / 16 * 16;
    float mu[kDim];
    for (int k = 0; k < kDim; ++k) mu[k] = (float)((double)col_sums_host[k] / (double)n_total);
    DevImage img[2];
    const uint8_t* descs[2] = {d_desc_i, d_desc_j};
    for (int k = 0; k < 2; ++k) {
        img[k] = DevImage{};
        img[k].desc = descs[k];
        img[k].key = reinterpret_cast<uint64_t*>(base + g.key[k]);
        img[k].code = reinterpret_cast<uint4*>(base + g.code[k]);
        img[k].scode = reinterpret_cast<uint4*>(base + g.scode[k]);
        img[k].sidx = reinterpret_cast<uint16_t*>(base + g.sidx[k]);
        img[k].off = reinterpret_cast<uint32_t*>(base + g.off[k]);
        img[k].hist = reinterpret_cast<uint32_t*>(base + g.hist[k]);
        img[k].brank = base + g.brank[k];
        img[k].norm = reinterpret_cast<uint32_t*>(base + g.norm[k]);
        img[k].n = n[k];
    }
    const int32_t batch[2] = {0, 1};
    const int32_t tiles[3] = {0, (n_i + kHashTile - 1) / kHashTile,
                              (n_i + kHashTile - 1) / kHashTile + (n_j + kHashTile - 1) / kHashTile};
    const int S = p->query_tile ? p->query_tile : kDefaultQueryTile;
    DevPair pair{};
    pair.i = 0;
    pair.j = 1;
    pair.row_off = 0;
    pair.item0 = 0;
    pair.nitems = (n_i + S - 1) / S;
    pair.ni = n_i;
    pair.rev = -1;

    cudaError_t e = cudaSuccess;
    auto h2d = [&](uint64_t off, const void* src, size_t bytes) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(base + off, src, bytes, cudaMemcpyHostToDevice, s);
    };
    {
        // weights W[128][P] laid out with P_pad columns (zero padded), then copied
        std::lock_guard<std::mutex> lock(g_setup_mu);
        cm_make_weights(p, g_w_host);
        for (int k = kDim - 1; k >= 0; --k)
            for (int h = P_pad - 1; h >= 0; --h) g_w_host[k * P_pad + h] = h < P ? g_w_host[k * P + h] : 0.f;
        h2d(g.W, g_w_host, (size_t)kDim * P_pad * 4);
    }
    h2d(g.mu, mu, sizeof mu);
    h2d(g.imgs, img, sizeof img);
    h2d(g.batch, batch, sizeof batch);
    h2d(g.tiles, tiles, sizeof tiles);
    h2d(g.pair, &pair, sizeof pair);
    // the array keeps the previous call's contents: clear the bucket counts and the work counter
    for (int k = 0; k < 2 && e == cudaSuccess; ++k)
        e = cudaMemsetAsync(base + g.hist[k], 0, (size_t)p->L * (1u << p->m) * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + g.counter, 0, 4, s);
    if (e != cudaSuccess) return fail(CM_ERR_CUDA, "cm_match_pair_noalloc: copy to scratch failed");

    HashLaunch h{};
    h.imgs = reinterpret_cast<const DevImage*>(base + g.imgs);
    h.batch = reinterpret_cast<const int32_t*>(base + g.batch);
    h.tile_pref = reinterpret_cast<const int32_t*>(base + g.tiles);
    h.n_batch = 2;
    h.n_tiles = tiles[2];
    h.W = reinterpret_cast<const float*>(base + g.W);
    h.mu = reinterpret_cast<const float*>(base + g.mu);
    h.L = p->L;
    h.m = p->m;
    h.P_pad = P_pad;
    h.rerank = p->rerank;
    if (h.n_tiles) {
        e = launch_hash(h, sms, s);
        if (e == cudaSuccess) e = launch_bucket(h, s);
    }
    if (e == cudaSuccess && pair.nitems > 0) {
        MatchLaunch m{};
        m.imgs = h.imgs;
        m.pairs = reinterpret_cast<const DevPair*>(base + g.pair);
        m.n_pairs = 1;
        m.n_items = pair.nitems;
        m.S = S;
        m.L = p->L;
        m.m = p->m;
        m.K = p->K;
        m.ratio_num = p->ratio_num;
        m.ratio_den = p->ratio_den;
        m.rerank = p->rerank;
        m.algo = CM_ALGO_WARP;
        m.counter = reinterpret_cast<unsigned*>(base + g.counter);
        m.out.best_j = d_best_j;
        m.out.d1sq = d_d1sq;
        m.out.d2sq = d_d2sq;
        e = launch_match_wq(m, sms, s);
    }
    if (e != cudaSuccess) return fail(CM_ERR_CUDA, "cm_match_pair_noalloc: kernel launch failed");
    return CM_OK;
}
