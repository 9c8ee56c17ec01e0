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
//
// The small tables reach the array through set-up kernels that take them as
// kernel arguments (copied at launch), so no host buffer of this call has to
// outlive it and the host never waits for the stream.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "cm_internal.h"

extern "C" cm_status cm_internal_fail(cm_status st, const char* msg);

namespace {

using namespace cm;

constexpr int kNoAllocMaxDesc = 8192;              // descriptors per image
constexpr size_t kNoAllocBytes = size_t(5) << 20;  // 5 MiB of device scratch
constexpr int kMaxDevices = 64;
constexpr int kWChunk = 7680;                      // weights per set-up launch (30 KB of kernel arguments)

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

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

// A slice of the weight matrix, passed by value.
struct WChunk {
    uint32_t at;     // byte offset in the array
    uint32_t count;  // floats
    float w[kWChunk];
};

// The per-call tables, passed by value, and the regions to clear.
struct Tables {
    Layout g;
    float mu[kDim];
    DevImage img[2];
    int32_t batch[2];
    int32_t tiles[3];
    DevPair pair;
    uint32_t hist_words;  // per image: L * 2^m bucket counts to zero
};

__global__ void k_noalloc_weights(WChunk c) {
    float* dst = reinterpret_cast<float*>(g_noalloc_scratch + c.at);
    for (uint32_t k = threadIdx.x; k < c.count; k += blockDim.x) dst[k] = c.w[k];
}

__global__ void k_noalloc_tables(Tables t) {
    unsigned char* a = g_noalloc_scratch;
    const int tid = threadIdx.x;
    for (int k = tid; k < kDim; k += blockDim.x) reinterpret_cast<float*>(a + t.g.mu)[k] = t.mu[k];
    if (tid < 2) {
        reinterpret_cast<DevImage*>(a + t.g.imgs)[tid] = t.img[tid];
        reinterpret_cast<int32_t*>(a + t.g.batch)[tid] = t.batch[tid];
    }
    if (tid < 3) reinterpret_cast<int32_t*>(a + t.g.tiles)[tid] = t.tiles[tid];
    if (tid == 0) {
        *reinterpret_cast<DevPair*>(a + t.g.pair) = t.pair;
        *reinterpret_cast<unsigned*>(a + t.g.counter) = 0u;   // the work counter starts at zero
    }
    // the array keeps the previous call's contents: bucket counts must start at zero
    for (int k = 0; k < 2; ++k)
        for (uint32_t w = tid; w < t.hist_words; w += blockDim.x) reinterpret_cast<uint32_t*>(a + t.g.hist[k])[w] = 0u;
}

cm_status fail(cm_status st, const char* msg) { return cm_internal_fail(st, msg); }

// Set-up of the array's device address, once per device and CUDA context: a
// context created after cudaDeviceReset holds a new copy of the array, which
// gets its own set-up.
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

std::mutex g_setup_mu;
struct DevSetup {
    unsigned long long ctx_id = 0;
    unsigned char* ptr = nullptr;
};
DevSetup g_setup[kMaxDevices];
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;
bool g_entry_looked_up = false;

cm_status scratch_address(int dev, unsigned char** out) {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_entry_looked_up) {
        g_entry_looked_up = true;
        void* f1 = nullptr;
        void* f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q2 == cudaDriverEntryPointSuccess) {
            g_ctx_current = reinterpret_cast<CtxGetCurrentFn>(f1);
            g_ctx_id = reinterpret_cast<CtxGetIdFn>(f2);
        }
    }
    unsigned long long id = 0;
    CUcontext ctx = nullptr;
    const bool have_id = g_ctx_current && g_ctx_id && g_ctx_current(&ctx) == CUDA_SUCCESS && ctx &&
                         g_ctx_id(ctx, &id) == CUDA_SUCCESS;
    DevSetup& d = g_setup[dev];
    if (!d.ptr || !have_id || d.ctx_id != id) {
        void* ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) return fail(CM_ERR_CUDA, "cm_match_pair_noalloc: cudaGetSymbolAddress failed");
        d.ptr = static_cast<unsigned char*>(ptr);
        d.ctx_id = have_id ? id : 0;
    }
    *out = d.ptr;
    return CM_OK;
}

}  // namespace

extern "C" cm_status cm_match_pair_noalloc(const cm_params* p, const uint8_t* d_desc_i, int32_t n_i,
                                           const uint8_t* d_desc_j, int32_t n_j, const uint64_t* col_sums_host,
                                           uint64_t n_total, int32_t* d_best_j, uint32_t* d_d1sq, uint32_t* d_d2sq,
                                           cm_stream stream) {
    cm_status st = cm_params_check(p);
    if (st != CM_OK) return st;
    if (p->rerank != CM_RERANK_FP32 && p->rerank != CM_RERANK_INT)
        return fail(CM_ERR_INVALID, "cm_match_pair_noalloc: only the FP32 and INT reranks are available");
    if (p->projection != CM_PROJ_FFMA)
        return fail(CM_ERR_INVALID, "cm_match_pair_noalloc: only the FP32 FFMA projection (CM_PROJ_FFMA) is available");
    if (p->algo == CM_ALGO_TC)
        return fail(CM_ERR_INVALID, "cm_match_pair_noalloc: the tensor-core scan needs a hand-over area; use TILE or WARP");
    if (n_i < 0 || n_j < 0 || n_i > kNoAllocMaxDesc || n_j > kNoAllocMaxDesc)
        return fail(CM_ERR_BUDGET, "cm_match_pair_noalloc: images are limited to 8192 descriptors each");
    if ((n_i && !d_desc_i) || (n_j && !d_desc_j) || !col_sums_host || !n_total || (n_i && !d_best_j))
        return fail(CM_ERR_INVALID, "cm_match_pair_noalloc: bad argument");
    const int n[2] = {n_i, n_j};
    const Layout g = layout(p, n);
    if (g.total > kNoAllocBytes)
        return fail(CM_ERR_BUDGET, "cm_match_pair_noalloc: parameters need more than the 5 MiB scratch");
    const int S = p->query_tile ? p->query_tile : kDefaultQueryTile;
    const bool tile = p->algo != CM_ALGO_WARP && match_smem_bytes(S, p->K) <= kMatchSmemLimit;
    if (p->algo == CM_ALGO_TILE && !tile)
        return fail(CM_ERR_INVALID, "cm_match_pair_noalloc: the tile mapping's shared memory does not fit this query tile");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fail(CM_ERR_CUDA, "cm_match_pair_noalloc: no current device");
    unsigned char* base = nullptr;
    if ((st = scratch_address(dev, &base)) != CM_OK) return st;
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);

    // weights W[128][P] with P_pad columns (zero padded), written by value in slices
    const int P = p->L * p->m + p->n_bits, P_pad = (P + 15) / 16 * 16;
    std::vector<float> W((size_t)kDim * P), Wp((size_t)kDim * P_pad, 0.f);
    cm_make_weights(p, W.data());
    for (int k = 0; k < kDim; ++k)
        for (int h = 0; h < P; ++h) Wp[(size_t)k * P_pad + h] = W[(size_t)k * P + h];
    cudaError_t e = cudaSuccess;
    {
        WChunk c;
        for (size_t f0 = 0; f0 < Wp.size() && e == cudaSuccess; f0 += kWChunk) {
            c.at = (uint32_t)(g.W + f0 * 4);
            c.count = (uint32_t)std::min<size_t>(kWChunk, Wp.size() - f0);
            std::memcpy(c.w, Wp.data() + f0, c.count * 4);
            k_noalloc_weights<<<1, 256, 0, s>>>(c);
            e = cudaGetLastError();
        }
    }
    Tables t{};
    t.g = g;
    for (int k = 0; k < kDim; ++k) t.mu[k] = (float)((double)col_sums_host[k] / (double)n_total);
    const uint8_t* descs[2] = {d_desc_i, d_desc_j};
    for (int k = 0; k < 2; ++k) {
        DevImage& im = t.img[k];
        im = DevImage{};
        im.desc = descs[k];
        im.key = reinterpret_cast<uint64_t*>(base + g.key[k]);
        im.code = reinterpret_cast<uint4*>(base + g.code[k]);
        im.scode = reinterpret_cast<uint4*>(base + g.scode[k]);
        im.sidx = reinterpret_cast<uint16_t*>(base + g.sidx[k]);
        im.off = reinterpret_cast<uint32_t*>(base + g.off[k]);
        im.hist = reinterpret_cast<uint32_t*>(base + g.hist[k]);
        im.brank = base + g.brank[k];
        im.norm = reinterpret_cast<uint32_t*>(base + g.norm[k]);
        im.n = n[k];
    }
    t.batch[0] = 0;
    t.batch[1] = 1;
    t.tiles[0] = 0;
    t.tiles[1] = (n_i + kHashTile - 1) / kHashTile;
    t.tiles[2] = t.tiles[1] + (n_j + kHashTile - 1) / kHashTile;
    t.pair = DevPair{};
    t.pair.i = 0;
    t.pair.j = 1;
    t.pair.row_off = 0;
    t.pair.item0 = 0;
    t.pair.nitems = (n_i + S - 1) / S;
    t.pair.ni = n_i;
    t.pair.rev = -1;
    t.hist_words = (uint32_t)(p->L << p->m);
    if (e == cudaSuccess) {
        k_noalloc_tables<<<1, 256, 0, s>>>(t);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return fail(CM_ERR_CUDA, "cm_match_pair_noalloc: set-up launch failed");

    HashLaunch h{};
    h.imgs = reinterpret_cast<const DevImage*>(base + g.imgs);
    h.batch = reinterpret_cast<const int32_t*>(base + g.batch);
    h.tile_pref = reinterpret_cast<const int32_t*>(base + g.tiles);
    h.n_batch = 2;
    h.n_tiles = t.tiles[2];
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
    if (e == cudaSuccess && t.pair.nitems > 0) {
        MatchLaunch m{};
        m.imgs = h.imgs;
        m.pairs = reinterpret_cast<const DevPair*>(base + g.pair);
        m.n_pairs = 1;
        m.n_items = t.pair.nitems;
        m.S = S;
        m.L = p->L;
        m.m = p->m;
        m.K = p->K;
        m.ratio_num = p->ratio_num;
        m.ratio_den = p->ratio_den;
        m.ratio_lo = ratio_band(p->ratio_num, p->ratio_den).lo;
        m.ratio_hi = ratio_band(p->ratio_num, p->ratio_den).hi;
        m.rerank = p->rerank;
        m.algo = tile ? CM_ALGO_TILE : CM_ALGO_WARP;
        m.counter = reinterpret_cast<unsigned*>(base + g.counter);
        m.out.best_j = d_best_j;
        m.out.d1sq = d_d1sq;
        m.out.d2sq = d_d2sq;
        e = tile ? launch_match(m, sms, s) : launch_match_wq(m, sms, s);
    }
    if (e != cudaSuccess) return fail(CM_ERR_CUDA, "cm_match_pair_noalloc: kernel launch failed");
    return CM_OK;
}
