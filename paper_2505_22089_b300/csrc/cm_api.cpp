// C-ABI entry points: parameters, projection weights, the arena-backed index,
// match plans.  Host C++; device work is enqueued through the launchers of
// cm_kernels.cu.  See include/cashmatch.h for the contract of each call.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <vector>

#include "cm_host.h"

using namespace cm;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_err;

cm_status cm::host_fail(cm_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}
#define fail ::cm::host_fail

extern "C" const char* cm_version(void) { return "cashmatch 0.1 (sm_103a)"; }
extern "C" cm_status cm_internal_fail(cm_status st, const char* msg) { return fail(st, "%s", msg); }
extern "C" const char* cm_last_error(void) { return g_err.c_str(); }

// ---------------------------------------------------------------------------
// parameters
// ---------------------------------------------------------------------------
extern "C" cm_status cm_params_default(cm_params* p) {
    if (!p) return fail(CM_ERR_INVALID, "cm_params_default: NULL");
    p->L = 6;
    p->m = 8;
    p->n_bits = 128;
    p->K = 8;
    p->ratio_num = 4;
    p->ratio_den = 5;
    p->seed = 0x5EED;
    p->rerank = CM_RERANK_FP32;
    p->query_tile = 0;
    p->algo = CM_ALGO_AUTO;
    p->projection = CM_PROJ_TC;
    return CM_OK;
}

extern "C" cm_status cm_params_check(const cm_params* p) {
    if (!p) return fail(CM_ERR_INVALID, "params: NULL");
    if (p->L < 1 || p->L > kMaxL) return fail(CM_ERR_INVALID, "params: L=%d not in 1..8", p->L);
    if (p->m < 0 || p->m > kMaxM) return fail(CM_ERR_INVALID, "params: m=%d not in 0..8", p->m);
    if (p->n_bits != 128) return fail(CM_ERR_INVALID, "params: n_bits=%d, only 128 is supported", p->n_bits);
    if (p->K != 2 && p->K != 4 && p->K != 8 && p->K != 16)
        return fail(CM_ERR_INVALID, "params: K=%d not in {2,4,8,16}", p->K);
    if (p->ratio_den < 1 || p->ratio_num < 0 || p->ratio_num > 4 * p->ratio_den)
        return fail(CM_ERR_INVALID, "params: ratio %d/%d out of range", p->ratio_num, p->ratio_den);
    if (p->rerank < CM_RERANK_FP32 || p->rerank > CM_RERANK_INT)
        return fail(CM_ERR_INVALID, "params: rerank mode %d not available", p->rerank);
    if (p->query_tile != 0 && (p->query_tile < 64 || p->query_tile > 8192 || p->query_tile % 64))
        return fail(CM_ERR_INVALID, "params: query_tile=%d must be 0 or a multiple of 64 in 64..8192",
                    p->query_tile);
    if (p->algo < CM_ALGO_AUTO || p->algo > CM_ALGO_BUCKET) return fail(CM_ERR_INVALID, "params: algo %d", p->algo);
    if (p->algo == CM_ALGO_TC && p->K < 4)
        return fail(CM_ERR_INVALID, "params: the tensor-core Hamming scan needs K in {4, 8, 16}");
    if (p->projection != CM_PROJ_TC && p->projection != CM_PROJ_FFMA)
        return fail(CM_ERR_INVALID, "params: projection %d", p->projection);
    const int S = query_tile(p);
    if ((p->rerank == CM_RERANK_BF16 || p->rerank == CM_RERANK_FP8) && p->algo == CM_ALGO_WARP)
        return fail(CM_ERR_INVALID, "params: the tensor-core reranks follow the bucket-major or tile scan (algo bucket, "
                                    "tile or auto)");
    if (p->algo == CM_ALGO_TILE && match_smem_bytes(S, p->K) > kMatchSmemLimit)
        return fail(CM_ERR_INVALID, "params: query_tile=%d with K=%d needs %zu bytes of shared memory (> 227 KB)", S,
                    p->K, match_smem_bytes(S, p->K));
    return CM_OK;
}

// ---------------------------------------------------------------------------
// projection weights: splitmix64 stream -> Box-Muller pairs -> float
// ---------------------------------------------------------------------------
namespace {
struct SplitMix64 {
    uint64_t x;
    uint64_t operator()() {
        x += 0x9E3779B97F4A7C15ull;
        uint64_t z = x;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
};
}  // namespace

extern "C" cm_status cm_make_weights(const cm_params* p, float* W) {
    cm_status st = cm_params_check(p);
    if (st != CM_OK) return st;
    if (!W) return fail(CM_ERR_INVALID, "cm_make_weights: NULL output");
    const int64_t n = (int64_t)kDim * proj_count(p);
    SplitMix64 g{p->seed};
    const double two_pi = 2.0 * 3.14159265358979323846;
    const double inv53 = 1.0 / 9007199254740992.0;
    for (int64_t e = 0; e < n; e += 2) {
        const uint64_t a = g(), b = g();
        const double u1 = (double)((a >> 11) + 1) * inv53;
        const double u2 = (double)(b >> 11) * inv53;
        const double radius = std::sqrt(-2.0 * std::log(u1));
        const double angle = two_pi * u2;
        W[e] = (float)(radius * std::cos(angle));
        if (e + 1 < n) W[e + 1] = (float)(radius * std::sin(angle));
    }
    return CM_OK;
}

// ---------------------------------------------------------------------------
// arena layout
// ---------------------------------------------------------------------------

extern "C" cm_status cm_image_bytes(const cm_params* p, int32_t n_desc, uint64_t* bytes) {
    cm_status st = cm_params_check(p);
    if (st != CM_OK) return st;
    if (!bytes || n_desc < 0 || n_desc > 65535) return fail(CM_ERR_INVALID, "cm_image_bytes: bad argument");
    *bytes = slot_layout(p, n_desc, false).total;
    return CM_OK;
}

extern "C" cm_status cm_plan_bytes(const cm_params* p, int64_t n_pairs, int64_t rows, int32_t max_query_rows,
                                   uint64_t* bytes) {
    cm_status st = cm_params_check(p);
    if (st != CM_OK) return st;
    if (!bytes || n_pairs < 0 || rows < 0 || max_query_rows < 0 || max_query_rows > 65535)
        return fail(CM_ERR_INVALID, "cm_plan_bytes: bad argument");
    *bytes = plan_bytes(p, n_pairs, rows, max_query_rows);
    return CM_OK;
}

extern "C" cm_status cm_index_bytes(const cm_params* p, int32_t n_images, const int32_t* n_desc, int32_t inplace,
                                    uint64_t* bytes) {
    cm_status st = cm_params_check(p);
    if (st != CM_OK) return st;
    if (!bytes || n_images < 0 || (n_images && !n_desc)) return fail(CM_ERR_INVALID, "cm_index_bytes: bad argument");
    uint64_t t = fixed_layout(p, n_images).total;
    for (int i = 0; i < n_images; ++i) {
        if (n_desc[i] < 0 || n_desc[i] > 65535) return fail(CM_ERR_INVALID, "image %d: %d descriptors", i, n_desc[i]);
        t += slot_layout(p, n_desc[i], inplace != 0).total;
    }
    *bytes = t + 64 * kAlign;
    return CM_OK;
}

// ---------------------------------------------------------------------------
// index
// ---------------------------------------------------------------------------
static cm_status upload_table(cm_index* ix, uint64_t off, const void* src, size_t bytes, cudaStream_t s) {
    CM_CUDA(ix->staging.upload(ix->arena + off, src, bytes, s));
    return CM_OK;
}

extern "C" cm_status cm_index_create(const cm_params* p, int32_t n_images, const int32_t* n_desc, void* d_arena,
                                     uint64_t arena_bytes, cm_index** out) {
    cm_status st = cm_params_check(p);
    if (st != CM_OK) return st;
    if (!out || !d_arena || n_images < 1 || !n_desc) return fail(CM_ERR_INVALID, "cm_index_create: bad argument");
    if (reinterpret_cast<uintptr_t>(d_arena) % kAlign) return fail(CM_ERR_INVALID, "arena must be 256-byte aligned");
    for (int i = 0; i < n_images; ++i)
        if (n_desc[i] < 0 || n_desc[i] > 65535)
            return fail(CM_ERR_INVALID, "image %d has %d descriptors (0..65535 supported)", i, n_desc[i]);
    cm_index* ix = new (std::nothrow) cm_index();
    if (!ix) return fail(CM_ERR_NOMEM, "cm_index_create: host allocation");
    ix->p = *p;
    ix->P = proj_count(p);
    ix->P_pad = proj_pad(p);
    ix->B = 1 << p->m;
    ix->n_images = n_images;
    ix->n_desc.assign(n_desc, n_desc + n_images);
    ix->arena = static_cast<uint8_t*>(d_arena);
    ix->arena_bytes = arena_bytes;
    ix->fx = fixed_layout(p, n_images);
    if (ix->fx.total > arena_bytes) {
        const unsigned long long need = ix->fx.total;
        delete ix;
        return fail(CM_ERR_BUDGET, "arena of %llu bytes is smaller than the index tables (%llu)",
                    (unsigned long long)arena_bytes, need);
    }
    ix->alloc.init(ix->fx.total, arena_bytes);
    ix->h_imgs.assign(n_images, DevImage{});
    for (int i = 0; i < n_images; ++i) ix->h_imgs[i].n = n_desc[i];
    ix->slot_at.assign(n_images, 0);
    ix->resident.assign(n_images, 0);
    ix->pending.assign(n_images, 0);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&ix->sms, cudaDevAttrMultiProcessorCount, dev);
    // weights, zero-padded to P_pad columns
    std::vector<float> W((size_t)kDim * ix->P), Wp((size_t)kDim * ix->P_pad, 0.f);
    cm_make_weights(p, W.data());
    for (int k = 0; k < kDim; ++k)
        for (int h = 0; h < ix->P; ++h) Wp[(size_t)k * ix->P_pad + h] = W[(size_t)k * ix->P + h];
    cudaError_t e = cudaMemcpy(ix->arena + ix->fx.W, Wp.data(), Wp.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(ix->arena + ix->fx.imgs, ix->h_imgs.data(), ix->h_imgs.size() * sizeof(DevImage),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(ix->arena + ix->fx.err, 0, 4);
    if (e != cudaSuccess) {
        delete ix;
        return fail(CM_ERR_CUDA, "cm_index_create: %s", cudaGetErrorString(e));
    }
    *out = ix;
    return CM_OK;
}

extern "C" void cm_index_destroy(cm_index* ix);

extern "C" cm_status cm_index_set_mean(cm_index* ix, const uint64_t* sums, uint64_t n_total, cm_stream stream) {
    if (!ix || !sums || !n_total) return fail(CM_ERR_INVALID, "cm_index_set_mean: bad argument");
    float mu[kDim];
    for (int k = 0; k < kDim; ++k) mu[k] = (float)((double)sums[k] / (double)n_total);
    cm_status st = upload_table(ix, ix->fx.mu, mu, sizeof mu, reinterpret_cast<cudaStream_t>(stream));
    if (st == CM_OK) {
        ix->mean_set = true;
        ix->sums_on_host = true;
        std::copy(sums, sums + kDim, ix->host_sums);
        ix->n_total = n_total;
    }
    return st;
}

extern "C" cm_status cm_index_col_sums(cm_index* ix, uint64_t* sums, uint64_t* n_total, cm_stream stream) {
    if (!ix || !sums) return fail(CM_ERR_INVALID, "cm_index_col_sums: bad argument");
    if (!ix->mean_set) return fail(CM_ERR_STATE, "cm_index_col_sums: no centring mean yet");
    if (ix->sums_on_host) {
        std::copy(ix->host_sums, ix->host_sums + kDim, sums);
    } else {
        cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
        CM_CUDA(cudaMemcpyAsync(sums, ix->arena + ix->fx.sums, kDim * 8, cudaMemcpyDeviceToHost, s));
        CM_CUDA(cudaStreamSynchronize(s));
    }
    if (n_total) *n_total = ix->n_total;
    return CM_OK;
}

extern "C" cm_status cm_index_mean_device(cm_index* ix, const uint8_t* d_desc, uint64_t n_rows, cm_stream stream) {
    if (!ix || (!d_desc && n_rows) || !n_rows) return fail(CM_ERR_INVALID, "cm_index_mean_device: bad argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned long long* sums = ix->at<unsigned long long>(ix->fx.sums);
    CM_CUDA(cudaMemsetAsync(sums, 0, kDim * 8, s));
    CM_CUDA(launch_colsum_rows(d_desc, n_rows, sums, s));
    CM_CUDA(launch_mean(sums, nullptr, n_rows, ix->at<float>(ix->fx.mu), s));
    ix->mean_set = true;
    ix->sums_on_host = false;
    ix->n_total = n_rows;
    return CM_OK;
}

namespace cm {
// Adds the exact column sums of the host rows of images ids[0..count) to the
// index's sums (fx.sums, not cleared here), copying them through the device
// staging block [stage, stage + stage_bytes) (a multiple of 128 bytes) in
// stream order.  Returns the rows summed in *rows.
cm_status index_stream_sums(cm_index* ix, int32_t count, const int32_t* ids, const uint8_t* const* desc_host,
                            uint8_t* stage, uint64_t stage_bytes, cudaStream_t s, uint64_t* rows) {
    const uint64_t rows_per_chunk = stage_bytes / kDim;
    if (!rows_per_chunk) return fail(CM_ERR_BUDGET, "centring: staging block of %llu bytes", (unsigned long long)stage_bytes);
    unsigned long long* sums = ix->at<unsigned long long>(ix->fx.sums);
    uint64_t fill = 0, total = 0;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < count && e == cudaSuccess; ++k) {
        const int i = ids[k];
        const uint64_t n = (uint64_t)ix->n_desc[i];
        if (n && !desc_host[i]) return fail(CM_ERR_INVALID, "centring: image %d has no rows", i);
        uint64_t done = 0;
        while (done < n && e == cudaSuccess) {
            const uint64_t take = std::min(n - done, rows_per_chunk - fill);
            e = cudaMemcpyAsync(stage + fill * kDim, desc_host[i] + done * kDim, take * kDim, cudaMemcpyHostToDevice, s);
            fill += take;
            done += take;
            if (fill == rows_per_chunk && e == cudaSuccess) {
                e = launch_colsum_rows(stage, fill, sums, s);
                fill = 0;
            }
        }
        total += n;
    }
    if (fill && e == cudaSuccess) e = launch_colsum_rows(stage, fill, sums, s);
    if (e != cudaSuccess) return fail(CM_ERR_CUDA, "centring: %s", cudaGetErrorString(e));
    *rows = total;
    return CM_OK;
}

// mu = sums / n_total from the index's sums (fx.sums), on the device.
cm_status index_mean_from_sums(cm_index* ix, uint64_t n_total, cudaStream_t s) {
    CM_CUDA(launch_mean(ix->at<unsigned long long>(ix->fx.sums), nullptr, n_total, ix->at<float>(ix->fx.mu), s));
    ix->mean_set = true;
    ix->sums_on_host = false;
    ix->n_total = n_total;
    return CM_OK;
}
}  // namespace cm

extern "C" cm_status cm_index_mean_host(cm_index* ix, const uint8_t* const* desc_host, cm_stream stream) {
    if (!ix || !desc_host) return fail(CM_ERR_INVALID, "cm_index_mean_host: bad argument");
    uint64_t total = 0;
    for (int i = 0; i < ix->n_images; ++i) {
        if (ix->n_desc[i] && !desc_host[i]) return fail(CM_ERR_INVALID, "cm_index_mean_host: image %d has no rows", i);
        total += (uint64_t)ix->n_desc[i];
    }
    if (!total) return fail(CM_ERR_INVALID, "cm_index_mean_host: the index has no rows");
    // staging: the largest block of up to 64 MiB (a multiple of 128-byte rows) the arena has free
    uint64_t chunk = std::min<uint64_t>(64ull << 20, align_up(total * kDim)), at = 0;
    while (chunk >= (1ull << 20) && !ix->alloc.alloc(chunk, &at)) chunk /= 2;
    if (chunk < (1ull << 20)) return fail(CM_ERR_BUDGET, "cm_index_mean_host: no 1 MiB of the arena is free");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    std::vector<int32_t> all(ix->n_images);
    for (int i = 0; i < ix->n_images; ++i) all[i] = i;
    uint64_t rows = 0;
    cudaError_t e = cudaMemsetAsync(ix->arena + ix->fx.sums, 0, kDim * 8, s);
    cm_status st = e == cudaSuccess ? index_stream_sums(ix, ix->n_images, all.data(), desc_host, ix->arena + at,
                                                        chunk / kDim * kDim, s, &rows)
                                    : fail(CM_ERR_CUDA, "cm_index_mean_host: %s", cudaGetErrorString(e));
    // later work on this stream is ordered after the sums: the block may be placed again at once
    ix->alloc.release(at);
    if (st != CM_OK) return st;
    return index_mean_from_sums(ix, total, s);
}

// Allocate slots, copy descriptors, refresh the device image table and the
// load-batch table.  Returns the batch's hash-tile count.
// Loading an image has three phases: placing its slot in the arena, copying
// its descriptors there, and publishing it (device table entry, cleared
// histograms, resident flag) before it is hashed.  cm_index_load runs them
// in a row on one stream; the pipeline runs the first two early, on a copy
// stream, for the next block row (index_prefetch / index_publish).
static cm_status check_loadable(cm_index* ix, int32_t count, const int32_t* ids, const uint8_t* const* desc,
                                int32_t mem) {
    if (count < 0 || (count && (!ids || !desc))) return fail(CM_ERR_INVALID, "load: bad argument");
    if (mem != CM_MEM_HOST && mem != CM_MEM_DEVICE && mem != CM_MEM_DEVICE_INPLACE)
        return fail(CM_ERR_INVALID, "load: bad memory kind %d", mem);
    std::vector<char> seen(ix->n_images, 0);
    for (int k = 0; k < count; ++k) {
        const int i = ids[k];
        if (i < 0 || i >= ix->n_images) return fail(CM_ERR_INVALID, "load: image id %d out of range", i);
        if (ix->resident[i] || ix->pending[i] || seen[i])
            return fail(CM_ERR_STATE, "load: image %d is already resident", i);
        if (!desc[k] && ix->n_desc[i]) return fail(CM_ERR_INVALID, "load: NULL descriptors for image %d", i);
        seen[i] = 1;
    }
    return CM_OK;
}

// Places the slots of ids (all or none); false when the arena has no room.
static bool place_slots(cm_index* ix, int32_t count, const int32_t* ids, bool inplace) {
    for (int k = 0; k < count; ++k) {
        const int i = ids[k];
        uint64_t at = 0;
        if (!ix->alloc.alloc(slot_layout(&ix->p, ix->n_desc[i], inplace).total, &at)) {
            for (int r = 0; r < k; ++r) {   // roll back this call's slots
                ix->alloc.release(ix->slot_at[ids[r]]);
                ix->pending[ids[r]] = 0;
            }
            return false;
        }
        ix->slot_at[i] = at;
        ix->pending[i] = 1;
    }
    return true;
}

static cm_status copy_descs(cm_index* ix, int32_t count, const int32_t* ids, const uint8_t* const* desc, int32_t mem,
                            cudaStream_t s) {
    if (mem == CM_MEM_DEVICE_INPLACE) return CM_OK;
    const cudaMemcpyKind kind = mem == CM_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    for (int k = 0; k < count; ++k) {
        const int i = ids[k];
        const int64_t n = ix->n_desc[i];
        if (n) CM_CUDA(cudaMemcpyAsync(ix->arena + ix->slot_at[i] + slot_layout(&ix->p, n, false).desc, desc[k],
                                       (size_t)n * kDim, kind, s));
    }
    return CM_OK;
}

// Fills the device-table entries of placed images, marks them resident and
// uploads the tables of the batch that hash_batch processes next.
static cm_status publish(cm_index* ix, int32_t count, const int32_t* ids, const uint8_t* const* desc, bool inplace,
                         cudaStream_t s, int* n_tiles_out, int* n_tiles128_out) {
    ++ix->generation;
    std::vector<int32_t> batch(count), tiles(count + 1, 0), tiles128(count + 1, 0);
    for (int k = 0; k < count; ++k) {
        const int i = ids[k];
        const int64_t n = ix->n_desc[i];
        const SlotLayout L = slot_layout(&ix->p, n, inplace);
        uint8_t* base = ix->arena + ix->slot_at[i];
        DevImage& e = ix->h_imgs[i];
        e.n = (int32_t)n;
        e.desc = inplace ? desc[k] : base + L.desc;
        e.key = reinterpret_cast<uint64_t*>(base + L.key);
        e.code = reinterpret_cast<uint4*>(base + L.code);
        e.scode = reinterpret_cast<uint4*>(base + L.scode);
        e.sidx = reinterpret_cast<uint16_t*>(base + L.sidx);
        e.off = reinterpret_cast<uint32_t*>(base + L.off);
        e.hist = reinterpret_cast<uint32_t*>(base + L.hist);
        e.brank = base + L.brank;
        e.norm = reinterpret_cast<uint32_t*>(base + L.norm);
        e.xq = L.xq ? base + L.xq : nullptr;
        e.xscale = L.xscale ? reinterpret_cast<float*>(base + L.xscale) : nullptr;
        ix->pending[i] = 0;
        ix->resident[i] = 1;
        batch[k] = i;
        tiles[k + 1] = tiles[k] + (int)((n + kHashTile - 1) / kHashTile);
        tiles128[k + 1] = tiles128[k] + (int)((n + 127) / 128);
        CM_CUDA(cudaMemsetAsync(e.hist, 0, (size_t)ix->p.L * ix->B * 4, s));
    }
    cm_status st = upload_table(ix, ix->fx.imgs, ix->h_imgs.data(), ix->h_imgs.size() * sizeof(DevImage), s);
    if (st == CM_OK) st = upload_table(ix, ix->fx.batch, batch.data(), batch.size() * 4, s);
    if (st == CM_OK) st = upload_table(ix, ix->fx.tiles, tiles.data(), tiles.size() * 4, s);
    if (st == CM_OK) st = upload_table(ix, ix->fx.tiles128, tiles128.data(), tiles128.size() * 4, s);
    if (st != CM_OK) return st;
    *n_tiles_out = tiles[count];
    *n_tiles128_out = tiles128[count];
    return CM_OK;
}

static cm_status stage_images(cm_index* ix, int32_t count, const int32_t* ids, const uint8_t* const* desc,
                              int32_t mem, cudaStream_t s, int* n_tiles_out, int* n_tiles128_out) {
    cm_status st = check_loadable(ix, count, ids, desc, mem);
    if (st != CM_OK) return st;
    const bool inplace = mem == CM_MEM_DEVICE_INPLACE;
    if (!place_slots(ix, count, ids, inplace)) {
        uint64_t need = 0;
        for (int k = 0; k < count; ++k) need += slot_layout(&ix->p, ix->n_desc[ids[k]], inplace).total;
        return fail(CM_ERR_BUDGET, "load: arena full while placing %d images (%llu bytes)", count,
                    (unsigned long long)need);
    }
    if ((st = copy_descs(ix, count, ids, desc, mem, s)) != CM_OK) {
        index_cancel_prefetch(ix, count, ids);
        return st;
    }
    return publish(ix, count, ids, desc, inplace, s, n_tiles_out, n_tiles128_out);
}

// The resident-set table used by cm_index_rehash.
static cm_status refresh_resident(cm_index* ix, cudaStream_t s, int* n_batch, int* n_tiles, uint64_t* rows) {
    std::vector<int32_t> batch, tiles(1, 0), tiles128(1, 0);
    uint64_t r = 0;
    for (int i = 0; i < ix->n_images; ++i) {
        if (!ix->resident[i]) continue;
        batch.push_back(i);
        tiles.push_back(tiles.back() + (ix->n_desc[i] + kHashTile - 1) / kHashTile);
        tiles128.push_back(tiles128.back() + (ix->n_desc[i] + 127) / 128);
        r += (uint64_t)ix->n_desc[i];
    }
    cm_status st = upload_table(ix, ix->fx.rbatch, batch.data(), batch.size() * 4, s);
    if (st == CM_OK) st = upload_table(ix, ix->fx.rtiles, tiles.data(), tiles.size() * 4, s);
    if (st == CM_OK) st = upload_table(ix, ix->fx.rtiles128, tiles128.data(), tiles128.size() * 4, s);
    *n_batch = (int)batch.size();
    *n_tiles = tiles.back();
    *rows = r;
    return st;
}

static cm_status hash_batch(cm_index* ix, const HashLaunch& h, cudaStream_t s) {
    if (h.n_batch == 0) return CM_OK;
    if (ix->p.projection == CM_PROJ_TC) {
        CM_CUDA(launch_bias(ix->at<float>(ix->fx.W), ix->at<float>(ix->fx.mu), ix->P_pad, ix->at<float>(ix->fx.bias), s));
        CM_CUDA(launch_hash_tc(h, ix->sms, s));
    } else {
        CM_CUDA(launch_hash(h, ix->sms, s));
    }
    CM_CUDA(launch_bucket(h, s));
    if (tc_rerank(&ix->p)) CM_CUDA(launch_xcopy(h, s));
    return CM_OK;
}

static int tiles_of(const cm_index* ix, int rows_per_tile) {
    int t = 0;
    for (int i = 0; i < ix->n_images; ++i)
        if (ix->resident[i]) t += (ix->n_desc[i] + rows_per_tile - 1) / rows_per_tile;
    return t;
}

extern "C" cm_status cm_index_check(cm_index* ix, cm_stream stream) {
    if (!ix) return fail(CM_ERR_INVALID, "cm_index_check: NULL index");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int err = 0;
    CM_CUDA(cudaMemcpyAsync(&err, ix->arena + ix->fx.err, 4, cudaMemcpyDeviceToHost, s));
    CM_CUDA(cudaStreamSynchronize(s));
    if (err) {
        CM_CUDA(cudaMemsetAsync(ix->arena + ix->fx.err, 0, 4, s));
        CM_CUDA(cudaStreamSynchronize(s));
        return fail(CM_ERR_TIMEOUT, "a bounded device wait gave up; the affected results are invalid");
    }
    return CM_OK;
}

extern "C" cm_status cm_index_load(cm_index* ix, int32_t count, const int32_t* ids, const uint8_t* const* desc,
                                   int32_t mem, cm_stream stream) {
    if (!ix) return fail(CM_ERR_INVALID, "cm_index_load: NULL index");
    if (!ix->mean_set) return fail(CM_ERR_STATE, "cm_index_load: centring mean not set");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int n_tiles = 0, n_tiles128 = 0;
    cm_status st = stage_images(ix, count, ids, desc, mem, s, &n_tiles, &n_tiles128);
    if (st != CM_OK) return st;
    int rb = 0, rt = 0;
    uint64_t rows = 0;
    st = refresh_resident(ix, s, &rb, &rt, &rows);
    if (st != CM_OK) return st;
    return hash_batch(ix, ix->hash_launch(false, count, n_tiles, n_tiles128), s);
}

namespace cm {

cm_status index_prefetch(cm_index* ix, int32_t count, const int32_t* ids, const uint8_t* const* desc,
                         cudaStream_t copy_stream, bool* placed) {
    *placed = false;
    cm_status st = check_loadable(ix, count, ids, desc, CM_MEM_HOST);
    if (st != CM_OK) return st;
    if (!place_slots(ix, count, ids, false)) return CM_OK;   // no room yet: the caller loads later
    if ((st = copy_descs(ix, count, ids, desc, CM_MEM_HOST, copy_stream)) != CM_OK) {
        index_cancel_prefetch(ix, count, ids);
        return st;
    }
    *placed = true;
    return CM_OK;
}

cm_status index_publish(cm_index* ix, int32_t count, const int32_t* ids, cudaStream_t s, bool centre_first) {
    for (int k = 0; k < count; ++k)
        if (ids[k] < 0 || ids[k] >= ix->n_images || !ix->pending[ids[k]])
            return fail(CM_ERR_STATE, "publish: image %d was not prefetched", ids[k]);
    int n_tiles = 0, n_tiles128 = 0;
    cm_status st = publish(ix, count, ids, nullptr, false, s, &n_tiles, &n_tiles128);
    if (st != CM_OK) return st;
    int rb = 0, rt = 0;
    uint64_t rows = 0;
    st = refresh_resident(ix, s, &rb, &rt, &rows);
    if (st != CM_OK) return st;
    const HashLaunch h = ix->hash_launch(false, count, n_tiles, n_tiles128);
    if (centre_first) {
        // the batch's column sums join those already in fx.sums; then the mean of every image
        uint64_t total = 0;
        for (int i = 0; i < ix->n_images; ++i) total += (uint64_t)ix->n_desc[i];
        if (n_tiles) CM_CUDA(launch_colsum_images(h, ix->at<unsigned long long>(ix->fx.sums), s));
        if ((st = index_mean_from_sums(ix, total, s)) != CM_OK) return st;
    }
    return hash_batch(ix, h, s);
}

void index_cancel_prefetch(cm_index* ix, int32_t count, const int32_t* ids) {
    for (int k = 0; k < count; ++k) {
        const int i = ids[k];
        if (i >= 0 && i < ix->n_images && ix->pending[i]) {
            ix->alloc.release(ix->slot_at[i]);
            ix->pending[i] = 0;
        }
    }
}

}  // namespace cm

extern "C" cm_status cm_index_rehash(cm_index* ix, cm_stream stream) {
    if (!ix) return fail(CM_ERR_INVALID, "cm_index_rehash: NULL index");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int nb = 0, nt = 0;
    uint64_t rows = 0;
    // the resident table is current after every load/evict; recount on the host only
    for (int i = 0; i < ix->n_images; ++i)
        if (ix->resident[i]) {
            ++nb;
            nt += (ix->n_desc[i] + kHashTile - 1) / kHashTile;
            rows += (uint64_t)ix->n_desc[i];
        }
    if (!nb) return fail(CM_ERR_STATE, "cm_index_rehash: no resident image");
    const HashLaunch h = ix->hash_launch(true, nb, nt, tiles_of(ix, 128));
    unsigned long long* sums = ix->at<unsigned long long>(ix->fx.sums);
    CM_CUDA(cudaMemsetAsync(sums, 0, kDim * 8, s));
    CM_CUDA(launch_colsum_images(h, sums, s));
    CM_CUDA(launch_mean(sums, nullptr, rows, ix->at<float>(ix->fx.mu), s));
    ix->mean_set = true;
    ix->sums_on_host = false;
    ix->n_total = rows;
    return hash_batch(ix, h, s);
}

extern "C" cm_status cm_index_col_sums_of(cm_index* ix, int32_t count, const int32_t* ids, uint64_t* d_sums,
                                          cm_stream stream) {
    if (!ix || count < 0 || (count && !ids) || !d_sums) return fail(CM_ERR_INVALID, "cm_index_col_sums_of: bad argument");
    std::vector<int32_t> batch(count), tiles(count + 1, 0);
    for (int k = 0; k < count; ++k) {
        const int i = ids[k];
        if (i < 0 || i >= ix->n_images) return fail(CM_ERR_INVALID, "cm_index_col_sums_of: image id %d", i);
        if (!ix->resident[i]) return fail(CM_ERR_STATE, "cm_index_col_sums_of: image %d is not resident", i);
        batch[k] = i;
        tiles[k + 1] = tiles[k] + (ix->n_desc[i] + kHashTile - 1) / kHashTile;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    CM_CUDA(cudaMemsetAsync(d_sums, 0, kDim * 8, s));
    if (!count || !tiles[count]) return CM_OK;
    cm_status st = upload_table(ix, ix->fx.batch, batch.data(), batch.size() * 4, s);
    if (st == CM_OK) st = upload_table(ix, ix->fx.tiles, tiles.data(), tiles.size() * 4, s);
    if (st != CM_OK) return st;
    CM_CUDA(launch_colsum_images(ix->hash_launch(false, count, tiles[count], 0), reinterpret_cast<unsigned long long*>(d_sums),
                                 s));
    return CM_OK;
}

extern "C" cm_status cm_index_set_mean_device(cm_index* ix, const uint64_t* d_sums, uint64_t n_total, cm_stream stream) {
    if (!ix || !d_sums || !n_total) return fail(CM_ERR_INVALID, "cm_index_set_mean_device: bad argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned long long* sums = ix->at<unsigned long long>(ix->fx.sums);
    CM_CUDA(cudaMemcpyAsync(sums, d_sums, kDim * 8, cudaMemcpyDeviceToDevice, s));
    CM_CUDA(launch_mean(sums, nullptr, n_total, ix->at<float>(ix->fx.mu), s));
    ix->mean_set = true;
    ix->sums_on_host = false;
    ix->n_total = n_total;
    return CM_OK;
}

extern "C" cm_status cm_index_hash(cm_index* ix, cm_stream stream) {
    if (!ix) return fail(CM_ERR_INVALID, "cm_index_hash: NULL index");
    if (!ix->mean_set) return fail(CM_ERR_STATE, "cm_index_hash: centring mean not set");
    int nb = 0, nt = 0;
    for (int i = 0; i < ix->n_images; ++i)
        if (ix->resident[i]) {
            ++nb;
            nt += (ix->n_desc[i] + kHashTile - 1) / kHashTile;
        }
    if (!nb) return fail(CM_ERR_STATE, "cm_index_hash: no resident image");
    return hash_batch(ix, ix->hash_launch(true, nb, nt, tiles_of(ix, 128)), reinterpret_cast<cudaStream_t>(stream));
}

extern "C" cm_status cm_index_evict(cm_index* ix, int32_t count, const int32_t* ids, cm_stream stream) {
    if (!ix || count < 0 || (count && !ids)) return fail(CM_ERR_INVALID, "cm_index_evict: bad argument");
    for (int k = 0; k < count; ++k) {
        const int i = ids[k];
        if (i < 0 || i >= ix->n_images) return fail(CM_ERR_INVALID, "evict: image id %d out of range", i);
        if (!ix->resident[i]) return fail(CM_ERR_STATE, "evict: image %d is not resident", i);
    }
    ++ix->generation;
    for (int k = 0; k < count; ++k) {
        const int i = ids[k];
        ix->alloc.release(ix->slot_at[i]);
        ix->resident[i] = 0;
        DevImage& e = ix->h_imgs[i];
        const int n = e.n;
        e = DevImage{};
        e.n = n;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cm_status st = upload_table(ix, ix->fx.imgs, ix->h_imgs.data(), ix->h_imgs.size() * sizeof(DevImage), s);
    int rb = 0, rt = 0;
    uint64_t rows = 0;
    if (st == CM_OK) st = refresh_resident(ix, s, &rb, &rt, &rows);
    return st;
}

extern "C" cm_status cm_build_index(const cm_params* p, int32_t n_images, const int32_t* n_desc,
                                    const uint8_t* desc, int32_t mem, void* d_arena, uint64_t arena_bytes,
                                    cm_stream stream, cm_index** out) {
    if (!out || !desc) return fail(CM_ERR_INVALID, "cm_build_index: bad argument");
    cm_index* ix = nullptr;
    cm_status st = cm_index_create(p, n_images, n_desc, d_arena, arena_bytes, &ix);
    if (st != CM_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    std::vector<int32_t> ids(n_images);
    std::vector<const uint8_t*> ptrs(n_images);
    uint64_t row = 0;
    for (int i = 0; i < n_images; ++i) {
        ids[i] = i;
        ptrs[i] = desc + row * kDim;
        row += (uint64_t)n_desc[i];
    }
    int n_tiles = 0, n_tiles128 = 0;
    st = stage_images(ix, n_images, ids.data(), ptrs.data(), mem, s, &n_tiles, &n_tiles128);
    int rb = 0, rt = 0;
    uint64_t rows = 0;
    if (st == CM_OK) st = refresh_resident(ix, s, &rb, &rt, &rows);
    if (st == CM_OK) {
        // centring mean over every descriptor of the index, then hash all images
        const HashLaunch h = ix->hash_launch(false, n_images, n_tiles, n_tiles128);
        unsigned long long* sums = ix->at<unsigned long long>(ix->fx.sums);
        cudaError_t e = cudaMemsetAsync(sums, 0, kDim * 8, s);
        if (e == cudaSuccess) e = launch_colsum_images(h, sums, s);
        if (e == cudaSuccess) e = launch_mean(sums, nullptr, rows, ix->at<float>(ix->fx.mu), s);
        if (e != cudaSuccess) st = fail(CM_ERR_CUDA, "cm_build_index: %s", cudaGetErrorString(e));
        ix->mean_set = true;
        ix->n_total = rows;
        if (st == CM_OK) st = hash_batch(ix, h, s);
    }
    if (st != CM_OK) {
        cm_index_destroy(ix);
        return st;
    }
    *out = ix;
    return CM_OK;
}

extern "C" cm_status cm_index_image_view(const cm_index* ix, int32_t image, const void** keys, const void** codes,
                                         const void** sorted_codes, const void** sorted_idx, const void** offsets) {
    if (!ix || image < 0 || image >= ix->n_images) return fail(CM_ERR_INVALID, "image_view: bad image");
    if (!ix->resident[image]) return fail(CM_ERR_STATE, "image_view: image %d not resident", image);
    const DevImage& e = ix->h_imgs[image];
    if (keys) *keys = e.key;
    if (codes) *codes = e.code;
    if (sorted_codes) *sorted_codes = e.scode;
    if (sorted_idx) *sorted_idx = e.sidx;
    if (offsets) *offsets = e.off;
    return CM_OK;
}

// ---------------------------------------------------------------------------
// match plans
// ---------------------------------------------------------------------------
namespace cm {
std::vector<int32_t> pair_order(const std::vector<DevPair>& tab, const std::vector<int32_t>& n_desc) {
    std::vector<int32_t> ord(tab.size());
    for (size_t k = 0; k < tab.size(); ++k) ord[k] = (int32_t)k;
    std::stable_sort(ord.begin(), ord.end(), [&](int32_t a, int32_t b) {
        return (int64_t)n_desc[tab[a].i] * n_desc[tab[a].j] > (int64_t)n_desc[tab[b].i] * n_desc[tab[b].j];
    });
    return ord;
}
}  // namespace cm

// Validates a pair list and fills its work table.  Returns the plan's device
// bytes (cm_plan_bytes) and its row / item counts.
static cm_status plan_table(const cm_index* ix, const cm_pair* pairs, int64_t n_pairs, int S, std::vector<DevPair>& tab,
                            int64_t* rows_out, int64_t* items_out, int32_t* max_ni_out) {
    tab.assign((size_t)n_pairs, DevPair{});
    int64_t rows = 0, items = 0;
    int32_t max_ni = 0;
    for (int64_t k = 0; k < n_pairs; ++k) {
        const int i = pairs[k].i, j = pairs[k].j;
        if (i < 0 || j < 0 || i >= ix->n_images || j >= ix->n_images)
            return fail(CM_ERR_INVALID, "plan: pair %lld (%d,%d) has an image id out of range", (long long)k, i, j);
        if (i == j) return fail(CM_ERR_INVALID, "plan: pair %lld matches image %d with itself", (long long)k, i);
        if (!ix->resident[i] || !ix->resident[j])
            return fail(CM_ERR_STATE, "plan: pair %lld (%d,%d) needs an image that is not resident", (long long)k, i,
                        j);
        DevPair& d = tab[k];
        d.i = i;
        d.j = j;
        d.row_off = rows;
        d.item0 = (int32_t)items;
        d.nitems = (ix->n_desc[i] + S - 1) / S;
        d.ni = ix->n_desc[i];
        rows += ix->n_desc[i];
        items += d.nitems;
        max_ni = std::max(max_ni, ix->n_desc[i]);
    }
    if (items > INT32_MAX / 2) return fail(CM_ERR_INVALID, "plan: too many work items");
    {   // the reverse of each pair within the plan (first occurrence), for cm_match_plan_mutual
        std::map<std::pair<int, int>, int64_t> first;
        for (int64_t k = 0; k < n_pairs; ++k) first.emplace(std::make_pair(tab[k].i, tab[k].j), k);
        for (int64_t k = 0; k < n_pairs; ++k) {
            auto it = first.find(std::make_pair(tab[k].j, tab[k].i));
            tab[k].rev = it == first.end() ? -1 : (int32_t)it->second;
        }
    }
    *rows_out = rows;
    *items_out = items;
    *max_ni_out = max_ni;
    return CM_OK;
}

extern "C" cm_status cm_match_plan_create(cm_index* ix, const cm_pair* pairs, int64_t n_pairs, cm_stream stream,
                                          cm_match_plan** out) {
    if (!ix || !out || n_pairs < 0 || (n_pairs && !pairs)) return fail(CM_ERR_INVALID, "plan: bad argument");
    const int S = query_tile(&ix->p);
    std::vector<DevPair> tab;
    int64_t rows = 0, items = 0;
    int32_t max_ni = 0;
    cm_status st0 = plan_table(ix, pairs, n_pairs, S, tab, &rows, &items, &max_ni);
    if (st0 != CM_OK) return st0;
    cm_match_plan* pl = new (std::nothrow) cm_match_plan();
    if (!pl) return fail(CM_ERR_NOMEM, "plan: host allocation");
    const uint64_t bytes = plan_bytes(&ix->p, n_pairs, rows, max_ni);
    if (ix->plan_reserve_bytes >= bytes && !ix->plan_reserve_busy) {   // the pipeline's reserved block
        pl->table_at = ix->plan_reserve_at;
        pl->reserved = true;
        ix->plan_reserve_busy = true;
    } else if (!ix->alloc.alloc(bytes, &pl->table_at)) {
        delete pl;
        return fail(CM_ERR_BUDGET, "plan: arena full (%llu bytes for the pair table)", (unsigned long long)bytes);
    }
    pl->ix = ix;
    pl->p = ix->p;
    pl->S = S;
    ix->plans.insert(pl);
    pl->n_pairs = n_pairs;
    pl->rows = rows;
    pl->n_items = (int32_t)items;
    pl->max_ni = max_ni;
    if (n_pairs) {
        cm_status st = upload_table(ix, pl->table_at, tab.data(), tab.size() * sizeof(DevPair),
                                    reinterpret_cast<cudaStream_t>(stream));
        if (st == CM_OK && resolved_algo(&pl->p, n_pairs) == CM_ALGO_BUCKET) {
            const std::vector<int32_t> ord = pair_order(tab, ix->n_desc);
            const uint64_t at = pl->table_at + align_up((uint64_t)n_pairs * sizeof(DevPair)) + kAlign +
                                hand_over(&pl->p, n_pairs, rows, max_ni).order;
            st = upload_table(ix, at, ord.data(), ord.size() * 4, reinterpret_cast<cudaStream_t>(stream));
        }
        if (st != CM_OK) {
            ix->alloc.release(pl->table_at);
            delete pl;
            return st;
        }
    }
    *out = pl;
    return CM_OK;
}

extern "C" int64_t cm_match_plan_rows(const cm_match_plan* pl) { return pl ? pl->rows : -1; }

extern "C" cm_status cm_match_plan_run(cm_match_plan* pl, const cm_match_out* out, cm_stream stream) {
    return cm_match_plan_run_marked(pl, out, nullptr, stream);
}

extern "C" cm_status cm_match_plan_run_marked(cm_match_plan* pl, const cm_match_out* out, void* scan_done,
                                              cm_stream stream) {
    if (!pl || !out || (!out->best_j && pl->rows)) return fail(CM_ERR_INVALID, "plan_run: bad argument");
    cm_index* ix = pl->ix;
    if (!ix) return fail(CM_ERR_STATE, "plan_run: the plan's index was destroyed");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaEvent_t mark = reinterpret_cast<cudaEvent_t>(scan_done);
    if (!pl->n_items) {
        if (mark) CM_CUDA(cudaEventRecord(mark, s));
        return CM_OK;
    }
    uint8_t* counter_ptr = pl->base() + align_up((uint64_t)pl->n_pairs * sizeof(DevPair));
    unsigned* counter = reinterpret_cast<unsigned*>(counter_ptr);
    CM_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned), s));
    MatchLaunch m{};
    m.imgs = ix->at<DevImage>(ix->fx.imgs);
    m.pairs = reinterpret_cast<const DevPair*>(pl->base());
    m.n_pairs = (int32_t)pl->n_pairs;
    m.n_items = pl->n_items;
    const cm_params& pp = pl->p;
    m.S = pl->S;
    m.L = pp.L;
    m.m = pp.m;
    m.K = pp.K;
    m.ratio_num = pp.ratio_num;
    m.ratio_den = pp.ratio_den;
    m.ratio_lo = ratio_band(pp.ratio_num, pp.ratio_den).lo;
    m.ratio_hi = ratio_band(pp.ratio_num, pp.ratio_den).hi;
    m.rerank = pp.rerank;
    m.counter = counter;
    m.out = *out;
    m.algo = resolved_algo(&pp, pl->n_pairs);
    if (m.algo == CM_ALGO_TILE && match_smem_bytes(m.S, m.K) > kMatchSmemLimit) m.algo = CM_ALGO_WARP;
    m.err = ix->at<int>(ix->fx.err);
    const HandOver ho = hand_over(&pp, pl->n_pairs, pl->rows, pl->max_ni);
    uint8_t* base = counter_ptr + kAlign;
    if (m.algo == CM_ALGO_BUCKET) {
        m.klists = reinterpret_cast<uint32_t*>(base + ho.klists);
        m.order = reinterpret_cast<const int32_t*>(base + ho.order);
    }
    auto scan = [&]() -> cudaError_t {
        switch (m.algo) {
            case CM_ALGO_BUCKET: return launch_match_bm(m, ix->sms, s);
            case CM_ALGO_TILE: return launch_match(m, ix->sms, s);
            default: return launch_match_wq(m, ix->sms, s);
        }
    };
    if (needs_hand_over(&pp)) {
        // a scan leaves each query's top-K in the plan's hand-over area, then a rerank launch
        m.topk16 = reinterpret_cast<uint16_t*>(base + ho.idx);
        m.hnorm = reinterpret_cast<uint32_t*>(base + ho.norm);
        m.hscale = pp.rerank == CM_RERANK_FP8 ? reinterpret_cast<float*>(base + ho.scale) : nullptr;
        if (m.algo == CM_ALGO_TC) {
            m.lists = reinterpret_cast<uint32_t*>(base + ho.lists);
            m.max_ni = pl->max_ni;
            CM_CUDA(launch_scan_tc(m, std::min(ix->sms, kMaxScanCtas), s));
        } else {
            CM_CUDA(scan());
        }
        if (mark) CM_CUDA(cudaEventRecord(mark, s));
        CM_CUDA(tc_rerank(&pp) ? launch_rerank_tc(m, ix->sms, s) : launch_rerank_cc(m, ix->sms, s));
        return CM_OK;
    }
    CM_CUDA(scan());
    if (mark) CM_CUDA(cudaEventRecord(mark, s));
    return CM_OK;
}

extern "C" cm_status cm_match_plan_compact(cm_match_plan* pl, const int32_t* d_best_j, uint32_t* d_counts,
                                           uint64_t* d_offsets, uint64_t* d_total, uint32_t* d_matches,
                                           uint64_t capacity, cm_stream stream) {
    if (!pl || !d_best_j || !d_counts || !d_offsets) return fail(CM_ERR_INVALID, "compact: bad argument");
    if (!pl->ix) return fail(CM_ERR_STATE, "compact: the plan's index was destroyed");
    cm_index* ix = pl->ix;
    CM_CUDA(launch_compact(reinterpret_cast<const DevPair*>(pl->base()), (int)pl->n_pairs,
                           ix->at<DevImage>(ix->fx.imgs), d_best_j, d_counts,
                           reinterpret_cast<unsigned long long*>(d_offsets), reinterpret_cast<unsigned long long*>(d_total),
                           d_matches, (unsigned long long)capacity, reinterpret_cast<cudaStream_t>(stream)));
    return CM_OK;
}

extern "C" cm_status cm_match_plan_mutual(cm_match_plan* pl, const int32_t* d_best_in, int32_t* d_best_out,
                                          cm_stream stream) {
    if (!pl || !d_best_in || !d_best_out || d_best_in == d_best_out)
        return fail(CM_ERR_INVALID, "mutual: bad argument (in and out must differ)");
    if (!pl->ix) return fail(CM_ERR_STATE, "mutual: the plan's index was destroyed");
    cm_index* ix = pl->ix;
    CM_CUDA(launch_mutual(reinterpret_cast<const DevPair*>(pl->base()), (int)pl->n_pairs,
                          ix->at<DevImage>(ix->fx.imgs), d_best_in, d_best_out, reinterpret_cast<cudaStream_t>(stream)));
    return CM_OK;
}

extern "C" void cm_match_plan_destroy(cm_match_plan* pl) {
    if (!pl) return;
    if (pl->ix) {
        if (pl->reserved)
            pl->ix->plan_reserve_busy = false;
        else
            pl->ix->alloc.release(pl->table_at);
        pl->ix->plans.erase(pl);
        ++pl->ix->generation;
    }
    delete pl;
}

extern "C" void cm_index_destroy(cm_index* ix) {
    if (!ix) return;
    for (cm_match_plan* pl : ix->plans) pl->ix = nullptr;  // a plan outliving its index becomes inert
    for (cm_sequence* q : ix->seqs) cm_sequence_detach(q);
    delete ix;
}

// Device bytes cm_match_pairs needs for a pair list (sizes only; residency is
// checked by the call itself).
static cm_status pairs_bytes(const cm_index* ix, const cm_pair* pairs, int64_t n_pairs, uint64_t* bytes) {
    int64_t rows = 0;
    int32_t max_ni = 0;
    for (int64_t k = 0; k < n_pairs; ++k) {
        const int i = pairs[k].i;
        if (i < 0 || i >= ix->n_images || pairs[k].j < 0 || pairs[k].j >= ix->n_images)
            return fail(CM_ERR_INVALID, "workspace: pair %lld has an image id out of range", (long long)k);
        rows += ix->n_desc[i];
        max_ni = std::max(max_ni, ix->n_desc[i]);
    }
    *bytes = plan_bytes(&ix->p, n_pairs, rows, max_ni);
    return CM_OK;
}

extern "C" cm_status cm_match_pairs_workspace_bytes(const cm_index* ix, const cm_pair* pairs, int64_t n_pairs,
                                                    uint64_t* bytes) {
    if (!ix || !bytes || n_pairs < 0 || (n_pairs && !pairs))
        return fail(CM_ERR_INVALID, "cm_match_pairs_workspace_bytes: bad argument");
    return pairs_bytes(ix, pairs, n_pairs, bytes);
}

extern "C" cm_status cm_index_workspace_bytes(const cm_index* ix, const cm_schedule* s, int32_t block,
                                              uint64_t* bytes) {
    if (!ix || !s || !bytes) return fail(CM_ERR_INVALID, "cm_index_workspace_bytes: bad argument");
    const int32_t R = cm_schedule_num_rows(s);
    if (block < -1 || block >= R) return fail(CM_ERR_INVALID, "cm_index_workspace_bytes: block %d of %d", block, R);
    int64_t n_all = 0;
    const cm_pair* all = schedule_pairs(s, &n_all);
    uint64_t most = 0;
    for (int32_t r = (block < 0 ? 0 : block); r < (block < 0 ? R : block + 1); ++r) {
        cm_schedule_row row{};
        cm_status st = cm_schedule_get_row(s, r, &row);
        if (st != CM_OK) return st;
        std::vector<cm_pair> rp((size_t)row.n_pairs);
        for (int64_t k = 0; k < row.n_pairs; ++k) {
            if (row.pairs[k] < 0 || row.pairs[k] >= n_all)
                return fail(CM_ERR_INVALID, "cm_index_workspace_bytes: row %d names pair %lld", r,
                            (long long)row.pairs[k]);
            rp[k] = all[row.pairs[k]];
        }
        uint64_t b = 0;
        if ((st = pairs_bytes(ix, rp.data(), row.n_pairs, &b)) != CM_OK) return st;
        most = std::max(most, b);
    }
    *bytes = most;
    return CM_OK;
}

extern "C" cm_status cm_match_pairs(cm_index* ix, const cm_pair* pairs, int64_t n_pairs, void* d_workspace,
                                    uint64_t ws_bytes, int32_t* d_best_j, uint32_t* d_d1sq, uint32_t* d_d2sq,
                                    cm_stream stream) {
    if (!ix || n_pairs < 0 || (n_pairs && !pairs)) return fail(CM_ERR_INVALID, "cm_match_pairs: bad argument");
    if (!d_workspace || reinterpret_cast<uintptr_t>(d_workspace) % kAlign)
        return fail(CM_ERR_INVALID, "cm_match_pairs: the workspace must be a 256-byte aligned device pointer");
    const int S = query_tile(&ix->p);
    std::vector<DevPair> tab;
    int64_t rows = 0, items = 0;
    int32_t max_ni = 0;
    cm_status st = plan_table(ix, pairs, n_pairs, S, tab, &rows, &items, &max_ni);
    if (st != CM_OK) return st;
    if (rows && !d_best_j) return fail(CM_ERR_INVALID, "cm_match_pairs: d_best_j is NULL");
    const uint64_t need = plan_bytes(&ix->p, n_pairs, rows, max_ni);
    if (ws_bytes < need)
        return fail(CM_ERR_BUDGET, "cm_match_pairs: workspace of %llu bytes, %llu needed", (unsigned long long)ws_bytes,
                    (unsigned long long)need);
    // a plan whose table lives in the caller's workspace: nothing of the arena
    // is taken, so the call returns as soon as the launches are enqueued
    cm_match_plan pl;
    pl.ix = ix;
    pl.p = ix->p;
    pl.S = S;
    pl.ext = static_cast<uint8_t*>(d_workspace);
    pl.n_pairs = n_pairs;
    pl.rows = rows;
    pl.n_items = (int32_t)items;
    pl.max_ni = max_ni;
    if (n_pairs) {
        CM_CUDA(ix->staging.upload(pl.ext, tab.data(), tab.size() * sizeof(DevPair),
                                   reinterpret_cast<cudaStream_t>(stream)));
        if (resolved_algo(&pl.p, n_pairs) == CM_ALGO_BUCKET) {
            const std::vector<int32_t> ord = pair_order(tab, ix->n_desc);
            CM_CUDA(ix->staging.upload(pl.ext + align_up((uint64_t)n_pairs * sizeof(DevPair)) + kAlign +
                                           hand_over(&pl.p, n_pairs, rows, max_ni).order,
                                       ord.data(), ord.size() * 4, reinterpret_cast<cudaStream_t>(stream)));
        }
    }
    cm_match_out out{};
    out.best_j = d_best_j;
    out.d1sq = d_d1sq;
    out.d2sq = d_d2sq;
    return cm_match_plan_run(&pl, &out, stream);
}

extern "C" void cm_free_index(cm_index* ix) { cm_index_destroy(ix); }
