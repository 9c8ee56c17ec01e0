// Exhaustive nearest neighbours of every query over all of the database
// image, for a list of pairs, with the exact ratio test: the matches cascade
// hashing would give with every database point a candidate (Sec. 2.3.1 with
// K = N_J), i.e. the quality ceiling against which the lookup's recall is
// measured.
//
// k_nn_exhaustive: a work item is a tile of 128 queries of one pair.  The
// tile is staged once as the A operand; the database image is walked in
// chunks of up to 256 rows, each staged as the B operand and multiplied on
// the tensor cores (BF16, FP32 accumulate).  The product gives
// t = |y|^2 - 2 x.y directly: K is 144, the 128 descriptor elements (x
// against -2 y) and a block of 16 in which A holds (2^16, 2^8, 1, 0, ..) and B
// the base-256 digits of |y|^2.  That block is issued first, so the
// accumulator starts at |y|^2 and only decreases, to t >= -|x|^2: every
// partial sum is an integer of magnitude below 2^23, so exact.  The epilogue
// keeps, per query, the smallest (t, j) and the second smallest t; with
// d^2 = |x|^2 + t (exact) the last chunk is followed by the exact integer
// ratio test.  Producers, the MMA issuer and
// the epilogue are separate warps with double-buffered operands and
// accumulators (see the kernel).
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "cm_host.h"
#include "cm_stage.cuh"
#include "cm_tc.cuh"

namespace cm {

namespace {

constexpr int kNnRows = 128;      // queries per work item (M)
constexpr int kNnChunk = 256;     // database rows per MMA (N)
constexpr int kNnPolls = 1 << 24;

struct NnPair {
    int32_t i, j;
    int64_t row_off;   // first output row
    int32_t item0;     // first work item
    int32_t pad;
};

// k_nn_tile writes each database image once as BF16 operand tiles of 256 rows
// (72 KB each) in the MMA's shared-memory layout; a row past the image has
// y = 0 and digits (255, 0, 0), so its t = 255 * 2^16 is above every real t
// (|t| <= 128 * 255^2 < 2^23) and it is never a neighbour.
//
// Warp roles of k_nn_exhaustive ((5 + 4 kNnSplit) warps, one CTA per SM):
//   warps 0-3  producers: stage each work item's 128 query rows (A, converted
//              from uint8); one thread copies each database tile with a bulk
//              copy into one of two B buffers;
//   warp 4     MMA issuer: one thread, each chunk into one of two TMEM
//              accumulators (2 x 256 columns), commits that free the B
//              buffer, fill the accumulator and, after an item, free A;
//   warps 5..  epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 (one query
//              each) for part (w - 5) / 4 of every chunk's columns (the
//              kNnSplit warps of a lane quarter split the chunk), keeps q1
//              (d^2, j) and q2's d^2, and the parts are merged for the outputs.
// Copies, MMA and epilogue of neighbouring chunks overlap.  Every wait is
// bounded and also gives up once another role has aborted.
constexpr int kNnProd = 128;
constexpr int kNnMmaWarp = 4;
constexpr int kNnSplit = 4;                  // epilogue warps per TMEM lane quarter
constexpr int kNnEpiWarps = 4 * kNnSplit;    // each on 1 / kNnSplit of a chunk's columns
constexpr int kNnPipeThreads = (5 + kNnEpiWarps) * 32;
constexpr int kNnK = kDim + 16;               // descriptor elements + the |y|^2 block
constexpr uint32_t kNnA = kNnRows * kNnK * 2, kNnB = kNnChunk * kNnK * 2;

__device__ __forceinline__ bool nn_wait(uint64_t* mbar, uint32_t parity, volatile int* abort_flag) {
    for (int it = 0; it < kNnPolls; it += 64) {
        if (tc::mbar_wait(mbar, parity, 64)) return true;
        if (*abort_flag) return false;
    }
    return false;
}

// One work item: a tile of up to 128 queries of one pair.
struct NnItem {
    int64_t oi, oj, row0;
    int ni, nj, q0, pj;
};

__device__ __forceinline__ NnItem nn_item(const NnPair* pairs, int n_pairs, const int64_t* img_off, int item) {
    int lo = 0, hi = n_pairs;   // last pair with item0 <= item
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (pairs[mid].item0 <= item) lo = mid; else hi = mid;
    }
    const NnPair P = pairs[lo];
    NnItem t;
    t.oi = img_off[P.i];
    t.oj = img_off[P.j];
    t.ni = (int)(img_off[P.i + 1] - t.oi);
    t.nj = (int)(img_off[P.j + 1] - t.oj);
    t.q0 = (item - P.item0) * kNnRows;
    t.row0 = P.row_off + t.q0;
    t.pj = P.j;
    return t;
}

// Named barrier 1 over the epilogue warps with an OR of a predicate.
__device__ __forceinline__ bool epi_bar_or(bool v) {
    uint32_t r;
    asm volatile("{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbarrier.cta.red.or.pred q, 1, %2, p;\n"
                 "selp.u32 %0, 1, 0, q;\n}\n"
                 : "=r"(r) : "r"((uint32_t)v), "n"(kNnEpiWarps * 32) : "memory");
    return r != 0;
}

__device__ __forceinline__ uint32_t row_norm(const uint8_t* row) {
    uint32_t nn = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(row) + c);
        nn = __dp4a(v.x, v.x, nn);
        nn = __dp4a(v.y, v.y, nn);
        nn = __dp4a(v.z, v.z, nn);
        nn = __dp4a(v.w, v.w, nn);
    }
    return nn;
}

// Bytes b0 and b0+1 of w, each times -2, as two BF16 values: 2^23 + b by one
// byte permute, then 2^24 - 2 (2^23 + b) = -2b exactly (at most 8
// significant bits, so the FP32 upper half is its exact BF16).
__device__ __forceinline__ uint32_t u8x2_to_bf16x2_m2(uint32_t w, int b0) {
    const float f0 = fmaf(__uint_as_float(__byte_perm(w, 0x4B000000u, 0x7540 + b0)), -2.f, 16777216.f);
    const float f1 = fmaf(__uint_as_float(__byte_perm(w, 0x4B000000u, 0x7541 + b0)), -2.f, 16777216.f);
    return __byte_perm(__float_as_uint(f0), __float_as_uint(f1), 0x7632);
}

__device__ __forceinline__ uint32_t bf16_hi(float f) { return __float_as_uint(f) >> 16; }

__global__ void __launch_bounds__(kNnChunk)
k_nn_tile(const uint8_t* __restrict__ desc, const int64_t* __restrict__ img_off, const int32_t* __restrict__ chunk_img,
          const int32_t* __restrict__ chunk_c0, unsigned char* __restrict__ tiles) {
    const int c = blockIdx.x, r = threadIdx.x;
    const int img = chunk_img[c];
    const int64_t o = img_off[img];
    const int n = (int)(img_off[img + 1] - o), row = chunk_c0[c] + r;
    const bool have = row < n;
    uint4 v[8];
    stage::load_row(desc + (size_t)(o + (have ? row : 0)) * kDim, have, v);
    unsigned char* tile = tiles + (size_t)c * kNnB;
    uint32_t nn = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        nn = __dp4a(v[k].x, v[k].x, nn);
        nn = __dp4a(v[k].y, v[k].y, nn);
        nn = __dp4a(v[k].z, v[k].z, nn);
        nn = __dp4a(v[k].w, v[k].w, nn);
        uint4 lo, hi;
        lo.x = u8x2_to_bf16x2_m2(v[k].x, 0); lo.y = u8x2_to_bf16x2_m2(v[k].x, 2);
        lo.z = u8x2_to_bf16x2_m2(v[k].y, 0); lo.w = u8x2_to_bf16x2_m2(v[k].y, 2);
        hi.x = u8x2_to_bf16x2_m2(v[k].z, 0); hi.y = u8x2_to_bf16x2_m2(v[k].z, 2);
        hi.z = u8x2_to_bf16x2_m2(v[k].w, 0); hi.w = u8x2_to_bf16x2_m2(v[k].w, 2);
        *reinterpret_cast<uint4*>(tile + tc::chunk_off(r, 2 * k, kNnChunk)) = lo;
        *reinterpret_cast<uint4*>(tile + tc::chunk_off(r, 2 * k + 1, kNnChunk)) = hi;
    }
    // |y|^2 <= 128 * 255^2 < 2^23: digits (|y|^2 >> 16, (|y|^2 >> 8) & 255, |y|^2 & 255)
    const uint32_t d0 = have ? nn >> 16 : 255u, d1 = have ? (nn >> 8) & 255u : 0u, d2 = have ? nn & 255u : 0u;
    uint4 dg;
    dg.x = bf16_hi((float)d0) | (bf16_hi((float)d1) << 16);
    dg.y = bf16_hi((float)d2);
    dg.z = 0;
    dg.w = 0;
    *reinterpret_cast<uint4*>(tile + tc::chunk_off(r, 16, kNnChunk)) = dg;
    *reinterpret_cast<uint4*>(tile + tc::chunk_off(r, 17, kNnChunk)) = make_uint4(0, 0, 0, 0);
}

// The 9 MMAs (K = 16 each) of one chunk: the |y|^2 block first (overwriting
// the accumulator), then the 8 descriptor blocks.
__device__ __forceinline__ void mma_chunk(uint32_t tmem_d, const unsigned char* A, const unsigned char* B) {
    constexpr uint32_t lbo_a = (kNnRows / 8) * 128, lbo_b = (kNnChunk / 8) * 128;
    const uint32_t a0 = tc::smem_addr(A), b0 = tc::smem_addr(B);
    constexpr uint32_t idesc = tc::idesc_f16(kNnRows, kNnChunk, 1);
    tc::mma_f16(tmem_d, tc::smem_desc(a0 + 16 * lbo_a, lbo_a, 128), tc::smem_desc(b0 + 16 * lbo_b, lbo_b, 128), idesc, 0);
#pragma unroll
    for (int ks = 0; ks < kDim / 16; ++ks)
        tc::mma_f16(tmem_d, tc::smem_desc(a0 + ks * 2 * lbo_a, lbo_a, 128), tc::smem_desc(b0 + ks * 2 * lbo_b, lbo_b, 128),
                    idesc, 1);
}

__device__ __forceinline__ float min3f(float a, float b, float c) {
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

__global__ void __launch_bounds__(kNnPipeThreads, 1)
k_nn_exhaustive(const uint8_t* __restrict__ desc, const int64_t* __restrict__ img_off, const NnPair* __restrict__ pairs,
                int n_pairs, int n_items, int ratio_num, int ratio_den, const unsigned char* __restrict__ tiles,
                const int64_t* __restrict__ tile_of, int32_t* __restrict__ best_j, uint32_t* __restrict__ d1sq,
                uint32_t* __restrict__ d2sq, int* err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* At = smem;                                   // 128 rows x K
    unsigned char* Bt = At + kNnA;                              // 2 x 256 rows x K
    uint64_t* bar = reinterpret_cast<uint64_t*>(Bt + 2 * kNnB);
    uint64_t *fullB = bar, *emptyB = bar + 2, *accFull = bar + 4, *accEmpty = bar + 6, *fullA = bar + 8,
             *emptyA = bar + 9;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    __shared__ float s_part_e1[kNnSplit - 1][kNnRows], s_part_e2[kNnSplit - 1][kNnRows];   // partial results
    __shared__ int s_part_j1[kNnSplit - 1][kNnRows];                                        // of parts 1..
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const float kInf = __uint_as_float(0x7F800000u);
    if (tid == 0) {
        for (int k = 0; k < 2; ++k) {
            tc::mbar_init(&fullB[k], 1);
            tc::mbar_init(&emptyB[k], 1);
            tc::mbar_init(&accFull[k], 1);
            tc::mbar_init(&accEmpty[k], kNnEpiWarps * 32);
        }
        tc::mbar_init(fullA, kNnProd);
        tc::mbar_init(emptyA, 1);
        s_abort = 0;
    }
    if (warp == kNnMmaWarp) tc::tmem_alloc(&s_tmem, 2 * kNnChunk);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = s_tmem;
    volatile int* abort_flag = &s_abort;
    auto give_up = [&]() {
        *abort_flag = 1;
        atomicExch(err, 1);
    };

    if (warp < 4) {
        // ---------------- producers
        {   // A's |y|^2 block, the same for every item: (2^16, 2^8, 1, 0, ..)
            const uint4 w = make_uint4(bf16_hi(65536.f) | (bf16_hi(256.f) << 16), bf16_hi(1.f), 0, 0);
            *reinterpret_cast<uint4*>(At + tc::chunk_off(tid, 16, kNnRows)) = w;
            *reinterpret_cast<uint4*>(At + tc::chunk_off(tid, 17, kNnRows)) = make_uint4(0, 0, 0, 0);
        }
        uint32_t g = 0, it = 0;
        bool ok = true;
        for (int item = blockIdx.x; item < n_items && ok; item += gridDim.x, ++it) {
            const NnItem t = nn_item(pairs, n_pairs, img_off, item);
            if (!nn_wait(emptyA, (it & 1u) ^ 1u, abort_flag)) { ok = false; break; }
            uint4 v[8];
            const bool qv = t.q0 + tid < t.ni;
            stage::load_row(desc + (size_t)(t.oi + t.q0 + (qv ? tid : 0)) * kDim, qv, v);
            stage::store_row(v, At, tid, kNnRows);
            tc::fence_proxy_async();
            tc::mbar_arrive(fullA);
            if (tid == 0) {   // the database tiles of this item, one bulk copy each
                const int64_t tb = tile_of[t.pj];
                for (int c0 = 0; c0 < t.nj; c0 += kNnChunk, ++g) {
                    const uint32_t s = g & 1u, ph = (g >> 1) & 1u;
                    if (!nn_wait(&emptyB[s], ph ^ 1u, abort_flag)) { ok = false; break; }
                    const int64_t c = tb + c0 / kNnChunk;
                    tc::mbar_arrive_expect_tx(&fullB[s], kNnB);
                    tc::bulk_g2s(Bt + s * kNnB, tiles + (size_t)c * kNnB, kNnB, &fullB[s]);
                }
            }
        }
        if (!ok) give_up();
    } else if (warp == kNnMmaWarp) {
        // ---------------- MMA issuer
        if (lane == 0) {
            uint32_t g = 0, it = 0;
            int64_t last = -1;   // the last chunk committed
            bool ok = true;
            for (int item = blockIdx.x; item < n_items && ok; item += gridDim.x, ++it) {
                const NnItem t = nn_item(pairs, n_pairs, img_off, item);
                if (!nn_wait(fullA, it & 1u, abort_flag)) { ok = false; break; }
                for (int c0 = 0; c0 < t.nj; c0 += kNnChunk, ++g) {
                    const uint32_t s = g & 1u, ph = (g >> 1) & 1u;
                    if (!nn_wait(&fullB[s], ph, abort_flag) || !nn_wait(&accEmpty[s], ph ^ 1u, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc::fence_after();
                    mma_chunk(tmem + s * kNnChunk, At, Bt + s * kNnB);   // whole tiles
                    tc::commit(&emptyB[s]);
                    tc::commit(&accFull[s]);
                    last = g;
                }
                if (ok) tc::commit(emptyA);   // A is free once this item's MMAs have read it
            }
            if (!ok) give_up();
            // the tensor memory is freed below: wait (bounded) for the last MMAs issued
            if (last >= 0) tc::mbar_wait(&accFull[last & 1], (uint32_t)(last >> 1) & 1u, kNnPolls);
        }
        __syncwarp();
    } else {
        // ---------------- epilogue: query row 32 (warp % 4) + lane of each item,
        // columns [part * H, part * H + H) of every chunk
        const int row = 32 * (warp & 3) + lane;
        const int part = (warp - 5) / 4;
        const uint32_t lane_base = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
        constexpr int H = kNnChunk / kNnSplit;
        uint32_t g = 0;
        bool ok = true;
        for (int item = blockIdx.x; item < n_items && ok; item += gridDim.x) {
            const NnItem t = nn_item(pairs, n_pairs, img_off, item);
            const int q = t.q0 + row;
            const bool qv = q < t.ni;
            const float nq = qv && part == 0 ? (float)row_norm(desc + (size_t)(t.oi + q) * kDim) : 0.f;
            float e1 = kInf, e2 = kInf;
            int j1 = -1;
            for (int c0 = 0; c0 < t.nj; c0 += kNnChunk, ++g) {
                const uint32_t s = g & 1u, ph = (g >> 1) & 1u;
                // every lane waits itself: its TMEM loads are ordered after the phase only if it saw it
                const bool got = nn_wait(&accFull[s], ph, abort_flag);
                if (!__all_sync(0xFFFFFFFFu, got)) { ok = false; break; }
                tc::fence_after();
                // the accumulator holds t = |y|^2 - 2 x.y (exact); d^2 = |x|^2 + t is
                // added at the end.  A group of 16 columns with no t below q2's is
                // skipped whole: it cannot change q1 or q2.
#pragma unroll
                for (int cc = part * H; cc < part * H + H; cc += 16) {
                    uint32_t acc[16];
                    tc::tmem_load16(lane_base + s * kNnChunk + cc, acc);
                    float tv[16];
#pragma unroll
                    for (int u = 0; u < 16; ++u) tv[u] = __uint_as_float(acc[u]);
                    const float m = fminf(min3f(min3f(tv[0], tv[1], tv[2]), min3f(tv[3], tv[4], tv[5]), min3f(tv[6], tv[7], tv[8])),
                                          min3f(min3f(tv[9], tv[10], tv[11]), min3f(tv[12], tv[13], tv[14]), tv[15]));
                    if (__any_sync(0xFFFFFFFFu, m < e2)) {
                        const int jb = c0 + cc;
#pragma unroll
                        for (int u = 0; u < 16; ++u) {
                            j1 = tv[u] < e1 ? jb + u : j1;   // columns in ascending j: a tie keeps the smaller j
                            e2 = fminf(e2, fmaxf(e1, tv[u]));
                            e1 = fminf(e1, tv[u]);
                        }
                    }
                }
                tc::fence_before();
                tc::mbar_arrive(&accEmpty[s]);
            }
            if (!ok) give_up();
            // merge the column parts of each row: parts 1.. post their partial
            // results, and one barrier of the epilogue warps both orders the
            // exchange and decides, the same way for every warp, whether to stop
            if (part > 0) {
                s_part_e1[part - 1][row] = e1;
                s_part_e2[part - 1][row] = e2;
                s_part_j1[part - 1][row] = j1;
            }
            if (epi_bar_or(!ok || *abort_flag)) break;
            if (part == 0 && qv) {
#pragma unroll
                for (int p = 0; p < kNnSplit - 1; ++p) {   // (q1, q2) of a union: ties keep the smaller j
                    const float f1 = s_part_e1[p][row], f2 = s_part_e2[p][row];
                    const int k1 = s_part_j1[p][row];
                    const bool take = f1 < e1 || (f1 == e1 && k1 >= 0 && (j1 < 0 || k1 < j1));
                    const float m2 = fminf(fmaxf(e1, f1), fminf(e2, f2));
                    j1 = take ? k1 : j1;
                    e1 = fminf(e1, f1);
                    e2 = m2;
                }
                const int64_t o = t.row0 + row;
                const bool has2 = t.nj >= 2;   // e2 is finite exactly when J has two rows
                const uint32_t u1 = j1 >= 0 ? (uint32_t)(e1 + nq) : 0xFFFFFFFFu,   // exact sums of integers
                               u2 = has2 ? (uint32_t)(e2 + nq) : 0xFFFFFFFFu;
                const bool pass = has2 && (int64_t)ratio_den * ratio_den * u1 < (int64_t)ratio_num * ratio_num * u2;
                best_j[o] = pass ? j1 : -1;
                if (d1sq) d1sq[o] = u1;
                if (d2sq) d2sq[o] = u2;
            }
            epi_bar_or(false);   // the parts are read before the next item overwrites them
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == kNnMmaWarp) tc::tmem_dealloc(tmem, 2 * kNnChunk);
}

// Workspace: error flag (fixed place), image offsets, pair records, the tile
// index of each image (-1: not a database image here), the chunk table, the
// database images' BF16 tiles (72 KB per 256 rows).
struct NnWork {
    uint64_t err, off, pairs, tile_of, chunk_img, chunk_c0, tiles, total;
};

NnWork nn_layout(int32_t n_images, int64_t n_pairs, int64_t n_chunks) {
    NnWork w{};
    w.err = 0;
    w.off = align_up(4);
    w.pairs = align_up(w.off + 8 * (uint64_t)(n_images + 1));
    w.tile_of = align_up(w.pairs + sizeof(NnPair) * (uint64_t)n_pairs);
    w.chunk_img = align_up(w.tile_of + 8 * (uint64_t)std::max(n_images, 1));
    w.chunk_c0 = align_up(w.chunk_img + 4 * (uint64_t)n_chunks);
    w.tiles = align_up(w.chunk_c0 + 4 * (uint64_t)n_chunks);
    w.total = align_up(w.tiles + (uint64_t)kNnB * (uint64_t)n_chunks);
    return w;
}

// The database images of the pair list in first-use order and their tiles.
struct NnTiles {
    std::vector<int64_t> tile_of;   // [n_images]
    std::vector<int32_t> chunk_img, chunk_c0;
};

cm_status nn_tiles(const int64_t* img_off, int32_t n_images, const cm_pair* pairs, int64_t n_pairs, NnTiles* t) {
    t->tile_of.assign((size_t)std::max(n_images, 0), -1);
    t->chunk_img.clear();
    t->chunk_c0.clear();
    for (int64_t k = 0; k < n_pairs; ++k) {
        const cm_pair pr = pairs[k];
        if (pr.i < 0 || pr.j < 0 || pr.i >= n_images || pr.j >= n_images)
            return host_fail(CM_ERR_INVALID, "cm_nn_pairs: pair %lld names an image out of range", (long long)k);
        if (t->tile_of[pr.j] >= 0) continue;
        t->tile_of[pr.j] = (int64_t)t->chunk_img.size();
        const int64_t n = img_off[pr.j + 1] - img_off[pr.j];
        for (int64_t c0 = 0; c0 < n; c0 += kNnChunk) {
            t->chunk_img.push_back(pr.j);
            t->chunk_c0.push_back((int32_t)c0);
        }
    }
    return CM_OK;
}

cm_status nn_check_offsets(const int64_t* img_off, int32_t n_images) {
    if (n_images < 0 || !img_off) return host_fail(CM_ERR_INVALID, "cm_nn_pairs: bad image offsets");
    if (img_off[0] != 0) return host_fail(CM_ERR_INVALID, "cm_nn_pairs: img_off[0] must be 0");
    for (int32_t i = 0; i < n_images; ++i)
        if (img_off[i + 1] < img_off[i] || img_off[i + 1] - img_off[i] > 65535)
            return host_fail(CM_ERR_INVALID, "cm_nn_pairs: img_off not ascending or an image above 65535 rows");
    return CM_OK;
}

}  // namespace

}  // namespace cm

using namespace cm;

extern "C" cm_status cm_nn_workspace_bytes(const int64_t* img_off, int32_t n_images, const cm_pair* pairs,
                                           int64_t n_pairs, uint64_t* bytes) {
    if (n_pairs < 0 || (n_pairs && !pairs) || !bytes) return host_fail(CM_ERR_INVALID, "cm_nn_workspace_bytes: bad argument");
    cm_status st = nn_check_offsets(img_off, n_images);
    if (st != CM_OK) return st;
    NnTiles t;
    if ((st = nn_tiles(img_off, n_images, pairs, n_pairs, &t)) != CM_OK) return st;
    *bytes = nn_layout(n_images, n_pairs, (int64_t)t.chunk_img.size()).total;
    return CM_OK;
}

extern "C" cm_status cm_nn_pairs(const uint8_t* desc, const int64_t* img_off, int32_t n_images, const cm_pair* pairs,
                                 int64_t n_pairs, int32_t ratio_num, int32_t ratio_den, void* d_work,
                                 uint64_t work_bytes, int32_t* best_j, uint32_t* d1sq, uint32_t* d2sq,
                                 cm_stream stream) {
    if (n_pairs < 0 || (n_pairs && (!pairs || !best_j)) || !d_work || ratio_num < 1 || ratio_den <= ratio_num ||
        ratio_den > 1024)
        return host_fail(CM_ERR_INVALID, "cm_nn_pairs: bad argument");
    cm_status st = nn_check_offsets(img_off, n_images);
    if (st != CM_OK) return st;
    NnTiles tl;
    if ((st = nn_tiles(img_off, n_images, pairs, n_pairs, &tl)) != CM_OK) return st;
    const int64_t n_chunks = (int64_t)tl.chunk_img.size();
    const NnWork w = nn_layout(n_images, n_pairs, n_chunks);
    if (work_bytes < w.total || (reinterpret_cast<uintptr_t>(d_work) & (kAlign - 1)))
        return host_fail(CM_ERR_BUDGET, "cm_nn_pairs: workspace smaller than cm_nn_workspace_bytes or not 256-byte aligned");
    std::vector<NnPair> rec((size_t)n_pairs);
    int64_t rows = 0, items = 0;
    for (int64_t k = 0; k < n_pairs; ++k) {
        const cm_pair pr = pairs[k];
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
    CM_CUDA(cudaMemcpyAsync(base + w.tile_of, tl.tile_of.data(), 8 * tl.tile_of.size(), cudaMemcpyHostToDevice, s));
    if (n_chunks) {
        CM_CUDA(cudaMemcpyAsync(base + w.chunk_img, tl.chunk_img.data(), 4 * (size_t)n_chunks, cudaMemcpyHostToDevice, s));
        CM_CUDA(cudaMemcpyAsync(base + w.chunk_c0, tl.chunk_c0.data(), 4 * (size_t)n_chunks, cudaMemcpyHostToDevice, s));
        k_nn_tile<<<(unsigned)n_chunks, kNnChunk, 0, s>>>(desc, reinterpret_cast<const int64_t*>(base + w.off),
                                                          reinterpret_cast<const int32_t*>(base + w.chunk_img),
                                                          reinterpret_cast<const int32_t*>(base + w.chunk_c0),
                                                          base + w.tiles);
        CM_CUDA(cudaGetLastError());
    }
    int dev = 0, sms = 148;
    CM_CUDA(cudaGetDevice(&dev));
    CM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // one CTA per SM: A and two B buffers in shared memory, two 256-column
    // accumulators (all of TMEM)
    const size_t smem = (size_t)kNnA + 2 * (size_t)kNnB + 16 * 8 + 1024;
    CM_CUDA(cudaFuncSetAttribute(k_nn_exhaustive, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int grid = (int)std::min<int64_t>(items, (int64_t)sms);
    k_nn_exhaustive<<<grid, kNnPipeThreads, smem, s>>>(
        desc, reinterpret_cast<const int64_t*>(base + w.off), reinterpret_cast<const NnPair*>(base + w.pairs),
        (int)n_pairs, (int)items, ratio_num, ratio_den, base + w.tiles, reinterpret_cast<const int64_t*>(base + w.tile_of),
        best_j, d1sq, d2sq, err);
    CM_CUDA(cudaGetLastError());
    return CM_OK;
}
