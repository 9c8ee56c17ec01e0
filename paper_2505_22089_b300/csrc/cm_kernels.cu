// Device kernels of the cascade-hashing matcher (sm_103a).
//
//  k_colsum_*   exact uint64 column sums of the descriptors (centring statistics)
//  k_mean       mu = sums / N (FP64 division, FP32 result)
//  k_hash       centring + projection onto the L*m coarse and 128 fine hyperplanes
//               (FP32 FFMA), sign bits -> bucket keys and codes, squared norms,
//               per-image bucket histograms (Sec. 2.3.1 steps (1)-(2); Sec. 2.3.2 step (1))
//  k_bucket     per (image, table): exclusive scan of the histogram and a stable
//               scatter of codes and indices into bucket order (the lookup tables
//               of Sec. 2.3.1 step (1))
//  k_match      persistent fused matcher over all pairs of a block: bucket lookup,
//               Hamming ranking to the top K, Euclidean rerank and ratio test
//               (Sec. 2.3.1 steps (1)-(4))
#include <cuda_runtime.h>
#include <cstdint>

#include "cm_internal.h"

namespace cm {

// ---------------------------------------------------------------------------
// centring statistics
// ---------------------------------------------------------------------------

// 256 threads: 32 rows x 8 chunks of 16 bytes per pass.
__device__ __forceinline__ void colsum_accum(uint4 v, uint32_t acc[16]) {
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int u = 0; u < 16; ++u) acc[u] += (w[u >> 2] >> (8 * (u & 3))) & 0xFFu;
}

__device__ __forceinline__ void colsum_flush(uint32_t acc[16], unsigned long long* sums) {
    __shared__ unsigned long long red[128];
    const int tid = threadIdx.x, c = tid & 7;
    if (tid < 128) red[tid] = 0ull;
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 16; ++u) atomicAdd(&red[16 * c + u], (unsigned long long)acc[u]);
    __syncthreads();
    if (tid < 128 && red[tid]) atomicAdd(&sums[tid], red[tid]);
}

__global__ void __launch_bounds__(256) k_colsum_rows(const uint8_t* __restrict__ desc, uint64_t n_rows,
                                                     unsigned long long* __restrict__ sums) {
    uint32_t acc[16] = {0};
    const int c = threadIdx.x & 7, r0 = threadIdx.x >> 3;
    // a thread adds at most n_rows / (32 * gridDim.x) rows of <= 255: bounded by the launch (< 2^32)
    for (uint64_t r = (uint64_t)blockIdx.x * 32 + r0; r < n_rows; r += (uint64_t)gridDim.x * 32) {
        uint4 v = __ldg(reinterpret_cast<const uint4*>(desc + r * kDim) + c);
        colsum_accum(v, acc);
    }
    colsum_flush(acc, sums);
}

__device__ __forceinline__ int find_batch(const int32_t* pref, int n, int tile) {
    int lo = 0, hi = n;  // pref[lo] <= tile < pref[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (pref[mid] <= tile) lo = mid; else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(256) k_colsum_images(HashLaunch h, unsigned long long* __restrict__ sums) {
    uint32_t acc[16] = {0};
    const int c = threadIdx.x & 7, r0 = threadIdx.x >> 3;
    for (int tile = blockIdx.x; tile < h.n_tiles; tile += gridDim.x) {
        const int b = find_batch(h.tile_pref, h.n_batch, tile);
        const DevImage& e = h.imgs[h.batch[b]];
        const int row0 = (tile - h.tile_pref[b]) * kHashTile;
        for (int d = r0; d < kHashTile; d += 32) {
            if (row0 + d < e.n) {
                uint4 v = __ldg(reinterpret_cast<const uint4*>(e.desc + (size_t)(row0 + d) * kDim) + c);
                colsum_accum(v, acc);
            }
        }
    }
    colsum_flush(acc, sums);
}

__global__ void k_count_rows(HashLaunch h, unsigned long long* n_total) {
    unsigned long long s = 0;
    for (int b = threadIdx.x; b < h.n_batch; b += blockDim.x) s += (unsigned long long)h.imgs[h.batch[b]].n;
    atomicAdd(n_total, s);
}

__global__ void k_mean(const unsigned long long* __restrict__ sums, const unsigned long long* __restrict__ n_dev,
                       uint64_t n_host, float* __restrict__ mu) {
    const int k = threadIdx.x;
    const double n = (double)(n_dev ? *n_dev : n_host);
    if (k < kDim) mu[k] = n > 0 ? (float)((double)sums[k] / n) : 0.f;
}

// ---------------------------------------------------------------------------
// hashing: keys, codes, norms, bucket histograms
// ---------------------------------------------------------------------------

__device__ __forceinline__ void put_bits(uint64_t w[3], int pos, uint64_t v, int len) {
    const int wi = pos >> 6, sh = pos & 63;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        if (q == wi) w[q] |= v << sh;
        if (q == wi + 1 && sh + len > 64) w[q] |= v >> (64 - sh);
    }
}

__device__ __forceinline__ uint32_t get_bits(const uint64_t w[3], int pos, int len) {
    const int wi = pos >> 6, sh = pos & 63;
    uint64_t lo = 0, hi = 0;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        if (q == wi) lo = w[q];
        if (q == wi + 1) hi = w[q];
    }
    uint64_t v = lo >> sh;
    if (sh && sh + len > 64) v |= hi << (64 - sh);
    const uint64_t mask = len >= 32 ? 0xFFFFFFFFull : ((1ull << len) - 1ull);
    return (uint32_t)(v & mask);
}

template <int NPG>
__global__ void __launch_bounds__(kHashThreads, 1) k_hash(HashLaunch h) {
    constexpr int P_pad = 4 * NPG;
    constexpr int XS = kDim + 1;                 // padded row of the transposed tile
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* Ws = reinterpret_cast<float*>(smem_raw);            // [128][P_pad]
    float* xs = Ws + kDim * P_pad;                             // [128][65] (transposed tile)
    uint64_t* pb = reinterpret_cast<uint64_t*>(xs + kDim * (kHashTile + 1));  // [64][4]
    uint32_t* hist = reinterpret_cast<uint32_t*>(pb + kHashTile * 4);        // [L][B]
    __shared__ float mus[kDim];
    (void)XS;

    const int tid = threadIdx.x;
    for (int e = tid; e < kDim * P_pad; e += kHashThreads) Ws[e] = h.W[e];
    if (tid < kDim) mus[tid] = h.mu[tid];
    const int B = 1 << h.m;
    const int LB = h.L * B;

    for (int tile = blockIdx.x; tile < h.n_tiles; tile += gridDim.x) {
        __syncthreads();
        const int bidx = find_batch(h.tile_pref, h.n_batch, tile);
        const DevImage e = h.imgs[h.batch[bidx]];
        const int row0 = (tile - h.tile_pref[bidx]) * kHashTile;
        const int nrows = min(kHashTile, e.n - row0);
        for (int b = tid; b < LB; b += kHashThreads) hist[b] = 0;

        // stage the tile, centred, transposed; squared norms on the way
        for (int idx = tid; idx < kHashTile * 8; idx += kHashThreads) {
            const int d = idx >> 3, c = idx & 7;
            const bool ok = d < nrows;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (ok) v = __ldg(reinterpret_cast<const uint4*>(e.desc + (size_t)(row0 + d) * kDim) + c);
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int k = 16 * c + u;
                const float xb = (float)((w[u >> 2] >> (8 * (u & 3))) & 0xFFu);
                xs[k * (kHashTile + 1) + d] = ok ? (xb - mus[k]) : 0.f;
            }
            unsigned nn = __dp4a(v.x, v.x, 0u);
            nn = __dp4a(v.y, v.y, nn);
            nn = __dp4a(v.z, v.z, nn);
            nn = __dp4a(v.w, v.w, nn);
            nn += __shfl_xor_sync(0xFFFFFFFFu, nn, 1);
            nn += __shfl_xor_sync(0xFFFFFFFFu, nn, 2);
            nn += __shfl_xor_sync(0xFFFFFFFFu, nn, 4);
            if (ok && c == 0 && e.norm) e.norm[row0 + d] = nn;
        }
        __syncthreads();

        // project: thread (d, g) computes projections g*NPG .. g*NPG+NPG-1 of row d
        const int d = tid & (kHashTile - 1), g = tid >> 6;
        float acc[NPG];
#pragma unroll
        for (int j = 0; j < NPG; ++j) acc[j] = 0.f;
        const float* wrow = Ws + g * NPG;
#pragma unroll 2
        for (int k = 0; k < kDim; ++k) {
            const float x = xs[k * (kHashTile + 1) + d];
            const float4* w4 = reinterpret_cast<const float4*>(wrow + k * P_pad);
#pragma unroll
            for (int j4 = 0; j4 < NPG / 4; ++j4) {
                const float4 wv = w4[j4];
                acc[4 * j4 + 0] = fmaf(wv.x, x, acc[4 * j4 + 0]);
                acc[4 * j4 + 1] = fmaf(wv.y, x, acc[4 * j4 + 1]);
                acc[4 * j4 + 2] = fmaf(wv.z, x, acc[4 * j4 + 2]);
                acc[4 * j4 + 3] = fmaf(wv.w, x, acc[4 * j4 + 3]);
            }
        }
        uint64_t bits = 0;
#pragma unroll
        for (int j = 0; j < NPG; ++j) bits |= (uint64_t)(acc[j] > 0.f) << j;
        pb[d * 4 + g] = bits;
        __syncthreads();

        if (tid < nrows) {
            uint64_t w[3] = {0, 0, 0};
#pragma unroll
            for (int q = 0; q < 4; ++q) put_bits(w, q * NPG, pb[tid * 4 + q], NPG);
            uint64_t keyword = 0;
            for (int t = 0; t < h.L; ++t) {
                const uint32_t kt = get_bits(w, t * h.m, h.m);
                keyword |= (uint64_t)kt << (8 * t);
                atomicAdd(&hist[t * B + kt], 1u);
            }
            const int cb = h.L * h.m;
            uint4 code;
            code.x = get_bits(w, cb + 0, 32);
            code.y = get_bits(w, cb + 32, 32);
            code.z = get_bits(w, cb + 64, 32);
            code.w = get_bits(w, cb + 96, 32);
            e.key[row0 + tid] = keyword;
            e.code[row0 + tid] = code;
        }
        __syncthreads();
        for (int b = tid; b < LB; b += kHashThreads)
            if (hist[b]) atomicAdd(&e.hist[b], hist[b]);
    }
}

// One warp per (image, table): bucket offsets + stable scatter into bucket order.
__global__ void __launch_bounds__(128) k_bucket(HashLaunch h) {
    __shared__ uint32_t base_s[4][256];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int wid = blockIdx.x * 4 + wib;
    if (wid >= h.n_batch * h.L) return;
    const int t = wid % h.L;
    const DevImage e = h.imgs[h.batch[wid / h.L]];
    const int B = 1 << h.m;
    uint32_t* base = base_s[wib];
    uint32_t* hist = e.hist + t * B;
    uint32_t* off = e.off + t * (B + 1);

    // exclusive scan of the B counts: lane owns buckets [lane*per, lane*per+per)
    const int per = (B + 31) / 32;
    uint32_t local = 0;
    for (int q = 0; q < per; ++q) {
        const int b = lane * per + q;
        if (b < B) local += hist[b];
    }
    uint32_t incl = local;
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
        const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, incl, s);
        if (lane >= s) incl += v;
    }
    uint32_t run = incl - local;
    for (int q = 0; q < per; ++q) {
        const int b = lane * per + q;
        if (b < B) {
            base[b] = run;
            off[b] = run;
            run += hist[b];
            hist[b] = 0;              // histograms are zero between hashing passes
        }
    }
    if (lane == 0) off[B] = (uint32_t)e.n;
    __syncwarp();

    const unsigned lt = (1u << lane) - 1u;
    uint4* scode = e.scode + (size_t)t * e.n;
    uint16_t* sidx = e.sidx + (size_t)t * e.n;
    for (int c0 = 0; c0 < e.n; c0 += 32) {
        const int i = c0 + lane;
        const unsigned vm = __ballot_sync(0xFFFFFFFFu, i < e.n);
        if (i < e.n) {
            const int k = (int)((e.key[i] >> (8 * t)) & 0xFFu);
            const unsigned peers = __match_any_sync(vm, k);
            const int rank = __popc(peers & lt);
            const uint32_t p0 = base[k];
            __syncwarp(vm);
            if (rank == 0) base[k] = p0 + __popc(peers);
            __syncwarp(vm);
            scode[p0 + rank] = e.code[i];
            sidx[p0 + rank] = (uint16_t)i;
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// matching
// ---------------------------------------------------------------------------

template <int K>
__device__ __forceinline__ void topk_insert(uint32_t (&s)[K], uint32_t key) {
    bool dup = false;
#pragma unroll
    for (int i = 0; i < K; ++i) dup |= (s[i] == key);
    if (dup) return;
#pragma unroll
    for (int i = K - 1; i > 0; --i) s[i] = (key < s[i - 1]) ? s[i - 1] : ((key < s[i]) ? key : s[i]);
    s[0] = min(s[0], key);
}

__device__ __forceinline__ int ham128(uint4 a, uint4 b) {
    return __popc(a.x ^ b.x) + __popc(a.y ^ b.y) + __popc(a.z ^ b.z) + __popc(a.w ^ b.w);
}

// Scan one bucket run [c0, c1) of the database image for one query.
template <int K>
__device__ __forceinline__ void scan_run(const uint4* __restrict__ codes, const uint16_t* __restrict__ idx,
                                         uint32_t c0, uint32_t c1, uint4 q, uint32_t (&s)[K]) {
    uint32_t kth_h = s[K - 1] >> 16;
    uint32_t c = c0;
    for (; c + 1 < c1; c += 2) {
        const uint4 v0 = __ldg(codes + c);
        const uint4 v1 = __ldg(codes + c + 1);
        const uint32_t h0 = (uint32_t)ham128(v0, q);
        const uint32_t h1 = (uint32_t)ham128(v1, q);
        if (min(h0, h1) <= kth_h) {
            if (h0 <= kth_h) {
                const uint32_t key = (h0 << 16) | __ldg(idx + c);
                if (key < s[K - 1]) topk_insert<K>(s, key);
            }
            if (h1 <= (s[K - 1] >> 16)) {
                const uint32_t key = (h1 << 16) | __ldg(idx + c + 1);
                if (key < s[K - 1]) topk_insert<K>(s, key);
            }
            kth_h = s[K - 1] >> 16;
        }
    }
    if (c < c1) {
        const uint4 v0 = __ldg(codes + c);
        const uint32_t h0 = (uint32_t)ham128(v0, q);
        if (h0 <= kth_h) {
            const uint32_t key = (h0 << 16) | __ldg(idx + c);
            if (key < s[K - 1]) topk_insert<K>(s, key);
        }
    }
}

// Exact ratio test dis(q1) < t_r dis(q2), t_r = num/den.  FP32 where the ratio is
// at least 1e-3 away from t_r (FP32 error is ~1e-7 there), FP64 re-check otherwise
// (d^2 < 2^24, so den^2 d1^2 and num^2 d2^2 are exact in FP64).
__device__ __forceinline__ bool ratio_pass(uint32_t d1, uint32_t d2, int num, int den, uint32_t& rechecks) {
    if (d2 == 0u) return false;
    const float r = sqrtf((float)d1 / (float)d2);
    const float tr = (float)num / (float)den;
    if (fabsf(r - tr) >= 1e-3f) return r < tr;
    ++rechecks;
    return (double)den * (double)den * (double)d1 < (double)num * (double)num * (double)d2;
}

__device__ __forceinline__ float byte_as_offset_float(uint32_t w, int b) {
    // 2^23 + byte, exactly; differences of two such values are exact
    return __uint_as_float(0x4B000000u | ((w >> (8 * b)) & 0xFFu));
}

template <int K>
__global__ void __launch_bounds__(kMatchThreads, 1) k_match(MatchLaunch ml) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int S = ml.S;
    uint32_t* st = reinterpret_cast<uint32_t*>(smem_raw);          // [S][K] running top-K keys (h<<16|j)
    uint4* qcode = reinterpret_cast<uint4*>(st + (size_t)S * K);  // [S]
    uint64_t* qkey = reinterpret_cast<uint64_t*>(qcode + S);      // [S]
    uint16_t* perm = reinterpret_cast<uint16_t*>(qkey + S);       // [S] table-order permutation
    uint16_t* rnk = perm + S;                                     // [S]
    uint32_t* hist = reinterpret_cast<uint32_t*>(rnk + S);        // [256]
    __shared__ int s_item;
    __shared__ uint32_t s_stats[2];

    const int tid = threadIdx.x;
    const int B = 1 << ml.m;
    if (tid < 2) s_stats[tid] = 0;
    uint32_t rechecks = 0, matches = 0;

    for (;;) {
        __syncthreads();
        if (tid == 0) s_item = (int)atomicAdd(ml.counter, 1u);
        __syncthreads();
        const int item = s_item;
        if (item >= ml.n_items) break;
        // pair of this item: last p with item0 <= item
        int lo = 0, hi = ml.n_pairs;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (ml.pairs[mid].item0 <= item) lo = mid; else hi = mid;
        }
        const DevPair P = ml.pairs[lo];
        const DevImage I = ml.imgs[P.i];
        const DevImage J = ml.imgs[P.j];
        const int q0 = (item - P.item0) * S;
        const int nq = min(S, I.n - q0);

        for (int q = tid; q < nq; q += kMatchThreads) {
            qcode[q] = I.code[q0 + q];
            qkey[q] = I.key[q0 + q];
        }
        for (int e = tid; e < nq * K; e += kMatchThreads) st[e] = kEmpty;
        __syncthreads();

        // Sec. 2.3.1 steps (1)-(3): one pass per hash table, queries in bucket order
        for (int t = 0; t < ml.L; ++t) {
            for (int b = tid; b < B; b += kMatchThreads) hist[b] = 0;
            __syncthreads();
            for (int q = tid; q < nq; q += kMatchThreads) {
                const int b = (int)((qkey[q] >> (8 * t)) & 0xFFu);
                rnk[q] = (uint16_t)atomicAdd(&hist[b], 1u);
            }
            __syncthreads();
            if (tid < 32) {
                const int per = (B + 31) / 32;
                uint32_t local = 0;
                for (int q = 0; q < per; ++q) {
                    const int b = tid * per + q;
                    if (b < B) local += hist[b];
                }
                uint32_t incl = local;
#pragma unroll
                for (int s = 1; s < 32; s <<= 1) {
                    const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, incl, s);
                    if (tid >= s) incl += v;
                }
                uint32_t run = incl - local;
                for (int q = 0; q < per; ++q) {
                    const int b = tid * per + q;
                    if (b < B) {
                        const uint32_t c = hist[b];
                        hist[b] = run;
                        run += c;
                    }
                }
            }
            __syncthreads();
            for (int q = tid; q < nq; q += kMatchThreads) {
                const int b = (int)((qkey[q] >> (8 * t)) & 0xFFu);
                perm[hist[b] + rnk[q]] = (uint16_t)q;
            }
            __syncthreads();

            const uint4* Jc = J.scode + (size_t)t * J.n;
            const uint16_t* Ji = J.sidx + (size_t)t * J.n;
            const uint32_t* Jo = J.off + t * (B + 1);
            for (int pos = tid; pos < nq; pos += kMatchThreads) {
                const int q = perm[pos];
                const int b = (int)((qkey[q] >> (8 * t)) & 0xFFu);
                const uint32_t c0 = __ldg(Jo + b), c1 = __ldg(Jo + b + 1);
                uint32_t s[K];
#pragma unroll
                for (int i = 0; i < K; ++i) s[i] = st[q * K + i];
                scan_run<K>(Jc, Ji, c0, c1, qcode[q], s);
#pragma unroll
                for (int i = 0; i < K; ++i) st[q * K + i] = s[i];
            }
            __syncthreads();
        }

        // Sec. 2.3.1 step (4): exact distances of the top K, q1 / q2, ratio test.
        // 8 lanes per query, 16 descriptor bytes per lane.
        const int g = tid >> 3, l8 = tid & 7;
        const int rounds = (nq + (kMatchThreads / 8) - 1) / (kMatchThreads / 8);
        for (int r = 0; r < rounds; ++r) {
            const int q = g + r * (kMatchThreads / 8);
            const bool active = q < nq;
            const int qq = active ? q : 0;
            const uint4 xv = __ldg(reinterpret_cast<const uint4*>(I.desc + (size_t)(q0 + qq) * kDim) + l8);
            float xf[16];
            if (ml.rerank == CM_RERANK_FP32) {
                const uint32_t xw[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
                for (int u = 0; u < 16; ++u) xf[u] = byte_as_offset_float(xw[u >> 2], u & 3);
            }
            uint32_t d1 = kEmpty, d2 = kEmpty;
            int j1 = -1, j2 = -1;
#pragma unroll 1
            for (int k = 0; k < K; ++k) {
                const uint32_t key = active ? st[qq * K + k] : kEmpty;
                const bool valid = key != kEmpty;
                const int j = valid ? (int)(key & 0xFFFFu) : 0;
                const uint8_t* yrow = valid ? (J.desc + (size_t)j * kDim) : (I.desc + (size_t)(q0 + qq) * kDim);
                const uint4 yv = __ldg(reinterpret_cast<const uint4*>(yrow) + l8);
                uint32_t dd;
                if (ml.rerank == CM_RERANK_FP32) {
                    const uint32_t yw[4] = {yv.x, yv.y, yv.z, yv.w};
                    float acc = 0.f;
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        const float df = byte_as_offset_float(yw[u >> 2], u & 3) - xf[u];
                        acc = fmaf(df, df, acc);
                    }
                    acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 1);
                    acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 2);
                    acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 4);
                    dd = (uint32_t)acc;
                } else {
                    uint32_t a0 = __vabsdiffu4(xv.x, yv.x), a1 = __vabsdiffu4(xv.y, yv.y);
                    uint32_t a2 = __vabsdiffu4(xv.z, yv.z), a3 = __vabsdiffu4(xv.w, yv.w);
                    uint32_t acc = __dp4a(a0, a0, 0u);
                    acc = __dp4a(a1, a1, acc);
                    acc = __dp4a(a2, a2, acc);
                    acc = __dp4a(a3, a3, acc);
                    acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 1);
                    acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 2);
                    acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 4);
                    dd = acc;
                }
                if (valid) {
                    if (j1 < 0 || dd < d1 || (dd == d1 && j < j1)) {
                        d2 = d1; j2 = j1; d1 = dd; j1 = j;
                    } else if (j2 < 0 || dd < d2 || (dd == d2 && j < j2)) {
                        d2 = dd; j2 = j;
                    }
                }
            }
            if (active) {
                const int64_t row = P.row_off + q0 + q;
                bool pass = false;
                if (j2 >= 0) pass = ratio_pass(d1, d2, ml.ratio_num, ml.ratio_den, rechecks);
                if (l8 == 0) {
                    ml.out.best_j[row] = pass ? j1 : -1;
                    if (ml.out.d1sq) ml.out.d1sq[row] = d1;
                    if (ml.out.d2sq) ml.out.d2sq[row] = d2;
                    matches += pass ? 1u : 0u;
                }
                if (ml.out.topk) {
                    for (int k = l8; k < K; k += 8) {
                        const uint32_t key = st[q * K + k];
                        ml.out.topk[row * K + k] = key == kEmpty ? -1 : (int)(key & 0xFFFFu);
                    }
                }
            }
        }
    }
    if (ml.out.stats) {
        // rechecks were counted by all 8 lanes of a group; keep lane 0's count
        if ((tid & 7) == 0) {
            atomicAdd(&s_stats[0], rechecks);
            atomicAdd(&s_stats[1], matches);
        }
        __syncthreads();
        if (tid == 0) {
            atomicAdd(&ml.out.stats[0], s_stats[0]);
            atomicAdd(&ml.out.stats[1], s_stats[1]);
        }
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

cudaError_t launch_colsum_rows(const uint8_t* desc, uint64_t n_rows, unsigned long long* sums, cudaStream_t s) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    uint64_t want = (n_rows + 31) / 32;
    int grid = (int)(want < (uint64_t)sms * 8 ? (want ? want : 1) : (uint64_t)sms * 8);
    k_colsum_rows<<<grid, 256, 0, s>>>(desc, n_rows, sums);
    return cudaGetLastError();
}

cudaError_t launch_colsum_images(const HashLaunch& h, unsigned long long* sums, cudaStream_t s) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int grid = h.n_tiles < sms * 8 ? (h.n_tiles ? h.n_tiles : 1) : sms * 8;
    k_colsum_images<<<grid, 256, 0, s>>>(h, sums);
    return cudaGetLastError();
}

cudaError_t launch_count_rows(const HashLaunch& h, unsigned long long* n_total, cudaStream_t s) {
    k_count_rows<<<1, 256, 0, s>>>(h, n_total);
    return cudaGetLastError();
}

cudaError_t launch_mean(const unsigned long long* sums, const unsigned long long* n_total_dev, uint64_t n_total,
                        float* mu, cudaStream_t s) {
    k_mean<<<1, kDim, 0, s>>>(sums, n_total_dev, n_total, mu);
    return cudaGetLastError();
}

int hash_npg(int P_pad) { return P_pad / 4; }

template <int NPG>
static cudaError_t launch_hash_t(const HashLaunch& h, int sms, cudaStream_t s) {
    const size_t smem = sizeof(float) * (size_t)kDim * 4 * NPG + sizeof(float) * kDim * (kHashTile + 1) +
                        sizeof(uint64_t) * kHashTile * 4 + sizeof(uint32_t) * kMaxL * 256;
    cudaError_t e = cudaFuncSetAttribute(k_hash<NPG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int grid = h.n_tiles < sms ? (h.n_tiles ? h.n_tiles : 1) : sms;
    k_hash<NPG><<<grid, kHashThreads, smem, s>>>(h);
    return cudaGetLastError();
}

cudaError_t launch_hash(const HashLaunch& h, int sms, cudaStream_t s) {
    switch (h.P_pad / 4) {
        case 32: return launch_hash_t<32>(h, sms, s);
        case 36: return launch_hash_t<36>(h, sms, s);
        case 40: return launch_hash_t<40>(h, sms, s);
        case 44: return launch_hash_t<44>(h, sms, s);
        case 48: return launch_hash_t<48>(h, sms, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_bucket(const HashLaunch& h, cudaStream_t s) {
    const int warps = h.n_batch * h.L;
    if (warps == 0) return cudaSuccess;
    k_bucket<<<(warps + 3) / 4, 128, 0, s>>>(h);
    return cudaGetLastError();
}

size_t match_smem_bytes(int S, int K) {
    return (size_t)S * K * 4 + (size_t)S * 16 + (size_t)S * 8 + (size_t)S * 2 * 2 + 256 * 4;
}

template <int K>
static cudaError_t launch_match_t(const MatchLaunch& m, int sms, cudaStream_t s) {
    const size_t smem = match_smem_bytes(m.S, K);
    cudaError_t e = cudaFuncSetAttribute(k_match<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int grid = m.n_items < sms ? (m.n_items ? m.n_items : 1) : sms;
    k_match<K><<<grid, kMatchThreads, smem, s>>>(m);
    return cudaGetLastError();
}

cudaError_t launch_match(const MatchLaunch& m, int sms, cudaStream_t s) {
    switch (m.K) {
        case 2: return launch_match_t<2>(m, sms, s);
        case 4: return launch_match_t<4>(m, sms, s);
        case 8: return launch_match_t<8>(m, sms, s);
        case 16: return launch_match_t<16>(m, sms, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace cm
