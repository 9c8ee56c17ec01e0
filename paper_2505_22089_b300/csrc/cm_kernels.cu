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
//  (the fused matcher k_match is in cm_match.cu)
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
        }
    }
    if (lane == 0) off[B] = (uint32_t)e.n;
    __syncwarp();
    // rank of each bucket by run length (ties by bucket id), for the match kernel's
    // query order; then clear the histogram (zero between hashing passes)
    for (int q = 0; q < per; ++q) {
        const int b = lane * per + q;
        if (b < B) {
            const uint32_t lb = hist[b];
            uint32_t r = 0;
            for (int b2 = 0; b2 < B; ++b2) {
                const uint32_t l2 = hist[b2];
                r += (l2 < lb || (l2 == lb && b2 < b)) ? 1u : 0u;
            }
            e.brank[t * 256 + b] = (uint8_t)r;
        }
    }
    __syncwarp();
    for (int q = 0; q < per; ++q) {
        const int b = lane * per + q;
        if (b < B) hist[b] = 0;
    }
    __syncwarp();

    const unsigned lt = (1u << lane) - 1u;
    uint4* scode = e.scode + (size_t)t * e.n;
    uint16_t* sidx = e.sidx + (size_t)t * e.n;
    // rows in groups of 32, U groups at a time: their keys and codes are loaded
    // before the first is scattered (the scatter is a chain through base[], the
    // loads are not), so one warp keeps U loads of each in flight
    constexpr int U = 8;
    for (int c0 = 0; c0 < e.n; c0 += 32 * U) {
        uint64_t kk[U];
        uint4 cc[U];
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const int i = c0 + 32 * q + lane;
            if (i < e.n) {
                kk[q] = e.key[i];
                cc[q] = e.code[i];
            }
        }
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const int i = c0 + 32 * q + lane;
            const unsigned vm = __ballot_sync(0xFFFFFFFFu, i < e.n);
            if (vm == 0u) break;   // the image's rows end in this group (uniform)
            if (i < e.n) {
                const int k = (int)((kk[q] >> (8 * t)) & 0xFFu);
                const unsigned peers = __match_any_sync(vm, k);
                const int rank = __popc(peers & lt);
                const uint32_t p0 = base[k];
                __syncwarp(vm);
                if (rank == 0) base[k] = p0 + __popc(peers);
                __syncwarp(vm);
                scode[p0 + rank] = cc[q];
                sidx[p0 + rank] = (uint16_t)i;
            }
            __syncwarp();
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

}  // namespace cm
