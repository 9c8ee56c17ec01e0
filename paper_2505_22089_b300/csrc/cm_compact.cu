// Compaction of a match launch's per-query decisions into per-pair match lists
// (the initial matches handed to outlier removal, Algorithm 1).
//
//   k_count   one CTA per pair: number of queries with best_j >= 0
//   k_scan    exclusive prefix of the counts (one CTA, chunked)
//   k_scatter one CTA per pair: matches (query << 16 | db index) in query order
// Every step is deterministic: a pair's list sits at its prefix offset.
#include <cuda_runtime.h>

#include <cstdint>

#include "cm_internal.h"

namespace cm {

namespace {

constexpr int kCompactThreads = 256;

__device__ __forceinline__ int block_sum(int v, int* red) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    if (lane == 0) red[w] = v;
    __syncthreads();
    int t = 0;
    if (threadIdx.x < 32) {
        t = threadIdx.x < kCompactThreads / 32 ? red[threadIdx.x] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xFFFFFFFFu, t, o);
    }
    __syncthreads();
    return t;
}

__global__ void __launch_bounds__(kCompactThreads) k_count(const DevPair* __restrict__ pairs, const DevImage* imgs,
                                                           const int32_t* __restrict__ best, uint32_t* __restrict__ counts) {
    __shared__ int red[kCompactThreads / 32];
    const DevPair P = pairs[blockIdx.x];
    const int n = imgs[P.i].n;
    int c = 0;
    for (int q = threadIdx.x; q < n; q += kCompactThreads) c += best[P.row_off + q] >= 0;
    const int t = block_sum(c, red);
    if (threadIdx.x == 0) counts[blockIdx.x] = (uint32_t)t;
}

// Exclusive prefix over n counts (single CTA; chunks of kCompactThreads).
__global__ void __launch_bounds__(kCompactThreads) k_scan(const uint32_t* __restrict__ counts, int n,
                                                          unsigned long long* __restrict__ offsets,
                                                          unsigned long long* __restrict__ total) {
    __shared__ unsigned long long part[kCompactThreads];
    __shared__ unsigned long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += kCompactThreads) {
        const int i = base + threadIdx.x;
        const unsigned long long v = i < n ? counts[i] : 0ull;
        part[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < kCompactThreads; o <<= 1) {   // Hillis-Steele inclusive scan
            const unsigned long long add = threadIdx.x >= o ? part[threadIdx.x - o] : 0ull;
            __syncthreads();
            part[threadIdx.x] += add;
            __syncthreads();
        }
        if (i < n) offsets[i] = carry + part[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == kCompactThreads - 1) carry += part[threadIdx.x];
        __syncthreads();
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void __launch_bounds__(kCompactThreads) k_scatter(const DevPair* __restrict__ pairs, const DevImage* imgs,
                                                             const int32_t* __restrict__ best,
                                                             const unsigned long long* __restrict__ offsets,
                                                             uint32_t* __restrict__ out, unsigned long long capacity) {
    __shared__ int red[kCompactThreads / 32];
    __shared__ int base_s;
    const DevPair P = pairs[blockIdx.x];
    const int n = imgs[P.i].n;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) base_s = 0;
    __syncthreads();
    unsigned long long pos0 = offsets[blockIdx.x];
    for (int q0 = 0; q0 < n; q0 += kCompactThreads) {
        const int q = q0 + threadIdx.x;
        const int j = q < n ? best[P.row_off + q] : -1;
        const bool m = j >= 0;
        const unsigned ballot = __ballot_sync(0xFFFFFFFFu, m);
        if (lane == 0) red[w] = __popc(ballot);
        __syncthreads();
        int before = 0, tot = 0;
        for (int k = 0; k < kCompactThreads / 32; ++k) {
            before += k < w ? red[k] : 0;
            tot += red[k];
        }
        if (m) {
            const unsigned long long p = pos0 + (unsigned long long)(base_s + before + __popc(ballot & ((1u << lane) - 1u)));
            if (p < capacity) out[p] = ((uint32_t)q << 16) | (uint32_t)j;
        }
        __syncthreads();
        if (threadIdx.x == 0) base_s += tot;
        __syncthreads();
    }
}

// Two-way consistency: a match q -> j of pair (I, J) stays only if the reverse
// pair (J, I) matched j back to q.  One CTA per pair; a pair without a reverse
// keeps its decisions.
__global__ void __launch_bounds__(kCompactThreads) k_mutual(const DevPair* __restrict__ pairs, const DevImage* imgs,
                                                            const int32_t* __restrict__ in, int32_t* __restrict__ out) {
    const DevPair P = pairs[blockIdx.x];
    const int n = imgs[P.i].n;
    const int nj = imgs[P.j].n;
    const int64_t back0 = P.rev >= 0 ? pairs[P.rev].row_off : 0;
    for (int q = threadIdx.x; q < n; q += kCompactThreads) {
        const int32_t j = in[P.row_off + q];
        int32_t keep = j;
        if (P.rev >= 0 && j >= 0) keep = (j < nj && in[back0 + j] == q) ? j : -1;
        out[P.row_off + q] = keep;
    }
}

}  // namespace

cudaError_t launch_mutual(const DevPair* pairs, int n_pairs, const DevImage* imgs, const int32_t* best_in,
                          int32_t* best_out, cudaStream_t s) {
    if (n_pairs <= 0) return cudaSuccess;
    k_mutual<<<n_pairs, kCompactThreads, 0, s>>>(pairs, imgs, best_in, best_out);
    return cudaGetLastError();
}

cudaError_t launch_compact(const DevPair* pairs, int n_pairs, const DevImage* imgs, const int32_t* best,
                           uint32_t* counts, unsigned long long* offsets, unsigned long long* total, uint32_t* out,
                           unsigned long long capacity, cudaStream_t s) {
    if (n_pairs <= 0) return cudaSuccess;
    k_count<<<n_pairs, kCompactThreads, 0, s>>>(pairs, imgs, best, counts);
    k_scan<<<1, kCompactThreads, 0, s>>>(counts, n_pairs, offsets, total);
    if (out) k_scatter<<<n_pairs, kCompactThreads, 0, s>>>(pairs, imgs, best, offsets, out, capacity);
    return cudaGetLastError();
}

}  // namespace cm
