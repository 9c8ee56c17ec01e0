// k_match_wq: the fused matcher with one warp per query (Sec. 2.3.1 steps (1)-(4)).
//
// The 32 lanes of a warp scan 32 candidates of one query's bucket run at a time
// (coalesced 16-byte code loads), so a top-K update is one warp operation
// instead of a divergent per-lane branch.  The running top-K list is
// distributed over lanes 0..K-1 (lane l holds the l-th smallest key
// Hamming << 16 | index, 0xFFFFFFFF = empty):
//   - candidates below the current K-th key are found with a ballot;
//   - a batch with many such candidates (the first batches of a query) is
//     merged in bulk: duplicates of listed keys are dropped, the batch is
//     bitonic-sorted across the warp and merged with the list;
//   - a batch with a few is inserted one key at a time with shuffles.
// Tables are scanned in order; a point met again in a later table has the same
// key and is dropped as a duplicate.  Step (4) reranks the K kept candidates
// with exact squared distances (4 lanes x 32 bytes per candidate) and applies
// the exact ratio test.
#include <cuda_runtime.h>
#include <cstdint>

#include "cm_internal.h"
#include "cm_ratio.cuh"

namespace cm {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kBulkHits = 6;   // batches with at least this many hits are merged in bulk

__device__ __forceinline__ uint32_t ham128(uint4 a, uint4 b) {
    return (uint32_t)(__popc(a.x ^ b.x) + __popc(a.y ^ b.y) + __popc(a.z ^ b.z) + __popc(a.w ^ b.w));
}

template <int K>
__device__ __forceinline__ uint32_t list_insert(uint32_t mykey, uint32_t k, int lane) {
    constexpr unsigned lowK = (1u << K) - 1u;
    if (__ballot_sync(kFull, mykey == k) & lowK) return mykey;
    const int pos = __popc(__ballot_sync(kFull, mykey < k) & lowK);
    const uint32_t up = __shfl_up_sync(kFull, mykey, 1);
    if (lane < K) mykey = lane > pos ? up : (lane == pos ? k : mykey);
    return mykey;
}

// Ascending bitonic sort of one value per lane across the warp.
__device__ __forceinline__ uint32_t warp_sort32(uint32_t v, int lane) {
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const uint32_t o = __shfl_xor_sync(kFull, v, j);
            const bool up = ((lane & k) == 0);
            const bool lower = ((lane & j) == 0);
            v = (lower == up) ? min(v, o) : max(v, o);
        }
    }
    return v;
}

// Merge a batch of candidate keys (one per lane, kEmpty where none) into the
// sorted list held in lanes 0..K-1.  The batch holds no repeated key.
template <int K>
__device__ __forceinline__ uint32_t list_merge(uint32_t mykey, uint32_t cand, int lane) {
    // drop candidates already listed (the same point from an earlier table)
#pragma unroll
    for (int i = 0; i < K; ++i) {
        const uint32_t li = __shfl_sync(kFull, mykey, i);
        if (cand == li) cand = kEmpty;
    }
    const uint32_t sorted = warp_sort32(cand, lane);
    // K smallest of two ascending K-lists: min(A_i, B_{K-1-i}) is bitonic, then sort it
    const uint32_t rev = __shfl_sync(kFull, sorted, (K - 1 - lane) & 31);
    uint32_t v = lane < K ? min(mykey, rev) : kEmpty;
#pragma unroll
    for (int j = K >> 1; j > 0; j >>= 1) {
        const uint32_t o = __shfl_xor_sync(kFull, v, j);
        v = ((lane & j) == 0) ? min(v, o) : max(v, o);
    }
    return lane < K ? v : kEmpty;
}

__device__ __forceinline__ float offset_byte(uint32_t w, int b) {
    return __uint_as_float(0x4B000000u | ((w >> (8 * b)) & 0xFFu));
}

// Squared distance over 32 bytes (two 16-byte words of each row).
__device__ __forceinline__ uint32_t seg_d2(uint4 x0, uint4 x1, uint4 y0, uint4 y1, bool fp32) {
    const uint32_t xw[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
    const uint32_t yw[8] = {y0.x, y0.y, y0.z, y0.w, y1.x, y1.y, y1.z, y1.w};
    if (fp32) {
        float acc = 0.f;
#pragma unroll
        for (int u = 0; u < 32; ++u) {
            const float d = offset_byte(yw[u >> 2], u & 3) - offset_byte(xw[u >> 2], u & 3);
            acc = fmaf(d, d, acc);
        }
        return (uint32_t)acc;  // exact: integer-valued, below 2^24
    }
    uint32_t acc = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        const uint32_t a = __vabsdiffu4(xw[w], yw[w]);
        acc = __dp4a(a, a, acc);
    }
    return acc;
}

template <int K>
__device__ __forceinline__ void match_query(const MatchLaunch& ml, const DevImage& I, const DevImage& J, int q,
                                            int64_t row, int lane, uint32_t& rechecks, uint32_t& matches) {
    const int L = ml.L;
    const int B1 = (1 << ml.m) + 1;
    const uint4 qc = I.code[q];
    const uint64_t qk = I.key[q];
    uint32_t c0 = 0, c1 = 0;
    if (lane < L) {
        const int b = (int)((qk >> (8 * lane)) & 0xFFu);
        const uint32_t* off = J.off + lane * B1;
        c0 = __ldg(off + b);
        c1 = __ldg(off + b + 1);
    }
    const size_t nJ = (size_t)J.n;
    uint32_t mykey = kEmpty, kth = kEmpty;
    for (int t = 0; t < L; ++t) {
        const uint32_t r0 = __shfl_sync(kFull, c0, t), r1 = __shfl_sync(kFull, c1, t);
        const uint4* codes = J.scode + (size_t)t * nJ;
        const uint16_t* idx = J.sidx + (size_t)t * nJ;
        for (uint32_t base = r0; base < r1; base += 32) {
            const uint32_t c = base + lane;
            const bool valid = c < r1;
            const uint4 x = valid ? __ldg(codes + c) : qc;
            const uint32_t h = ham128(x, qc);
            uint32_t key = kEmpty;
            if (valid && h <= (kth >> 16)) {
                key = (h << 16) | (uint32_t)__ldg(idx + c);
                if (key >= kth) key = kEmpty;
            }
            const unsigned hits = __ballot_sync(kFull, key != kEmpty);
            if (hits) {
                if (__popc(hits) >= kBulkHits) {
                    mykey = list_merge<K>(mykey, key, lane);
                } else {
                    unsigned m = hits;
                    while (m) {
                        const int src = __ffs(m) - 1;
                        m &= m - 1;
                        mykey = list_insert<K>(mykey, __shfl_sync(kFull, key, src), lane);
                    }
                }
                kth = __shfl_sync(kFull, mykey, K - 1);
            }
        }
    }

    // step (4): exact distances of the kept candidates; 4 lanes x 32 bytes per candidate
    const bool fp32 = ml.rerank == CM_RERANK_FP32;
    const int seg = lane & 3;
    const uint4* xrow = reinterpret_cast<const uint4*>(I.desc + (size_t)q * kDim) + 2 * seg;
    const uint4 x0 = __ldg(xrow), x1 = __ldg(xrow + 1);
    constexpr int ROUNDS = K > 8 ? 2 : 1;
    uint32_t dr[ROUNDS];
#pragma unroll
    for (int r = 0; r < ROUNDS; ++r) {
        const int k = (lane >> 2) + 8 * r;
        const uint32_t kk = __shfl_sync(kFull, mykey, k);
        const bool valid = k < K && kk != kEmpty;
        const uint8_t* yb = valid ? J.desc + (size_t)(kk & 0xFFFFu) * kDim : I.desc + (size_t)q * kDim;
        const uint4* yrow = reinterpret_cast<const uint4*>(yb) + 2 * seg;
        uint32_t d = seg_d2(x0, x1, __ldg(yrow), __ldg(yrow + 1), fp32);
        d += __shfl_xor_sync(kFull, d, 1);
        d += __shfl_xor_sync(kFull, d, 2);
        dr[r] = d;
    }
    uint32_t myd = __shfl_sync(kFull, dr[0], 4 * (lane & 7));
    if (ROUNDS > 1) {
        const uint32_t d1 = __shfl_sync(kFull, dr[ROUNDS - 1], 4 * (lane & 7));
        if (lane >= 8) myd = d1;
    }
    const bool have = lane < K && mykey != kEmpty;
    const unsigned long long mine = have ? (((unsigned long long)myd << 16) | (mykey & 0xFFFFu)) : ~0ull;
    unsigned long long m1 = mine;
#pragma unroll
    for (int o = K / 2; o > 0; o >>= 1) m1 = min(m1, __shfl_xor_sync(kFull, m1, o));
    unsigned long long m2 = mine == m1 ? ~0ull : mine;
#pragma unroll
    for (int o = K / 2; o > 0; o >>= 1) m2 = min(m2, __shfl_xor_sync(kFull, m2, o));
    if (lane == 0) {
        const bool h1 = m1 != ~0ull, h2 = m2 != ~0ull;
        const uint32_t d1 = h1 ? (uint32_t)(m1 >> 16) : kEmpty;
        const uint32_t d2 = h2 ? (uint32_t)(m2 >> 16) : kEmpty;
        const bool ok = h2 && ratio_pass(d1, d2, ml.ratio_num, ml.ratio_den, ml.ratio_lo, ml.ratio_hi, rechecks);
        ml.out.best_j[row] = ok ? (int32_t)(m1 & 0xFFFFu) : -1;
        if (ml.out.d1sq) ml.out.d1sq[row] = d1;
        if (ml.out.d2sq) ml.out.d2sq[row] = d2;
        matches += ok ? 1u : 0u;
    }
    if (ml.out.topk && lane < K) ml.out.topk[row * K + lane] = mykey == kEmpty ? -1 : (int32_t)(mykey & 0xFFFFu);
}

template <int K>
__global__ void __launch_bounds__(kWqThreads, kWqBlocksPerSM) k_match_wq(MatchLaunch ml) {
    __shared__ int s_item;
    __shared__ uint32_t s_stats[2];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid < 2) s_stats[tid] = 0;
    uint32_t rechecks = 0, matches = 0;
    for (;;) {
        __syncthreads();
        if (tid == 0) s_item = (int)atomicAdd(ml.counter, 1u);
        __syncthreads();
        const int item = s_item;
        if (item >= ml.n_items) break;
        int lo = 0, hi = ml.n_pairs;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (ml.pairs[mid].item0 <= item) lo = mid; else hi = mid;
        }
        const DevPair P = ml.pairs[lo];
        const DevImage I = ml.imgs[P.i];
        const DevImage J = ml.imgs[P.j];
        const int q0 = (item - P.item0) * ml.S;
        const int nq = min(ml.S, I.n - q0);
        const uint16_t* order = I.sidx;   // table-0 bucket order: neighbouring warps share runs
        for (int pos = warp; pos < nq; pos += kWqThreads / 32) {
            const int q = order[q0 + pos];
            match_query<K>(ml, I, J, q, P.row_off + q, lane, rechecks, matches);
        }
    }
    if (ml.out.stats) {
        if (lane == 0) {
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

template <int K>
cudaError_t launch_t(const MatchLaunch& m, int sms, cudaStream_t s) {
    const int cap = sms * kWqBlocksPerSM;
    const int grid = m.n_items < cap ? (m.n_items ? m.n_items : 1) : cap;
    k_match_wq<K><<<grid, kWqThreads, 0, s>>>(m);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_match_wq(const MatchLaunch& m, int sms, cudaStream_t s) {
    switch (m.K) {
        case 2: return launch_t<2>(m, sms, s);
        case 4: return launch_t<4>(m, sms, s);
        case 8: return launch_t<8>(m, sms, s);
        case 16: return launch_t<16>(m, sms, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace cm
