// k_match: persistent fused cascade-hashing matcher over every pair of a block
// (Sec. 2.3.1 steps (1)-(4)).
//
// Work items are (pair, tile of S queries), fetched by CTAs from an atomic
// counter so uneven images balance.  A CTA of 1024 threads keeps the running
// top-K of its S queries in shared memory and makes one pass per hash table:
//   - the tile's queries are counting-sorted by their bucket in table t, so the
//     lanes of a warp mostly share a bucket and read the same run of the
//     database image's bucket-sorted codes (coalesced / broadcast loads);
//   - buckets are taken in order of their run length in the database image, so
//     the lanes of a warp also have runs of about the same length;
//   - each lane walks its query's run: 128-bit Hamming distance with POPC.
//     While a query's list is not full its candidates are inserted directly (all
//     lanes do so together); afterwards a candidate whose Hamming distance is not
//     above the K-th kept one is only recorded (distance, run offset) in a
//     per-lane shared-memory buffer;
//   - the warp flushes the buffers into the sorted per-lane top-K lists in
//     lockstep when one fills up and at the end of the run, resolving the
//     database index and the exact (Hamming << 16 | index) order there.  A key
//     already present (the same point met in an earlier table) is skipped.
// Step (4) then computes exact squared distances of each query's K kept
// candidates (8 lanes per query), selects q1, q2 by (d^2, index) and applies the
// ratio test exactly (FP64 re-check within 1e-3 of the threshold).
#include <cuda_runtime.h>
#include <cstdint>

#include "cm_internal.h"
#include "cm_ratio.cuh"

namespace cm {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kUnroll = 4;        // candidates per lane per loop step
constexpr int kHitCap = 16;       // per-lane hit buffer (shared memory)
constexpr int kFill = 16;         // first candidates of a query inserted directly

// Insert key into the ascending list s unless already present.  For sorted s,
// max(s[i-1], min(s[i], key)) shifts everything above key up one slot.
template <int K>
__device__ __forceinline__ void topk_insert(uint32_t (&s)[K], uint32_t key) {
    bool dup = false;
#pragma unroll
    for (int i = 0; i < K; ++i) dup |= (s[i] == key);
    if (dup) return;
#pragma unroll
    for (int i = K - 1; i > 0; --i) s[i] = max(s[i - 1], min(s[i], key));
    s[0] = min(s[0], key);
}

__device__ __forceinline__ uint32_t ham128(uint4 a, uint4 b) {
    return (uint32_t)(__popc(a.x ^ b.x) + __popc(a.y ^ b.y) + __popc(a.z ^ b.z) + __popc(a.w ^ b.w));
}

// Lockstep flush of the buffered hits (Hamming << 16 | run offset) of every lane.
// Database indices of 8 entries are requested together, then merged.
template <int K>
__device__ __forceinline__ void flush_hits(const uint32_t* __restrict__ buf, int cnt, const uint16_t* __restrict__ idx,
                                           uint32_t c0, uint32_t (&s)[K]) {
    const int cmax = (int)__reduce_max_sync(kFull, (unsigned)cnt);
    for (int e0 = 0; e0 < cmax; e0 += 8) {
        uint32_t key[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            key[u] = kEmpty;
            if (e0 + u < cnt) {
                const uint32_t v = buf[(e0 + u) * kMatchThreads];
                key[u] = (v & 0xFFFF0000u) | (uint32_t)__ldg(idx + c0 + (v & 0xFFFFu));
            }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (key[u] < s[K - 1]) topk_insert<K>(s, key[u]);
    }
}

// One table pass for one query per lane: walk the run [c0, c1) of the database
// image's bucket-sorted codes.  Warp-uniform loop (idle lanes pass c0 == c1);
// `buf` is this lane's column of the shared hit buffer.
template <int K>
__device__ __forceinline__ void scan_run(const uint4* __restrict__ codes, const uint16_t* __restrict__ idx,
                                         uint32_t c0, uint32_t c1, uint4 q, uint32_t (&s)[K], uint32_t* buf) {
    const uint32_t len = c1 - c0;
    const uint32_t lmax = __reduce_max_sync(kFull, len);
    uint32_t i = 0;
    // while a list is not full every candidate is a hit for every lane: insert
    // directly, 8 candidates' loads at a time
    if (__any_sync(kFull, s[K - 1] == kEmpty)) {
        const uint32_t n = min(lmax, (uint32_t)kFill);
        for (; i < n; i += 8) {
            uint32_t key[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                key[u] = kEmpty;
                if (i + u < min(len, n)) {
                    const uint32_t h = ham128(__ldg(codes + c0 + i + u), q);
                    key[u] = (h << 16) | (uint32_t)__ldg(idx + c0 + i + u);
                }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (key[u] < s[K - 1]) topk_insert<K>(s, key[u]);
        }
        i = n;
    }
    uint32_t kth = s[K - 1];
    int cnt = 0;
    // common part: every lane has kUnroll candidates left (no per-candidate predicates)
    const uint32_t lmin = __reduce_min_sync(kFull, len);
    for (; i + kUnroll <= lmin; i += kUnroll) {
        uint4 x[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) x[u] = __ldg(codes + c0 + i + u);
        const uint32_t kh = kth >> 16;
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const uint32_t h = ham128(x[u], q);
            if (h <= kh) {
                buf[cnt * kMatchThreads] = (h << 16) | (i + u);
                ++cnt;
            }
        }
        if (__any_sync(kFull, cnt > kHitCap - kUnroll)) {
            flush_hits<K>(buf, cnt, idx, c0, s);
            cnt = 0;
            kth = s[K - 1];
        }
    }
    // ragged part
    for (; i < lmax; i += kUnroll) {
        uint4 x[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) x[u] = (i + u < len) ? __ldg(codes + c0 + i + u) : q;
        const uint32_t kh = kth >> 16;
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const uint32_t h = ham128(x[u], q);
            if (i + u < len && h <= kh) {
                buf[cnt * kMatchThreads] = (h << 16) | (i + u);
                ++cnt;
            }
        }
        if (__any_sync(kFull, cnt > kHitCap - kUnroll)) {
            flush_hits<K>(buf, cnt, idx, c0, s);
            cnt = 0;
            kth = s[K - 1];
        }
    }
    if (__any_sync(kFull, cnt > 0)) flush_hits<K>(buf, cnt, idx, c0, s);
}


__device__ __forceinline__ float offset_byte(uint32_t w, int b) {
    // 2^23 + byte exactly; the difference of two such values is exact
    return __uint_as_float(0x4B000000u | ((w >> (8 * b)) & 0xFFu));
}

template <int K>
__global__ void __launch_bounds__(kMatchThreads, 1) k_match(MatchLaunch ml) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int S = ml.S;
    uint32_t* st = reinterpret_cast<uint32_t*>(smem_raw);          // [S][K] running top-K keys
    uint4* qcode = reinterpret_cast<uint4*>(st + (size_t)S * K);  // [S]
    uint64_t* qkey = reinterpret_cast<uint64_t*>(qcode + S);      // [S]
    uint16_t* perm = reinterpret_cast<uint16_t*>(qkey + S);       // [S] table-order permutation
    uint16_t* rnk = perm + S;                                     // [S]
    uint32_t* hist = reinterpret_cast<uint32_t*>(rnk + S);        // [256]
    uint32_t* order = hist + 256;                                 // [256] bucket -> rank by run length
    uint32_t* hitbuf = order + 256;                               // [kHitCap][kMatchThreads]
    __shared__ int s_item;
    __shared__ uint32_t s_stats[3];

    const int tid = threadIdx.x, lane = tid & 31;
    const int B = 1 << ml.m;
    const bool tcr = ml.rerank == CM_RERANK_BF16 || ml.rerank == CM_RERANK_FP8;
    if (tid < 3) s_stats[tid] = 0;
    uint32_t rechecks = 0, matches = 0, swaps = 0;

    for (;;) {
        __syncthreads();
        if (tid == 0) s_item = (int)atomicAdd(ml.counter, 1u);
        __syncthreads();
        const int item = s_item;
        if (item >= ml.n_items) break;
        int lo = 0, hi = ml.n_pairs;  // last pair with item0 <= item
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

        // Sec. 2.3.1 steps (1)-(3): one pass per hash table.  Queries are grouped
        // by bucket, buckets ordered by the length of their run in J, so a warp's
        // lanes share runs and have runs of about the same length.
        for (int t = 0; t < ml.L; ++t) {
            const uint32_t* Jo = J.off + t * (B + 1);
            for (int b = tid; b < B; b += kMatchThreads) {
                hist[b] = 0;
                order[b] = J.brank[t * 256 + b];
            }
            __syncthreads();
            for (int q = tid; q < nq; q += kMatchThreads) {
                const int b = (int)order[(qkey[q] >> (8 * t)) & 0xFFu];
                rnk[q] = (uint16_t)atomicAdd(&hist[b], 1u);
            }
            __syncthreads();
            if (tid < 32) {
                const int per = (B + 31) / 32;
                uint32_t local = 0;
                for (int k = 0; k < per; ++k) {
                    const int b = tid * per + k;
                    if (b < B) local += hist[b];
                }
                uint32_t incl = local;
#pragma unroll
                for (int s = 1; s < 32; s <<= 1) {
                    const uint32_t v = __shfl_up_sync(kFull, incl, s);
                    if (tid >= s) incl += v;
                }
                uint32_t run = incl - local;
                for (int k = 0; k < per; ++k) {
                    const int b = tid * per + k;
                    if (b < B) {
                        const uint32_t c = hist[b];
                        hist[b] = run;
                        run += c;
                    }
                }
            }
            __syncthreads();
            for (int q = tid; q < nq; q += kMatchThreads) {
                const int b = (int)order[(qkey[q] >> (8 * t)) & 0xFFu];
                perm[hist[b] + rnk[q]] = (uint16_t)q;
            }
            __syncthreads();

            const uint4* Jc = J.scode + (size_t)t * J.n;
            const uint16_t* Ji = J.sidx + (size_t)t * J.n;
            // warp-uniform: every lane runs every round (idle lanes with an empty run).
            // Odd rounds run backwards so each thread pairs a short run with a long one.
            for (int base = 0; base < nq; base += kMatchThreads) {
                const int pos = base + (((base / kMatchThreads) & 1) ? kMatchThreads - 1 - tid : tid);
                const bool active = pos < nq;
                const int q = active ? perm[pos] : 0;
                uint32_t c0 = 0, c1 = 0;
                uint4 qc = make_uint4(0, 0, 0, 0);
                uint32_t s[K];
#pragma unroll
                for (int i = 0; i < K; ++i) s[i] = kEmpty;
                if (active) {
                    const int b = (int)((qkey[q] >> (8 * t)) & 0xFFu);
                    c0 = __ldg(Jo + b);
                    c1 = __ldg(Jo + b + 1);
                    qc = qcode[q];
#pragma unroll
                    for (int i = 0; i < K; ++i) s[i] = st[q * K + i];
                }
                scan_run<K>(Jc, Ji, c0, c1, qc, s, hitbuf + tid);
                if (active) {
#pragma unroll
                    for (int i = 0; i < K; ++i) st[q * K + i] = s[i];
                }
            }
            __syncthreads();
        }

        // Tensor-core forms: step (4) runs in k_rerank_tc; hand over the top-K lists
        if (tcr) {
            // each kept candidate with its squared norm (and FP8 scale): the rerank then
            // reads one contiguous record per candidate instead of gathering them
            const int64_t r0 = P.row_off + q0;
            const bool fp8 = ml.rerank == CM_RERANK_FP8;
#pragma unroll 4
            for (int e = tid; e < nq * K; e += kMatchThreads) {
                const uint32_t key = st[e];
                const bool hv = key != kEmpty;
                const int j = (int)(key & 0xFFFFu);
                ml.topk16[r0 * K + e] = hv ? (uint16_t)j : (uint16_t)0xFFFFu;
                ml.hnorm[r0 * K + e] = hv ? __ldg(J.norm + j) : 0u;
                if (fp8) ml.hscale[r0 * K + e] = hv ? __ldg(J.xscale + j) : 0.f;
                if (ml.out.topk) ml.out.topk[r0 * K + e] = hv ? j : -1;
            }
            continue;
        }
        // Sec. 2.3.1 step (4) on CUDA cores: exact distances of the top K, q1 / q2, ratio test.
        // 8 lanes per query, 16 descriptor bytes per lane.
        const int g = tid >> 3, l8 = tid & 7;
        const int rounds = (nq + (kMatchThreads / 8) - 1) / (kMatchThreads / 8);
        for (int r = 0; r < rounds; ++r) {
            const int q = g + r * (kMatchThreads / 8);
            const bool active = q < nq;
            const int qq = active ? q : 0;
            const uint4 xv = __ldg(reinterpret_cast<const uint4*>(I.desc + (size_t)(q0 + qq) * kDim) + l8);
            const uint32_t xw[4] = {xv.x, xv.y, xv.z, xv.w};
            uint32_t d1 = kEmpty, d2 = kEmpty;
            int j1 = -1, j2 = -1;
            // candidate rows are requested in batches of up to 8 before any is used
            constexpr int CH = K < 8 ? K : 8;
#pragma unroll
            for (int k0 = 0; k0 < K; k0 += CH) {
            uint4 yv[CH];
            int jk[CH];
#pragma unroll
            for (int k = 0; k < CH; ++k) {
                const uint32_t key = active ? st[qq * K + k0 + k] : kEmpty;
                jk[k] = key != kEmpty ? (int)(key & 0xFFFFu) : -1;
                const uint8_t* yrow = jk[k] >= 0 ? (J.desc + (size_t)jk[k] * kDim) : (I.desc + (size_t)(q0 + qq) * kDim);
                yv[k] = __ldg(reinterpret_cast<const uint4*>(yrow) + l8);
            }
#pragma unroll
            for (int k = 0; k < CH; ++k) {
                uint32_t dd;
                if (ml.rerank == CM_RERANK_FP32) {
                    const uint32_t yw[4] = {yv[k].x, yv[k].y, yv[k].z, yv[k].w};
                    float acc = 0.f;
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        const float df = offset_byte(yw[u >> 2], u & 3) - offset_byte(xw[u >> 2], u & 3);
                        acc = fmaf(df, df, acc);
                    }
                    acc += __shfl_xor_sync(kFull, acc, 1);
                    acc += __shfl_xor_sync(kFull, acc, 2);
                    acc += __shfl_xor_sync(kFull, acc, 4);
                    dd = (uint32_t)acc;   // exact: integer-valued, below 2^24
                } else {
                    const uint32_t a0 = __vabsdiffu4(xv.x, yv[k].x), a1 = __vabsdiffu4(xv.y, yv[k].y);
                    const uint32_t a2 = __vabsdiffu4(xv.z, yv[k].z), a3 = __vabsdiffu4(xv.w, yv[k].w);
                    uint32_t acc = __dp4a(a0, a0, 0u);
                    acc = __dp4a(a1, a1, acc);
                    acc = __dp4a(a2, a2, acc);
                    acc = __dp4a(a3, a3, acc);
                    acc += __shfl_xor_sync(kFull, acc, 1);
                    acc += __shfl_xor_sync(kFull, acc, 2);
                    acc += __shfl_xor_sync(kFull, acc, 4);
                    dd = acc;
                }
                const int j = jk[k];
                if (j >= 0) {
                    if (j1 < 0 || dd < d1 || (dd == d1 && j < j1)) {
                        d2 = d1; j2 = j1; d1 = dd; j1 = j;
                    } else if (j2 < 0 || dd < d2 || (dd == d2 && j < j2)) {
                        d2 = dd; j2 = j;
                    }
                }
            }
            }
            if (active) {
                const int64_t row = P.row_off + q0 + q;
                bool pass = false;
                uint32_t rc = 0;
                if (j2 >= 0) pass = ratio_pass(d1, d2, ml.ratio_num, ml.ratio_den, ml.ratio_lo, ml.ratio_hi, rc);
                if (l8 == 0) rechecks += rc;
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
        if (rechecks) atomicAdd(&s_stats[0], rechecks);
        if (matches) atomicAdd(&s_stats[1], matches);
        if (swaps) atomicAdd(&s_stats[2], swaps);
        __syncthreads();
        if (tid == 0) {
            atomicAdd(&ml.out.stats[0], s_stats[0]);
            atomicAdd(&ml.out.stats[1], s_stats[1]);
            atomicAdd(&ml.out.stats[2], s_stats[2]);
        }
    }
    (void)lane;
}

size_t match_smem_bytes(int S, int K) {
    return (size_t)S * K * 4 + (size_t)S * 16 + (size_t)S * 8 + (size_t)S * 2 * 2 + 2 * 256 * 4 +
           (size_t)kHitCap * kMatchThreads * 4;
}

template <int K>
static cudaError_t launch_match_t(const MatchLaunch& m, int sms, cudaStream_t s) {
    const size_t smem = match_smem_bytes(m.S, K);
    cudaError_t e = cudaFuncSetAttribute(k_match<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = m.n_items < sms ? (m.n_items ? m.n_items : 1) : sms;
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
