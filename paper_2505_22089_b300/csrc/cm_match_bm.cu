// k_match_bm: the fused cascade-hashing matcher in bucket-major order
// (Sec. 2.3.1 steps (1)-(4)), the default thread mapping.
//
// Step (1) pairs each query with the database points of its bucket in every
// table.  Both images already hold, per table, their descriptors' codes and
// indices sorted by bucket (the lookup tables built on load), so for table t
// and bucket b the queries Q_b and the candidates D_b are two contiguous runs
// and step (1)-(3) over them is a dense |Q_b| x |D_b| block of Hamming
// distances.  The kernel walks those blocks directly, with no per-launch
// sorting of queries:
//   - a CTA owns one pair at a time and sweeps the L tables in order, so each
//     query's running top-K list (kept in the plan's list area, [rows][K]
//     keys Hamming << 16 | index) is updated by one table after the other;
//   - the units of a table are (bucket, 32 consecutive queries of its run),
//     dealt to warps by a shared counter, buckets with the longest database
//     runs first; lane l owns query l of the unit, its code and its list in
//     registers;
//   - the unit's database run is staged chunk by chunk into the warp's two
//     shared-memory buffers by bulk copies (cp.async.bulk, completing on an
//     mbarrier), the next chunk in flight while the current one is scanned;
//     every lane reads the same candidate code (a broadcast), so the 32 lanes
//     run the same loop with no divergence;
//   - a candidate whose distance is not above the K-th kept one is recorded
//     (key with its database index, read from the staged index window) in
//     the lane's column of a shared hit buffer, and the warp merges the
//     buffers into the lists in lockstep; a key already present (the same
//     point met in an earlier table) is skipped.
// Step (4) then reranks each query's K kept candidates exactly (8 lanes per
// query) and applies the exact ratio test, or, for the tensor-core reranks,
// writes the hand-over k_rerank_tc reads (index, squared norm, FP8 scale).
// CTAs take the pairs largest first (the plan's order), so the last pairs
// dealt, which set the launch's tail, are small.
#include <cuda_runtime.h>
#include <cstdint>

#include "cm_internal.h"
#include "cm_ratio.cuh"
#include "cm_tc.cuh"

namespace cm {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kWarps = kBmThreads / 32;
constexpr int kChunk = 64;                         // database candidates per staged chunk
constexpr int kIdxBytes = kChunk * 2 + 32;         // index window, widened to 16-byte bounds
constexpr int kBufBytes = kChunk * 16 + kIdxBytes; // one staging buffer: codes then indices
constexpr int kHitCap = 16;                        // per-lane hit buffer
constexpr int kWaitPolls = 1 << 22;                // bounded mbarrier wait (each poll may sleep ~0.5 us)

static_assert(kBufBytes % 16 == 0, "staging buffers keep 16-byte alignment");

// 128-bit Hamming distance with three population counts instead of four: the
// four XOR words are added bitwise by a carry-save step (s, c1, c2 with
// w0 + w1 + w2 + w3 = s + 2 c1 + 2 c2 per bit position), so the count is
// popc(s) + 2 (popc(c1) + popc(c2)).  POPC runs at a quarter of the rate of
// the logic ops that replace one of them (16 against 64 per clock per SM).
__device__ __forceinline__ uint32_t ham128(uint4 a, uint4 b) {
    const uint32_t w0 = a.x ^ b.x, w1 = a.y ^ b.y, w2 = a.z ^ b.z, w3 = a.w ^ b.w;
    const uint32_t s1 = w0 ^ w1 ^ w2, c1 = (w0 & w1) | (w2 & (w0 ^ w1));
    const uint32_t s2 = s1 ^ w3, c2 = s1 & w3;
    return (uint32_t)__popc(s2) + 2u * (uint32_t)(__popc(c1) + __popc(c2));
}

// Insert key into the ascending list s unless already present.  check = false
// skips the presence test: in the first table a database point meets each
// query at most once (it lies in one bucket of that table), so no key repeats.
template <int K>
__device__ __forceinline__ void topk_insert(uint32_t (&s)[K], uint32_t key, bool check) {
    if (check) {
        bool dup = false;
#pragma unroll
        for (int i = 0; i < K; ++i) dup |= (s[i] == key);
        if (dup) return;
    }
#pragma unroll
    for (int i = K - 1; i > 0; --i) s[i] = max(s[i - 1], min(s[i], key));
    s[0] = min(s[0], key);
}

// Lockstep merge of every lane's buffered keys into its list.
template <int K>
__device__ __forceinline__ void flush(const uint32_t* __restrict__ col, int cnt, uint32_t (&s)[K], bool check) {
    const int cmax = (int)__reduce_max_sync(kFull, (unsigned)cnt);
    for (int e = 0; e < cmax; ++e) {
        const uint32_t key = e < cnt ? col[e * kBmThreads] : kEmpty;
        if (key < s[K - 1]) topk_insert<K>(s, key, check);
    }
}

template <int K>
__device__ __forceinline__ void load_list(const uint32_t* p, uint32_t (&s)[K]) {
    if constexpr (K >= 4) {
#pragma unroll
        for (int i = 0; i < K; i += 4) {
            const uint4 v = *reinterpret_cast<const uint4*>(p + i);
            s[i] = v.x; s[i + 1] = v.y; s[i + 2] = v.z; s[i + 3] = v.w;
        }
    } else {
        const uint2 v = *reinterpret_cast<const uint2*>(p);
        s[0] = v.x; s[1] = v.y;
    }
}

template <int K>
__device__ __forceinline__ void store_list(uint32_t* p, const uint32_t (&s)[K]) {
    if constexpr (K >= 4) {
#pragma unroll
        for (int i = 0; i < K; i += 4) *reinterpret_cast<uint4*>(p + i) = make_uint4(s[i], s[i + 1], s[i + 2], s[i + 3]);
    } else {
        *reinterpret_cast<uint2*>(p) = make_uint2(s[0], s[1]);
    }
}

// Waits (sleeping) for the phase of a staging barrier; false after the poll limit.
__device__ __forceinline__ bool stage_wait(uint64_t* mbar, uint32_t parity) {
    for (int it = 0; it < kWaitPolls; ++it)
        if (tc::mbar_try_wait_sleep(mbar, parity, 500)) return true;
    return false;
}

__device__ __forceinline__ float offset_byte(uint32_t w, int b) {
    return __uint_as_float(0x4B000000u | ((w >> (8 * b)) & 0xFFu));   // 2^23 + byte, exact
}

}  // namespace

size_t match_bm_smem_bytes() {
    return (size_t)kWarps * 2 * kBufBytes + (size_t)kWarps * 2 * 8 + (size_t)kHitCap * kBmThreads * 4 + 256 * 4 +
           3 * 260 * 4;
}

template <int K>
__global__ void __launch_bounds__(kBmThreads, 2) k_match_bm(MatchLaunch ml) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* bufs = smem_raw;                                                       // [warps][2][kBufBytes]
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem_raw + (size_t)kWarps * 2 * kBufBytes);   // [warps][2]
    uint32_t* hitbuf = reinterpret_cast<uint32_t*>(mbar + kWarps * 2);                   // [kHitCap][threads]
    uint32_t* order = hitbuf + kHitCap * kBmThreads;                                     // [256] rank -> bucket
    uint32_t* upre = order + 256;                                                        // [B + 1] unit prefix
    uint32_t* sIo = upre + 260;                                                          // [B + 1] this table's
    uint32_t* sJo = sIo + 260;                                                           // bucket offsets, I and J
    __shared__ int s_item;
    __shared__ unsigned s_unit;
    __shared__ uint32_t s_stats[3];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int B = 1 << ml.m;
    const bool tcr = ml.rerank == CM_RERANK_BF16 || ml.rerank == CM_RERANK_FP8;
    uint64_t* wm = mbar + warp * 2;
    unsigned char* wb = bufs + (size_t)warp * 2 * kBufBytes;
    uint32_t* col = hitbuf + tid;
    if (lane == 0) {
        tc::mbar_init(&wm[0], 1);
        tc::mbar_init(&wm[1], 1);
    }
    if (tid < 3) s_stats[tid] = 0;
    __syncthreads();
    uint32_t seq = 0;        // chunks this warp has staged so far: buffer seq & 1, phase (seq >> 1) & 1
    bool failed = false;     // a staging wait gave up: this warp does no more work
    uint32_t rechecks = 0, matches = 0;

    for (;;) {
        __syncthreads();
        if (tid == 0) s_item = (int)atomicAdd(ml.counter, 1u);
        __syncthreads();
        const int item = s_item;
        if (item >= ml.n_pairs) break;
        const DevPair P = ml.pairs[ml.order ? ml.order[item] : item];   // largest pairs first
        const DevImage I = ml.imgs[P.i];
        const DevImage J = ml.imgs[P.j];
        const int nq = I.n;
        if (nq == 0) continue;
        uint32_t* lists = ml.klists + (size_t)P.row_off * K;

        // Sec. 2.3.1 steps (1)-(3), one table after the other
        for (int t = 0; t < ml.L; ++t) {
            const uint32_t* Io = I.off + t * (B + 1);
            const uint32_t* Jo = J.off + t * (B + 1);
            if (tid < B) order[B - 1 - J.brank[t * 256 + tid]] = (uint32_t)tid;   // longest database run first
            if (tid <= B) {   // the units read their runs' bounds from shared memory
                sIo[tid] = Io[tid];
                sJo[tid] = Jo[tid];
            }
            __syncthreads();
            if (warp == 0) {
                // units per bucket rank: ceil(|Q_b| / 32) where the bucket has candidates (in the first
                // table every query gets a unit, which also initialises its list)
                const int per = (B + 31) / 32;
                uint32_t local = 0;
                for (int k = 0; k < per; ++k) {
                    const int r = lane * per + k;
                    if (r < B) {
                        const uint32_t b = order[r];
                        const uint32_t qn = sIo[b + 1] - sIo[b], dn = sJo[b + 1] - sJo[b];
                        local += (qn && (dn || t == 0)) ? (qn + 31) / 32 : 0u;
                    }
                }
                uint32_t incl = local;
#pragma unroll
                for (int s = 1; s < 32; s <<= 1) {
                    const uint32_t v = __shfl_up_sync(kFull, incl, s);
                    if (lane >= s) incl += v;
                }
                uint32_t run = incl - local;
                for (int k = 0; k < per; ++k) {
                    const int r = lane * per + k;
                    if (r < B) {
                        upre[r] = run;
                        const uint32_t b = order[r];
                        const uint32_t qn = sIo[b + 1] - sIo[b], dn = sJo[b + 1] - sJo[b];
                        run += (qn && (dn || t == 0)) ? (qn + 31) / 32 : 0u;
                    }
                }
                if (lane == 31) upre[B] = run;
                if (lane == 0) s_unit = 0;
            }
            __syncthreads();
            const uint32_t total = upre[B];
            const uint4* Ic = I.scode + (size_t)t * I.n;
            const uint16_t* Ii = I.sidx + (size_t)t * I.n;
            const uint4* Jc = J.scode + (size_t)t * J.n;
            const uint16_t* Ji = J.sidx + (size_t)t * J.n;
            while (!failed) {
                uint32_t u = 0;
                if (lane == 0) u = atomicAdd(&s_unit, 1u);
                u = __shfl_sync(kFull, u, 0);
                if (u >= total) break;
                int lo = 0, hi = B;   // upre[lo] <= u < upre[lo + 1]
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (upre[mid] <= u) lo = mid; else hi = mid;
                }
                const uint32_t b = order[lo];
                const uint32_t pos = sIo[b] + (u - upre[lo]) * 32 + lane;
                const bool active = pos < sIo[b + 1];
                uint32_t q = 0;
                uint4 qc = make_uint4(0, 0, 0, 0);
                uint32_t s[K];
#pragma unroll
                for (int i = 0; i < K; ++i) s[i] = kEmpty;
                if (active) {
                    q = Ii[pos];
                    qc = Ic[pos];
                    if (t > 0) load_list<K>(lists + (size_t)q * K, s);
                }
                const uint32_t d0 = sJo[b], nd = sJo[b + 1] - d0;
                const int nch = (int)((nd + kChunk - 1) / kChunk);
                // lane 0 stages chunk c of the run into buffer (seq + c) & 1
                auto issue = [&](int c) {
                    const uint32_t c0 = d0 + (uint32_t)c * kChunk;
                    const uint32_t n = min((uint32_t)kChunk, nd - (uint32_t)c * kChunk);
                    const uintptr_t i0 = reinterpret_cast<uintptr_t>(Ji + c0) & ~(uintptr_t)15;
                    const uintptr_t i1 = (reinterpret_cast<uintptr_t>(Ji + c0 + n) + 15) & ~(uintptr_t)15;
                    const uint32_t k = (seq + (uint32_t)c) & 1u;
                    unsigned char* dst = wb + k * kBufBytes;
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    tc::mbar_arrive_expect_tx(&wm[k], n * 16u + (uint32_t)(i1 - i0));
                    tc::bulk_g2s(dst, Jc + c0, n * 16u, &wm[k]);
                    tc::bulk_g2s(dst + kChunk * 16, reinterpret_cast<const void*>(i0), (uint32_t)(i1 - i0), &wm[k]);
                };
                if (nch > 0 && lane == 0) issue(0);
                uint32_t kh = s[K - 1] >> 16;
                int cnt = 0;
                int c = 0;
                for (; c < nch; ++c) {
                    const uint32_t cur = seq + (uint32_t)c;
                    if (c + 1 < nch && lane == 0) issue(c + 1);
                    if (!__all_sync(kFull, stage_wait(&wm[cur & 1u], (cur >> 1) & 1u))) {
                        failed = true;
                        break;
                    }
                    const unsigned char* buf = wb + (cur & 1u) * kBufBytes;
                    const uint4* sc = reinterpret_cast<const uint4*>(buf);
                    const unsigned char* sj = buf + kChunk * 16 +
                                              (reinterpret_cast<uintptr_t>(Ji + d0 + (uint32_t)c * kChunk) & 15);
                    const int n = (int)min((uint32_t)kChunk, nd - (uint32_t)c * kChunk);
                    int i = 0;
                    // a candidate whose distance is not above the K-th kept one is buffered with its
                    // index (the index is read only for those; the exact key order is settled in flush)
                    for (; i + 4 <= n; i += 4) {
                        // room for this step's 4 hits in every lane's buffer (counts carry over chunks)
                        if (__any_sync(kFull, cnt > kHitCap - 4)) {
                            flush<K>(col, cnt, s, t > 0);
                            cnt = 0;
                            kh = s[K - 1] >> 16;
                        }
                        uint4 x[4];
#pragma unroll
                        for (int v = 0; v < 4; ++v) x[v] = sc[i + v];
#pragma unroll
                        for (int v = 0; v < 4; ++v) {
                            const uint32_t h = ham128(x[v], qc);
                            if (active && h <= kh) {
                                col[cnt * kBmThreads] =
                                    (h << 16) | (uint32_t)*reinterpret_cast<const uint16_t*>(sj + 2 * (i + v));
                                ++cnt;
                            }
                        }
                    }
                    for (; i < n; ++i) {
                        if (__any_sync(kFull, cnt > kHitCap - 1)) {
                            flush<K>(col, cnt, s, t > 0);
                            cnt = 0;
                            kh = s[K - 1] >> 16;
                        }
                        const uint32_t h = ham128(sc[i], qc);
                        if (active && h <= kh) {
                            col[cnt * kBmThreads] = (h << 16) | (uint32_t)*reinterpret_cast<const uint16_t*>(sj + 2 * i);
                            ++cnt;
                        }
                    }
                    __syncwarp();   // every lane is done with this buffer before it is staged again
                }
                if (failed) {
                    // the copies this warp has in flight land before the CTA can finish
                    const uint32_t cur = seq + (uint32_t)c;
                    stage_wait(&wm[cur & 1u], (cur >> 1) & 1u);
                    if (c + 1 < nch) stage_wait(&wm[(cur + 1) & 1u], ((cur + 1) >> 1) & 1u);
                    if (lane == 0) atomicExch(ml.err, 1);
                    break;
                }
                seq += (uint32_t)nch;
                if (__any_sync(kFull, cnt > 0)) flush<K>(col, cnt, s, t > 0);
                if (active) store_list<K>(lists + (size_t)q * K, s);
            }
            __syncthreads();
        }

        if (tcr) {
            // step (4) runs in k_rerank_tc: hand over each kept candidate's index, squared norm
            // (and FP8 scale), read while the pair's lists and J's norms are in L2
            const int64_t r0 = P.row_off;
            const bool fp8 = ml.rerank == CM_RERANK_FP8;
            const int ne = nq * K;
            // the next entry's key is loaded before this entry's stores (a store could alias
            // it, so the compiler would not move the load up by itself)
            uint32_t key = tid < ne ? lists[tid] : kEmpty;
            for (int e = tid; e < ne; e += kBmThreads) {
                const uint32_t key_next = e + kBmThreads < ne ? lists[e + kBmThreads] : kEmpty;
                const bool hv = key != kEmpty;
                const int j = (int)(key & 0xFFFFu);
                const uint32_t nv = hv ? __ldg(J.norm + j) : 0u;
                const float sv = fp8 && hv ? __ldg(J.xscale + j) : 0.f;
                ml.topk16[r0 * K + e] = hv ? (uint16_t)j : (uint16_t)0xFFFFu;
                ml.hnorm[r0 * K + e] = nv;
                if (fp8) ml.hscale[r0 * K + e] = sv;
                if (ml.out.topk) ml.out.topk[r0 * K + e] = hv ? j : -1;
                key = key_next;
            }
            continue;
        }
        // Sec. 2.3.1 step (4) on CUDA cores: exact distances of the top K, q1 / q2, ratio test.
        // 8 lanes per query, 16 descriptor bytes per lane.
        const int g = tid >> 3, l8 = tid & 7;
        constexpr int kPerRound = kBmThreads / 8;
        const int rounds = (nq + kPerRound - 1) / kPerRound;
        for (int r = 0; r < rounds; ++r) {
            const int q = g + r * kPerRound;
            const bool active = q < nq;
            const int qq = active ? q : 0;
            const uint4 xv = __ldg(reinterpret_cast<const uint4*>(I.desc + (size_t)qq * kDim) + l8);
            const uint32_t xw[4] = {xv.x, xv.y, xv.z, xv.w};
            uint32_t d1 = kEmpty, d2 = kEmpty;
            int j1 = -1, j2 = -1;
            constexpr int CH = K < 8 ? K : 8;
#pragma unroll
            for (int k0 = 0; k0 < K; k0 += CH) {
                uint4 yv[CH];
                int jk[CH];
#pragma unroll
                for (int k = 0; k < CH; ++k) {
                    const uint32_t key = active ? lists[(size_t)qq * K + k0 + k] : kEmpty;
                    jk[k] = key != kEmpty ? (int)(key & 0xFFFFu) : -1;
                    const uint8_t* yrow = jk[k] >= 0 ? (J.desc + (size_t)jk[k] * kDim) : (I.desc + (size_t)qq * kDim);
                    yv[k] = __ldg(reinterpret_cast<const uint4*>(yrow) + l8);
                }
#pragma unroll
                for (int k = 0; k < CH; ++k) {
                    uint32_t dd;
                    if (ml.rerank == CM_RERANK_FP32) {
                        const uint32_t yw[4] = {yv[k].x, yv[k].y, yv[k].z, yv[k].w};
                        float acc = 0.f;
#pragma unroll
                        for (int v = 0; v < 16; ++v) {
                            const float df = offset_byte(yw[v >> 2], v & 3) - offset_byte(xw[v >> 2], v & 3);
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
                const int64_t row = P.row_off + q;
                bool pass = false;
                uint32_t rc = 0;
                if (j2 >= 0) pass = ratio_pass(d1, d2, ml.ratio_num, ml.ratio_den, ml.ratio_lo, ml.ratio_hi, rc);
                if (l8 == 0) {
                    rechecks += rc;
                    ml.out.best_j[row] = pass ? j1 : -1;
                    if (ml.out.d1sq) ml.out.d1sq[row] = d1;
                    if (ml.out.d2sq) ml.out.d2sq[row] = d2;
                    matches += pass ? 1u : 0u;
                }
                if (ml.out.topk) {
                    for (int k = l8; k < K; k += 8) {
                        const uint32_t key = lists[(size_t)q * K + k];
                        ml.out.topk[row * K + k] = key == kEmpty ? -1 : (int)(key & 0xFFFFu);
                    }
                }
            }
        }
    }
    if (ml.out.stats) {
        if (rechecks) atomicAdd(&s_stats[0], rechecks);
        if (matches) atomicAdd(&s_stats[1], matches);
        __syncthreads();
        if (tid == 0) {
            atomicAdd(&ml.out.stats[0], s_stats[0]);
            atomicAdd(&ml.out.stats[1], s_stats[1]);
        }
    }
}

template <int K>
static cudaError_t launch_bm_t(const MatchLaunch& m, int sms, cudaStream_t s) {
    const size_t smem = match_bm_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(k_match_bm<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = m.n_pairs < 2 * sms ? (m.n_pairs ? m.n_pairs : 1) : 2 * sms;
    k_match_bm<K><<<grid, kBmThreads, smem, s>>>(m);
    return cudaGetLastError();
}

cudaError_t launch_match_bm(const MatchLaunch& m, int sms, cudaStream_t s) {
    switch (m.K) {
        case 2: return launch_bm_t<2>(m, sms, s);
        case 4: return launch_bm_t<4>(m, sms, s);
        case 8: return launch_bm_t<8>(m, sms, s);
        case 16: return launch_bm_t<16>(m, sms, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace cm
