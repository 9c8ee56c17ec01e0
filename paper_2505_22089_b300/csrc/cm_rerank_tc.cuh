// Tensor-core rerank of a tile of queries (Sec. 2.3.1 step (4)), included by cm_match.cu.
//
// A sub-tile holds QS = 128 / K queries: its A operand is their K candidate
// rows each (128 rows), its B operand the QS query rows (padded to NB >= 16
// rows); one tcgen05.mma chain (M = 128, N = NB, K = 128) gives every
// candidate's dot product with every query of the sub-tile, of which row r
// needs column r / K.  Several sub-tiles share one round: all threads stage
// them into the shared memory the table passes no longer use, one thread
// issues the MMAs and commits to an mbarrier, and warps 0-3 (one TMEM lane =
// one candidate row per thread) read the dot products back.
//   BF16: descriptors are exact in BF16 and the dot is an exact integer in
//         FP32, so d^2 = |x|^2 + |y|^2 - 2 x.y is exact.
//   FP8:  rows are scaled by max/448 and rounded to E4M3; the approximate d^2
//         picks q1, q2, which are then re-scored exactly on CUDA cores (FP32
//         exact on integers); a re-score that reverses their order is counted.
// The ratio test is the same exact test as the CUDA-core forms.
#pragma once
#include <cuda_fp8.h>

#include "cm_tc.cuh"

namespace cm {

constexpr int kTcWaitPolls = 1 << 24;

template <int K, bool FP8>
struct RerankShape {
    static constexpr int QS = 128 / K;                 // queries per sub-tile
    static constexpr int NB = QS < 16 ? 16 : QS;       // B rows = MMA N
    static constexpr int EB = FP8 ? 1 : 2;             // bytes per element
    static constexpr uint32_t A_BYTES = 128u * 128u * EB;
    static constexpr uint32_t B_BYTES = (uint32_t)NB * 128u * EB;
    static constexpr uint32_t SLOT = A_BYTES + B_BYTES;
    static constexpr int ROWS = 128 + NB;              // staged rows per sub-tile
    static constexpr int MAX_SLOTS = (256 / NB) < 6 ? (256 / NB) : 6;  // TMEM: 256 columns
};

__device__ __forceinline__ uint32_t tc_bf16x2(uint32_t w, int b0) {
    const float f0 = __uint_as_float(0x4B000000u | ((w >> (8 * b0)) & 0xFFu)) - 8388608.f;
    const float f1 = __uint_as_float(0x4B000000u | ((w >> (8 * (b0 + 1))) & 0xFFu)) - 8388608.f;
    return __byte_perm(__float_as_uint(f0), __float_as_uint(f1), 0x7632);
}

__device__ __forceinline__ uint32_t tc_e4m3x4(uint32_t w, float inv) {
    const float a = (float)(w & 0xFFu) * inv, b = (float)((w >> 8) & 0xFFu) * inv;
    const float c = (float)((w >> 16) & 0xFFu) * inv, d = (float)(w >> 24) * inv;
    const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3);
    const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(c, d), __NV_SATFINITE, __NV_E4M3);
    return lo | (hi << 16);
}

__device__ __forceinline__ uint32_t row_max_u8(uint4 v) {
    uint32_t m = __vmaxu4(__vmaxu4(v.x, v.y), __vmaxu4(v.z, v.w));
    m = __vmaxu4(m, m >> 16);
    m = __vmaxu4(m, m >> 8);
    return m & 0xFFu;
}

// exact squared distance over `nb` bytes (nb multiple of 16) of two rows
__device__ __forceinline__ uint32_t exact_d2(const uint8_t* x, const uint8_t* y, int nb) {
    uint32_t acc = 0;
    for (int o = 0; o < nb; o += 16) {
        const uint4 a = __ldg(reinterpret_cast<const uint4*>(x + o));
        const uint4 b = __ldg(reinterpret_cast<const uint4*>(y + o));
        const uint32_t d0 = __vabsdiffu4(a.x, b.x), d1 = __vabsdiffu4(a.y, b.y);
        const uint32_t d2 = __vabsdiffu4(a.z, b.z), d3 = __vabsdiffu4(a.w, b.w);
        acc = __dp4a(d0, d0, acc);
        acc = __dp4a(d1, d1, acc);
        acc = __dp4a(d2, d2, acc);
        acc = __dp4a(d3, d3, acc);
    }
    return acc;
}

template <int K, bool FP8>
__device__ void rerank_tc(const MatchLaunch& ml, const DevPair& P, const DevImage& I, const DevImage& J, int q0,
                          int nq, const uint32_t* __restrict__ st, unsigned char* region, uint32_t region_bytes,
                          float* scales, uint32_t* norms, uint32_t tmem, uint64_t* mbar, uint32_t& parity, uint32_t& rechecks,
                          uint32_t& matches, uint32_t& swaps) {
    using RS = RerankShape<K, FP8>;
    constexpr int QS = RS::QS, NB = RS::NB;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int slots = (int)(region_bytes / RS::SLOT);
    slots = slots < RS::MAX_SLOTS ? slots : RS::MAX_SLOTS;
    const uint32_t idesc = FP8 ? tc::idesc_e4m3(128, NB) : tc::idesc_f16(128, NB, 1);

    for (int base = 0; base < nq; base += slots * QS) {
        // ---- stage: rows of every slot, 8 threads x 16 bytes per row; each thread
        // requests up to 4 segments before converting any.  Row norms and (FP8)
        // row scales are reduced over the 8 lanes of a row into shared memory.
        const int total = slots * RS::ROWS * 8;   // a multiple of 32: every warp is full or idle
        for (int f0 = tid; f0 < total; f0 += 4 * kMatchThreads) {
            uint4 v[4];
            bool real[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int f = f0 + u * kMatchThreads;
                const int seg = f & 7, rr = f >> 3;
                const int s = rr / RS::ROWS, r = rr % RS::ROWS;
                const uint8_t* src = nullptr;
                if (f < total) {
                    if (r < 128) {
                        const int qi = base + s * QS + r / K;
                        if (qi < nq) {
                            const uint32_t key = st[qi * K + (r % K)];
                            if (key != kEmpty) src = J.desc + (size_t)(key & 0xFFFFu) * kDim;
                        }
                    } else {
                        const int n = r - 128, qi = base + s * QS + n;
                        if (n < QS && qi < nq) src = I.desc + (size_t)(q0 + qi) * kDim;
                    }
                }
                real[u] = src != nullptr;
                v[u] = src ? __ldg(reinterpret_cast<const uint4*>(src) + seg) : make_uint4(0, 0, 0, 0);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int f = f0 + u * kMatchThreads;
                if (f >= total) break;               // uniform per warp
                const int seg = f & 7, rr = f >> 3;
                const int s = rr / RS::ROWS, r = rr % RS::ROWS;
                unsigned char* slot = region + (size_t)s * RS::SLOT;
                unsigned char* tile = r < 128 ? slot : slot + RS::A_BYTES;
                const int trow = r < 128 ? r : r - 128, trows = r < 128 ? 128 : NB;
                unsigned nn = __dp4a(v[u].x, v[u].x, 0u);
                nn = __dp4a(v[u].y, v[u].y, nn);
                nn = __dp4a(v[u].z, v[u].z, nn);
                nn = __dp4a(v[u].w, v[u].w, nn);
                nn += __shfl_xor_sync(0xFFFFFFFFu, nn, 1);
                nn += __shfl_xor_sync(0xFFFFFFFFu, nn, 2);
                nn += __shfl_xor_sync(0xFFFFFFFFu, nn, 4);
                if (seg == 0) norms[s * RS::ROWS + r] = nn;
                if (!FP8) {
                    uint4 lo, hi;
                    lo.x = tc_bf16x2(v[u].x, 0); lo.y = tc_bf16x2(v[u].x, 2);
                    lo.z = tc_bf16x2(v[u].y, 0); lo.w = tc_bf16x2(v[u].y, 2);
                    hi.x = tc_bf16x2(v[u].z, 0); hi.y = tc_bf16x2(v[u].z, 2);
                    hi.z = tc_bf16x2(v[u].w, 0); hi.w = tc_bf16x2(v[u].w, 2);
                    *reinterpret_cast<uint4*>(tile + tc::chunk_off(trow, 2 * seg, trows)) = lo;
                    *reinterpret_cast<uint4*>(tile + tc::chunk_off(trow, 2 * seg + 1, trows)) = hi;
                } else {
                    uint32_t mx = row_max_u8(v[u]);
                    mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, 1));
                    mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, 2));
                    mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, 4));
                    const float scale = mx ? (float)mx / 448.f : 1.f;
                    const float inv = 1.f / scale;
                    uint4 o;
                    o.x = tc_e4m3x4(v[u].x, inv); o.y = tc_e4m3x4(v[u].y, inv);
                    o.z = tc_e4m3x4(v[u].z, inv); o.w = tc_e4m3x4(v[u].w, inv);
                    *reinterpret_cast<uint4*>(tile + tc::chunk_off(trow, seg, trows)) = o;
                    if (seg == 0) scales[s * RS::ROWS + r] = real[u] ? scale : 0.f;
                }
            }
        }
        tc::fence_proxy_async();
        __syncthreads();

        // ---- MMA: one thread, every slot, then one commit
        if (tid == 0) {
            tc::fence_after();
            constexpr uint32_t lboA = 16 * 128, lboB = (uint32_t)(NB / 8) * 128;
            for (int s = 0; s < slots; ++s) {
                const uint32_t a0 = tc::smem_addr(region + (size_t)s * RS::SLOT);
                const uint32_t b0 = a0 + RS::A_BYTES;
                const uint32_t d = tmem + (uint32_t)(s * NB);
                if (!FP8) {
#pragma unroll
                    for (int ks = 0; ks < 8; ++ks)      // K = 16 per MMA: chunks 2ks, 2ks+1
                        tc::mma_f16(d, tc::smem_desc(a0 + ks * 2 * lboA, lboA, 128),
                                    tc::smem_desc(b0 + ks * 2 * lboB, lboB, 128), idesc, ks != 0);
                } else {
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks)      // K = 32 per MMA: chunks 2ks, 2ks+1 (16 bytes each)
                        tc::mma_f8f6f4(d, tc::smem_desc(a0 + ks * 2 * lboA, lboA, 128),
                                       tc::smem_desc(b0 + ks * 2 * lboB, lboB, 128), idesc, ks != 0);
                }
            }
            tc::commit(mbar);
        }
        const bool ok = tc::mbar_wait(mbar, parity, kTcWaitPolls);
        parity ^= 1u;
        if (__syncthreads_or(!ok)) {
            if (tid == 0 && ml.err) atomicExch(ml.err, 1);
            tc::mbar_wait(mbar, parity ^ 1u, kTcWaitPolls);
            return;
        }
        tc::fence_after();

        // ---- epilogue: warps 0-3, thread = TMEM lane = candidate row
        if (warp < 4) {
            const int r = tid;                    // 0..127
            const int k = r % K, c = r / K;       // candidate slot, query column
            const int chunk = (32 * warp / K) / 16;
            for (int s = 0; s < slots; ++s) {
                const int qi = base + s * QS + c;
                uint32_t v[16];
                tc::tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(s * NB + 16 * chunk), v);
                tc::tmem_wait_ld();
                float dot = 0.f;
#pragma unroll
                for (int jj = 0; jj < 16; ++jj)
                    if (jj == (c & 15)) dot = __uint_as_float(v[jj]);
                const bool qv = qi < nq;
                const uint32_t key = qv ? st[qi * K + k] : kEmpty;
                const bool have = key != kEmpty;
                const int j = have ? (int)(key & 0xFFFFu) : 0;
                const int64_t row = P.row_off + q0 + (qv ? qi : 0);
                uint64_t mine = ~0ull;
                if (have) {
                    const float ny = (float)norms[s * RS::ROWS + r], nx = (float)norms[s * RS::ROWS + 128 + c];
                    if (!FP8) {
                        const uint32_t d2 = (uint32_t)(nx + ny - 2.f * dot);   // exact: integers below 2^24
                        mine = ((uint64_t)d2 << 32) | (uint32_t)j;
                    } else {
                        const float sxy = scales[s * RS::ROWS + r] * scales[s * RS::ROWS + 128 + c];
                        const float d2a = fmaxf(nx + ny - 2.f * dot * sxy, 0.f);
                        mine = ((uint64_t)__float_as_uint(d2a) << 32) | (uint32_t)j;
                    }
                }
                // q1, q2 over the K lanes of this query
                uint64_t m1 = mine;
#pragma unroll
                for (int o = K / 2; o > 0; o >>= 1) m1 = min(m1, __shfl_xor_sync(0xFFFFFFFFu, m1, o));
                uint64_t m2 = mine == m1 ? ~0ull : mine;
#pragma unroll
                for (int o = K / 2; o > 0; o >>= 1) m2 = min(m2, __shfl_xor_sync(0xFFFFFFFFu, m2, o));
                int j1 = m1 != ~0ull ? (int)(m1 & 0xFFFFu) : -1;
                int j2 = m2 != ~0ull ? (int)(m2 & 0xFFFFu) : -1;
                uint32_t d1 = j1 >= 0 ? (uint32_t)(m1 >> 32) : kEmpty;
                uint32_t d2 = j2 >= 0 ? (uint32_t)(m2 >> 32) : kEmpty;
                if (FP8) {
                    // exact re-score of q1 and q2: half of the K lanes per row
                    constexpr int LPR = K / 2 > 0 ? K / 2 : 1;     // lanes per row
                    constexpr int NBYTES = 128 / LPR;
                    const int half = k / LPR, part = k % LPR;
                    const int jr = half == 0 ? j1 : j2;
                    uint32_t e = 0;
                    if (qv && jr >= 0)
                        e = exact_d2(I.desc + (size_t)(q0 + qi) * kDim + part * NBYTES,
                                     J.desc + (size_t)jr * kDim + part * NBYTES, NBYTES);
#pragma unroll
                    for (int o = LPR / 2; o > 0; o >>= 1) e += __shfl_xor_sync(0xFFFFFFFFu, e, o);
                    const int gbase = lane & ~(K - 1);
                    const uint32_t e1 = __shfl_sync(0xFFFFFFFFu, e, gbase);
                    const uint32_t e2 = __shfl_sync(0xFFFFFFFFu, e, gbase + LPR);
                    d1 = j1 >= 0 ? e1 : kEmpty;
                    d2 = j2 >= 0 ? e2 : kEmpty;
                    if (j2 >= 0 && (d2 < d1 || (d2 == d1 && j2 < j1))) {   // the re-score reverses q1, q2
                        const uint32_t td = d1; d1 = d2; d2 = td;
                        const int tj = j1; j1 = j2; j2 = tj;
                        if (k == 0 && qv) ++swaps;
                    }
                }
                if (k == 0 && qv) {
                    bool pass = false;
                    if (j2 >= 0) pass = ratio_pass(d1, d2, ml.ratio_num, ml.ratio_den, rechecks);
                    ml.out.best_j[row] = pass ? j1 : -1;
                    if (ml.out.d1sq) ml.out.d1sq[row] = d1;
                    if (ml.out.d2sq) ml.out.d2sq[row] = d2;
                    matches += pass ? 1u : 0u;
                }
                if (ml.out.topk && qv) ml.out.topk[row * K + k] = have ? j : -1;
            }
        }
        tc::fence_before();
        __syncthreads();
    }
}

}  // namespace cm
