// k_rerank_cc: Sec. 2.3.1 step (4) on CUDA cores for a launch whose scan left
// each query's top-K in the hand-over area (the tensor-core Hamming scan).
// Exact squared distances of the K kept candidates, 8 lanes per query and 16
// descriptor bytes per lane (FP32 on exact integers, or byte SIMD for the
// integer form), q1 / q2 by (d^2, index), the exact ratio test.  Groups of 32
// queries are dealt round-robin to the CTAs.
#include <cuda_runtime.h>

#include <cstdint>

#include "cm_internal.h"
#include "cm_ratio.cuh"

namespace cm {

namespace {

constexpr int kRcThreads = 256;
constexpr int kRcQ = kRcThreads / 8;   // queries per group

__device__ __forceinline__ float rc_byte(uint32_t w, int b) {
    // 2^23 + byte exactly; the difference of two such values is exact
    return __uint_as_float(0x4B000000u | ((w >> (8 * b)) & 0xFFu));
}

template <int K>
__global__ void __launch_bounds__(kRcThreads) k_rerank_cc(MatchLaunch ml) {
    const int tid = threadIdx.x, g8 = tid >> 3, l8 = tid & 7;
    __shared__ uint32_t s_stats[2];
    if (tid < 2) s_stats[tid] = 0;
    __syncthreads();
    uint32_t rechecks = 0, matches = 0;
    const int per_item = ml.S / kRcQ;
    const int n_grp = ml.n_items * per_item;
    int pair = -1, item_end = 0, item0 = 0, n_i = 0, n_j = 0;
    int64_t row_off = 0;
    const uint8_t *Id = nullptr, *Jd = nullptr;
    for (int u = blockIdx.x; u < n_grp; u += gridDim.x) {
        const int item = u / per_item;
        while (item >= item_end && pair + 1 < ml.n_pairs) {   // the CTA's sequence only moves forward
            ++pair;
            const DevPair P = ml.pairs[pair];
            item0 = P.item0;
            item_end = P.item0 + P.nitems;
            row_off = P.row_off;
            const DevImage& I = ml.imgs[P.i];
            n_i = I.n;
            Id = I.desc;
            Jd = ml.imgs[P.j].desc;
            n_j = ml.imgs[P.j].n;
        }
        const int q = (item - item0) * ml.S + (u % per_item) * kRcQ + g8;
        const bool active = item < item_end && q < n_i;
        const int qq = active ? q : 0;
        const int64_t row = row_off + qq;
        uint4 xv = make_uint4(0, 0, 0, 0);
        if (active) xv = __ldg(reinterpret_cast<const uint4*>(Id + (size_t)qq * kDim) + l8);
        uint32_t d1 = kEmpty, d2 = kEmpty;
        int j1 = -1, j2 = -1;
        constexpr int CH = K < 8 ? K : 8;   // candidate rows requested together
#pragma unroll
        for (int k0 = 0; k0 < K; k0 += CH) {
            uint4 yv[CH];
            int jk[CH];
#pragma unroll
            for (int k = 0; k < CH; ++k) {
                const uint16_t j = active ? ml.topk16[row * K + k0 + k] : (uint16_t)0xFFFFu;
                jk[k] = j != 0xFFFFu && (int)j < n_j ? (int)j : -1;   // an index out of range: recorded below
                if (j != 0xFFFFu && (int)j >= n_j && ml.err) atomicExch(ml.err, 2);
                const uint8_t* yrow = jk[k] >= 0 ? Jd + (size_t)jk[k] * kDim : Id + (size_t)qq * kDim;
                yv[k] = active ? __ldg(reinterpret_cast<const uint4*>(yrow) + l8) : make_uint4(0, 0, 0, 0);
            }
#pragma unroll
            for (int k = 0; k < CH; ++k) {
                uint32_t dd;
                if (ml.rerank == CM_RERANK_FP32) {
                    const uint32_t xw[4] = {xv.x, xv.y, xv.z, xv.w};
                    const uint32_t yw[4] = {yv[k].x, yv[k].y, yv[k].z, yv[k].w};
                    float acc = 0.f;
#pragma unroll
                    for (int v = 0; v < 16; ++v) {
                        const float df = rc_byte(yw[v >> 2], v & 3) - rc_byte(xw[v >> 2], v & 3);
                        acc = fmaf(df, df, acc);
                    }
                    acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 1);
                    acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 2);
                    acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 4);
                    dd = (uint32_t)acc;   // exact: integer-valued, below 2^24
                } else {
                    const uint32_t a0 = __vabsdiffu4(xv.x, yv[k].x), a1 = __vabsdiffu4(xv.y, yv[k].y);
                    const uint32_t a2 = __vabsdiffu4(xv.z, yv[k].z), a3 = __vabsdiffu4(xv.w, yv[k].w);
                    uint32_t acc = __dp4a(a0, a0, 0u);
                    acc = __dp4a(a1, a1, acc);
                    acc = __dp4a(a2, a2, acc);
                    acc = __dp4a(a3, a3, acc);
                    acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 1);
                    acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 2);
                    acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 4);
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
        if (active && l8 == 0) {
            bool pass = false;
            if (j2 >= 0) pass = ratio_pass(d1, d2, ml.ratio_num, ml.ratio_den, ml.ratio_lo, ml.ratio_hi, rechecks);
            ml.out.best_j[row] = pass ? j1 : -1;
            if (ml.out.d1sq) ml.out.d1sq[row] = d1;
            if (ml.out.d2sq) ml.out.d2sq[row] = d2;
            matches += pass ? 1u : 0u;
        }
    }
    if (ml.out.stats) {
        if (rechecks) atomicAdd(&s_stats[0], rechecks);
        if (matches) atomicAdd(&s_stats[1], matches);
        __syncthreads();
        if (tid == 0) {
            if (s_stats[0]) atomicAdd(&ml.out.stats[0], s_stats[0]);
            if (s_stats[1]) atomicAdd(&ml.out.stats[1], s_stats[1]);
        }
    }
}

template <int K>
cudaError_t launch_k(const MatchLaunch& m, int sms, cudaStream_t s) {
    const int n_grp = m.n_items * (m.S / kRcQ);
    const int grid = n_grp < sms * 8 ? (n_grp ? n_grp : 1) : sms * 8;
    k_rerank_cc<K><<<grid, kRcThreads, 0, s>>>(m);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_rerank_cc(const MatchLaunch& m, int sm_count, cudaStream_t s) {
    if (m.n_items == 0) return cudaSuccess;
    switch (m.K) {
        case 2: return launch_k<2>(m, sm_count, s);
        case 4: return launch_k<4>(m, sm_count, s);
        case 8: return launch_k<8>(m, sm_count, s);
        case 16: return launch_k<16>(m, sm_count, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace cm
