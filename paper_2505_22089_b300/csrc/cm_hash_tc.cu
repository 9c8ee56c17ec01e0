// k_hash_tc: bucket keys and codes with the projection on the tensor cores.
//
// For a tile of 128 descriptors the projections s = (x - mu) . W (Sec. 2.3.1
// steps (1)-(2)) are one dense 128 x P x 128 contraction.  x is an integer
// 0..255, exact in BF16; W (FP32) is split into three BF16 parts
// W = W0 + W1 + W2 (W1, W2 the rounding residuals), so every product is exact
// and the FP32 accumulation over the 3 x 128 terms carries FP32-level error.
// The centring is folded into a per-projection bias b = mu . W (FP64), giving
// s = x . W - b.  One elected thread issues the 3 x 8 tcgen05.mma (M = 128,
// N = P, K = 16) into a TMEM accumulator; the 4 warps read their 32 lanes back
// (one descriptor per thread), take the sign bits, and write keys, codes and
// bucket histograms exactly as the CUDA-core kernel does.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "cm_internal.h"
#include "cm_tc.cuh"

namespace cm {

namespace {

constexpr int kTcThreads = 128;
constexpr int kTcRows = 128;         // descriptors per tile (M)
constexpr int kWaitPolls = 1 << 24;  // bound of every mbarrier wait

__device__ __forceinline__ int find_tile_image(const int32_t* pref, int n, int tile) {
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (pref[mid] <= tile) lo = mid; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ uint32_t bits_at(const uint32_t (&w)[6], int pos, int len) {
    if (len == 0) return 0u;
    const int wi = pos >> 5, sh = pos & 31;
    uint32_t lo = 0, hi = 0;
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        if (q == wi) lo = w[q];
        if (q == wi + 1) hi = w[q];
    }
    uint32_t v = lo >> sh;
    if (sh && sh + len > 32) v |= hi << (32 - sh);
    return len >= 32 ? v : (v & ((1u << len) - 1u));
}

// two bytes of w (selected by byte index b0, b0+1) -> two packed BF16 values
__device__ __forceinline__ uint32_t bytes_to_bf16x2(uint32_t w, int b0) {
    const float f0 = __uint_as_float(0x4B000000u | ((w >> (8 * b0)) & 0xFFu)) - 8388608.f;
    const float f1 = __uint_as_float(0x4B000000u | ((w >> (8 * (b0 + 1))) & 0xFFu)) - 8388608.f;
    // an integer 0..255 has at most 8 significant bits: its FP32 upper half is its exact BF16
    return __byte_perm(__float_as_uint(f0), __float_as_uint(f1), 0x7632);
}

template <int NP>
__global__ void __launch_bounds__(kTcThreads, 1) k_hash_tc(HashLaunch h) {
    constexpr uint32_t kPart = (uint32_t)NP * 256;      // one BF16 part of W: NP rows x 128 k
    constexpr uint32_t kLboB = (uint32_t)(NP / 8) * 128;
    constexpr uint32_t kLboA = (uint32_t)(kTcRows / 8) * 128;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* Wt = smem;                                          // 3 parts
    unsigned char* At = Wt + 3 * kPart;                                // 32 KB
    uint32_t* hist = reinterpret_cast<uint32_t*>(At + kTcRows * 256);  // [L][B]
    float* bias = reinterpret_cast<float*>(hist + kMaxL * 256);        // [NP]
    uint64_t* mbar = reinterpret_cast<uint64_t*>(bias + kMaxP);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
    const int tid = threadIdx.x, warp = tid >> 5;

    for (int e = tid; e < kDim * NP; e += kTcThreads) {
        const int k = e / NP, n = e % NP;
        const float w = h.W[e];
        const __nv_bfloat16 p0 = __float2bfloat16_rn(w);
        const float r1 = w - __bfloat162float(p0);
        const __nv_bfloat16 p1 = __float2bfloat16_rn(r1);
        const __nv_bfloat16 p2 = __float2bfloat16_rn(r1 - __bfloat162float(p1));
        const uint32_t off = tc::chunk_off(n, k >> 3, NP) + (k & 7) * 2;
        *reinterpret_cast<__nv_bfloat16*>(Wt + off) = p0;
        *reinterpret_cast<__nv_bfloat16*>(Wt + kPart + off) = p1;
        *reinterpret_cast<__nv_bfloat16*>(Wt + 2 * kPart + off) = p2;
    }
    for (int n = tid; n < NP; n += kTcThreads) bias[n] = h.bias[n];
    if (tid == 0) tc::mbar_init(mbar, 1);
    if (warp == 0) tc::tmem_alloc(tslot, 256);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t idesc = tc::idesc_f16(kTcRows, NP, 1);
    const int B = 1 << h.m, LB = h.L * B;
    uint32_t parity = 0;

    // The tile's image, first row and rows, and thread tid's descriptor row of it
    // (zeros past the image).  Each tile's row is loaded one tile ahead, so the
    // loads are in flight while the tile before is converted, multiplied and signed.
    auto tile_of = [&](int tile, DevImage& e, int& row0, int& nrows) {
        const int bidx = find_tile_image(h.tile_pref128, h.n_batch, tile);
        e = h.imgs[h.batch[bidx]];
        row0 = (tile - h.tile_pref128[bidx]) * kTcRows;
        nrows = min(kTcRows, e.n - row0);
    };
    auto load_row = [&](const DevImage& e, int row0, int nrows, uint4 (&v)[8]) {
        const bool have = tid < nrows;
        const uint4* src = reinterpret_cast<const uint4*>(e.desc + (size_t)(row0 + (have ? tid : 0)) * kDim);
#pragma unroll
        for (int c = 0; c < 8; ++c) v[c] = have ? __ldg(src + c) : make_uint4(0, 0, 0, 0);
    };
    DevImage e_next{};
    int row0_next = 0, nrows_next = 0;
    uint4 v_next[8];
    if (blockIdx.x < h.n_tiles128) {
        tile_of(blockIdx.x, e_next, row0_next, nrows_next);
        load_row(e_next, row0_next, nrows_next, v_next);
    }

    for (int tile = blockIdx.x; tile < h.n_tiles128; tile += gridDim.x) {
        const DevImage e = e_next;
        const int row0 = row0_next, nrows = nrows_next;
        uint4 vrow[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) vrow[c] = v_next[c];
        if (tile + (int)gridDim.x < h.n_tiles128) {   // the next tile's row, loaded during this one
            tile_of(tile + (int)gridDim.x, e_next, row0_next, nrows_next);
            load_row(e_next, row0_next, nrows_next, v_next);
        }
        for (int b = tid; b < LB; b += kTcThreads) hist[b] = 0;

        // stage: thread tid converts descriptor row0 + tid to BF16 in the operand layout
        const bool have = tid < nrows;
        unsigned nn = 0;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const uint4 v = vrow[c];
            nn = __dp4a(v.x, v.x, nn);
            nn = __dp4a(v.y, v.y, nn);
            nn = __dp4a(v.z, v.z, nn);
            nn = __dp4a(v.w, v.w, nn);
            // 16 bytes = two 8-element chunks (2c, 2c+1)
            uint4 lo, hi;
            lo.x = bytes_to_bf16x2(v.x, 0); lo.y = bytes_to_bf16x2(v.x, 2);
            lo.z = bytes_to_bf16x2(v.y, 0); lo.w = bytes_to_bf16x2(v.y, 2);
            hi.x = bytes_to_bf16x2(v.z, 0); hi.y = bytes_to_bf16x2(v.z, 2);
            hi.z = bytes_to_bf16x2(v.w, 0); hi.w = bytes_to_bf16x2(v.w, 2);
            *reinterpret_cast<uint4*>(At + tc::chunk_off(tid, 2 * c, kTcRows)) = lo;
            *reinterpret_cast<uint4*>(At + tc::chunk_off(tid, 2 * c + 1, kTcRows)) = hi;
        }
        if (have && e.norm) e.norm[row0 + tid] = nn;
        tc::fence_proxy_async();
        __syncthreads();

        if (tid == 0) {
            tc::fence_after();
            const uint32_t a0 = tc::smem_addr(At), w0 = tc::smem_addr(Wt);
#pragma unroll
            for (int p = 0; p < 3; ++p) {
#pragma unroll
                for (int ks = 0; ks < kDim / 16; ++ks) {
                    const uint64_t ad = tc::smem_desc(a0 + ks * 2 * kLboA, kLboA, 128);
                    const uint64_t bd = tc::smem_desc(w0 + p * kPart + ks * 2 * kLboB, kLboB, 128);
                    tc::mma_f16(tmem, ad, bd, idesc, (p | ks) != 0);
                }
            }
            tc::commit(mbar);
        }
        const bool ok = tc::mbar_wait(mbar, parity, kWaitPolls);
        parity ^= 1u;
        if (__syncthreads_or(!ok)) {
            // the accumulator never completed: report, give the MMA a last bounded wait, stop
            if (tid == 0) atomicExch(h.err, 1);
            tc::mbar_wait(mbar, parity ^ 1u, kWaitPolls);
            break;
        }
        tc::fence_after();

        // epilogue: this thread's lane = descriptor row0 + tid; signs of s = acc - b
        uint32_t w6[6] = {0, 0, 0, 0, 0, 0};
        const uint32_t lane_base = tmem + ((uint32_t)(32 * warp) << 16);
#pragma unroll
        for (int c = 0; c < NP / 16; ++c) {
            uint32_t v[16];
            tc::tmem_load16(lane_base + 16 * c, v);
            uint32_t bits = 0;
#pragma unroll
            for (int j = 0; j < 16; ++j) bits |= (uint32_t)(__uint_as_float(v[j]) - bias[16 * c + j] > 0.f) << j;
            w6[c >> 1] |= bits << (16 * (c & 1));
        }
        if (have) {
            uint64_t keyword = 0;
            for (int t = 0; t < h.L; ++t) {
                const uint32_t kt = bits_at(w6, t * h.m, h.m);
                keyword |= (uint64_t)kt << (8 * t);
                atomicAdd(&hist[t * B + kt], 1u);
            }
            const int cb = h.L * h.m;
            uint4 code;
            code.x = bits_at(w6, cb, 32);
            code.y = bits_at(w6, cb + 32, 32);
            code.z = bits_at(w6, cb + 64, 32);
            code.w = bits_at(w6, cb + 96, 32);
            e.key[row0 + tid] = keyword;
            e.code[row0 + tid] = code;
        }
        tc::fence_before();
        __syncthreads();  // TMEM and the A tile are reused by the next tile; histogram complete
        for (int b = tid; b < LB; b += kTcThreads)
            if (hist[b]) atomicAdd(&e.hist[b], hist[b]);
        __syncthreads();
    }
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

__global__ void k_bias(const float* __restrict__ W, const float* __restrict__ mu, int P_pad, float* __restrict__ bias) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= P_pad) return;
    double s = 0.0;
    for (int k = 0; k < kDim; ++k) s += (double)W[k * P_pad + n] * (double)mu[k];
    bias[n] = (float)s;
}

template <int NP>
cudaError_t launch_t(const HashLaunch& h, int sms, cudaStream_t s) {
    const size_t smem = 3 * (size_t)NP * 256 + kTcRows * 256 + kMaxL * 256 * 4 + kMaxP * 4 + 64;
    cudaError_t e = cudaFuncSetAttribute(k_hash_tc<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = h.n_tiles128 < sms ? (h.n_tiles128 ? h.n_tiles128 : 1) : sms;
    k_hash_tc<NP><<<grid, kTcThreads, smem, s>>>(h);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_bias(const float* W, const float* mu, int P_pad, float* bias, cudaStream_t s) {
    k_bias<<<1, kMaxP, 0, s>>>(W, mu, P_pad, bias);
    return cudaGetLastError();
}

cudaError_t launch_hash_tc(const HashLaunch& h, int sms, cudaStream_t s) {
    if (h.n_tiles128 == 0) return cudaSuccess;
    switch (h.P_pad) {
        case 128: return launch_t<128>(h, sms, s);
        case 144: return launch_t<144>(h, sms, s);
        case 160: return launch_t<160>(h, sms, s);
        case 176: return launch_t<176>(h, sms, s);
        case 192: return launch_t<192>(h, sms, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace cm
