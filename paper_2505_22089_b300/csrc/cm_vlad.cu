// VLAD image encoding (Sec. 2.1): the retrieval front end that turns each
// image's descriptors into one vector, from which the view graph's pairs are
// retrieved.
//
// k_vlad_assign: nearest codeword of every descriptor.  With x and the
// codewords c on the integer grid 0..255 (exact in BF16), the dot products
// x.c of a tile of 128 descriptors against all C codewords are one
// 128 x C x 128 tcgen05 contraction; every partial sum is an integer below
// 2^24, so the FP32 accumulator is exact and so is |c|^2 - 2 x.c (its
// magnitude stays below 2^24).  The argmin over c of that value (ties to the
// smaller c) is the exact nearest codeword.  The codebook is converted once
// per CTA and stays in shared memory; each CTA converts its tiles' rows,
// one thread issues the 8 MMAs, the 4 warps read their lanes back.
//
// k_vlad_accum: one CTA per image sums x per codeword in shared memory
// (integer atomics, exact), forms the residual sums r_c = sum x - n_c * c,
// takes the signed square root of every component and L2-normalises the
// vector (FP64 sum of squares).
#include <cuda_runtime.h>

#include <cstdint>

#include "cm_host.h"
#include "cm_stage.cuh"
#include "cm_tc.cuh"

namespace cm {

namespace {

constexpr int kVaThreads = 128;
constexpr int kVaRows = 128;            // descriptors per tile (M)
constexpr int kVaMaxC = 256;            // codewords (N <= 256)
constexpr int kVaPolls = 1 << 24;       // bound of every mbarrier wait
constexpr int kAcThreads = 512;

using stage::load_row;

__global__ void __launch_bounds__(kVaThreads, 3)
k_vlad_assign(const uint8_t* __restrict__ desc, int64_t n_rows, const uint8_t* __restrict__ codebook, int C, int NC,
              int tcols, uint16_t* __restrict__ assign, int* err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* Bt = smem;                                   // NC x 256 B
    unsigned char* At = Bt + (size_t)NC * 256;                  // 128 x 256 B
    float* cn = reinterpret_cast<float*>(At + kVaRows * 256);   // [NC] |c|^2
    uint64_t* mbar = reinterpret_cast<uint64_t*>(cn + kVaMaxC);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
    const int tid = threadIdx.x, warp = tid >> 5;

    for (int r = tid; r < NC; r += kVaThreads) {
        uint4 v[8];
        load_row(codebook + (size_t)(r < C ? r : 0) * kDim, r < C, v);
        const uint32_t nn = stage::store_row(v, Bt, r, NC);
        cn[r] = r < C ? (float)nn : __uint_as_float(0x7F800000u);   // exact below 2^24; padding: +inf
    }
    if (tid == 0) tc::mbar_init(mbar, 1);
    if (warp == 0) tc::tmem_alloc(tslot, tcols);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;
    const int64_t n_tiles = (n_rows + kVaRows - 1) / kVaRows;
    uint32_t parity = 0;

    // the next tile's row is loaded while this tile's MMA and epilogue run
    uint4 raw[8];
    {
        const int64_t row = (int64_t)blockIdx.x * kVaRows + tid;
        load_row(desc + (size_t)(row < n_rows ? row : 0) * kDim, blockIdx.x < n_tiles && row < n_rows, raw);
    }
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int64_t row = tile * kVaRows + tid;
        const bool have = row < n_rows;
        stage::store_row(raw, At, tid, kVaRows);
        {
            const int64_t nrow = (tile + gridDim.x) * kVaRows + tid;
            const bool nhave = tile + gridDim.x < n_tiles && nrow < n_rows;
            load_row(desc + (size_t)(nhave ? nrow : 0) * kDim, nhave, raw);
        }
        tc::fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after();
            stage::mma_128xN(tmem, At, Bt, NC);
            tc::commit(mbar);
        }
        const bool ok = tc::mbar_wait(mbar, parity, kVaPolls);
        parity ^= 1u;
        if (__syncthreads_or(!ok)) {
            // the accumulator never completed: report, give the MMA a last bounded wait, stop
            if (tid == 0) atomicExch(err, 1);
            tc::mbar_wait(mbar, parity ^ 1u, kVaPolls);
            break;
        }
        tc::fence_after();
        // this thread's lane = row; argmin over c of |c|^2 - 2 x.c, ties to the smaller c
        // (padded codewords carry |c|^2 = +inf and never win)
        const uint32_t lane = tmem + ((uint32_t)(32 * warp) << 16);
        float best = __uint_as_float(0x7F800000u);
        int bc = 0;
        for (int c0 = 0; c0 < NC; c0 += 16) {
            uint32_t v[16];
            tc::tmem_load16(lane + c0, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const float d = fmaf(-2.f, __uint_as_float(v[j]), cn[c0 + j]);   // exact: integers below 2^24
                bc = d < best ? c0 + j : bc;
                best = fminf(best, d);
            }
        }
        if (have) assign[row] = (uint16_t)bc;
        tc::fence_before();
        __syncthreads();   // TMEM and the A tile are reused by the next tile
    }
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, tcols);
}

__global__ void __launch_bounds__(kAcThreads)
k_vlad_accum(const uint8_t* __restrict__ desc, const int64_t* __restrict__ img_off, const uint8_t* __restrict__ codebook,
             int C, const uint16_t* __restrict__ assign, float* __restrict__ vlad, int* err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    int32_t* acc = reinterpret_cast<int32_t*>(smem);   // [C][128]
    int32_t* cnt = acc + C * kDim;                      // [C]
    double* red = reinterpret_cast<double*>(cnt + ((C + 1) & ~1));   // [kAcThreads / 32]
    const int tid = threadIdx.x, img = blockIdx.x;
    const int64_t r0 = img_off[img], nr = img_off[img + 1] - r0;
    for (int e = tid; e < C * kDim; e += kAcThreads) acc[e] = 0;
    for (int c = tid; c < C; c += kAcThreads) cnt[c] = 0;
    __syncthreads();
    // A warp takes 32 consecutive rows: lane l loads the l-th word of each
    // (32 independent coalesced loads in flight) and the row's codeword; then
    // per row, lane l gathers bytes l, l+32, l+64, l+96 by shuffles and adds
    // them, so each atomic instruction touches 32 consecutive words.
    const int lane = tid & 31, warp = tid >> 5;
    for (int64_t g = (int64_t)warp * 32; g < nr; g += kAcThreads) {
        const int rows = nr - g < 32 ? (int)(nr - g) : 32;
        uint32_t w[32];
#pragma unroll
        for (int k = 0; k < 32; ++k)
            w[k] = k < rows ? __ldg(reinterpret_cast<const uint32_t*>(desc + (size_t)(r0 + g + k) * kDim) + lane) : 0u;
        const int cl = lane < rows ? assign[r0 + g + lane] : 0;
        if (lane < rows && cl >= C) atomicExch(err, 2);   // cannot happen for k_vlad_assign's output
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            const int c = __shfl_sync(0xFFFFFFFFu, cl, k);
            if (k >= rows || c >= C) continue;   // uniform over the warp
            int32_t* a = acc + c * kDim + lane;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t word = __shfl_sync(0xFFFFFFFFu, w[k], (lane >> 2) + 8 * q);
                atomicAdd(a + 32 * q, (int32_t)((word >> (8 * (lane & 3))) & 0xFFu));
            }
            if (lane == 0) atomicAdd(cnt + c, 1);
        }
    }
    __syncthreads();
    // residuals, signed square roots (kept in place as floats), sum of squares
    float* s = reinterpret_cast<float*>(acc);
    double ss = 0.0;
    for (int e = tid; e < C * kDim; e += kAcThreads) {
        const int c = e >> 7;
        const int32_t r = acc[e] - cnt[c] * (int32_t)codebook[e];
        const float q = sqrtf((float)(r < 0 ? -r : r));
        const float v = r < 0 ? -q : q;
        s[e] = v;
        ss += (double)v * (double)v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xFFFFFFFFu, ss, o);
    if ((tid & 31) == 0) red[tid >> 5] = ss;
    __syncthreads();
    double tot = 0.0;
    for (int w = 0; w < kAcThreads / 32; ++w) tot += red[w];
    const float inv = tot > 0.0 ? (float)(1.0 / sqrt(tot)) : 0.f;
    float* out = vlad + (size_t)img * C * kDim;
    for (int e = tid; e < C * kDim; e += kAcThreads) out[e] = s[e] * inv;
}

// Workspace: the error flag first (a fixed place, read by cm_workspace_status),
// then the device copy of the image offsets, then the assignments when the
// caller does not take them.
struct VladWork {
    uint64_t err, off, assign, total;
};

VladWork vlad_layout(int32_t n_images, int64_t n_rows) {
    VladWork w{};
    w.err = 0;
    w.off = align_up(4);
    w.assign = align_up(w.off + 8 * (uint64_t)(n_images + 1));
    w.total = align_up(w.assign + 2 * (uint64_t)n_rows);
    return w;
}

}  // namespace

}  // namespace cm

using namespace cm;

extern "C" cm_status cm_vlad_workspace_bytes(int32_t n_images, int64_t n_rows, uint64_t* bytes) {
    if (n_images < 0 || n_rows < 0 || !bytes) return host_fail(CM_ERR_INVALID, "cm_vlad_workspace_bytes: bad argument");
    *bytes = vlad_layout(n_images, n_rows).total;
    return CM_OK;
}

extern "C" cm_status cm_vlad_encode(const uint8_t* desc, const int64_t* img_off, int32_t n_images,
                                    const uint8_t* codebook, int32_t n_codewords, void* d_work, uint64_t work_bytes,
                                    uint16_t* assign, float* vlad, cm_stream stream) {
    if (n_images < 0 || !img_off || n_codewords < 1 || n_codewords > kVaMaxC || !codebook || !d_work ||
        (n_images > 0 && !vlad))
        return host_fail(CM_ERR_INVALID, "cm_vlad_encode: bad argument");
    if (img_off[0] != 0) return host_fail(CM_ERR_INVALID, "cm_vlad_encode: img_off[0] must be 0");
    for (int32_t i = 0; i < n_images; ++i)
        if (img_off[i + 1] < img_off[i]) return host_fail(CM_ERR_INVALID, "cm_vlad_encode: img_off not ascending");
    const int64_t n_rows = img_off[n_images];
    if (n_rows > 0 && !desc) return host_fail(CM_ERR_INVALID, "cm_vlad_encode: desc is NULL");
    const VladWork w = vlad_layout(n_images, n_rows);
    if (work_bytes < w.total || (reinterpret_cast<uintptr_t>(d_work) & (kAlign - 1)))
        return host_fail(CM_ERR_BUDGET, "cm_vlad_encode: workspace smaller than cm_vlad_workspace_bytes or not 256-byte aligned");
    if (n_images == 0) return CM_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned char* base = static_cast<unsigned char*>(d_work);
    int64_t* off = reinterpret_cast<int64_t*>(base + w.off);
    int* err = reinterpret_cast<int*>(base + w.err);
    uint16_t* asg = assign ? assign : reinterpret_cast<uint16_t*>(base + w.assign);
    CM_CUDA(cudaMemcpyAsync(off, img_off, 8 * (size_t)(n_images + 1), cudaMemcpyHostToDevice, s));
    CM_CUDA(cudaMemsetAsync(err, 0, 4, s));
    int dev = 0, sms = 148;
    CM_CUDA(cudaGetDevice(&dev));
    CM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (n_rows > 0) {
        const int NC = (n_codewords + 15) / 16 * 16;
        int tcols = 32;
        while (tcols < NC) tcols <<= 1;
        // at most 512 / tcols CTAs per SM, so that their TMEM allocations always fit together
        const size_t per_sm = 228 * 1024, max_ctas = 512 / tcols;
        size_t smem = (size_t)NC * 256 + kVaRows * 256 + kVaMaxC * 4 + 64;
        smem = std::max(smem, per_sm / (max_ctas + 1) + 1024);
        CM_CUDA(cudaFuncSetAttribute(k_vlad_assign, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        const int64_t n_tiles = (n_rows + kVaRows - 1) / kVaRows;
        const int grid = (int)std::min<int64_t>(n_tiles, (int64_t)std::min<size_t>(max_ctas, per_sm / smem) * sms);
        k_vlad_assign<<<grid, kVaThreads, smem, s>>>(desc, n_rows, codebook, n_codewords, NC, tcols, asg, err);
        CM_CUDA(cudaGetLastError());
    }
    const size_t smem2 = (size_t)n_codewords * kDim * 4 + ((n_codewords + 1) & ~1) * 4 + (kAcThreads / 32) * 8;
    CM_CUDA(cudaFuncSetAttribute(k_vlad_accum, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2));
    k_vlad_accum<<<n_images, kAcThreads, smem2, s>>>(desc, off, codebook, n_codewords, asg, vlad, err);
    CM_CUDA(cudaGetLastError());
    return CM_OK;
}

extern "C" cm_status cm_workspace_status(const void* d_work, cm_stream stream) {
    if (!d_work || (reinterpret_cast<uintptr_t>(d_work) & (kAlign - 1)))
        return host_fail(CM_ERR_INVALID, "cm_workspace_status: bad workspace");
    int flag = 0;
    CM_CUDA(cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)));
    CM_CUDA(cudaMemcpy(&flag, d_work, 4, cudaMemcpyDeviceToHost));
    if (flag == 1) return host_fail(CM_ERR_TIMEOUT, "a bounded device wait gave up");
    if (flag != 0) return host_fail(CM_ERR_STATE, "a device-side bounds check failed");
    return CM_OK;
}
