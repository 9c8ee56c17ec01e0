// cm_probe_int: throughput of the integer operations the candidate scan is
// made of, measured on the device with the SM's own cycle counter.
//
// One CTA of 1024 threads per SM runs `iters` steps of 8 independent chains
// per thread (enough independent work per scheduler to reach the pipe's
// rate).  Each CTA reads clock64() before and after its loop; the result is
// operations (or candidate evaluations) per clock per SM, from the CTA with
// the median cycle count.  The bodies:
//   CM_PROBE_POPC   x = popc(x) + x               (1 POPC + 1 IADD per step)
//   CM_PROBE_LOP3   x = (x ^ y) & z ^ x ...       (1 LOP3 per step)
//   CM_PROBE_HAM4   one 128-bit Hamming distance: 4 XOR, 4 POPC, 3 IADD
//   CM_PROBE_HAM3   the same distance through a carry-save sum: 8 LOP3,
//                   3 POPC, 2 IADD (popc(s) + 2 popc(c1) + 2 popc(c2))
// The values are kept live by an XOR into one output word per thread.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <vector>

#include "cm_host.h"

namespace {

constexpr int kProbeThreads = 1024;

template <int KIND>
__global__ void __launch_bounds__(kProbeThreads, 1) k_probe(int iters, uint32_t seed, unsigned long long* cycles,
                                                           uint32_t* sink) {
    uint32_t x[8], q[4];
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = seed * (threadIdx.x + 1) + 0x9E3779B9u * (c + 1);
#pragma unroll
    for (int w = 0; w < 4; ++w) q[w] = seed ^ (0x85EBCA6Bu * (w + 7) + threadIdx.x);
    __syncthreads();
    const unsigned long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            if (KIND == CM_PROBE_POPC) {
                x[c] = (uint32_t)__popc(x[c]) + x[c];
            } else if (KIND == CM_PROBE_LOP3) {
                uint32_t r;
                asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(r) : "r"(x[c]), "r"(q[c & 3]), "r"(x[(c + 1) & 7]));
                x[c] = r;
            } else if (KIND == CM_PROBE_HAM4) {
                const uint32_t a = x[c], b = a * 0x01000193u;   // a second "code" word pair from the chain
                const uint32_t h = (uint32_t)(__popc(a ^ q[0]) + __popc(b ^ q[1]) + __popc((a + 1) ^ q[2]) +
                                              __popc((b + 1) ^ q[3]));
                x[c] = a + h;
            } else {   // CM_PROBE_HAM3
                const uint32_t a = x[c], b = a * 0x01000193u;
                const uint32_t w0 = a ^ q[0], w1 = b ^ q[1], w2 = (a + 1) ^ q[2], w3 = (b + 1) ^ q[3];
                const uint32_t s1 = w0 ^ w1 ^ w2, c1 = (w0 & w1) | (w2 & (w0 ^ w1));
                const uint32_t s2 = s1 ^ w3, c2 = s1 & w3;
                const uint32_t h = (uint32_t)__popc(s2) + 2u * (uint32_t)(__popc(c1) + __popc(c2));
                x[c] = a + h;
            }
        }
    }
    const unsigned long long t1 = clock64();
    uint32_t acc = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) acc ^= x[c];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

}  // namespace

extern "C" cm_status cm_probe_int(int32_t kind, int32_t iters, void* d_work, uint64_t work_bytes, cm_stream stream,
                                  double* per_clock_per_sm) {
    if (kind < CM_PROBE_POPC || kind > CM_PROBE_HAM3 || iters < 1 || iters > (1 << 24) || !d_work || !per_clock_per_sm)
        return host_fail(CM_ERR_INVALID, "cm_probe_int: bad argument");
    int dev = 0, sms = 0;
    CM_CUDA(cudaGetDevice(&dev));
    CM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const uint64_t need = (uint64_t)sms * 8 + (uint64_t)sms * kProbeThreads * 4;
    if (work_bytes < need) return host_fail(CM_ERR_BUDGET, "cm_probe_int: workspace %llu bytes, %llu needed",
                                            (unsigned long long)work_bytes, (unsigned long long)need);
    auto* cycles = static_cast<unsigned long long*>(d_work);
    auto* sink = reinterpret_cast<uint32_t*>(static_cast<uint8_t*>(d_work) + (uint64_t)sms * 8);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    switch (kind) {
        case CM_PROBE_POPC: k_probe<CM_PROBE_POPC><<<sms, kProbeThreads, 0, s>>>(iters, 12345u, cycles, sink); break;
        case CM_PROBE_LOP3: k_probe<CM_PROBE_LOP3><<<sms, kProbeThreads, 0, s>>>(iters, 12345u, cycles, sink); break;
        case CM_PROBE_HAM4: k_probe<CM_PROBE_HAM4><<<sms, kProbeThreads, 0, s>>>(iters, 12345u, cycles, sink); break;
        default: k_probe<CM_PROBE_HAM3><<<sms, kProbeThreads, 0, s>>>(iters, 12345u, cycles, sink); break;
    }
    CM_CUDA(cudaGetLastError());
    std::vector<unsigned long long> c((size_t)sms);
    CM_CUDA(cudaMemcpyAsync(c.data(), cycles, (size_t)sms * 8, cudaMemcpyDeviceToHost, s));
    CM_CUDA(cudaStreamSynchronize(s));
    std::sort(c.begin(), c.end());
    const double med = (double)c[c.size() / 2];
    // one operation (POPC, LOP3) or one 128-bit distance per chain step
    *per_clock_per_sm = med > 0 ? (double)kProbeThreads * 8.0 * iters / med : 0.0;
    return CM_OK;
}
