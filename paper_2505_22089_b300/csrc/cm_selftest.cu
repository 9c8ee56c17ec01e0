// cm_selftest_wait: runs the library's bounded-wait path on the device
// without any fault.  One CTA allocates tensor memory like the tcgen05
// kernels, thread 0 waits on an mbarrier that nothing arrives on with the
// same bounded poll helper every kernel uses, gives up after `polls` polls,
// records the timeout in the status word, and the CTA frees its tensor
// memory and returns.  The host reads the status and reports CM_ERR_TIMEOUT,
// as it does for a real launch whose wait ran out; the context stays usable.
#include <cuda_runtime.h>

#include <cstdint>

#include "cm_host.h"
#include "cm_tc.cuh"

namespace cm {
namespace {

__global__ void k_wait_probe(int polls, int* status) {
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tslot;
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) tc::mbar_init(&mbar, 1);
    if (warp == 0) tc::tmem_alloc(&tslot, 32);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    bool ok = true;
    if (threadIdx.x == 0) ok = tc::mbar_wait(&mbar, 0, polls);   // phase 0 never completes
    if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicExch(status, 1);
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tslot, 32);
}

}  // namespace
}  // namespace cm

using namespace cm;

extern "C" cm_status cm_selftest_wait(int32_t polls, cm_stream stream) {
    if (polls < 1 || polls > (1 << 24)) return host_fail(CM_ERR_INVALID, "cm_selftest_wait: polls out of range");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int* d_status = nullptr;
    CM_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&d_status), sizeof(int), s));
    cudaError_t e = cudaMemsetAsync(d_status, 0, sizeof(int), s);
    if (e == cudaSuccess) {
        k_wait_probe<<<1, 64, 0, s>>>(polls, d_status);
        e = cudaGetLastError();
    }
    int status = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&status, d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFreeAsync(d_status, s);
    if (e != cudaSuccess) return host_fail(CM_ERR_CUDA, "cm_selftest_wait: %s", cudaGetErrorString(e));
    return status ? host_fail(CM_ERR_TIMEOUT, "cm_selftest_wait: the bounded wait gave up after %d polls", polls)
                  : CM_OK;
}
