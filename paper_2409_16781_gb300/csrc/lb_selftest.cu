// lb_selftest.cu -- a self-test of the library's failure path for device
// waits: the TMA pipeline kernels wait on shared-memory mbarriers for bulk
// copies, and every such wait is bounded (mbar_wait) so that a copy that
// never completes makes the kernel set an error word and return instead of
// hanging the GPU.  lb_selftest_wait exercises exactly that bounded wait on
// a barrier that nothing ever signals, with a short deadline, and reports
// LB_ETIMEOUT -- the failure is produced by design, without a fault.
#include <cmath>

#include "lbgb.h"
#include "lb_internal.h"
#include "lb_mbarrier.cuh"

namespace lbgb {

__global__ void wait_selftest_kernel(uint64_t deadline_ns, int* __restrict__ result) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(smem_addr(&bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // no thread arrives on the barrier: its phase 0 never completes
        const bool completed = mbar_wait(smem_addr(&bar), 0, deadline_ns);
        *result = completed ? 1 : 2;
    }
}

}  // namespace lbgb

extern "C" int lb_selftest_wait(double seconds, void* stream) {
    using namespace lbgb;
    if (!(seconds > 0.0) || !(seconds <= 5.0) || !std::isfinite(seconds)) return LB_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int* d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(int));
    if (e != cudaSuccess) return LB_ENOMEM;
    int result = 0;
    e = cudaMemsetAsync(d, 0, sizeof(int), st);
    if (e == cudaSuccess) {
        wait_selftest_kernel<<<1, 32, 0, st>>>((uint64_t)(seconds * 1e9), d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&result, d, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d);
    if (e != cudaSuccess) return LB_ECUDA;
    return result == 2 ? LB_ETIMEOUT : (result == 1 ? LB_OK : LB_ECUDA);
}
