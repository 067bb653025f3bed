// k_selftest.cu -- device self-test of the bounded-wait failure path: an mbarrier phase that
// expects 16 bytes no copy will ever deliver.  The wait must give up after its cycle budget
// and report KERR_TMA_TIMEOUT through global memory; nothing traps and the context stays usable.
#include <cuda_runtime.h>

#include "../../include/mmfd.h"
#include "solver.h"
#include "tma.cuh"

namespace mmfd {

__global__ void k_selftest_wait(long long budget, int* status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        mbar_arrive_expect_tx(&bar, 16u);  // arrival done, 16 bytes of transaction never arrive
    }
    __syncwarp();
    const bool ok = mbar_wait_bounded(&bar, 0u, budget);
    if (threadIdx.x == 0) *status = ok ? KERR_NONE : KERR_TMA_TIMEOUT;
}

}  // namespace mmfd

extern "C" int mmfd_selftest_wait_timeout(void* stream, long long budget_cycles) {
    using namespace mmfd;
    if (budget_cycles <= 0) return set_error(MMFD_ERR_ARG, "budget must be positive");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int* d = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&d), sizeof(int), s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync");
    cudaMemsetAsync(d, 0xff, sizeof(int), s);
    k_selftest_wait<<<1, 32, 0, s>>>(budget_cycles, d);
    e = cudaGetLastError();
    int h = -1;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFreeAsync(d, s);
    if (e != cudaSuccess) return cuda_fail(e, "self-test kernel");
    if (h == KERR_TMA_TIMEOUT) return set_error(MMFD_ERR_TIMEOUT, "bounded wait ran out as designed");
    return h == KERR_NONE ? MMFD_OK : set_error(MMFD_ERR_CUDA, "self-test kernel did not report");
}
