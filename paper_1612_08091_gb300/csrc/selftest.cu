// selftest.cu -- the device-side bounded wait, made to run out.
//
// Every kernel that waits on an mbarrier (bulk copies, tensor-core
// commits) polls it a bounded number of times and, on time-out, raises an
// error flag that the host turns into QSIM_ETIMEOUT, leaving the context
// usable.  This entry point runs that same wait (mbar_wait) on a barrier
// that nothing arrives on, so the time-out path can be exercised without
// faulting or hanging the GPU.
#include <cuda_runtime.h>

#include "../../include/qsim.h"
#include "common.cuh"
#include "tc_common.cuh"

using namespace qsim_tc;

namespace {

__global__ void k_wait_selftest(uint32_t limit, unsigned int *flag) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const bool ok = mbar_wait(&bar, 0, limit);  // phase 0 never completes: no arrival
    if (!ok) atomicOr(flag, 1u);
}

}  // namespace

extern "C" int qsim_selftest_wait_timeout(unsigned int limit, void *stream, double *ms) {
    if (limit < 1 || limit > (1u << 20)) return QSIM_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned int *d_flag = nullptr;
    if (cudaMalloc((void **)&d_flag, sizeof(unsigned int)) != cudaSuccess) {
        cudaGetLastError();
        return QSIM_ENOMEM;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = QSIM_ECUDA;
    unsigned int h_flag = 0;
    if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess &&
        cudaMemsetAsync(d_flag, 0, sizeof(unsigned int), st) == cudaSuccess &&
        cudaEventRecord(e0, st) == cudaSuccess) {
        k_wait_selftest<<<1, 32, 0, st>>>(limit, d_flag);
        if (cudaGetLastError() == cudaSuccess && cudaEventRecord(e1, st) == cudaSuccess &&
            cudaMemcpyAsync(&h_flag, d_flag, sizeof(unsigned int), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
            cudaStreamSynchronize(st) == cudaSuccess) {
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            if (ms) *ms = (double)t;
            rc = h_flag ? QSIM_ETIMEOUT : QSIM_OK;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(d_flag);
    return rc;
}
