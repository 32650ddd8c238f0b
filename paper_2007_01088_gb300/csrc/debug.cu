// Diagnostic entry point: a bounded device wait made to run out.
//
// Every spin-wait in the library's kernels is bounded: after its limit the
// kernel records the failure in a device status word and returns, and the
// host call reports CC3_ERR_TIMEOUT while the CUDA context stays usable.
// This call exercises that path on its own, with nothing else in flight: one
// thread waits on an mbarrier that nothing ever arrives on.
#include <cuda_runtime.h>

#include "cc3_internal.h"
#include "sm100_prims.cuh"

namespace {

__global__ void wait_timeout_kernel(unsigned long long limit_ns, int *status) {
  using namespace cc3::sm100;
  __shared__ __align__(8) uint64_t bar;
  __shared__ volatile int err;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    err = 0;
    fence_barrier_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait(&bar, 0, &err, limit_ns)) atomicExch(status, err ? err : 1);
}

}  // namespace

extern "C" int cc3_debug_wait_timeout(double limit_s) {
  if (!(limit_s >= 1e-6 && limit_s <= 1.0)) return CC3_FAIL(CC3_ERR_ARG, "limit outside [1 us, 1 s]");
  int *status = nullptr;
  if (cudaMalloc(&status, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return CC3_FAIL(CC3_ERR_OOM, "status word");
  }
  int h = 0;
  cudaError_t e = cudaMemset(status, 0, sizeof(int));
  if (e == cudaSuccess) {
    wait_timeout_kernel<<<1, 32>>>((unsigned long long)(limit_s * 1e9), status);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(&h, status, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(status);
  if (e != cudaSuccess) return CC3_FAIL(CC3_ERR_CUDA, cudaGetErrorString(e));
  return h ? CC3_FAIL(CC3_ERR_TIMEOUT, "the bounded wait gave up") : CC3_OK;
}
