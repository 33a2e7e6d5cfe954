// selftest.cu -- exercise the bounded-wait failure path on the device
// without a fault: a kernel waits on an mbarrier phase that nothing
// completes, with a small clock budget, and must give up, set the error
// word and return.
#include <cuda_runtime.h>

#include "internal.h"
#include "tma.cuh"

namespace vofl {
namespace {

__global__ void k_wait_selftest(int* err, long long budget) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  // no thread arrives and no copy is issued: phase 0 never completes
  mbar_wait_bounded(&bar, 0, err, budget);
}

}  // namespace
}  // namespace vofl

extern "C" int vofl_selftest_bounded_wait(int* gave_up) {
  using namespace vofl;
  if (!gave_up) return VOFL_EINVAL;
  *gave_up = 0;
  int* d_err = nullptr;
  if (dev_malloc(&d_err, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return VOFL_ENOMEM;
  }
  int rc = VOFL_OK;
  cudaMemset(d_err, 0, sizeof(int));
  k_wait_selftest<<<1, 32>>>(d_err, 2000000LL);  // ~1 ms budget
  count_launch();
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    rc = VOFL_ECUDA;
  } else {
    int h = 0;
    if (cudaMemcpy(&h, d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) rc = VOFL_ECUDA;
    *gave_up = h;
  }
  dev_free(d_err);
  return rc;
}
