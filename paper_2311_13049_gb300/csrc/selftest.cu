// selftest.cu -- exercise the bounded-wait failure paths on the device
// without a fault: a kernel waits on an mbarrier phase that nothing
// completes, and a two-CTA kernel waits at the grid-wide barrier of the
// cooperative forward launch, which its second CTA never reaches; with a
// small clock budget each must give up, set its error word and return.
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

__global__ void k_grid_barrier_selftest(unsigned long long* ctr, int* err, long long budget) {
  if (blockIdx.x == 1) return;  // never arrives
  grid_barrier_bounded(ctr, err, budget);
}

}  // namespace
}  // namespace vofl

extern "C" int vofl_selftest_bounded_wait(int* gave_up) {
  using namespace vofl;
  if (!gave_up) return VOFL_EINVAL;
  *gave_up = 0;
  // [0]: mbarrier wait's error word, [1]: grid barrier's, then from [2]
  // the barrier's count and generation (two 8-byte words)
  int* d_buf = nullptr;
  if (dev_malloc(&d_buf, 8 * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return VOFL_ENOMEM;
  }
  int rc = VOFL_OK;
  cudaMemset(d_buf, 0, 8 * sizeof(int));
  unsigned long long* d_ctr = reinterpret_cast<unsigned long long*>(d_buf + 2);
  k_wait_selftest<<<1, 32>>>(d_buf, 2000000LL);  // ~1 ms budget
  k_grid_barrier_selftest<<<2, 32>>>(d_ctr, d_buf + 1, 2000000LL);
  count_launch(2);
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    rc = VOFL_ECUDA;
  } else {
    int h[2] = {0, 0};
    if (cudaMemcpy(h, d_buf, 2 * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) rc = VOFL_ECUDA;
    *gave_up = (h[0] && h[1]) ? 1 : 0;
  }
  dev_free(d_buf);
  return rc;
}
