// Diagnostics entry point: one kernel that waits, with the bounded mbarrier wait the
// tensor-core kernels and the cluster eigensolver use, on a barrier that another
// thread of the block may or may not arrive on. A wait that gives up returns and
// reports through a status word, which the host turns into LR_ETIMEOUT: the context
// stays usable, so the failure path can be exercised without faulting the device.
#include <stdint.h>

#include "common.cuh"
#include "kernels.h"
#include "lret.h"
#include "tc_common.cuh"

namespace {

__global__ void k_selftest_wait(long long polls, int arrive, int* __restrict__ status) {
  __shared__ __align__(8) uint64_t mbar;
  const uint32_t a = lret::tc::smem_u32(&mbar);
  if (threadIdx.x == 0) {
    lret::tc::mbar_init(a, 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  __syncthreads();
  if (threadIdx.x == 1 && arrive) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
  if (threadIdx.x == 0) *status = lret::tc::mbar_wait_n(a, 0u, polls) ? 0 : 1;
}

}  // namespace

extern "C" int lr_selftest_wait(long long polls, int arrive, void* stream) {
  if (polls < 1) return LR_EINVAL;
  const cudaStream_t s = (cudaStream_t)stream;
  int* d_status = nullptr;
  if (cudaMalloc((void**)&d_status, sizeof(int)) != cudaSuccess) return LR_ENOMEM;
  int h_status = -1;
  k_selftest_wait<<<1, 32, 0, s>>>(polls, arrive ? 1 : 0, d_status);
  lret::note_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_status, d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d_status);
  if (e != cudaSuccess) {
    lret::set_error("%s%s", "lr_selftest_wait: ", cudaGetErrorString(e));
    return LR_ECUDA;
  }
  return h_status == 0 ? LR_OK : LR_ETIMEOUT;
}
