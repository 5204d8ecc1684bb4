// Diagnostic of the library's bounded device waits (the mbarrier waits of the
// TMA-staged tile solve).  One block waits on an mbarrier phase that no copy
// ever completes: thread 0 announces a transaction count, no copy is issued,
// so the phase stays open; the wait gives up after the given number of SM
// clock cycles, records ST_TIMEOUT in the status word (which pm_check reports
// as PM_ERR_TIMEOUT) and the block invalidates the barrier and returns.
// Nothing is in flight when it exits: no fault, no hang, the context stays
// usable.
#include <cuda_runtime.h>

#include "pm_common.cuh"
#include "tma.cuh"

namespace pm {

__global__ void k_wait_probe(int* status, long long limit) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    tma::mbar_init(&bar, 1);
    tma::fence_barrier_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) tma::mbar_arrive_expect_tx(&bar, 16u);   // 16 bytes that no copy delivers
  const int gave_up = tma::mbar_wait(&bar, 0, limit) ? 0 : 1;
  if (__syncthreads_or(gave_up) && threadIdx.x == 0) atomicOr(status, ST_TIMEOUT);
  __syncthreads();
  if (threadIdx.x == 0) asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" ::"r"(tma::smem_u32(&bar)) : "memory");
}

cudaError_t launch_wait_probe(int* status, long long limit, cudaStream_t st) {
  k_wait_probe<<<1, 32, 0, st>>>(status, limit);
  return cudaGetLastError();
}

}  // namespace pm
