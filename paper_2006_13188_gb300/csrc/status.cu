// Self-test of the device-side failure path: a kernel whose only wait can
// never complete.  One thread initialises a shared-memory mbarrier that
// expects one arrival and then waits for its phase with the plan's bounded
// wait; no copy, no tensor-core work and no other thread will ever arrive,
// so the wait runs out its budget, records EXT_ERR_TIMEOUT in the status word
// and returns.  Nothing asynchronous is in flight when it gives up.
#include "internal.h"
#include "tc_common.cuh"

__global__ void k_selftest_timeout(int* err) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x != 0) return;
  const uint32_t addr = tc::smem_u32(&bar);
  tc::mbar_init(addr, 1);
  tc::mbar_wait_bounded(addr, 0, 1000000000ull, err, EXT_ERR_TIMEOUT);
}

void launch_selftest_timeout(int* err, cudaStream_t st) { k_selftest_timeout<<<1, 32, 0, st>>>(err); }
