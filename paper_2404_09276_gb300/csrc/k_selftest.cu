// Self-test of the bounded-wait path that every pipelined kernel of the
// library uses: one thread waits on a shared-memory mbarrier that nothing
// ever arrives on, with a poll bound; when the bound runs out it writes the
// error word and the kernel returns, so the host sees DASHSVD_ETIMEOUT and
// the context stays usable. Nothing faults, traps or spins without a bound.
#include "internal.cuh"
#include "tc_common.cuh"

namespace dsvd {
namespace {

__global__ void bounded_wait_selftest_kernel(uint32_t polls, int* err) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    tc::fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // phase 0 of a fresh barrier completes only after one arrival, which never comes
    if (!tc::mbar_wait(&bar, 0u, polls)) atomicExch(err, 1);
  }
}

}  // namespace

cudaError_t launch_bounded_wait_selftest(uint32_t polls, int* err, cudaStream_t st) {
  bounded_wait_selftest_kernel<<<1, 32, 0, st>>>(polls, err);
  return cudaGetLastError();
}

}  // namespace dsvd
