// Self-test of the bounded device waits (delimit_selftest_wait_timeout in
// include/delimit.h): failure detection exercised without a GPU fault.
#include "kernels.h"
#include "tc_gemm.h"
#include "tc_ptx.cuh"

namespace delimit {

// Self-test of the bounded waits: one thread waits, through the same wait_bounded the
// kernels use, on an mbarrier that nothing arrives at; when the limit runs out the
// wait records `code` in the error word and the kernel returns.
__global__ void wait_probe_kernel(int* err, int code) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  const uint32_t b = ptx::smem_u32(&bar);
  ptx::mbar_init(b, 1);
  ptx::fence_mbar_init();
  ptx::wait_bounded(b, 0, nullptr, err, code);
}

cudaError_t launch_wait_probe(int* err, int code, cudaStream_t st) {
  wait_probe_kernel<<<1, 32, 0, st>>>(err, code);
  count_launch();
  return cudaGetLastError();
}

}  // namespace delimit
