// Self-test of failure detection without a GPU fault: one thread waits, in the form of the
// library's single-flag waits (acquire load, back-off, wall-clock deadline of DevCtrl::wait_ns),
// on a flag that nothing sets.  It gives up at the deadline, records ST_TIMEOUT in the status
// word and returns, so the host sees the error status and the context stays usable.  The
// multi-CTA forms (the Jacobi exchanges and the tensor-core pipeline) are exercised by the
// same entry point with one signal withheld inside those kernels (DevCtrl::test_fault).
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace eamps {
namespace {

__global__ void wait_probe_kernel(const unsigned* __restrict__ flag, unsigned target, DevCtrl* __restrict__ ctrl) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const unsigned long long end = wait_deadline(ctrl);
  int polls = 0;
  for (;;) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(flag) : "memory");
    if (v >= target) return;
    if (++polls > 64) __nanosleep(20);
    if ((*(volatile int*)&ctrl->status & ST_TIMEOUT) || global_ns() > end) {
      atomicOr(&ctrl->status, ST_TIMEOUT);
      return;
    }
  }
}

}  // namespace

cudaError_t wait_probe(const unsigned* flag, unsigned target, DevCtrl* ctrl, cudaStream_t st) {
  wait_probe_kernel<<<1, 32, 0, st>>>(flag, target, ctrl);
  return cudaGetLastError();
}

}  // namespace eamps
