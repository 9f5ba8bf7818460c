// Self-test of failure detection without a GPU fault: a wait of the form every waiting kernel
// of the library uses (acquire load of a flag, back-off, iteration limit), on a flag that nothing
// sets.  It gives up after `limit` iterations, records ST_TIMEOUT in the status word and returns,
// so the host sees the error status and the context stays usable.
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace eamps {
namespace {

__global__ void wait_probe_kernel(const unsigned* __restrict__ flag, unsigned target, long long limit,
                                  DevCtrl* __restrict__ ctrl) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  long long spins = 0;
  for (;;) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(flag) : "memory");
    if (v >= target) return;
    if (++spins > 64) __nanosleep(20);
    if (spins > limit) {
      atomicOr(&ctrl->status, ST_TIMEOUT);
      return;
    }
  }
}

}  // namespace

cudaError_t wait_probe(const unsigned* flag, unsigned target, long long limit, DevCtrl* ctrl, cudaStream_t st) {
  wait_probe_kernel<<<1, 32, 0, st>>>(flag, target, limit, ctrl);
  return cudaGetLastError();
}

}  // namespace eamps
