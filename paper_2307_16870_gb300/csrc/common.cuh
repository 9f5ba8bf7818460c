// Shared device-side definitions of the EA-MPS library: complex arithmetic on
// float2/double2, the device control block that holds the FP64 bookkeeping of
// the entanglement-aware truncation, and a bounded grid barrier.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace eamps {

// ----------------------------------------------------------------- complex
template <class R> struct C2;
template <> struct C2<float> { using T = float2; };
template <> struct C2<double> { using T = double2; };
template <class R> using cplx = typename C2<R>::T;

template <class R> __host__ __device__ __forceinline__ cplx<R> mk(R re, R im) {
  cplx<R> z; z.x = re; z.y = im; return z;
}
template <class Z> __host__ __device__ __forceinline__ Z cadd(Z a, Z b) { a.x += b.x; a.y += b.y; return a; }
template <class Z> __host__ __device__ __forceinline__ Z csub(Z a, Z b) { a.x -= b.x; a.y -= b.y; return a; }
template <class Z> __host__ __device__ __forceinline__ Z cmul(Z a, Z b) {
  Z z; z.x = a.x * b.x - a.y * b.y; z.y = a.x * b.y + a.y * b.x; return z;
}
// conj(a) * b
template <class Z> __host__ __device__ __forceinline__ Z cmulc(Z a, Z b) {
  Z z; z.x = a.x * b.x + a.y * b.y; z.y = a.x * b.y - a.y * b.x; return z;
}
template <class Z> __host__ __device__ __forceinline__ Z cconj(Z a) { a.y = -a.y; return a; }
template <class Z, class R> __host__ __device__ __forceinline__ Z cscale(Z a, R s) { a.x *= s; a.y *= s; return a; }
// acc += a * b
template <class Z> __host__ __device__ __forceinline__ void cfma(Z& acc, Z a, Z b) {
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
}

// ---------------------------------------------------------- status bits
enum : int {
  ST_NOT_CONVERGED = 1,
  ST_NONFINITE = 2,
  ST_TIMEOUT = 4,
  ST_CHI_CAP = 8,
  ST_BAD_ARG = 16,
};

// Device control block: FP64 bookkeeping of the entanglement-aware run and
// the per-gate outputs of the selection kernel.  One per handle.
struct DevCtrl {
  // schedule and inferred fidelity (Eq. prod / Eq. uniform / Fig. 1)
  double product;      // running product of truncation fidelities
  double lognorm;      // MPO: log of the norm factor folded out at every cut
  double f_min;
  double f0;           // F_min^(1/n)
  long long n_2q;
  long long n_done;    // truncations performed so far
  int strategy;
  int fixed_chi;
  int chi_max;
  int mixed_fid;
  int kind;
  int status;          // sticky ST_* bits
  // outputs of the last selection
  int k;
  int rank_bound;
  int cap_hit;
  int sweeps;          // Jacobi sweeps used by the last SVD
  double f, f_t, W, Wk;
  // grid barrier and sweep bookkeeping of the cooperative Jacobi kernel
  unsigned bar_count;
  unsigned bar_gen;
  unsigned rot[3];
  unsigned pad_;
  // wall-clock limit of every device-side wait, nanoseconds (0: kWaitNs)
  unsigned long long wait_ns;
  // failure self-test only (mps_selftest_timeout): which multi-CTA kernel withholds one signal
  int test_fault;
  int pad2_;
  // statistics accumulated over Jacobi launches (reset by the host)
  unsigned long long jac_sweeps;
  double jac_flops;
};

// Wall-clock limit of the waits: %globaltimer nanoseconds, so the budget of a wait depends neither
// on the SM clock nor on the cost of one poll.  DevCtrl::wait_ns overrides it per handle.
constexpr unsigned long long kWaitNs = 2000000000ull;
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned long long wait_deadline(const DevCtrl* ctrl) {
  const unsigned long long w = *(volatile const unsigned long long*)&ctrl->wait_ns;
  return global_ns() + (w ? w : kWaitNs);
}

// Grid-wide barrier for a cooperative launch of nblocks CTAs.  Returns false
// (and sets ST_TIMEOUT) if the wait passed its wall-clock deadline or another
// wait of the handle gave up; callers then return without further waits.
__device__ __forceinline__ bool grid_barrier(DevCtrl* ctrl, unsigned nblocks) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned* vgen = &ctrl->bar_gen;
    unsigned g = *vgen;
    __threadfence();
    unsigned arrived = atomicAdd(&ctrl->bar_count, 1u);
    if (arrived == nblocks - 1) {
      atomicExch(&ctrl->bar_count, 0u);
      __threadfence();
      atomicAdd(&ctrl->bar_gen, 1u);
    } else {
      const unsigned long long end = wait_deadline(ctrl);
      while (*vgen == g) {
        __nanosleep(32);
        if ((*(volatile int*)&ctrl->status & ST_TIMEOUT) || global_ns() > end) {
          atomicOr(&ctrl->status, ST_TIMEOUT);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    if (*(volatile int*)&ctrl->status & ST_TIMEOUT) ok = 0;
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

template <class R> __device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace eamps
