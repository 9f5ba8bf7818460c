// One-sided (Hestenes) Jacobi SVD of the two-site matrix theta ("Truncation
// fidelity" section: the bond is truncated from the SVD of the contraction of
// both tensors neighbouring it).
//
// Design (sm_103a):
//  * The c columns are split into nb = 2P blocks of w columns; each of the P
//    CTAs of a cooperative launch holds one block pair in shared memory.
//  * A sweep visits every column pair once: the blocks meet in a round-robin
//    tournament (circle method, nb-1 rounds); inside a round a CTA rotates all
//    w*w cross pairs of its two blocks (w steps of w disjoint pairs), and in
//    round 0 also the pairs inside each block.
//  * One warp per column pair: lane-strided dot products, warp-shuffle
//    reduction, the 2x2 complex rotation applied by the same lanes.  No
//    shared-memory traffic between lanes of a pair.
//  * Between rounds the blocks go back to global memory (L2-resident) and the
//    CTAs meet at a bounded grid barrier; after the last round of a sweep the
//    rotation count decides convergence for every CTA at once.
//  * A pair is rotated only when |a^dagger b| > tol |a||b|, tol = 4 sqrt(l)
//    eps: below that the inner product is rounding noise.
#include <algorithm>
#include <cmath>
#include <cfloat>

#include "kernels.h"

namespace eamps {

namespace {

__device__ __forceinline__ int rr_player(int n, int r, int pos) {
  return pos == 0 ? 0 : ((pos - 1 + r) % (n - 1)) + 1;
}

template <class R> struct Eps;
template <> struct Eps<float> { static constexpr float v = FLT_EPSILON; };
template <> struct Eps<double> { static constexpr double v = DBL_EPSILON; };

// Orthogonalise columns x and y (length L, of which the first l enter the
// inner products).  Returns 1 if a rotation was applied.
template <class R>
__device__ __forceinline__ int rotate_pair(cplx<R>* __restrict__ x, cplx<R>* __restrict__ y, int l, int L,
                                           R tol, int lane) {
  R a = 0, b = 0, gr = 0, gi = 0;
  for (int i = lane; i < l; i += 32) {
    cplx<R> u = x[i], v = y[i];
    a = fma(u.x, u.x, fma(u.y, u.y, a));
    b = fma(v.x, v.x, fma(v.y, v.y, b));
    gr = fma(u.x, v.x, fma(u.y, v.y, gr));
    gi = fma(u.x, v.y, fma(-u.y, v.x, gi));
  }
  a = warp_sum(a); b = warp_sum(b); gr = warp_sum(gr); gi = warp_sum(gi);
  R g = sqrt(gr * gr + gi * gi);
  if (!(a > 0) || !(b > 0) || !(g > tol * sqrt(a) * sqrt(b))) return 0;
  R zeta = (b - a) / (2 * g);
  R t = (zeta >= 0 ? R(1) : R(-1)) / (fabs(zeta) + sqrt(R(1) + zeta * zeta));
  R cs = R(1) / sqrt(R(1) + t * t);
  R sn = cs * t;
  R er = gr / g, ei = gi / g;   // e^{i phi}, phi = arg(a^dagger b)
  // x' = cs x - sn e^{-i phi} y ;  y' = sn e^{i phi} x + cs y
  for (int i = lane; i < L; i += 32) {
    cplx<R> u = x[i], v = y[i];
    R cyr = er * v.x + ei * v.y, cyi = er * v.y - ei * v.x;
    R exr = er * u.x - ei * u.y, exi = er * u.y + ei * u.x;
    x[i] = mk<R>(cs * u.x - sn * cyr, cs * u.y - sn * cyi);
    y[i] = mk<R>(sn * exr + cs * v.x, sn * exi + cs * v.y);
  }
  return 1;
}

template <class R>
struct JArgs {
  cplx<R>* X; long long ldx; int l; int c;
  cplx<R>* W; long long ldw;
  int w; int nb; int max_sweeps; R tol;
  DevCtrl* ctrl;
};

template <class R>
__device__ void load_pair(const JArgs<R>& p, cplx<R>* slots, int* gcol, int L, int bA, int bB) {
  const int w = p.w;
  for (int s = threadIdx.x; s < 2 * w; s += blockDim.x) {
    int g = (s < w) ? bA * w + s : bB * w + (s - w);
    gcol[s] = g < p.c ? g : -1;
  }
  __syncthreads();
  const long long total = (long long)2 * w * L;
  for (long long e = threadIdx.x; e < total; e += blockDim.x) {
    int s = (int)(e / L), i = (int)(e % L);
    int g = gcol[s];
    cplx<R> v = mk<R>(0, 0);
    if (g >= 0) v = (i < p.l) ? p.X[g * p.ldx + i] : p.W[g * p.ldw + (i - p.l)];
    slots[(long long)s * L + i] = v;
  }
  __syncthreads();
}

template <class R>
__device__ void store_pair(const JArgs<R>& p, const cplx<R>* slots, const int* gcol, int L) {
  const int w = p.w;
  const long long total = (long long)2 * w * L;
  for (long long e = threadIdx.x; e < total; e += blockDim.x) {
    int s = (int)(e / L), i = (int)(e % L);
    int g = gcol[s];
    if (g < 0) continue;
    cplx<R> v = slots[(long long)s * L + i];
    if (i < p.l) p.X[g * p.ldx + i] = v; else p.W[g * p.ldw + (i - p.l)] = v;
  }
  __syncthreads();
}

template <class R>
__global__ void __launch_bounds__(256) jacobi_kernel(JArgs<R> p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int w = p.w, nb = p.nb, P = nb / 2;
  const int L = p.l + (p.W ? p.c : 0);
  cplx<R>* slots = reinterpret_cast<cplx<R>*>(smem_raw);
  int* gcol = reinterpret_cast<int*>(slots + (long long)2 * w * L);
  __shared__ unsigned rot_s;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int cta = blockIdx.x;
  const int wpad = w + (w & 1);   // even player count for the intra-block tournament

  int bA = rr_player(nb, 0, cta), bB = rr_player(nb, 0, nb - 1 - cta);
  unsigned long long rot_total = 0;   // thread 0: rotations of this CTA over all sweeps
  bool loaded = false;
  int sweep = 0;
  bool converged = false;
  for (sweep = 0; sweep < p.max_sweeps; ++sweep) {
    if (threadIdx.x == 0) rot_s = 0;
    __syncthreads();
    for (int r = 0; r < nb - 1; ++r) {
      bA = rr_player(nb, r, cta);
      bB = rr_player(nb, r, nb - 1 - cta);
      if (P > 1 || !loaded) { load_pair(p, slots, gcol, L, bA, bB); loaded = true; }
      unsigned my_rot = 0;
      if (r == 0) {
        // pairs inside each block: round robin over wpad players, both blocks at once
        const int half = wpad / 2;
        for (int t = 0; t < wpad - 1; ++t) {
          for (int pi = warp; pi < 2 * half; pi += nwarps) {
            int blk = pi / half, i = pi % half;
            int s1 = rr_player(wpad, t, i), s2 = rr_player(wpad, t, wpad - 1 - i);
            if (s1 >= w || s2 >= w) continue;
            s1 += blk * w; s2 += blk * w;
            if (gcol[s1] < 0 || gcol[s2] < 0) continue;
            my_rot += rotate_pair<R>(slots + (long long)s1 * L, slots + (long long)s2 * L, p.l, L, p.tol, lane);
          }
          __syncthreads();
        }
      }
      // cross pairs between the two blocks
      for (int t = 0; t < w; ++t) {
        for (int i = warp; i < w; i += nwarps) {
          int s1 = i, s2 = w + (i + t) % w;
          if (gcol[s1] < 0 || gcol[s2] < 0) continue;
          my_rot += rotate_pair<R>(slots + (long long)s1 * L, slots + (long long)s2 * L, p.l, L, p.tol, lane);
        }
        __syncthreads();
      }
      if (lane == 0 && my_rot) atomicAdd(&rot_s, my_rot);
      if (P > 1) {
        store_pair(p, slots, gcol, L);
        if (r == nb - 2 && threadIdx.x == 0) atomicAdd(&p.ctrl->rot[sweep % 3], rot_s);
        if (!grid_barrier(p.ctrl, P)) return;
        if (r == 0 && cta == 0 && threadIdx.x == 0) p.ctrl->rot[(sweep + 1) % 3] = 0u;
      } else {
        __syncthreads();
      }
    }
    unsigned total = (P > 1) ? *(volatile unsigned*)&p.ctrl->rot[sweep % 3] : rot_s;
    if (threadIdx.x == 0) rot_total += rot_s;
    __syncthreads();
    if (total == 0) { converged = true; break; }
  }
  if (P == 1 && loaded) store_pair(p, slots, gcol, L);
  if (threadIdx.x == 0) {
    // algorithmic flops: 16 l per visited pair (three complex inner products),
    // 24 L per rotation applied (two complex column updates of length L)
    atomicAdd(&p.ctrl->jac_flops, 24.0 * (double)L * (double)rot_total);
  }
  if (cta == 0 && threadIdx.x == 0) {
    const int used = converged ? sweep + 1 : sweep;
    p.ctrl->sweeps = used;
    atomicAdd(&p.ctrl->jac_sweeps, (unsigned long long)used);
    atomicAdd(&p.ctrl->jac_flops, 16.0 * (double)p.l * 0.5 * (double)p.c * (double)(p.c - 1) * (double)used);
    if (!converged) atomicOr(&p.ctrl->status, ST_NOT_CONVERGED);
  }
}

}  // namespace

template <class R> int jacobi_max_ctas(size_t smem) {
  int per_sm = 0;
  if (cudaFuncSetAttribute(jacobi_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_kernel<R>, 256, smem) != cudaSuccess) return 0;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return per_sm * sms;
}

template <class R>
JacobiPlan jacobi_plan(int l, int c, bool accumulate, int sm_count, int max_ctas) {
  JacobiPlan plan;
  const size_t budget = 200 * 1024;
  const size_t col_bytes = (size_t)(l + (accumulate ? c : 0)) * sizeof(cplx<R>);
  int w_fit = (int)std::max<size_t>(1, budget / (2 * col_bytes + 8));
  int half = (c + 1) / 2;
  if (half <= w_fit && c <= 128) {
    plan.w = std::max(1, half);        // one CTA holds every column: no grid barrier at all
    plan.nb = 2;
  } else {
    int target = std::max(1, std::min(sm_count, max_ctas));
    int w = (c + 2 * target - 1) / (2 * target);
    w = std::max(1, std::min(w, w_fit));
    int P = (c + 2 * w - 1) / (2 * w);
    if (P > target) {  // smem too small for the spread: fall back to the largest fitting block
      w = w_fit;
      P = (c + 2 * w - 1) / (2 * w);
    }
    plan.w = w;
    plan.nb = 2 * P;
  }
  plan.smem = (size_t)2 * plan.w * (l + (accumulate ? c : 0)) * sizeof(cplx<R>) + 2 * plan.w * sizeof(int) + 16;
  return plan;
}

template <class R>
cudaError_t jacobi_launch(const JacobiPlan& plan, cplx<R>* X, long long ldx, int l, int c,
                          cplx<R>* W, long long ldw, int max_sweeps, DevCtrl* ctrl, cudaStream_t st) {
  if (c <= 1) {
    // a single column is already "orthogonal"
    return cudaSuccess;
  }
  cudaError_t e = cudaFuncSetAttribute(jacobi_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plan.smem);
  if (e != cudaSuccess) return e;
  // reset barrier and sweep counters (bar_count, bar_gen, rot[3] are contiguous)
  e = cudaMemsetAsync(&ctrl->bar_count, 0, 5 * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  JArgs<R> a;
  a.X = X; a.ldx = ldx; a.l = l; a.c = c; a.W = W; a.ldw = ldw;
  a.w = plan.w; a.nb = plan.nb; a.max_sweeps = max_sweeps;
  a.tol = R(4) * std::sqrt(R(std::max(l, 1))) * Eps<R>::v;
  a.ctrl = ctrl;
  void* args[] = {&a};
  const int P = plan.nb / 2;
  if (P == 1) return cudaLaunchKernel((void*)jacobi_kernel<R>, dim3(1), dim3(256), args, plan.smem, st);
  return cudaLaunchCooperativeKernel((void*)jacobi_kernel<R>, dim3(P), dim3(256), args, plan.smem, st);
}

template JacobiPlan jacobi_plan<float>(int, int, bool, int, int);
template JacobiPlan jacobi_plan<double>(int, int, bool, int, int);
template cudaError_t jacobi_launch<float>(const JacobiPlan&, cplx<float>*, long long, int, int, cplx<float>*,
                                          long long, int, DevCtrl*, cudaStream_t);
template cudaError_t jacobi_launch<double>(const JacobiPlan&, cplx<double>*, long long, int, int, cplx<double>*,
                                           long long, int, DevCtrl*, cudaStream_t);
template int jacobi_max_ctas<float>(size_t);
template int jacobi_max_ctas<double>(size_t);

}  // namespace eamps
