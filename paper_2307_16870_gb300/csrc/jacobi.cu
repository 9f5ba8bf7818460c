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
#include <cfloat>
#include <cmath>
#include <cstdlib>
#include <type_traits>

#include <cooperative_groups.h>

#include "kernels.h"

namespace eamps {

namespace {

__device__ __forceinline__ int rr_player(int n, int r, int pos) {
  return pos == 0 ? 0 : ((pos - 1 + r) % (n - 1)) + 1;
}

template <class R> struct Eps;
template <> struct Eps<float> { static constexpr float v = FLT_EPSILON; };
template <> struct Eps<double> { static constexpr double v = DBL_EPSILON; };

// Parameters of the 2x2 complex Jacobi rotation that makes columns with squared
// norms a, b and inner product gr + i gi orthogonal; false when the pair is
// already orthogonal to the tolerance.  FP64: IEEE operations; FP32: fast
// reciprocal square roots (the rotation only has to be close to unitary).
template <class R>
__device__ __forceinline__ bool rot_params(R a, R b, R gr, R gi, R tol, R& cs, R& sn, R& er, R& ei);
template <>
__device__ __forceinline__ bool rot_params<double>(double a, double b, double gr, double gi, double tol, double& cs,
                                                   double& sn, double& er, double& ei) {
  const double g = sqrt(gr * gr + gi * gi);
  if (!(a > 0) || !(b > 0) || !(g > tol * sqrt(a) * sqrt(b))) return false;
  const double zeta = (b - a) / (2 * g);
  const double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
  cs = 1.0 / sqrt(1.0 + t * t);
  sn = cs * t;
  er = gr / g;
  ei = gi / g;
  return true;
}
template <>
__device__ __forceinline__ bool rot_params<float>(float a, float b, float gr, float gi, float tol, float& cs,
                                                  float& sn, float& er, float& ei) {
  const float g2 = gr * gr + gi * gi;
  if (!(a > 0.f) || !(b > 0.f) || !(g2 > tol * tol * a * b)) return false;
  const float rg = rsqrtf(g2);
  const float zeta = 0.5f * (b - a) * rg;
  const float z2 = 1.f + zeta * zeta;
  const float t = __fdividef(zeta >= 0.f ? 1.f : -1.f, fabsf(zeta) + z2 * rsqrtf(z2));
  cs = rsqrtf(1.f + t * t);
  sn = cs * t;
  er = gr * rg;
  ei = gi * rg;
  return true;
}

// FP32 rotation of the register-resident kernels in the form the column update uses:
// cs = cos, (al, be) = sin * e^{i phi} split into real and imaginary parts.  With
// u = b - a, v = 2|g| and D = |u| + sqrt(u^2 + v^2): tan = sign(u) v / D, so
// cs = D / sqrt(D^2 + v^2) and sin e^{i phi} = sign(u) 2 g / sqrt(D^2 + v^2) -- the same
// angle as rot_params<float>, with two reciprocal square roots instead of four
// dependent special-function operations.  cs^2 + |sin|^2 = 1 to rsqrt accuracy.
__device__ __forceinline__ bool rot_params_fused(float a, float b, float gr, float gi, float tol, float& cs, float& al,
                                                 float& be) {
  const float g2 = gr * gr + gi * gi;
  if (!(a > 0.f) || !(b > 0.f) || !(g2 > tol * tol * a * b)) return false;
  const float u = b - a;
  const float x = fmaf(u, u, 4.f * g2);
  const float h = x * rsqrtf(x);
  const float D = fabsf(u) + h;
  const float r = rsqrtf(fmaf(D, D, 4.f * g2));
  const float s2 = (u >= 0.f) ? 2.f * r : -2.f * r;
  cs = D * r;
  al = s2 * gr;
  be = s2 * gi;
  return true;
}

// Orthogonalise columns x and y (length L, of which the first l enter the
// inner products).  Returns 0 when no rotation was applied, 1 for a rotation of a pair
// whose cosine was at most tol_stop, 2 for a larger one.
template <class R>
__device__ __forceinline__ int rotate_pair(cplx<R>* __restrict__ x, cplx<R>* __restrict__ y, int l, int L,
                                           R tol, R tol_stop, int lane) {
  R a = 0, b = 0, gr = 0, gi = 0;
  for (int i = lane; i < l; i += 32) {
    cplx<R> u = x[i], v = y[i];
    a = fma(u.x, u.x, fma(u.y, u.y, a));
    b = fma(v.x, v.x, fma(v.y, v.y, b));
    gr = fma(u.x, v.x, fma(u.y, v.y, gr));
    gi = fma(u.x, v.y, fma(-u.y, v.x, gi));
  }
  a = warp_sum(a); b = warp_sum(b); gr = warp_sum(gr); gi = warp_sum(gi);
  R cs, sn, er, ei;
  if (!rot_params<R>(a, b, gr, gi, tol, cs, sn, er, ei)) return 0;
  const int large = (gr * gr + gi * gi > tol_stop * tol_stop * a * b) ? 2 : 1;
  // x' = cs x - sn e^{-i phi} y ;  y' = sn e^{i phi} x + cs y
  for (int i = lane; i < L; i += 32) {
    cplx<R> u = x[i], v = y[i];
    R cyr = er * v.x + ei * v.y, cyi = er * v.y - ei * v.x;
    R exr = er * u.x - ei * u.y, exi = er * u.y + ei * u.x;
    x[i] = mk<R>(cs * u.x - sn * cyr, cs * u.y - sn * cyi);
    y[i] = mk<R>(sn * exr + cs * v.x, sn * exi + cs * v.y);
  }
  return large;
}

template <class R>
struct JArgs {
  cplx<R>* X; long long ldx; int l; int c;
  cplx<R>* W; long long ldw;
  int w; int nb; int max_sweeps; R tol;
  R tol_stop;          // a sweep whose largest pair cosine is at most this ends the iteration
  DevCtrl* ctrl;
  cplx<R>* xch;        // exchange slots: [2 parities][nb positions][w columns][L]
  unsigned* flags;     // per position: 1 + the last round whose block was published
};

__device__ __forceinline__ void st_release(unsigned* a, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(a), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned* a) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
  return v;
}
__device__ __forceinline__ unsigned atom_add_release(unsigned* a, unsigned v) {
  unsigned old;
  asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(a), "r"(v) : "memory");
  return old;
}

// Thread 0 waits until *a >= target, for at most the handle's wall-clock wait limit (or until
// another wait of the handle has given up); the whole CTA then proceeds.
__device__ __forceinline__ bool cta_wait_geq(const unsigned* a, unsigned target, DevCtrl* ctrl) {
  __shared__ int ok_s;
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned long long end = wait_deadline(ctrl);
    int polls = 0;
    while (ld_acquire(a) < target) {
      if (++polls > 64) __nanosleep(20);
      if ((*(volatile int*)&ctrl->status & ST_TIMEOUT) || global_ns() > end) {
        atomicOr(&ctrl->status, ST_TIMEOUT);
        ok = 0;
        break;
      }
    }
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// Thread 0 only: wait until *a >= target, bounded as cta_wait_geq (sets ST_TIMEOUT and returns
// false on expiry).
__device__ __forceinline__ bool spin_geq(const unsigned* a, unsigned target, DevCtrl* ctrl) {
  const unsigned long long end = wait_deadline(ctrl);
  int polls = 0;
  while (ld_acquire(a) < target) {
    if (++polls > 64) __nanosleep(20);
    if ((*(volatile int*)&ctrl->status & ST_TIMEOUT) || global_ns() > end) {
      atomicOr(&ctrl->status, ST_TIMEOUT);
      return false;
    }
  }
  return true;
}

// Bulk (TMA, untiled) copies between the exchange slots and shared memory.  Both
// addresses are 16-byte aligned and the size is a multiple of 16 bytes.
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void xbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
  // make the initialised barrier visible to the async proxy that completes the copies
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void xbar_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void xbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
// Wait for the phase of the given parity, bounded by the handle's wall-clock wait limit; false
// on expiry.
__device__ __forceinline__ bool xbar_wait(uint64_t* bar, uint32_t parity, const DevCtrl* ctrl) {
  const unsigned long long end = wait_deadline(ctrl);
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done) : "r"(smem_addr(bar)), "r"(parity) : "memory");
    if (done) return true;
    if (global_ns() > end) return false;
  }
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void bulk_store(void* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_addr(src)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// Wait until at most N committed bulk groups of this thread are pending (older ones complete).
template <int N>
__device__ __forceinline__ void bulk_wait() { asm volatile("cp.async.bulk.wait_group %0;" ::"n"(N) : "memory"); }
// Make completed bulk stores visible at GPU scope, then release a flag.
__device__ __forceinline__ void publish_flag(unsigned* flag, unsigned v) {
  asm volatile("fence.proxy.async.global;" ::: "memory");
  __threadfence();
  st_release(flag, v);
}

template <class R>
__device__ void load_pair(const JArgs<R>& p, cplx<R>* slots, int* gcol, int L, int bA, int bB) {
  const int w = p.w;
  for (int s = threadIdx.x; s < 2 * w; s += blockDim.x) {
    int g = (s < w) ? bA * w + s : bB * w + (s - w);
    gcol[s] = g < p.c ? g : -1;
  }
  __syncthreads();
  // one warp per column, lanes along the rows (coalesced, no index division)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int s = warp; s < 2 * w; s += nwarps) {
    const int g = gcol[s];
    cplx<R>* dst = slots + (long long)s * L;
    if (g < 0) {
      for (int i = lane; i < L; i += 32) dst[i] = mk<R>(0, 0);
      continue;
    }
    const cplx<R>* xs = p.X + (long long)g * p.ldx;
    for (int i = lane; i < p.l; i += 32) dst[i] = __ldcg(xs + i);
    if (p.W) {
      const cplx<R>* ws = p.W + (long long)g * p.ldw;
      for (int i = lane; i < p.c; i += 32) dst[p.l + i] = __ldcg(ws + i);
    }
  }
  __syncthreads();
}

template <class R>
__device__ void store_pair(const JArgs<R>& p, const cplx<R>* slots, const int* gcol, int L) {
  const int w = p.w;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int s = warp; s < 2 * w; s += nwarps) {
    const int g = gcol[s];
    if (g < 0) continue;
    const cplx<R>* src = slots + (long long)s * L;
    cplx<R>* xd = p.X + (long long)g * p.ldx;
    for (int i = lane; i < p.l; i += 32) __stcg(xd + i, src[i]);
    if (p.W) {
      cplx<R>* wd = p.W + (long long)g * p.ldw;
      for (int i = lane; i < p.c; i += 32) __stcg(wd + i, src[p.l + i]);
    }
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
  __shared__ unsigned rot_s, big_s;   // rotations of this CTA in the sweep, those above tol_stop
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int cta = blockIdx.x;
  const int wpad = w + (w & 1);   // even player count for the intra-block tournament

  int bA = rr_player(nb, 0, cta), bB = rr_player(nb, 0, nb - 1 - cta);
  unsigned long long rot_total = 0;   // thread 0: rotations of this CTA over all sweeps
  bool loaded = false;
  int sweep = 0;
  bool converged = false;
  for (sweep = 0; sweep < p.max_sweeps; ++sweep) {
    if (threadIdx.x == 0) { rot_s = 0; big_s = 0; }
    __syncthreads();
    for (int r = 0; r < nb - 1; ++r) {
      bA = rr_player(nb, r, cta);
      bB = rr_player(nb, r, nb - 1 - cta);
      if (P > 1 || !loaded) { load_pair(p, slots, gcol, L, bA, bB); loaded = true; }
      unsigned my_rot = 0, my_big = 0;
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
            const int rc = rotate_pair<R>(slots + (long long)s1 * L, slots + (long long)s2 * L, p.l, L, p.tol,
                                          p.tol_stop, lane);
            my_rot += rc != 0;
            my_big += rc == 2;
          }
          __syncthreads();
        }
      }
      // cross pairs between the two blocks
      for (int t = 0; t < w; ++t) {
        for (int i = warp; i < w; i += nwarps) {
          int s1 = i, s2 = w + (i + t) % w;
          if (gcol[s1] < 0 || gcol[s2] < 0) continue;
          const int rc = rotate_pair<R>(slots + (long long)s1 * L, slots + (long long)s2 * L, p.l, L, p.tol,
                                        p.tol_stop, lane);
          my_rot += rc != 0;
          my_big += rc == 2;
        }
        __syncthreads();
      }
      if (lane == 0 && my_rot) atomicAdd(&rot_s, my_rot);
      if (lane == 0 && my_big) atomicAdd(&big_s, my_big);
      if (P > 1) {
        store_pair(p, slots, gcol, L);
        if (r == nb - 2 && threadIdx.x == 0) atomicAdd(&p.ctrl->rot[sweep % 3], big_s);
        if (!grid_barrier(p.ctrl, P)) return;
        if (r == 0 && cta == 0 && threadIdx.x == 0) p.ctrl->rot[(sweep + 1) % 3] = 0u;
      } else {
        __syncthreads();
      }
    }
    unsigned total = (P > 1) ? *(volatile unsigned*)&p.ctrl->rot[sweep % 3] : big_s;
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


// Copy n complex entries global -> shared (or shared -> global) with eight loads in
// flight per lane; lanes of one warp stride over the column.
template <class Z, bool kFromGlobal>
__device__ __forceinline__ void warp_copy(Z* __restrict__ dst, const Z* __restrict__ src, int n, int lane) {
  constexpr int U = 8;
  for (int i0 = lane; i0 < n; i0 += 32 * U) {
    Z v[U];
#pragma unroll
    for (int j = 0; j < U; ++j) {
      const int i = i0 + 32 * j;
      if (i < n) v[j] = kFromGlobal ? __ldcg(src + i) : src[i];
    }
#pragma unroll
    for (int j = 0; j < U; ++j) {
      const int i = i0 + 32 * j;
      if (i < n) {
        if (kFromGlobal) dst[i] = v[j];
        else __stcg(dst + i, v[j]);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Register-resident kernels (complex64).
//
// Column layout in shared memory and in the exchange slots: ld = 32 * RPL rows,
// zero padded.  Rows [0, l) hold the column of X; when the rotations are
// accumulated, rows [lw, lw + c) hold the column of W, lw = l rounded up to a
// multiple of 32; every other row is zero.  Zero rows stay zero under the
// rotations, so loads and stores need no per-row bounds test, and the inner
// products run over the first kl = lw / 32 rows of each lane (all RPL rows
// when nothing is accumulated).  Columns past c are zero too: their squared
// norm is zero, so the rotation test skips every pair they are in.

// Column g of X (and of W) into a padded slot column; g < 0: a zero column.
template <int RPL>
__device__ __forceinline__ void fill_column(float2* __restrict__ dst, const JArgs<float>& p, int g, int lw, int lane) {
  constexpr int ld = 32 * RPL;
  if (g < 0) {
    for (int i = lane; i < ld; i += 32) dst[i] = make_float2(0.f, 0.f);
    return;
  }
  warp_copy<float2, true>(dst, p.X + (long long)g * p.ldx, p.l, lane);
  const int wend = p.W ? lw + p.c : p.l;
  for (int i = p.l + lane; i < lw && p.W; i += 32) dst[i] = make_float2(0.f, 0.f);
  if (p.W) warp_copy<float2, true>(dst + lw, p.W + (long long)g * p.ldw, p.c, lane);
  for (int i = wend + lane; i < ld; i += 32) dst[i] = make_float2(0.f, 0.f);
}

// Padded slot column back to column g of X (and of W).
__device__ __forceinline__ void drain_column(const float2* __restrict__ src, const JArgs<float>& p, int g, int lw,
                                             int lane) {
  if (g < 0) return;
  warp_copy<float2, false>(p.X + (long long)g * p.ldx, src, p.l, lane);
  if (p.W) warp_copy<float2, false>(p.W + (long long)g * p.ldw, src + lw, p.c, lane);
}

// Sum of each of N = 4 or 8 values over the 32 lanes of a warp, returned in every lane.
// Reduce-scatter (each halving level sends half of the remaining values), a butterfly on
// the single value left, then a broadcast: 2N - 1 + 5 - log2 N shuffles instead of 5 N.
template <int N>
__device__ __forceinline__ void warp_allreduce(float (&v)[N], int lane) {
  static_assert(N == 4 || N == 8, "four or eight values");
  constexpr int LOG = (N == 4) ? 2 : 3;
  float cur[N];
#pragma unroll
  for (int i = 0; i < N; ++i) cur[i] = v[i];
#pragma unroll
  for (int lev = 0; lev < LOG; ++lev) {
    const int half = (N >> lev) / 2;
    const int o = 16 >> lev;
    const bool upper = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const float send = upper ? cur[i] : cur[i + half];
      const float keep = upper ? cur[i + half] : cur[i];
      cur[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
#pragma unroll
  for (int o = 16 >> LOG; o > 0; o >>= 1) cur[0] += __shfl_xor_sync(0xffffffffu, cur[0], o);
  // lane holds the sum of value (lane >> (5 - LOG))
#pragma unroll
  for (int i = 0; i < N; ++i) v[i] = __shfl_sync(0xffffffffu, cur[0], i << (5 - LOG));
}

// The w*w cross pairs of one round.  The NW warps form SP groups of NW / SP; warp pw of group h
// keeps rows [h RPL / SP, (h + 1) RPL / SP) (per lane) of A columns ia = pw*AP + a in registers;
// at step t it takes the same rows of B column w + (ia + t) mod w, which warp pw + 1 (mod NW / SP)
// of its group released at step t - 1.  With SP > 1 the SP warps of a pair add their partial sums
// through shared memory, in the same order, so that they apply the same rotation.  Returns the
// rotations applied by this warp (counted by group 0 only).
template <int NW, int RPL, int AP, int SP>
__device__ __forceinline__ unsigned cross_phase(float2* __restrict__ slots, int w, int kl, float tol, float tol_stop,
                                                int lane, int warp, unsigned& big) {
  constexpr int ld = 32 * RPL;
  constexpr int NP = NW / SP;    // pairs in flight (warps per group)
  constexpr int RH = RPL / SP;   // rows per lane of one warp
  static_assert(NP * SP == NW && RH * SP == RPL, "the row split divides warps and rows");
  static_assert(SP == 1 || NP <= 15, "one named barrier per pair");
  __shared__ float part[SP > 1 ? 2 : 1][NP * AP][SP][4];   // by step parity
  const int pw = warp % NP, h = warp / NP, k0 = h * RH;
  float2 A[AP][RH], B[AP][RH];
  int ib[AP];
#pragma unroll
  for (int a = 0; a < AP; ++a) {
    ib[a] = pw * AP + a;
    const float2* src = slots + ib[a] * ld + lane;
#pragma unroll
    for (int k = 0; k < RH; ++k) A[a][k] = src[32 * (k0 + k)];
  }
  unsigned my_rot = 0;
  for (int t = 0; t < w; ++t) {
    float2* bcol[AP];
#pragma unroll
    for (int a = 0; a < AP; ++a) {
      bcol[a] = slots + (w + ib[a]) * ld + lane;
#pragma unroll
      for (int k = 0; k < RH; ++k) B[a][k] = bcol[a][32 * (k0 + k)];
    }
    // packed two-wide FP32: (u.re*u.re, u.im*u.im) style partial sums
    float2 d2a[AP], d2b[AP], g2a[AP], g2b[AP];
#pragma unroll
    for (int a = 0; a < AP; ++a) {
      d2a[a] = make_float2(0.f, 0.f); d2b[a] = d2a[a]; g2a[a] = d2a[a]; g2b[a] = d2a[a];
    }
#pragma unroll
    for (int k = 0; k < RH; ++k) {
      if (k0 + k < kl) {
#pragma unroll
        for (int a = 0; a < AP; ++a) {
          const float2 u = A[a][k], v = B[a][k];
          d2a[a] = __ffma2_rn(u, u, d2a[a]);
          d2b[a] = __ffma2_rn(v, v, d2b[a]);
          g2a[a] = __ffma2_rn(u, v, g2a[a]);                         // (u.re v.re, u.im v.im)
          g2b[a] = __ffma2_rn(u, make_float2(v.y, v.x), g2b[a]);      // (u.re v.im, u.im v.re)
        }
      }
    }
    float s[4 * AP];
#pragma unroll
    for (int a = 0; a < AP; ++a) {
      s[4 * a + 0] = d2a[a].x + d2a[a].y;
      s[4 * a + 1] = d2b[a].x + d2b[a].y;
      s[4 * a + 2] = g2a[a].x + g2a[a].y;      // Re(u^dagger v)
      s[4 * a + 3] = g2b[a].x - g2b[a].y;      // Im(u^dagger v)
    }
    warp_allreduce<4 * AP>(s, lane);
    if constexpr (SP > 1) {
      float (*pt)[SP][4] = part[t & 1];
      if (lane == 0) {
#pragma unroll
        for (int i = 0; i < 4 * AP; ++i) pt[pw * AP + i / 4][h][i % 4] = s[i];
      }
      // only the SP warps of this pair meet here (named barrier 1 + pw; 0 is the CTA barrier)
      asm volatile("bar.sync %0, %1;" ::"r"(1 + pw), "r"(32 * SP) : "memory");
#pragma unroll
      for (int i = 0; i < 4 * AP; ++i) {
        float acc = pt[pw * AP + i / 4][0][i % 4];
#pragma unroll
        for (int hh = 1; hh < SP; ++hh) acc += pt[pw * AP + i / 4][hh][i % 4];
        s[i] = acc;
      }
    }
#pragma unroll
    for (int a = 0; a < AP; ++a) {
      float cs, al, be;
      if (rot_params_fused(s[4 * a], s[4 * a + 1], s[4 * a + 2], s[4 * a + 3], tol, cs, al, be)) {
        if (h == 0)
          big += (s[4 * a + 2] * s[4 * a + 2] + s[4 * a + 3] * s[4 * a + 3] >
                  tol_stop * tol_stop * s[4 * a] * s[4 * a + 1]) ? 1u : 0u;
        // x' = cs x - sn e^{-i phi} y = cs x - al y - be (y.im, -y.re)
        // y' = sn e^{i phi} x + cs y = al x + be (-x.im, x.re) + cs y,  al + i be = sn e^{i phi}
        const float2 csv = make_float2(cs, cs), mal = make_float2(-al, -al), pal = make_float2(al, al);
        const float2 pbe = make_float2(-be, be);
#pragma unroll
        for (int k = 0; k < RH; ++k) {
          const float2 u = A[a][k], v = B[a][k];
          float2 nu = __fmul2_rn(u, csv);
          nu = __ffma2_rn(v, mal, nu);
          nu = __ffma2_rn(make_float2(v.y, v.x), pbe, nu);
          float2 nv = __fmul2_rn(v, csv);
          nv = __ffma2_rn(u, pal, nv);
          nv = __ffma2_rn(make_float2(u.y, u.x), pbe, nv);
          A[a][k] = nu;
          bcol[a][32 * (k0 + k)] = nv;
        }
        if (h == 0) ++my_rot;
      }
      ib[a] = (ib[a] + 1 == w) ? 0 : ib[a] + 1;
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < AP; ++a) {
    float2* dst = slots + (pw * AP + a) * ld + lane;
#pragma unroll
    for (int k = 0; k < RH; ++k) dst[32 * (k0 + k)] = A[a][k];
  }
  return my_rot;
}

// Pairs inside each of the two blocks (round 0 of a sweep): round robin over wpad players,
// both blocks at once, one warp per pair.
__device__ __forceinline__ unsigned intra_phase(float2* slots, const int* gcol, int w, int ld, int lrows, float tol,
                                                float tol_stop, int lane, int warp, int nwarps, unsigned& big) {
  const int wpad = w + (w & 1);
  const int half = wpad / 2;
  unsigned my_rot = 0;
  for (int t = 0; t < wpad - 1; ++t) {
    for (int pi = warp; pi < 2 * half; pi += nwarps) {
      const int blk = pi / half, i = pi % half;
      int s1 = rr_player(wpad, t, i), s2 = rr_player(wpad, t, wpad - 1 - i);
      if (s1 >= w || s2 >= w) continue;
      s1 += blk * w; s2 += blk * w;
      if (gcol[s1] < 0 || gcol[s2] < 0) continue;
      const int rc = rotate_pair<float>(slots + (long long)s1 * ld, slots + (long long)s2 * ld, lrows, ld, tol,
                                        tol_stop, lane);
      my_rot += rc != 0;
      big += rc == 2;
    }
    __syncthreads();
  }
  return my_rot;
}

// Register-resident kernel with point-to-point exchange.  CTA i always holds
// the positions i (block A) and nb-1-i (block B) of the circle-method
// tournament; after every round the blocks shift by one position, so each
// CTA takes its next blocks from its two neighbours.  A CTA publishes its two
// blocks into double-buffered exchange slots and releases a per-position
// flag; its neighbours acquire the flag before reading.  Double buffering is
// enough because every writer also reads from the CTA that reads its slot,
// so it cannot finish two rounds before that reader has taken the block.  The
// only grid-wide synchronisation is one counter barrier per sweep for the
// convergence vote.
//
// Blocks move by bulk copies (one per block and direction): the publishing
// thread drains its stores before the release, and the reading thread orders
// its bulk load after the acquire with a proxy fence.
template <class R, int NW, int RPL, int AP, int SP>
__global__ void __launch_bounds__(NW * 32) jacobi_kernel3(JArgs<R> p) {
  static_assert(std::is_same<R, float>::value, "register-resident kernels are complex64");
  constexpr int ld = 32 * RPL;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int w = p.w, nb = p.nb, P = nb / 2;
  const int lw = (p.l + 31) & ~31;
  const int kl = p.W ? lw / 32 : RPL;
  float2* slots = reinterpret_cast<float2*>(smem_raw);
  int* gcol = reinterpret_cast<int*>(slots + (long long)2 * w * ld);
  __shared__ unsigned rot_s, big_s;   // rotations in the sweep, those above tol_stop (the vote)
  __shared__ unsigned total_s;
  __shared__ __align__(8) uint64_t xbar;   // completion of the incoming bulk copies
  __shared__ int xok_s;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int cta = blockIdx.x;
  const int pos[2] = {cta, nb - 1 - cta};
  const long long blk = (long long)w * ld;   // entries per block
  const uint32_t blk_bytes = (uint32_t)(blk * (long long)sizeof(float2));
  const bool bulk = P > 1 && (reinterpret_cast<uintptr_t>(p.xch) & 15) == 0 && blk_bytes < (1u << 19);
  uint32_t xphase = 0;
  if (bulk && threadIdx.x == 0) xbar_init(&xbar);
  unsigned long long rot_total = 0;
  bool converged = false;
  int sweep = 0;
  unsigned rnd = 0;   // rounds completed over all sweeps
  const bool withhold = cta == 0 && *(volatile const int*)&p.ctrl->test_fault == 1;

  // round 0 of the first sweep: position q holds player q
  for (int s = threadIdx.x; s < 2 * w; s += blockDim.x) {
    const int g = pos[s / w] * w + (s % w);
    gcol[s] = g < p.c ? g : -1;
  }
  __syncthreads();
  for (int s = warp; s < 2 * w; s += NW) fill_column<RPL>(slots + (long long)s * ld, p, gcol[s], lw, lane);
  __syncthreads();

  for (sweep = 0; sweep < p.max_sweeps; ++sweep) {
    if (threadIdx.x == 0) { rot_s = 0; big_s = 0; }
    __syncthreads();
    for (int r = 0; r < nb - 1; ++r, ++rnd) {
      if (rnd > 0 && P > 1) {
        // take the blocks that moved into my positions
        if (bulk) {
          if (threadIdx.x == 0) {
            // both sources first: a copy is issued only once every source block is published,
            // so a wait that gives up never leaves a copy in flight into this CTA
            int ok = 1;
            for (int h = 0; h < 2 && ok; ++h) {
              if (pos[h] == 0) continue;                  // block 0 never moves
              const int src = (pos[h] == nb - 1) ? 1 : pos[h] + 1;
              if (!spin_geq(p.flags + src, rnd, p.ctrl)) ok = 0;
            }
            if (ok) {
              asm volatile("fence.proxy.async.global;" ::: "memory");
              for (int h = 0; h < 2; ++h) {
                if (pos[h] == 0) continue;
                const int src = (pos[h] == nb - 1) ? 1 : pos[h] + 1;
                xbar_expect(&xbar, blk_bytes);
                bulk_load(slots + h * blk, p.xch + ((long long)((rnd - 1) & 1) * nb + src) * blk, blk_bytes, &xbar);
              }
            }
            xbar_arrive(&xbar);   // the phase completes when the issued copies (if any) have landed
            xok_s = ok;
          }
          // every thread waits only for copies that were issued from published sources
          const bool landed = xbar_wait(&xbar, xphase, p.ctrl);
          xphase ^= 1u;
          if (__syncthreads_or(!landed)) {
            if (threadIdx.x == 0) atomicOr(&p.ctrl->status, ST_TIMEOUT);
            xbar_wait(&xbar, xphase ^ 1u, p.ctrl);   // one more bounded wait for them to land
            return;
          }
          if (!xok_s) return;
        } else {
          for (int h = 0; h < 2; ++h) {
            if (pos[h] == 0) continue;
            const int src = (pos[h] == nb - 1) ? 1 : pos[h] + 1;
            if (!cta_wait_geq(p.flags + src, rnd, p.ctrl)) return;
            const float2* from = p.xch + ((long long)((rnd - 1) & 1) * nb + src) * blk;
            for (int s = warp; s < w; s += NW)
              warp_copy<float2, true>(slots + (long long)(h * w + s) * ld, from + (long long)s * ld, ld, lane);
          }
        }
        for (int s = threadIdx.x; s < 2 * w; s += blockDim.x) {
          const int g = rr_player(nb, r, pos[s / w]) * w + (s % w);
          gcol[s] = g < p.c ? g : -1;
        }
        __syncthreads();
      }
      unsigned my_rot = 0, my_big = 0;
      if (r == 0) my_rot += intra_phase(slots, gcol, w, ld, 32 * kl, p.tol, p.tol_stop, lane, warp, NW, my_big);
      my_rot += cross_phase<NW, RPL, AP, SP>(slots, w, kl, p.tol, p.tol_stop, lane, warp, my_big);
      if (lane == 0 && my_rot) atomicAdd(&rot_s, my_rot);
      if (lane == 0 && my_big) atomicAdd(&big_s, my_big);
      // shared-memory writes above must be visible to the bulk stores below
      if (bulk) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      // failure self-test: CTA 0 withholds its publications (a later one would also satisfy a
      // wait for an earlier round), so its neighbours' waits run out
      if (P > 1 && !withhold) {
        // publish both blocks of this round (block 0 stays in CTA 0)
        float2* to = p.xch + (long long)(rnd & 1) * nb * blk;
        if (bulk) {
          if (threadIdx.x == 0) {
            // one bulk group per block, each flag released as soon as its own block has landed;
            // the final wait also ends the reads of shared memory before the next loads
            if (pos[0] != 0) { bulk_store(to + (long long)pos[0] * blk, slots, blk_bytes); bulk_commit(); }
            bulk_store(to + (long long)pos[1] * blk, slots + blk, blk_bytes);
            bulk_commit();
            if (pos[0] != 0) { bulk_wait<1>(); publish_flag(p.flags + pos[0], rnd + 1); }
            bulk_wait<0>();
            publish_flag(p.flags + pos[1], rnd + 1);
          }
        } else {
          for (int h = 0; h < 2; ++h) {
            if (pos[h] == 0) continue;
            float2* base = to + (long long)pos[h] * blk;
            for (int s = warp; s < w; s += NW)
              warp_copy<float2, false>(base + (long long)s * ld, slots + (long long)(h * w + s) * ld, ld, lane);
          }
          __syncthreads();
          if (threadIdx.x == 0) {
            __threadfence();
            if (pos[0] != 0) st_release(p.flags + pos[0], rnd + 1);
            st_release(p.flags + pos[1], rnd + 1);
          }
        }
      }
    }
    // convergence vote over all CTAs: one counter barrier per sweep
    if (P > 1) {
      if (threadIdx.x == 0) {
        atomicAdd(&p.ctrl->rot[sweep % 3], big_s);
        const unsigned old = atom_add_release(&p.ctrl->bar_count, 1u);
        total_s = (old / (unsigned)P + 1u) * (unsigned)P;   // arrivals that complete this barrier
      }
      __syncthreads();
      if (!cta_wait_geq(&p.ctrl->bar_count, total_s, p.ctrl)) return;
      if (threadIdx.x == 0) {
        total_s = ld_acquire(&p.ctrl->rot[sweep % 3]);
        if (cta == 0) p.ctrl->rot[(sweep + 2) % 3] = 0u;
      }
      __syncthreads();
    } else {
      if (threadIdx.x == 0) total_s = big_s;
      __syncthreads();
    }
    if (threadIdx.x == 0) rot_total += rot_s;
    const unsigned total = total_s;
    __syncthreads();
    if (total == 0) { converged = true; break; }
  }
  // final blocks back to their columns
  for (int s = warp; s < 2 * w; s += NW) drain_column(slots + (long long)s * ld, p, gcol[s], lw, lane);
  const double L = (double)p.l + (p.W ? (double)p.c : 0.0);
  if (threadIdx.x == 0) atomicAdd(&p.ctrl->jac_flops, 24.0 * L * (double)rot_total);
  if (cta == 0 && threadIdx.x == 0) {
    const int used = converged ? sweep + 1 : sweep;
    p.ctrl->sweeps = used;
    atomicAdd(&p.ctrl->jac_sweeps, (unsigned long long)used);
    atomicAdd(&p.ctrl->jac_flops, 16.0 * (double)p.l * 0.5 * (double)p.c * (double)(p.c - 1) * (double)used);
    if (!converged) atomicOr(&p.ctrl->status, ST_NOT_CONVERGED);
  }
}

// Cluster-resident kernel: the whole matrix lives in the shared memory of
// one thread-block cluster (P <= 16 CTAs).  After every round each CTA reads
// the blocks that shift into its positions straight from its neighbours'
// shared memory (distributed shared memory) into registers, between two
// hardware cluster barriers; no global-memory traffic, no flags.
template <class R, int NW, int RPL, int AP>
__global__ void __launch_bounds__(NW * 32) jacobi_cluster_kernel(JArgs<R> p) {
  static_assert(std::is_same<R, float>::value, "register-resident kernels are complex64");
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  constexpr int ld = 32 * RPL;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int w = p.w, nb = p.nb, P = nb / 2;
  const int lw = (p.l + 31) & ~31;
  const int kl = p.W ? lw / 32 : RPL;
  float2* slots = reinterpret_cast<float2*>(smem_raw);
  int* gcol = reinterpret_cast<int*>(slots + (long long)2 * w * ld);
  __shared__ unsigned rot_s, big_s, vote_s;
  __shared__ unsigned rot_slot[2], big_slot[2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int cta = (int)cluster.block_rank();
  const int pos[2] = {cta, nb - 1 - cta};
  unsigned long long rot_total = 0;
  bool converged = false;
  int sweep = 0;

  // sources of the blocks that move into my positions: (rank, half) of position src
  auto holder = [&](int q, int& rank, int& half) {
    if (q < P) { rank = q; half = 0; } else { rank = nb - 1 - q; half = 1; }
  };
  int srank[2], shalf[2];
  {
    const int srcA = cta + 1;                              // position cta + 1 (P -> own bottom)
    holder(srcA, srank[0], shalf[0]);
    const int srcB = (pos[1] == nb - 1) ? 1 : pos[1] + 1;  // position nb-1 takes from position 1
    holder(srcB, srank[1], shalf[1]);
  }

  for (int s = threadIdx.x; s < 2 * w; s += blockDim.x) {
    const int g = pos[s / w] * w + (s % w);
    gcol[s] = g < p.c ? g : -1;
  }
  if (threadIdx.x == 0) { rot_slot[0] = 0; rot_slot[1] = 0; big_slot[0] = 0; big_slot[1] = 0; vote_s = 0; }
  __syncthreads();
  for (int s = warp; s < 2 * w; s += NW) fill_column<RPL>(slots + (long long)s * ld, p, gcol[s], lw, lane);
  __syncthreads();

  for (sweep = 0; sweep < p.max_sweeps; ++sweep) {
    if (threadIdx.x == 0) { rot_s = 0; big_s = 0; }
    __syncthreads();
    for (int r = 0; r < nb - 1; ++r) {
      unsigned my_rot = 0, my_big = 0;
      if (r == 0) my_rot += intra_phase(slots, gcol, w, ld, 32 * kl, p.tol, p.tol_stop, lane, warp, NW, my_big);
      my_rot += cross_phase<NW, RPL, AP, 1>(slots, w, kl, p.tol, p.tol_stop, lane, warp, my_big);
      if (lane == 0 && my_rot) atomicAdd(&rot_s, my_rot);
      if (lane == 0 && my_big) atomicAdd(&big_s, my_big);
      __syncthreads();
      const bool last = (r == nb - 2);
      if (last && threadIdx.x == 0) { rot_slot[sweep & 1] = rot_s; big_slot[sweep & 1] = big_s; }
      if (P > 1) {
        cluster.sync();   // every CTA finished the round: its shared blocks are final
        // Two phases, one block staged in registers at a time.  Phase 1: CTAs 1..P-1 take the
        // block for their A half (position i+1), CTA 0 takes position 1's block for its B half
        // and keeps it in registers to the end (its own B half is still read in phase 2).
        // Phase 2: CTAs 1..P-1 take the block for their B half (position nb-i).
        float2 in[AP][RPL];
        {
          const int rk = (cta == 0) ? srank[1] : srank[0];
          const int hf = (cta == 0) ? shalf[1] : shalf[0];
          const float2* remote = cluster.map_shared_rank(slots, rk);
#pragma unroll
          for (int a = 0; a < AP; ++a) {
            const float2* src = remote + (long long)(hf * w + warp * AP + a) * ld + lane;
#pragma unroll
            for (int k = 0; k < RPL; ++k) in[a][k] = src[32 * k];
          }
        }
        unsigned vote = 0;
        if (last && threadIdx.x == 0) {
          for (int q = 0; q < P; ++q) vote += cluster.map_shared_rank(big_slot, q)[sweep & 1];
        }
        cluster.sync();   // phase-1 sources read
        if (cta != 0) {
#pragma unroll
          for (int a = 0; a < AP; ++a) {
            float2* dst = slots + (long long)(warp * AP + a) * ld + lane;
#pragma unroll
            for (int k = 0; k < RPL; ++k) dst[32 * k] = in[a][k];
          }
          const float2* remote = cluster.map_shared_rank(slots, srank[1]);
#pragma unroll
          for (int a = 0; a < AP; ++a) {
            const float2* src = remote + (long long)(shalf[1] * w + warp * AP + a) * ld + lane;
#pragma unroll
            for (int k = 0; k < RPL; ++k) in[a][k] = src[32 * k];
          }
        }
        cluster.sync();   // phase-2 sources read
#pragma unroll
        for (int a = 0; a < AP; ++a) {
          float2* dst = slots + (long long)(w + warp * AP + a) * ld + lane;
#pragma unroll
          for (int k = 0; k < RPL; ++k) dst[32 * k] = in[a][k];
        }
        const int rn = last ? 0 : r + 1;
        for (int s = threadIdx.x; s < 2 * w; s += blockDim.x) {
          const int g = rr_player(nb, rn, pos[s / w]) * w + (s % w);
          gcol[s] = g < p.c ? g : -1;
        }
        if (last && threadIdx.x == 0) vote_s = vote;
        __syncthreads();
      }
    }
    if (threadIdx.x == 0) rot_total += (P > 1) ? rot_slot[sweep & 1] : rot_s;
    const unsigned total = (P > 1) ? vote_s : big_s;   // rotations above tol_stop: cluster-wide or this CTA's
    __syncthreads();
    if (total == 0) { converged = true; break; }
  }
  // final blocks back to their columns
  for (int s = warp; s < 2 * w; s += NW) drain_column(slots + (long long)s * ld, p, gcol[s], lw, lane);
  const double L = (double)p.l + (p.W ? (double)p.c : 0.0);
  if (threadIdx.x == 0) atomicAdd(&p.ctrl->jac_flops, 24.0 * L * (double)rot_total);
  if (cta == 0 && threadIdx.x == 0) {
    const int used = converged ? sweep + 1 : sweep;
    p.ctrl->sweeps = used;
    atomicAdd(&p.ctrl->jac_sweeps, (unsigned long long)used);
    atomicAdd(&p.ctrl->jac_flops, 16.0 * (double)p.l * 0.5 * (double)p.c * (double)(p.c - 1) * (double)used);
    if (!converged) atomicOr(&p.ctrl->status, ST_NOT_CONVERGED);
  }
  cluster.sync();   // no CTA leaves while others may still read its shared memory
}

// Kernel variants of the register-resident form, indexed by (warps, rows per lane / 32, columns
// per warp, warps sharing the rows of a column pair).  Block width w = nw / sp * ap.
struct Variant { int nw, rpl, ap; const void* fn; int sp = 1; };

#define EAMPS_V(NW, RPL, AP) {NW, RPL, AP, (const void*)jacobi_kernel3<float, NW, RPL, AP, 1>}
#define EAMPS_S(NW, RPL, AP, SP) {NW, RPL, AP, (const void*)jacobi_kernel3<float, NW, RPL, AP, SP>, SP}
const Variant kVariants[] = {
    EAMPS_V(4, 4, 1),  EAMPS_V(8, 4, 1),  EAMPS_V(16, 4, 1),  EAMPS_V(8, 4, 2),  EAMPS_V(16, 4, 2),
    EAMPS_V(4, 8, 1),  EAMPS_V(8, 8, 1),  EAMPS_V(16, 8, 1),  EAMPS_V(4, 8, 2),  EAMPS_V(8, 8, 2), EAMPS_V(16, 8, 2),
    EAMPS_V(4, 12, 1), EAMPS_V(8, 12, 1), EAMPS_V(4, 12, 2),  EAMPS_V(8, 12, 2),
    EAMPS_V(4, 16, 1), EAMPS_V(8, 16, 1), EAMPS_V(16, 16, 1), EAMPS_V(4, 16, 2), EAMPS_V(8, 16, 2),
    EAMPS_V(4, 24, 1), EAMPS_V(8, 24, 1),
    EAMPS_V(4, 32, 1), EAMPS_V(8, 32, 1),
    // rows split over two warps: 8 columns per block on 16 warps
    EAMPS_S(16, 16, 1, 2), EAMPS_S(16, 8, 1, 2),
};
#undef EAMPS_V
#undef EAMPS_S

#define EAMPS_C(NW, RPL) {NW, RPL, 1, (const void*)jacobi_cluster_kernel<float, NW, RPL, 1>}
const Variant kClusterVariants[] = {
    EAMPS_C(8, 4),  EAMPS_C(16, 4), EAMPS_C(8, 8),  EAMPS_C(16, 8), EAMPS_C(8, 12),
    EAMPS_C(8, 16), EAMPS_C(16, 16), EAMPS_C(8, 24), EAMPS_C(8, 32),
};
#undef EAMPS_C

const Variant* find_cluster_variant(int nw, int rpl) {
  for (const Variant& v : kClusterVariants)
    if (v.nw == nw && v.rpl == rpl) return &v;
  return nullptr;
}

const Variant* find_variant(int nw, int rpl, int ap, int sp = 1) {
  for (const Variant& v : kVariants)
    if (v.nw == nw && v.rpl == rpl && v.ap == ap && v.sp == sp) return &v;
  return nullptr;
}

}  // namespace

namespace {

// Rows per lane of the register-resident kernels for padded columns of L rows (0: too long).
int rows_per_lane(int L) {
  for (int r : {4, 8, 12, 16, 24, 32})
    if (32 * r >= L) return r;
  return 0;
}

}  // namespace

template <class R>
int jacobi_max_ctas(const JacobiPlan& plan) {
  const void* fn = plan.fn ? plan.fn : (const void*)jacobi_kernel<R>;
  if (allow_dynamic_smem(fn) != cudaSuccess) return 0;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, plan.threads, plan.smem) != cudaSuccess) return 0;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return per_sm * sms;
}

// Block width, CTA count and kernel variant for one SVD.
//  * complex64 with columns of at most 1024 rows (accumulated rotations included): the
//    register-resident kernel; one CTA when every column fits it, else about
//    c / (2 w) CTAs with w = 8 columns per block.
//  * otherwise (complex128, longer columns): the shared-memory kernel.
template <class R>
JacobiPlan jacobi_plan(int l, int c, bool accumulate, int sm_count, int max_ctas, int kind) {
  JacobiPlan plan;
  const bool no_split = (kind & kJacobiNoSplit) != 0 || (kind & 7) == kJacobiTournamentUnsplit;
  kind &= 7;
  const int L = l + (accumulate ? c : 0);
  // block Jacobi with Gram-matrix inner sweeps over clusters across the GPU (jacobi_gram.cu)
  if (std::is_same<R, float>::value && kind != kJacobiTournament && kind != kJacobiTournamentUnsplit &&
      c >= (kind == kJacobiGram ? 64 : kGramMinCols) &&
      jacobi_gram_plan(l, c, accumulate, std::min(sm_count, max_ctas), plan))
    return plan;
  const size_t budget = 200 * 1024;
  // register-resident kernels: padded columns (W rows start at l rounded up to 32)
  const int Lreg = accumulate ? ((l + 31) & ~31) + c : l;
  const int rpl = rows_per_lane(Lreg);
  const size_t col_bytes = (size_t)32 * rpl * sizeof(cplx<R>);
  if (std::is_same<R, float>::value && rpl > 0 && rpl <= 16) {
    // whole matrix in one cluster of at most 16 CTAs with 8 warps each (w = 8), i.e. up to 256
    // columns; wider blocks (16 warps) were measured slower than the point-to-point kernel on
    // more SMs, because a step's latency grows with the warps that share an SM
    const int nw = 8;
    const Variant* v = find_cluster_variant(nw, rpl);
    if (v) {
      const int w = v->nw;
      const int P = (c + 2 * w - 1) / (2 * w);
      const size_t smem = (size_t)2 * w * col_bytes + 2 * w * sizeof(int) + 16;
      if (P >= 2 && P <= 16 && smem <= 200 * 1024) {
        plan.w = w;
        plan.nb = 2 * P;
        plan.smem = smem;
        plan.fn = v->fn;
        plan.threads = v->nw * 32;
        plan.cluster = P;
        plan.ld = 32 * rpl;
        return plan;
      }
    }
  }
  if (std::is_same<R, float>::value && rpl > 0) {
    const int target = std::max(1, std::min(sm_count, max_ctas));
    // single CTA: the widest variant whose columns fit
    const int single_max = 64;
    const Variant* v = nullptr;
    int w = 0;
    if (c <= single_max) {
      const int cand_nw[] = {16, 8, 4};
      for (int ap : {2, 1}) {
        for (int nw : cand_nw) {
          const Variant* cv = find_variant(nw, rpl, ap);
          if (!cv) continue;
          const int cw = nw * ap;
          if (2 * cw >= c && (size_t)2 * cw * col_bytes + 2 * cw * 4 + 16 <= budget) {
            if (!v || cw < w) { v = cv; w = cw; }   // the narrowest single-CTA variant that holds all columns
          }
        }
      }
    }
    int nb = 2;
    if (!v) {
      const int nw = 8, ap = 1;
      v = find_variant(nw, rpl, ap);
      if (!v) v = find_variant(8, rpl, 1);
      w = v->nw * v->ap;
      int P = (c + 2 * w - 1) / (2 * w);
      while (P > target && v) {   // too many CTAs: widen the blocks
        const Variant* wider = find_variant(v->nw * 2, rpl, v->ap);
        if (!wider) wider = find_variant(v->nw, rpl, v->ap * 2);
        if (!wider) break;
        v = wider;
        w = v->nw * v->ap;
        P = (c + 2 * w - 1) / (2 * w);
      }
      nb = 2 * P;
      // the same blocks on twice the warps: the rows of each column pair split over two warps
      if (!no_split && v->nw == 8 && v->ap == 1 && v->sp == 1)
        if (const Variant* sv = find_variant(16, rpl, 1, 2)) v = sv;
    }
    const size_t smem = (size_t)2 * w * col_bytes + 2 * w * sizeof(int) + 16;
    if (v && smem <= 227 * 1024) {
      plan.w = w;
      plan.nb = nb;
      plan.smem = smem;
      plan.fn = v->fn;
      plan.threads = v->nw * 32;
      plan.ld = 32 * rpl;
      return plan;
    }
  }
  // shared-memory kernel
  const size_t col_bytes_v1 = (size_t)L * sizeof(cplx<R>);
  int w_fit = (int)std::max<size_t>(1, budget / (2 * col_bytes_v1 + 8));
  int half = (c + 1) / 2;
  if (half <= w_fit && c <= 128) {
    plan.w = std::max(1, half);
    plan.nb = 2;
  } else {
    int target = std::max(1, std::min(sm_count, max_ctas));
    int w = (c + 2 * target - 1) / (2 * target);
    w = std::max(1, std::min(w, w_fit));
    int P = (c + 2 * w - 1) / (2 * w);
    if (P > target) {
      w = w_fit;
      P = (c + 2 * w - 1) / (2 * w);
    }
    plan.w = w;
    plan.nb = 2 * P;
  }
  plan.smem = (size_t)2 * plan.w * L * sizeof(cplx<R>) + 2 * plan.w * sizeof(int) + 16;
  plan.ld = L;
  plan.fn = (const void*)jacobi_kernel<R>;
  plan.threads = 256;
  return plan;
}

template <class R>
cudaError_t jacobi_launch(const JacobiPlan& plan, cplx<R>* X, long long ldx, int l, int c,
                          cplx<R>* W, long long ldw, int max_sweeps, DevCtrl* ctrl, cplx<R>* xch,
                          size_t xch_cap, unsigned* flags, int flags_cap, cudaStream_t st) {
  if (c <= 1) return cudaSuccess;   // a single column is already orthogonal
  if (plan.gram_R > 0) {
    if constexpr (std::is_same<R, float>::value)
      return jacobi_gram_launch(plan, X, ldx, l, c, W, ldw, max_sweeps, ctrl, xch, xch_cap, flags, flags_cap, st);
    return cudaErrorInvalidValue;
  }
  if ((size_t)2 * plan.nb * plan.w * (size_t)plan.ld > xch_cap || plan.nb > flags_cap) return cudaErrorInvalidValue;
  cudaError_t e = allow_dynamic_smem(plan.fn);
  if (e != cudaSuccess) return e;
  // reset barrier and sweep counters (bar_count, bar_gen, rot[3] are contiguous) and the position flags
  e = cudaMemsetAsync(&ctrl->bar_count, 0, 5 * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(flags, 0, sizeof(unsigned) * plan.nb, st);
  if (e != cudaSuccess) return e;
  JArgs<R> a;
  a.X = X; a.ldx = ldx; a.l = l; a.c = c; a.W = W; a.ldw = ldw;
  a.w = plan.w; a.nb = plan.nb; a.max_sweeps = max_sweeps;
  a.tol = R(4) * std::sqrt(R(std::max(l, 1))) * Eps<R>::v;
  // quadratic convergence: after a sweep whose pair cosines were all at most sqrt(tol), the next
  // sweep's are at the rounding level, so that sweep is not run
  a.tol_stop = plan.early_stop ? std::sqrt(a.tol) : a.tol;
  a.ctrl = ctrl;
  a.xch = xch;
  a.flags = flags;
  void* args[] = {&a};
  const int P = plan.nb / 2;
  if (plan.cluster > 0) {
    if (plan.cluster > 8) {
      e = cudaFuncSetAttribute(plan.fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(P);
    cfg.blockDim = dim3(plan.threads);
    cfg.dynamicSmemBytes = plan.smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = P;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, plan.fn, args);
  }
  if (P == 1) return cudaLaunchKernel(plan.fn, dim3(1), dim3(plan.threads), args, plan.smem, st);
  return cudaLaunchCooperativeKernel(plan.fn, dim3(P), dim3(plan.threads), args, plan.smem, st);
}

template JacobiPlan jacobi_plan<float>(int, int, bool, int, int, int);
template JacobiPlan jacobi_plan<double>(int, int, bool, int, int, int);
template cudaError_t jacobi_launch<float>(const JacobiPlan&, cplx<float>*, long long, int, int, cplx<float>*,
                                          long long, int, DevCtrl*, cplx<float>*, size_t, unsigned*, int,
                                          cudaStream_t);
template cudaError_t jacobi_launch<double>(const JacobiPlan&, cplx<double>*, long long, int, int, cplx<double>*,
                                           long long, int, DevCtrl*, cplx<double>*, size_t, unsigned*, int,
                                           cudaStream_t);
template int jacobi_max_ctas<float>(const JacobiPlan&);
template int jacobi_max_ctas<double>(const JacobiPlan&);

}  // namespace eamps
