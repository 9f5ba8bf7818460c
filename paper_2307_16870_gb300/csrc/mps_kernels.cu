// Small kernels of the two-site update: gate upload, theta with the gate,
// FP64 bond selection (sort + prefix sums + the entanglement-aware rule +
// fidelity bookkeeping), column extraction into site tensors, and the
// observables.
#include <cmath>

#include "kernels.h"

namespace eamps {

namespace {

struct GateParam { double v[512]; };   // up to 16 x 16 complex, passed by value with the launch

template <class R>
__global__ void gate_from_param(GateParam g, int d2, cplx<R>* dst) {
  for (int i = threadIdx.x; i < d2 * d2; i += blockDim.x) dst[i] = mk<R>((R)g.v[2 * i], (R)g.v[2 * i + 1]);
}

template <class R>
__global__ void gate_from_device(const double* __restrict__ src, int d2, cplx<R>* dst) {
  for (int i = threadIdx.x; i < d2 * d2; i += blockDim.x) dst[i] = mk<R>((R)src[2 * i], (R)src[2 * i + 1]);
}

// One thread per (a, b): all d*d physical entries of theta at that (a, b).
template <class R, int D>
__global__ void gate_theta_kernel(const cplx<R>* __restrict__ T, int chiL, int chiR, const cplx<R>* __restrict__ G,
                                  cplx<R>* __restrict__ X, int xmode, cplx<R>* __restrict__ theta) {
  __shared__ cplx<R> Gs[D * D * D * D];
  for (int i = threadIdx.x; i < D * D * D * D; i += blockDim.x) Gs[i] = G[i];
  __syncthreads();
  const long long total = (long long)chiL * chiR;
  const long long m = (long long)D * chiL, n = (long long)D * chiR;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int a = (int)(e / chiR), b = (int)(e % chiR);
    cplx<R> in[D * D];
#pragma unroll
    for (int t = 0; t < D * D; ++t) in[t] = T[((long long)a * D * D + t) * chiR + b];
#pragma unroll
    for (int s1 = 0; s1 < D; ++s1)
#pragma unroll
      for (int s2 = 0; s2 < D; ++s2) {
        cplx<R> acc = mk<R>(0, 0);
#pragma unroll
        for (int t = 0; t < D * D; ++t) cfma(acc, Gs[(s1 * D + s2) * D * D + t], in[t]);
        const long long row = (long long)a * D + s1, col = (long long)s2 * chiR + b;
        if (theta) theta[row * n + col] = acc;
        if (xmode == 0) X[col * m + row] = acc;
        else X[row * n + col] = cconj(acc);
      }
  }
}

template <class R>
__device__ __forceinline__ bool before_key(double ka, int ia, double kb, int ib) {
  return ka > kb || (ka == kb && ia < ib);
}

// Single CTA of 1024 threads.  Shared: key[n2], idx[n2], cum[n2] (n2 = power of two >= c).
template <class R>
__global__ void __launch_bounds__(1024) select_kernel(int c, int n2, DevCtrl* ctrl, double target,
                                                      double* __restrict__ s_sorted, int* __restrict__ perm) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* key = reinterpret_cast<double*>(smem_raw);
  double* cum = key + n2;
  int* idx = reinterpret_cast<int*>(cum + n2);
  __shared__ double part[1024];
  __shared__ int kcount;
  __shared__ double thr_s;
  const int tid = threadIdx.x;
  // 1. squared column norms (FP64, computed across the GPU into s_sorted by colnorm_kernel)
  for (int j = tid; j < n2; j += blockDim.x) {
    key[j] = (j < c) ? s_sorted[j] : -1.0;
    idx[j] = j;
  }
  __syncthreads();
  // 2. bitonic sort, decreasing key, ties by increasing index
  for (int k = 2; k <= n2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < n2; i += blockDim.x) {
        int ixj = i ^ j;
        if (ixj > i) {
          bool desc = ((i & k) == 0);
          double ki = key[i], kx = key[ixj];
          int ii = idx[i], ix = idx[ixj];
          bool sw = desc ? before_key<R>(kx, ix, ki, ii) : before_key<R>(ki, ii, kx, ix);
          if (sw) { key[i] = kx; key[ixj] = ki; idx[i] = ix; idx[ixj] = ii; }
        }
      }
      __syncthreads();
    }
  }
  // 3. inclusive prefix sums of the sorted weights (FP64)
  const int chunk = (n2 + 1023) / 1024;
  double run = 0.0;
  const int lo = tid * chunk;
  for (int j = lo; j < lo + chunk && j < n2; ++j) { run += (j < c) ? key[j] : 0.0; cum[j] = run; }
  part[tid] = run;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    double v = (tid >= off) ? part[tid - off] : 0.0;
    __syncthreads();
    part[tid] += v;
    __syncthreads();
  }
  const double base = (tid > 0) ? part[tid - 1] : 0.0;
  for (int j = lo; j < lo + chunk && j < n2; ++j) cum[j] += base;
  __syncthreads();
  // 4. target and threshold (thread 0)
  if (tid == 0) {
    const double W = cum[c - 1];
    double ft;
    if (target >= 0.0) ft = target >= 1.0 ? 1.0 : target;
    else if (ctrl->f_min >= 1.0) ft = 1.0;
    else if (ctrl->product < ctrl->f_min) ft = 1.0;
    else {
      long long rem = ctrl->n_2q - ctrl->n_done;
      if (rem < 1) rem = 1;
      if (ctrl->strategy == 0) ft = ctrl->f0;
      else if (ctrl->strategy == 1) ft = pow(ctrl->f_min / ctrl->product, 1.0 / (double)rem);
      else ft = ctrl->f_min / (ctrl->product * pow(ctrl->f0, (double)(rem - 1)));
      if (ft > 1.0) ft = 1.0;
    }
    ctrl->f_t = ft;
    ctrl->W = W;
    thr_s = (ctrl->mixed_fid == 1 ? ft * ft : ft) * W;
    kcount = 0;
  }
  __syncthreads();
  const double thr = thr_s;
  int mine = 0;
  for (int j = lo; j < lo + chunk && j < c; ++j) mine += (cum[j] < thr) ? 1 : 0;
  if (mine) atomicAdd(&kcount, mine);
  __syncthreads();
  if (tid == 0) {
    const double W = ctrl->W;
    const double ft = ctrl->f_t;
    int k;
    if (ctrl->fixed_chi > 0) k = min(ctrl->fixed_chi, c);
    else if (ft >= 1.0) k = c;
    else k = min(max(kcount + 1, 1), c);
    int cap = 0;
    if (ctrl->chi_max > 0 && k > ctrl->chi_max) { k = ctrl->chi_max; cap = 1; }
    double wk = cum[k - 1];
    double f = (W > 0.0) ? wk / W : 1.0;
    if (ctrl->mixed_fid == 1) f = sqrt(f);
    if (!isfinite(W) || !isfinite(wk) || !(wk > 0.0)) {
      atomicOr(&ctrl->status, ST_NONFINITE);
      f = 0.0;
      wk = 1.0;
    }
    ctrl->k = k;
    ctrl->rank_bound = c;
    ctrl->cap_hit = cap;
    if (cap) atomicOr(&ctrl->status, ST_CHI_CAP);
    ctrl->Wk = wk;
    ctrl->f = f;
    ctrl->product *= f;
    ctrl->n_done += 1;
    if (ctrl->kind == 1) ctrl->lognorm += 0.5 * log(wk);
  }
  for (int j = tid; j < c; j += blockDim.x) { s_sorted[j] = sqrt(key[j]); perm[j] = idx[j]; }
}

template <class R>
__global__ void colnorm_kernel(const cplx<R>* __restrict__ Y, long long ldy, int l, int c, double* __restrict__ out,
                               int squared) {
  const int lane = threadIdx.x & 31;
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j >= c) return;
  const cplx<R>* col = Y + (long long)j * ldy;
  double s = 0.0;
  for (int i = lane; i < l; i += 32) { cplx<R> v = col[i]; s += (double)v.x * v.x + (double)v.y * v.y; }
  s = warp_sum(s);
  if (lane == 0) out[j] = squared ? s : sqrt(s);
}

template <class R>
__global__ void extract_kernel(cplx<R>* __restrict__ out, long long o_js, long long o_rs, int kout, int rows,
                               const cplx<R>* __restrict__ src, long long s_js, long long s_rs,
                               const int* __restrict__ perm, int conj, const double* __restrict__ svals,
                               int wk_scale, const DevCtrl* __restrict__ ctrl) {
  __shared__ cplx<R> tile[32][33];   // [j][r]
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int r0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
  const double gscale = wk_scale ? 1.0 / sqrt(ctrl->Wk) : 1.0;
  const bool load_j_fast = (s_js == 1 && s_rs != 1 && perm == nullptr);
  for (int a = ty; a < 32; a += 8) {
    const int jj = load_j_fast ? tx : a, rr = load_j_fast ? a : tx;
    const int j = j0 + jj, r = r0 + rr;
    if (j < kout && r < rows) {
      const long long col = perm ? perm[j] : j;
      cplx<R> v = src[col * s_js + (long long)r * s_rs];
      if (conj) v.y = -v.y;
      double sc = gscale;
      if (svals) { const double s = svals[j]; sc = (s > 0.0) ? sc / s : 0.0; }
      tile[jj][rr] = cscale(v, (R)sc);
    }
  }
  __syncthreads();
  const bool store_j_fast = (o_js == 1 && o_rs != 1);
  for (int a = ty; a < 32; a += 8) {
    const int jj = store_j_fast ? tx : a, rr = store_j_fast ? a : tx;
    const int j = j0 + jj, r = r0 + rr;
    if (j < kout && r < rows) out[(long long)j * o_js + (long long)r * o_rs] = tile[jj][rr];
  }
}

template <class R>
__global__ void identity_kernel(cplx<R>* W, long long ld, int c) {
  const long long total = (long long)c * c;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int col = (int)(e / c), row = (int)(e % c);
    W[col * ld + row] = mk<R>(row == col ? 1 : 0, 0);
  }
}

template <class R, int D>
__global__ void apply_local_kernel(cplx<R>* A, int chiL, int chiR, const cplx<R>* __restrict__ G) {
  const long long total = (long long)chiL * chiR;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int a = (int)(e / chiR), b = (int)(e % chiR);
    cplx<R> in[D];
#pragma unroll
    for (int t = 0; t < D; ++t) in[t] = A[((long long)a * D + t) * chiR + b];
#pragma unroll
    for (int s = 0; s < D; ++s) {
      cplx<R> acc = mk<R>(0, 0);
#pragma unroll
      for (int t = 0; t < D; ++t) cfma(acc, G[s * D + t], in[t]);
      A[((long long)a * D + s) * chiR + b] = acc;
    }
  }
}

template <class R>
__global__ void __launch_bounds__(1024) renorm_kernel(cplx<R>* A, long long count, DevCtrl* ctrl) {
  __shared__ double red[32];
  __shared__ double scale_s;
  double s = 0.0;
  for (long long i = threadIdx.x; i < count; i += blockDim.x) { cplx<R> v = A[i]; s += (double)v.x * v.x + (double)v.y * v.y; }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) {
      if (!(v > 0.0) || !isfinite(v)) { atomicOr(&ctrl->status, ST_NONFINITE); scale_s = 1.0; }
      else { scale_s = 1.0 / sqrt(v); ctrl->lognorm += 0.5 * log(v); }
    }
  }
  __syncthreads();
  const R sc = (R)scale_s;
  for (long long i = threadIdx.x; i < count; i += blockDim.x) A[i] = cscale(A[i], sc);
}

template <class R>
__global__ void local_expect_kernel(const cplx<R>* __restrict__ T, int chiL, int D, int chiR,
                                    const cplx<R>* __restrict__ O, double2* out) {
  __shared__ double red_r[32], red_i[32];
  double accr = 0.0, acci = 0.0;
  const long long total = (long long)chiL * chiR;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int a = (int)(e / chiR), b = (int)(e % chiR);
    for (int s = 0; s < D; ++s) {
      cplx<R> x = T[((long long)a * D + s) * chiR + b];
      double yr = 0.0, yi = 0.0;
      for (int t = 0; t < D; ++t) {
        cplx<R> o = O[s * D + t], v = T[((long long)a * D + t) * chiR + b];
        yr += (double)o.x * v.x - (double)o.y * v.y;
        yi += (double)o.x * v.y + (double)o.y * v.x;
      }
      accr += (double)x.x * yr + (double)x.y * yi;   // conj(x) * y
      acci += (double)x.x * yi - (double)x.y * yr;
    }
  }
  accr = warp_sum(accr); acci = warp_sum(acci);
  if ((threadIdx.x & 31) == 0) { red_r[threadIdx.x >> 5] = accr; red_i[threadIdx.x >> 5] = acci; }
  __syncthreads();
  if (threadIdx.x < 32) {
    double vr = (threadIdx.x < (blockDim.x >> 5)) ? red_r[threadIdx.x] : 0.0;
    double vi = (threadIdx.x < (blockDim.x >> 5)) ? red_i[threadIdx.x] : 0.0;
    vr = warp_sum(vr); vi = warp_sum(vi);
    if (threadIdx.x == 0) { atomicAdd(&out->x, vr); atomicAdd(&out->y, vi); }
  }
}

// Sequential transfer along the chain in one CTA; FP64 vectors.
template <class R>
__global__ void __launch_bounds__(1024) chain_kernel(int N, const cplx<R>* const* __restrict__ sites,
                                                     const int* __restrict__ bonds, int d,
                                                     const double2* __restrict__ w, int q2,
                                                     const double2* __restrict__ w2, double2* work, int max_chi,
                                                     double2* out) {
  double2* v = work;
  double2* vn = work + max_chi;
  double2* z = work + 2 * max_chi;
  if (threadIdx.x == 0) v[0] = make_double2(1.0, 0.0);
  __syncthreads();
  for (int i = 0; i < N; ++i) {
    const int cl = bonds[i], cr = bonds[i + 1];
    const cplx<R>* A = sites[i];
    if (i == q2) {
      const cplx<R>* B = sites[i + 1];
      const int cr2 = bonds[i + 2];
      // z[u, c] = sum_a sum_t v[a] w2[t, u] A[a, t, c]
      for (int e = threadIdx.x; e < d * cr; e += blockDim.x) {
        const int u = e / cr, cc = e % cr;
        double zr = 0.0, zi = 0.0;
        for (int a = 0; a < cl; ++a) {
          const double2 va = v[a];
          for (int t = 0; t < d; ++t) {
            const double2 ww = w2[t * d + u];
            const cplx<R> x = A[((long long)a * d + t) * cr + cc];
            const double pr = va.x * ww.x - va.y * ww.y, pi = va.x * ww.y + va.y * ww.x;
            zr += pr * x.x - pi * x.y;
            zi += pr * x.y + pi * x.x;
          }
        }
        z[e] = make_double2(zr, zi);
      }
      __syncthreads();
      for (int b = threadIdx.x; b < cr2; b += blockDim.x) {
        double ar = 0.0, ai = 0.0;
        for (int u = 0; u < d; ++u)
          for (int cc = 0; cc < cr; ++cc) {
            const double2 zz = z[u * cr + cc];
            const cplx<R> x = B[((long long)cc * d + u) * cr2 + b];
            ar += zz.x * x.x - zz.y * x.y;
            ai += zz.x * x.y + zz.y * x.x;
          }
        vn[b] = make_double2(ar, ai);
      }
      ++i;
    } else {
      for (int b = threadIdx.x; b < cr; b += blockDim.x) {
        double ar = 0.0, ai = 0.0;
        for (int a = 0; a < cl; ++a) {
          const double2 va = v[a];
          for (int t = 0; t < d; ++t) {
            const double2 ww = w[(long long)i * d + t];
            if (ww.x == 0.0 && ww.y == 0.0) continue;
            const double pr = va.x * ww.x - va.y * ww.y, pi = va.x * ww.y + va.y * ww.x;
            const cplx<R> x = A[((long long)a * d + t) * cr + b];
            ar += pr * x.x - pi * x.y;
            ai += pr * x.y + pi * x.x;
          }
        }
        vn[b] = make_double2(ar, ai);
      }
    }
    __syncthreads();
    double2* tmp = v; v = vn; vn = tmp;
  }
  if (threadIdx.x == 0) *out = v[0];
}

// Product state: site i = (1, d, 1) with entry t = 0 equal to 1.
template <class R>
__global__ void product_state_kernel(cplx<R>* const* sites, int N, int d) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < N * d; e += gridDim.x * blockDim.x)
    sites[e / d][e % d] = mk<R>((e % d) == 0 ? 1 : 0, 0);
}

template <class R>
__global__ void from_double_kernel(const double2* __restrict__ src, cplx<R>* __restrict__ dst, long long count) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x)
    dst[i] = mk<R>((R)src[i].x, (R)src[i].y);
}

template <class R>
__global__ void to_double_kernel(const cplx<R>* __restrict__ src, double2* __restrict__ dst, long long count) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x)
    dst[i] = make_double2((double)src[i].x, (double)src[i].y);
}

inline int grid_for(long long work, int threads) {
  long long g = (work + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > 4096) g = 4096;
  return (int)g;
}

}  // namespace

template <class R>
cudaError_t load_gate_param(const double* host_op, int d2, cplx<R>* dst, cudaStream_t st) {
  GateParam g;
  for (int i = 0; i < 2 * d2 * d2; ++i) g.v[i] = host_op[i];
  gate_from_param<R><<<1, 256, 0, st>>>(g, d2, dst);
  return cudaGetLastError();
}

template <class R>
cudaError_t load_gate_device(const double* dev_op, int d2, cplx<R>* dst, cudaStream_t st) {
  gate_from_device<R><<<1, 256, 0, st>>>(dev_op, d2, dst);
  return cudaGetLastError();
}

template <class R>
cudaError_t gate_theta(const cplx<R>* T, int chiL, int d, int chiR, const cplx<R>* G, cplx<R>* X, int xmode,
                       cplx<R>* theta, cudaStream_t st) {
  const int grid = grid_for((long long)chiL * chiR, 256);
  if (d == 2) gate_theta_kernel<R, 2><<<grid, 256, 0, st>>>(T, chiL, chiR, G, X, xmode, theta);
  else gate_theta_kernel<R, 4><<<grid, 256, 0, st>>>(T, chiL, chiR, G, X, xmode, theta);
  return cudaGetLastError();
}

template <class R>
cudaError_t select_bond(const cplx<R>* Y, long long ldy, int l, int c, DevCtrl* ctrl, double target,
                        double* s_sorted, int* perm, cudaStream_t st) {
  int n2 = 32;
  while (n2 < c) n2 <<= 1;
  if (n2 > 8192) return cudaErrorInvalidValue;
  size_t smem = (size_t)n2 * (2 * sizeof(double) + sizeof(int));
  cudaError_t e = allow_dynamic_smem((const void*)select_kernel<R>);
  if (e != cudaSuccess) return e;
  // squared norms in FP64, one warp per column across (c + 7) / 8 CTAs, into s_sorted; the
  // selection reads them into shared memory before it writes the sorted values there
  colnorm_kernel<R><<<(c + 7) / 8, 256, 0, st>>>(Y, ldy, l, c, s_sorted, 1);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  select_kernel<R><<<1, 1024, smem, st>>>(c, n2, ctrl, target, s_sorted, perm);
  return cudaGetLastError();
}

template <class R>
cudaError_t column_norms(const cplx<R>* Y, long long ldy, int l, int c, double* norms, cudaStream_t st) {
  colnorm_kernel<R><<<(c + 7) / 8, 256, 0, st>>>(Y, ldy, l, c, norms, 0);
  return cudaGetLastError();
}

template <class R>
cudaError_t extract_columns(cplx<R>* out, long long o_js, long long o_rs, int kout, int rows,
                            const cplx<R>* src, long long s_js, long long s_rs, const int* perm, int conj,
                            const double* svals, int wk_scale, const DevCtrl* ctrl, cudaStream_t st) {
  if (kout <= 0 || rows <= 0) return cudaSuccess;
  dim3 grid((rows + 31) / 32, (kout + 31) / 32);
  extract_kernel<R><<<grid, dim3(32, 8), 0, st>>>(out, o_js, o_rs, kout, rows, src, s_js, s_rs, perm, conj, svals,
                                                  wk_scale, ctrl);
  return cudaGetLastError();
}

template <class R>
cudaError_t set_identity(cplx<R>* W, long long ld, int c, cudaStream_t st) {
  identity_kernel<R><<<grid_for((long long)c * c, 256), 256, 0, st>>>(W, ld, c);
  return cudaGetLastError();
}

template <class R>
cudaError_t apply_local(cplx<R>* A, int chiL, int d, int chiR, const cplx<R>* G, cudaStream_t st) {
  const int grid = grid_for((long long)chiL * chiR, 256);
  if (d == 2) apply_local_kernel<R, 2><<<grid, 256, 0, st>>>(A, chiL, chiR, G);
  else apply_local_kernel<R, 4><<<grid, 256, 0, st>>>(A, chiL, chiR, G);
  return cudaGetLastError();
}

template <class R>
cudaError_t renormalise_site(cplx<R>* A, long long count, DevCtrl* ctrl, cudaStream_t st) {
  renorm_kernel<R><<<1, 1024, 0, st>>>(A, count, ctrl);
  return cudaGetLastError();
}

template <class R>
cudaError_t local_expect(const cplx<R>* T, int chiL, int D, int chiR, const cplx<R>* O, double2* out,
                         cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double2), st);
  if (e != cudaSuccess) return e;
  local_expect_kernel<R><<<grid_for((long long)chiL * chiR, 256), 256, 0, st>>>(T, chiL, D, chiR, O, out);
  return cudaGetLastError();
}

template <class R>
cudaError_t chain_contract(int N, const cplx<R>* const* sites, const int* bonds, int d, const double2* w, int q2,
                           const double2* w2, double2* work, int max_chi, double2* out, cudaStream_t st) {
  chain_kernel<R><<<1, 1024, 0, st>>>(N, sites, bonds, d, w, q2, w2, work, max_chi, out);
  return cudaGetLastError();
}

template <class R>
__global__ void triu_extract_kernel(cplx<R>* __restrict__ dst, long long d_rs, long long d_cs,
                                    const cplx<R>* __restrict__ src, long long ld, int rows, int cols, int conj) {
  const long long total = (long long)rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e / rows), r = (int)(e % rows);
    cplx<R> v = mk<R>(0, 0);
    if (r <= j) {
      v = src[(long long)j * ld + r];
      if (conj) v.y = -v.y;
    }
    dst[(long long)r * d_rs + (long long)j * d_cs] = v;
  }
}

template <class R>
cudaError_t triu_extract(cplx<R>* dst, long long d_rs, long long d_cs, const cplx<R>* src, long long ld, int rows,
                         int cols, int conj, cudaStream_t st) {
  const long long total = (long long)rows * cols;
  if (total <= 0) return cudaSuccess;
  triu_extract_kernel<R><<<grid_for(total, 256), 256, 0, st>>>(dst, d_rs, d_cs, src, ld, rows, cols, conj);
  return cudaGetLastError();
}

template <class R>
__global__ void scale_lambda_kernel(cplx<R>* __restrict__ Y, long long ld, int rows, int cols,
                                    const double* __restrict__ lam, int d, int by_row) {
  const long long total = (long long)rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e / rows), r = (int)(e % rows);
    const R f = (R)lam[(by_row ? r : j) / d];
    cplx<R>& y = Y[(long long)j * ld + r];
    y.x *= f;
    y.y *= f;
  }
}

template <class R>
cudaError_t scale_by_lambda(cplx<R>* Y, long long ld, int rows, int cols, const double* lam, int d, int by_row,
                            cudaStream_t st) {
  const long long total = (long long)rows * cols;
  if (total <= 0) return cudaSuccess;
  scale_lambda_kernel<R><<<grid_for(total, 256), 256, 0, st>>>(Y, ld, rows, cols, lam, d, by_row);
  return cudaGetLastError();
}

__global__ void store_lambda_kernel(double* __restrict__ lam_out, const double* __restrict__ s_sorted,
                                    const DevCtrl* __restrict__ ctrl, int cap) {
  const int k = min(ctrl->k, cap);
  const double inv = 1.0 / sqrt(ctrl->Wk);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) lam_out[i] = s_sorted[i] * inv;
}

cudaError_t store_lambda(double* lam_out, const double* s_sorted, const DevCtrl* ctrl, int cap, cudaStream_t st) {
  store_lambda_kernel<<<grid_for(cap, 256), 256, 0, st>>>(lam_out, s_sorted, ctrl, cap);
  return cudaGetLastError();
}

template <class R>
cudaError_t product_state(cplx<R>* const* sites, int N, int d, cudaStream_t st) {
  product_state_kernel<R><<<grid_for((long long)N * d, 256), 256, 0, st>>>(sites, N, d);
  return cudaGetLastError();
}

template <class R>
cudaError_t from_double(const double2* src, cplx<R>* dst, long long count, cudaStream_t st) {
  from_double_kernel<R><<<grid_for(count, 256), 256, 0, st>>>(src, dst, count);
  return cudaGetLastError();
}

template <class R>
cudaError_t to_double(const cplx<R>* src, double2* dst, long long count, cudaStream_t st) {
  to_double_kernel<R><<<grid_for(count, 256), 256, 0, st>>>(src, dst, count);
  return cudaGetLastError();
}

#define EAMPS_INST(R)                                                                                           \
  template cudaError_t load_gate_param<R>(const double*, int, cplx<R>*, cudaStream_t);                         \
  template cudaError_t load_gate_device<R>(const double*, int, cplx<R>*, cudaStream_t);                        \
  template cudaError_t gate_theta<R>(const cplx<R>*, int, int, int, const cplx<R>*, cplx<R>*, int, cplx<R>*,    \
                                     cudaStream_t);                                                             \
  template cudaError_t select_bond<R>(const cplx<R>*, long long, int, int, DevCtrl*, double, double*, int*,     \
                                      cudaStream_t);                                                            \
  template cudaError_t column_norms<R>(const cplx<R>*, long long, int, int, double*, cudaStream_t);            \
  template cudaError_t extract_columns<R>(cplx<R>*, long long, long long, int, int, const cplx<R>*, long long,  \
                                          long long, const int*, int, const double*, int, const DevCtrl*,       \
                                          cudaStream_t);                                                        \
  template cudaError_t set_identity<R>(cplx<R>*, long long, int, cudaStream_t);                                \
  template cudaError_t apply_local<R>(cplx<R>*, int, int, int, const cplx<R>*, cudaStream_t);                  \
  template cudaError_t renormalise_site<R>(cplx<R>*, long long, DevCtrl*, cudaStream_t);                      \
  template cudaError_t local_expect<R>(const cplx<R>*, int, int, int, const cplx<R>*, double2*, cudaStream_t); \
  template cudaError_t chain_contract<R>(int, const cplx<R>* const*, const int*, int, const double2*, int,      \
                                         const double2*, double2*, int, double2*, cudaStream_t);               \
  template cudaError_t to_double<R>(const cplx<R>*, double2*, long long, cudaStream_t);                        \
  template cudaError_t scale_by_lambda<R>(cplx<R>*, long long, int, int, const double*, int, int, cudaStream_t); \
  template cudaError_t triu_extract<R>(cplx<R>*, long long, long long, const cplx<R>*, long long, int, int, int, \
                                      cudaStream_t);                                                          \
  template cudaError_t product_state<R>(cplx<R>* const*, int, int, cudaStream_t);                            \
  template cudaError_t from_double<R>(const double2*, cplx<R>*, long long, cudaStream_t);

EAMPS_INST(float)
EAMPS_INST(double)

}  // namespace eamps
