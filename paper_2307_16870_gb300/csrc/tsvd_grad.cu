// Kernels of the differentiable two-site update: ordering and selection of singular values for
// a stand-alone truncated SVD, and the pieces of its reverse-mode derivative.
//
// The paper differentiates nothing; the update it truncates (the two-site SVD of Eq. svd with
// the cut of the "Entanglement-aware" section) is differentiated here as follows.  With
// A = U S V^H (m x n, c = min(m, n), all c singular triplets, s descending), the update keeps
// k triplets and writes
//     A_q = U_k                         (m x k)
//     A_p = diag(sigma) V_k^H,  sigma_i = s_i / sqrt(W_k),  W_k = sum_{i<k} s_i^2   (k x n).
// Cotangents follow the convention gbar = dL/dRe + i dL/dIm of a real loss L, so that
// dL = Re sum conj(gbar) dX.  Given Abar_q, Abar_p:
//     sigmabar_i = Re (Abar_p V)_ii,   Vbar = Abar_p^H diag(sigma)  (columns >= k zero)
//     sbar_l     = sigmabar_l / sqrt(W_k) - s_l (sum_i sigmabar_i s_i) / W_k^(3/2)
//     Ubar       = Abar_q                                         (columns >= k zero)
// and, with Ju = U^H Ubar, Jv = V^H Vbar, F_ij = 1 / (s_j^2 - s_i^2) (i != j, broadened to
// (s_j^2 - s_i^2) / ((s_j^2 - s_i^2)^2 + eps)), F_ii = 0:
//     G = (F o (Ju - Ju^H)) S + S (F o (Jv - Jv^H)) + diag(sbar) + i diag((Im Ju_ii - Im Jv_ii) / (2 s_i))
//     Abar = U G V^H + (1 - U U^H) Ubar S^-1 V^H + U S^-1 Vbar^H (1 - V V^H).
// The first line is the first-order perturbation of the singular triplets (off-diagonal part
// from U^H dA V = dP S + dS - S dQ with dP, dQ anti-Hermitian; the diagonal imaginary part is
// the phase freedom of each pair u_i, v_i, which a phase-invariant loss sees only through the
// difference of the two phases).  Zero cotangents on the discarded columns make the same formula
// the exact derivative of the truncated outputs, couplings between kept and discarded values
// included.  Only one complement term is needed: the factor computed by the Jacobi rotations
// (V when m >= n, U when m < n) is square and unitary; the other is P / s with zero columns where
// s = 0, which the complement term covers.
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace eamps {
namespace {

inline int blocks_for(long long work, int threads) {
  long long b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 4096) b = 4096;
  return (int)b;
}

// descending order of s (NaN ordered last, ties by index): perm[rank] = i, s_sorted[rank] = s_i
__global__ void rank_sort_kernel(const double* __restrict__ s, int c, int* __restrict__ perm,
                                 double* __restrict__ s_sorted) {
  for (int i = threadIdx.x; i < c; i += blockDim.x) {
    const double si = isnan(s[i]) ? -1.0 : s[i];
    int rank = 0;
    for (int j = 0; j < c; ++j) {
      const double sj = isnan(s[j]) ? -1.0 : s[j];
      rank += (sj > si) || (sj == si && j < i);
    }
    perm[rank] = i;
    s_sorted[rank] = s[i];
  }
}

// k = smallest count with W_k >= target * W (all c when target >= 1), at most the number of
// values above rank_tol * s_0 and at most max_k (> 0), at least 1; sums in index order (FP64)
__global__ void select_values_kernel(const double* __restrict__ s, int c, double target, int max_k,
                                     double rank_tol, double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double W = 0.0;
  for (int i = 0; i < c; ++i) W += s[i] * s[i];
  int k = c;
  if (target < 1.0) {
    double cum = 0.0;
    for (int i = 0; i < c; ++i) {
      cum += s[i] * s[i];
      if (cum >= target * W) { k = i + 1; break; }
    }
  }
  int nz = 0;
  for (int i = 0; i < c; ++i) nz += s[i] > rank_tol * s[0];
  if (k > nz) k = nz;
  if (max_k > 0 && k > max_k) k = max_k;
  if (k < 1) k = 1;
  double Wk = 0.0;
  for (int i = 0; i < k; ++i) Wk += s[i] * s[i];
  out[0] = (double)k;
  out[1] = W > 0.0 ? Wk / W : 1.0;
  out[2] = W;
  out[3] = Wk;
}

// sbar (c) from Abar_p and V: one CTA, thread i handles kept value i
template <class R>
__global__ void __launch_bounds__(1024) tsvd_sbar_kernel(int n, int c, int k, const cplx<R>* __restrict__ V,
                                                         const double* __restrict__ s,
                                                         const cplx<R>* __restrict__ Ap_bar,
                                                         double* __restrict__ sbar, double* __restrict__ wk_out) {
  __shared__ double red[32];
  __shared__ double Wk_s;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    double w = 0.0;
    for (int i = 0; i < k; ++i) w += s[i] * s[i];
    Wk_s = w;
    wk_out[0] = w;
  }
  __syncthreads();
  const double Wk = Wk_s, rw = 1.0 / sqrt(Wk);
  double part = 0.0;
  for (int i = tid; i < c; i += blockDim.x) {
    double sig = 0.0;
    if (i < k && Ap_bar)
      for (int j = 0; j < n; ++j) {
        const cplx<R> a = Ap_bar[(long long)i * n + j], v = V[(long long)j * c + i];
        sig += (double)a.x * v.x - (double)a.y * v.y;   // Re(a v)
      }
    sbar[i] = sig;   // sigmabar for now
    part += sig * s[i];
  }
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if (lane == 0) red[warp] = part;
  __syncthreads();
  if (warp == 0) {
    double v = (lane < (int)(blockDim.x >> 5)) ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[0] = v;
  }
  __syncthreads();
  const double t = red[0];
  for (int i = tid; i < c; i += blockDim.x)
    sbar[i] = (i < k) ? sbar[i] * rw - s[i] * t * rw / Wk : 0.0;
}

// Ubar (m x c) = Abar_q padded with zero columns; Vbar (n x c): Vbar[j, i] = sigma_i conj(Abar_p[i, j])
template <class R>
__global__ void tsvd_pad_kernel(int m, int n, int c, int k, const double* __restrict__ s,
                                const double* __restrict__ wk, const cplx<R>* __restrict__ Aq_bar,
                                const cplx<R>* __restrict__ Ap_bar, cplx<R>* __restrict__ Ubar,
                                cplx<R>* __restrict__ Vbar) {
  const double rw = 1.0 / sqrt(wk[0]);
  const long long nu = (long long)m * c, total = nu + (long long)n * c;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    if (e < nu) {
      const int r = (int)(e / c), i = (int)(e % c);
      Ubar[e] = (i < k && Aq_bar) ? Aq_bar[(long long)r * k + i] : mk<R>(0, 0);
    } else {
      const long long f = e - nu;
      const int j = (int)(f / c), i = (int)(f % c);
      cplx<R> v = mk<R>(0, 0);
      if (i < k && Ap_bar) v = cscale(cconj(Ap_bar[(long long)i * n + j]), (R)(s[i] * rw));
      Vbar[f] = v;
    }
  }
}

// Y (rows x c, row-major): column i scaled by 1/s_i for i < k, zero otherwise (and where s_i = 0)
template <class R>
__global__ void tsvd_scale_kernel(cplx<R>* __restrict__ Y, int rows, int c, int k, const double* __restrict__ s) {
  const long long total = (long long)rows * c;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % c);
    const double inv = (i < k && s[i] > 0.0) ? 1.0 / s[i] : 0.0;
    Y[e] = cscale(Y[e], (R)inv);
  }
}

// G (c x c, row-major) from Ju, Jv, s, sbar and the complement correction Zc (Zu, or Zv^H when
// zc_adjoint), all row-major c x c
template <class R>
__global__ void tsvd_core_kernel(int c, const cplx<R>* __restrict__ Ju, const cplx<R>* __restrict__ Jv,
                                 const double* __restrict__ s, const double* __restrict__ sbar, double eps,
                                 const cplx<R>* __restrict__ Zc, int zc_adjoint, cplx<R>* __restrict__ G) {
  const long long total = (long long)c * c;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / c), j = (int)(e % c);
    const long long t = (long long)j * c + i;   // transposed position
    double gr, gi;
    if (i == j) {
      gr = sbar[i];
      gi = s[i] > 0.0 ? ((double)Ju[e].y - (double)Jv[e].y) / (2.0 * s[i]) : 0.0;
    } else {
      const double si = s[i], sj = s[j];
      const double dd = sj * sj - si * si;
      const double den = dd * dd + eps;
      const double F = den > 0.0 ? dd / den : 0.0;
      // (Ju - Ju^H)_ij and (Jv - Jv^H)_ij
      const double aur = (double)Ju[e].x - (double)Ju[t].x, aui = (double)Ju[e].y + (double)Ju[t].y;
      const double avr = (double)Jv[e].x - (double)Jv[t].x, avi = (double)Jv[e].y + (double)Jv[t].y;
      gr = F * (aur * sj + si * avr);
      gi = F * (aui * sj + si * avi);
    }
    if (Zc) {
      if (zc_adjoint) { gr -= (double)Zc[t].x; gi += (double)Zc[t].y; }
      else { gr -= (double)Zc[e].x; gi -= (double)Zc[e].y; }
    }
    G[e] = mk<R>((R)gr, (R)gi);
  }
}

// dst[r * ldd + j] += op(src[r * s_rs + j * s_cs]), op = conj when conj
template <class R>
__global__ void cadd_kernel(cplx<R>* __restrict__ dst, long long ldd, int rows, int cols,
                            const cplx<R>* __restrict__ src, long long s_rs, long long s_cs, int conj) {
  const long long total = (long long)rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e / cols), j = (int)(e % cols);
    cplx<R> v = src[(long long)r * s_rs + (long long)j * s_cs];
    if (conj) v.y = -v.y;
    cplx<R>& d = dst[(long long)r * ldd + j];
    d = cadd(d, v);
  }
}

}  // namespace

cudaError_t rank_sort(const double* s, int c, int* perm, double* s_sorted, cudaStream_t st) {
  rank_sort_kernel<<<1, 1024, 0, st>>>(s, c, perm, s_sorted);
  return cudaGetLastError();
}

cudaError_t select_values(const double* s_sorted, int c, double target, int max_k, double rank_tol, double* out,
                          cudaStream_t st) {
  select_values_kernel<<<1, 32, 0, st>>>(s_sorted, c, target, max_k, rank_tol, out);
  return cudaGetLastError();
}

template <class R>
cudaError_t tsvd_cotangents(int m, int n, int c, int k, const cplx<R>* V, const double* s, const cplx<R>* Aq_bar,
                            const cplx<R>* Ap_bar, cplx<R>* Ubar, cplx<R>* Vbar, double* sbar, double* wk,
                            cudaStream_t st) {
  tsvd_sbar_kernel<R><<<1, 1024, 0, st>>>(n, c, k, V, s, Ap_bar, sbar, wk);
  tsvd_pad_kernel<R><<<blocks_for((long long)(m + n) * c, 256), 256, 0, st>>>(m, n, c, k, s, wk, Aq_bar, Ap_bar,
                                                                              Ubar, Vbar);
  return cudaGetLastError();
}

template <class R>
cudaError_t tsvd_scale(cplx<R>* Y, int rows, int c, int k, const double* s, cudaStream_t st) {
  tsvd_scale_kernel<R><<<blocks_for((long long)rows * c, 256), 256, 0, st>>>(Y, rows, c, k, s);
  return cudaGetLastError();
}

template <class R>
cudaError_t tsvd_core(int c, const cplx<R>* Ju, const cplx<R>* Jv, const double* s, const double* sbar, double eps,
                      const cplx<R>* Zc, int zc_adjoint, cplx<R>* G, cudaStream_t st) {
  tsvd_core_kernel<R><<<blocks_for((long long)c * c, 256), 256, 0, st>>>(c, Ju, Jv, s, sbar, eps, Zc, zc_adjoint, G);
  return cudaGetLastError();
}

template <class R>
cudaError_t cadd_strided(cplx<R>* dst, long long ldd, int rows, int cols, const cplx<R>* src, long long s_rs,
                         long long s_cs, int conj, cudaStream_t st) {
  cadd_kernel<R><<<blocks_for((long long)rows * cols, 256), 256, 0, st>>>(dst, ldd, rows, cols, src, s_rs, s_cs, conj);
  return cudaGetLastError();
}

#define EAMPS_TSVD_INST(R)                                                                                        \
  template cudaError_t tsvd_cotangents<R>(int, int, int, int, const cplx<R>*, const double*, const cplx<R>*,     \
                                          const cplx<R>*, cplx<R>*, cplx<R>*, double*, double*, cudaStream_t);    \
  template cudaError_t tsvd_scale<R>(cplx<R>*, int, int, int, const double*, cudaStream_t);                      \
  template cudaError_t tsvd_core<R>(int, const cplx<R>*, const cplx<R>*, const double*, const double*, double,   \
                                    const cplx<R>*, int, cplx<R>*, cudaStream_t);                                 \
  template cudaError_t cadd_strided<R>(cplx<R>*, long long, int, int, const cplx<R>*, long long, long long, int,  \
                                       cudaStream_t);

EAMPS_TSVD_INST(float)
EAMPS_TSVD_INST(double)

}  // namespace eamps
