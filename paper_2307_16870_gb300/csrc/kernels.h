// Launchers of the EA-MPS device kernels (host-callable, templated on the real type).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace eamps {

// ------------------------------------------------------------ Jacobi SVD
// One-sided Jacobi on the c columns (length l, column j at X + j*ldx) of X:
// on return X V = Y (mutually orthogonal columns, |Y_j| = singular value j,
// unordered).  If W != nullptr the rotations are also applied to the c x c
// matrix W (column j at W + j*ldw), which must hold the identity on entry, so
// that W = V.  Cooperative launch; status bits and sweep count go to ctrl.
// Allow `fn` the largest dynamic shared memory the device offers (opt-in maximum minus the
// kernel's static shared memory).  Always the same value for a given kernel, so concurrent
// host threads that launch it with different dynamic sizes cannot undo each other's setting.
inline cudaError_t allow_dynamic_smem(const void* fn) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, fn);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

// dst(r, j) = op(src[j * ld + r]) for r <= j, 0 below the diagonal (r < rows, j < cols), with
// dst(r, j) at dst + r * d_rs + j * d_cs and op = conjugation when conj: the triangular factor of
// a column-major QR result, written in any layout (e.g. its adjoint with d_rs = 1-style strides).
template <class R>
cudaError_t triu_extract(cplx<R>* dst, long long d_rs, long long d_cs, const cplx<R>* src, long long ld, int rows,
                         int cols, int conj, cudaStream_t st);

// Vidal / Hastings form: element (r, j) of the column-major Y (leading dimension ld) times
// lam[r / d] (by_row) or lam[j / d] (columns), lam FP64.
template <class R>
cudaError_t scale_by_lambda(cplx<R>* Y, long long ld, int rows, int cols, const double* lam, int d, int by_row,
                            cudaStream_t st);
// lam_out[i] = s_sorted[i] / sqrt(ctrl->Wk) for i < ctrl->k (the renormalised kept values).
cudaError_t store_lambda(double* lam_out, const double* s_sorted, const DevCtrl* ctrl, int cap, cudaStream_t st);

// Householder QR of the l x c complex64 matrix X (column-major, leading dimension ldx), in place:
// R in the upper trapezoid, the reflector vectors (unit leading entry implicit) below the
// diagonal, tau (min(l, c) entries) and the block-reflector factors Tm (32 x 32 per panel of
// 32 columns).  Rows l <= qr_max_rows().  One launch is one thread-block cluster of ctas CTAs
// (qr_ctas(); at most qr_max_ctas()), so it waits on no other work of the device.
int qr_max_rows();
int qr_max_ctas();
int qr_ctas(int l, int c, int max_ctas);
cudaError_t qr_factor(float2* X, long long ldx, int l, int c, float2* tau, float2* Tm, DevCtrl* ctrl, int ctas,
                      cudaStream_t st);
// Q (l x min(l, c), column-major, leading dimension ldq) from the reflectors left by qr_factor.
cudaError_t qr_form_q(const float2* X, long long ldx, int l, int c, const float2* Tm, float2* Q, long long ldq,
                      DevCtrl* ctrl, int ctas, cudaStream_t st);

struct JacobiPlan {
  int w = 1;               // columns per block
  int nb = 2;              // number of blocks (even); CTAs = nb / 2
  size_t smem = 0;         // dynamic shared memory per CTA
  const void* fn = nullptr;  // kernel variant
  int threads = 256;
  int cluster = 0;           // > 0: cluster-resident kernel, one cluster of this many CTAs
  int ld = 0;                // column stride (complex entries) in shared memory and the exchange slots
  int gram_R = 0;            // > 0: block Jacobi with Gram-matrix inner sweeps (jacobi_gram.cu), one
                             // cluster of gram_R CTAs per slot of two 16-column blocks, nb / 2 slots
  int gram_mr = 0;           // rows of the stacked [X; W] held by each CTA of that kernel
  bool early_stop = true;    // end after the first sweep whose pair cosines are all <= sqrt(tol);
                             // false: only after a sweep with no rotation above tol
};
// kind: kJacobiAuto (the fixed rule, used where the engine has no measured choice for the shape:
// the Gram-matrix block kernel from kGramMinCols columns on, else the tournament kernels), kJacobiTournament (the cluster / point-to-point kernels only), kJacobiGram
// (the Gram-matrix block kernel whenever a layout fits, from 64 columns on).  Measured on GB300
// (complex64, square theta): the two layouts take the same time at 512 columns (7.7 ms, 13 sweeps)
// and the Gram kernel wins at 1024 (21.2 ms against 24.9 ms); below 512 the tournament kernels win.
// kJacobiTournamentUnsplit: the tournament kernels with one warp per column pair throughout
// (kJacobiTournament splits the rows of each pair over two warps in the point-to-point kernel at
// 256 and 512 rows).
// kJacobiNoSplit (a flag added to any kind): no row split either (a handle that runs beside others:
// the split variant's 512-thread CTAs hold a whole SM's registers and leave no room for the others').
enum { kJacobiAuto = 0, kJacobiTournament = 1, kJacobiGram = 2, kJacobiTournamentUnsplit = 3, kJacobiNoSplit = 8 };
constexpr int kGramMinCols = 1024;
template <class R>
JacobiPlan jacobi_plan(int l, int c, bool accumulate, int sm_count, int max_ctas, int kind = kJacobiAuto);
// xch: exchange slots of the multi-CTA kernels (2 * nb * w * plan.ld complex entries at
// most xch_cap); flags: nb position flags (at most flags_cap).
template <class R>
cudaError_t jacobi_launch(const JacobiPlan& plan, cplx<R>* X, long long ldx, int l, int c,
                          cplx<R>* W, long long ldw, int max_sweeps, DevCtrl* ctrl, cplx<R>* xch,
                          size_t xch_cap, unsigned* flags, int flags_cap, cudaStream_t st);
template <class R> int jacobi_max_ctas(const JacobiPlan& plan);
// CTAs of one launch of the plan (all co-resident: they wait on one another).
inline int jacobi_plan_ctas(const JacobiPlan& plan) {
  if (plan.gram_R > 0) return plan.nb / 2 * plan.gram_R;
  return plan.cluster > 0 ? plan.cluster : plan.nb / 2;
}
// Block one-sided Jacobi with Gram-matrix inner sweeps (complex64, c >= 64 columns): fills plan
// and returns true when a layout of at most max_ctas co-resident CTAs exists.
bool jacobi_gram_plan(int l, int c, bool accumulate, int max_ctas, JacobiPlan& plan);
cudaError_t jacobi_gram_launch(const JacobiPlan& plan, float2* X, long long ldx, int l, int c, float2* W,
                               long long ldw, int max_sweeps, DevCtrl* ctrl, float2* xch, size_t xch_cap,
                               unsigned* flags, int flags_cap, cudaStream_t st);

// ------------------------------------------------------------ CUDA-core GEMM
// C = alpha * op(A) * op(B); op(A)[i,k] = A[i*a_rs + k*a_cs] (conjugated if conjA).
template <class R>
cudaError_t cgemm_simt(int M, int N, int K, R alpha,
                       const cplx<R>* A, long long a_rs, long long a_cs, int conjA,
                       const cplx<R>* B, long long b_rs, long long b_cs, int conjB,
                       cplx<R>* C, long long c_rs, long long c_cs, cudaStream_t st);

// ------------------------------------------------------------ small kernels
// gate (d2 x d2, row-major complex doubles) -> device buffer in precision R
template <class R>
cudaError_t load_gate_param(const double* host_op, int d2, cplx<R>* dst, cudaStream_t st);
template <class R>
cudaError_t load_gate_device(const double* dev_op, int d2, cplx<R>* dst, cudaStream_t st);

// theta[(a s1),(s2 b)] = sum_{t1 t2} G[(s1 s2),(t1 t2)] T[a,t1,t2,b];  writes X (xmode 0: theta
// column-major, ld = m; xmode 1: conj(theta) row-major = theta^dagger column-major, ld = n) and
// optionally theta row-major.
template <class R>
cudaError_t gate_theta(const cplx<R>* T, int chiL, int d, int chiR, const cplx<R>* G,
                       cplx<R>* X, int xmode, cplx<R>* theta, cudaStream_t st);

// Sort the column norms of Y (FP64) in decreasing order, choose the bond (entanglement-aware rule,
// fixed chi or cap), update the FP64 product / schedule / log-norm in ctrl, and write the sorted
// singular values and the permutation.  c <= 8192.
template <class R>
cudaError_t select_bond(const cplx<R>* Y, long long ldy, int l, int c, DevCtrl* ctrl, double target,
                        double* s_sorted, int* perm, cudaStream_t st);

// FP64 norms of the c columns (length l) of Y.
template <class R>
cudaError_t column_norms(const cplx<R>* Y, long long ldy, int l, int c, double* norms, cudaStream_t st);

// out[j*o_js + r*o_rs] = scale_j * op(src[col(j)*s_js + r*s_rs]) for j < kout, r < rows, where
// col(j) = perm ? perm[j] : j, op = conj if conj, scale_j = (svals ? 1/svals[j] (0 if svals[j]==0) : 1)
// * (wk_scale ? 1/sqrt(ctrl->Wk) : 1).
template <class R>
cudaError_t extract_columns(cplx<R>* out, long long o_js, long long o_rs, int kout, int rows,
                            const cplx<R>* src, long long s_js, long long s_rs, const int* perm, int conj,
                            const double* svals, int wk_scale, const DevCtrl* ctrl, cudaStream_t st);

// Identity into a c x c column-major matrix (ld).
template <class R>
cudaError_t set_identity(cplx<R>* W, long long ld, int c, cudaStream_t st);

// A'[a,s,b] = sum_t G[s,t] A[a,t,b] in place, site (chiL, d, chiR).
template <class R>
cudaError_t apply_local(cplx<R>* A, int chiL, int d, int chiR, const cplx<R>* G, cudaStream_t st);

// Normalise a site to unit Frobenius norm (FP64), lognorm += log(norm).
template <class R>
cudaError_t renormalise_site(cplx<R>* A, long long count, DevCtrl* ctrl, cudaStream_t st);

// sum_{a,b,s,t} conj(T[a,s,b]) O[s,t] T[a,t,b] (FP64) into *out (double2, device); O is D x D.
template <class R>
cudaError_t local_expect(const cplx<R>* T, int chiL, int D, int chiR, const cplx<R>* O, double2* out,
                         cudaStream_t st);

// Transfer contraction along the chain: v <- v * sum_t w_i[t] A_i[:,t,:], with an optional
// two-site weight w2 (d x d, indices (t_q, t_q+1)) replacing the weights of sites q, q+1.
// sites: device array of N site pointers; bonds: device, N+1 entries.
template <class R>
cudaError_t chain_contract(int N, const cplx<R>* const* sites, const int* bonds, int d,
                           const double2* w, int q2, const double2* w2, double2* work, int max_chi,
                           double2* out, cudaStream_t st);

// Product state |0...0> (or vec(|0..0><0..0|)): site i = (1, d, 1), entry 0 = 1.
template <class R>
cudaError_t product_state(cplx<R>* const* sites, int N, int d, cudaStream_t st);

// Convert complex128 to the working precision.
template <class R>
cudaError_t from_double(const double2* src, cplx<R>* dst, long long count, cudaStream_t st);

// Convert a site to complex128.
template <class R>
cudaError_t to_double(const cplx<R>* src, double2* dst, long long count, cudaStream_t st);

// ------------------------------------------------ differentiable two-site update (tsvd_grad.cu)
// Descending order of c values: perm[rank] = i, s_sorted[rank] = s[i] (one CTA, c <= a few 1000).
cudaError_t rank_sort(const double* s, int c, int* perm, double* s_sorted, cudaStream_t st);
// Truncation of sorted values: out = {k, W_k/W, W, W_k} (device), k from target, rank_tol, max_k.
cudaError_t select_values(const double* s_sorted, int c, double target, int max_k, double rank_tol, double* out,
                          cudaStream_t st);
// Cotangents of the full factors from those of A_q = U_k and A_p = diag(s_k / sqrt(W_k)) V_k^H:
// Ubar (m x c), Vbar (n x c), sbar (c), W_k into wk[0]; row-major, zero beyond column k.
template <class R>
cudaError_t tsvd_cotangents(int m, int n, int c, int k, const cplx<R>* V, const double* s, const cplx<R>* Aq_bar,
                            const cplx<R>* Ap_bar, cplx<R>* Ubar, cplx<R>* Vbar, double* sbar, double* wk,
                            cudaStream_t st);
// Y (rows x c) column i scaled by 1/s_i for i < k (zero otherwise).
template <class R>
cudaError_t tsvd_scale(cplx<R>* Y, int rows, int c, int k, const double* s, cudaStream_t st);
// Core matrix G (c x c) of the SVD adjoint, minus Zc (or Zc^H when zc_adjoint).
template <class R>
cudaError_t tsvd_core(int c, const cplx<R>* Ju, const cplx<R>* Jv, const double* s, const double* sbar, double eps,
                      const cplx<R>* Zc, int zc_adjoint, cplx<R>* G, cudaStream_t st);
// Wait of one thread for *flag >= target, bounded by ctrl->wait_ns; ST_TIMEOUT in ctrl->status
// on expiry (selftest.cu).
cudaError_t wait_probe(const unsigned* flag, unsigned target, DevCtrl* ctrl, cudaStream_t st);
// dst (rows x cols, ld ldd) += op(src) with src(r, j) at src + r * s_rs + j * s_cs.
template <class R>
cudaError_t cadd_strided(cplx<R>* dst, long long ldd, int rows, int cols, const cplx<R>* src, long long s_rs,
                         long long s_cs, int conj, cudaStream_t st);

}  // namespace eamps
