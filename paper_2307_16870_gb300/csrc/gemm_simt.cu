// Strided complex GEMM on the CUDA cores: C = alpha * op(A) * op(B).
// Used for the FP64 (complex128) path and as the FP32 reference path of the
// contractions; the complex64 production path runs on the tensor cores.
#include "kernels.h"

namespace eamps {

namespace {

constexpr int BM = 64, BN = 64, BK = 16;

template <class R>
__global__ void __launch_bounds__(256) cgemm_kernel(int M, int N, int K, R alpha,
    const cplx<R>* __restrict__ A, long long a_rs, long long a_cs, int conjA,
    const cplx<R>* __restrict__ B, long long b_rs, long long b_cs, int conjB,
    cplx<R>* __restrict__ C, long long c_rs, long long c_cs) {
  __shared__ cplx<R> As[BK][BM + 1];
  __shared__ cplx<R> Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  cplx<R> acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = mk<R>(0, 0);
  const bool a_row_fast = (a_rs == 1);
  const bool b_col_fast = (b_cs == 1);
  for (int k0 = 0; k0 < K; k0 += BK) {
    for (int e = tid; e < BM * BK; e += 256) {
      int row, kk;
      if (a_row_fast) { row = e % BM; kk = e / BM; } else { kk = e % BK; row = e / BK; }
      int gi = m0 + row, gk = k0 + kk;
      cplx<R> v = mk<R>(0, 0);
      if (gi < M && gk < K) { v = A[gi * a_rs + gk * a_cs]; if (conjA) v.y = -v.y; }
      As[kk][row] = v;
    }
    for (int e = tid; e < BN * BK; e += 256) {
      int col, kk;
      if (b_col_fast) { col = e % BN; kk = e / BN; } else { kk = e % BK; col = e / BK; }
      int gj = n0 + col, gk = k0 + kk;
      cplx<R> v = mk<R>(0, 0);
      if (gj < N && gk < K) { v = B[gk * b_rs + gj * b_cs]; if (conjB) v.y = -v.y; }
      Bs[kk][col] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      cplx<R> a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) cfma(acc[i][j], a[i], b[j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int gi = m0 + ty + 16 * i, gj = n0 + tx + 16 * j;
      if (gi < M && gj < N) C[gi * c_rs + gj * c_cs] = cscale(acc[i][j], alpha);
    }
}

}  // namespace

template <class R>
cudaError_t cgemm_simt(int M, int N, int K, R alpha,
                       const cplx<R>* A, long long a_rs, long long a_cs, int conjA,
                       const cplx<R>* B, long long b_rs, long long b_cs, int conjB,
                       cplx<R>* C, long long c_rs, long long c_cs, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM);
  cgemm_kernel<R><<<grid, 256, 0, st>>>(M, N, K, alpha, A, a_rs, a_cs, conjA, B, b_rs, b_cs, conjB, C, c_rs, c_cs);
  return cudaGetLastError();
}

template cudaError_t cgemm_simt<float>(int, int, int, float, const cplx<float>*, long long, long long, int,
                                       const cplx<float>*, long long, long long, int, cplx<float>*, long long,
                                       long long, cudaStream_t);
template cudaError_t cgemm_simt<double>(int, int, int, double, const cplx<double>*, long long, long long, int,
                                        const cplx<double>*, long long, long long, int, cplx<double>*, long long,
                                        long long, cudaStream_t);

}  // namespace eamps
