// Complex64 GEMM on the 5th-generation tensor cores (tcgen05, kind::tf32) with
// the 3xTF32 split: each FP32 operand x = hi + lo (hi = x rounded to TF32),
// A B ~ Ahi Bhi + Ahi Blo + Alo Bhi, accumulated in FP32 in tensor memory.
#pragma once

#include <cuda_runtime.h>

namespace eamps {

struct TcGemm;

// Workspace for operands of up to max_elems complex entries each.  nullptr on failure.
TcGemm* tc_create(size_t max_elems);
void tc_destroy(TcGemm* g);

// C = alpha * op(A) * op(B) with the strided conventions of cgemm_simt (complex64).
// *launched receives the number of kernels launched; a device-side wait that
// timed out sets ST_TIMEOUT in *status (device int).
cudaError_t tc_gemm(TcGemm* g, int M, int N, int K, float alpha,
                    const float2* A, long long a_rs, long long a_cs, int conjA,
                    const float2* B, long long b_rs, long long b_cs, int conjB,
                    float2* C, long long c_rs, long long c_cs, cudaStream_t st, int* launched, int* status);

// The same product on caller-provided packing buffers (each large enough for
// M x pad32(2K) and 2N x pad32(2K) floats); allocates nothing.
cudaError_t tc_gemm_raw(float* ah, float* al, float* bh, float* bl, int M, int N, int K, float alpha,
                        const float2* A, long long a_rs, long long a_cs, int conjA, const float2* B, long long b_rs,
                        long long b_cs, int conjB, float2* C, long long c_rs, long long c_cs, cudaStream_t st,
                        int* launched, int* status);
// Failure self-test: the same kernel with CTA (0, 0)'s loads withheld, so that its tensor-core
// issuer's bounded wait (wait_ns) runs out: ST_TIMEOUT in *status, every role returns, the
// tensor memory is released.  Row-major A (M x K), B (K x N), C (M x N).
cudaError_t tc_gemm_selftest(TcGemm* g, int M, int N, int K, const float2* A, const float2* B, float2* C,
                             cudaStream_t st, int* status, unsigned long long wait_ns);
const void* tc_gemm_kernel_entry();
int tc_gemm_smem_bytes();

// Whether the workspace holds the packed operands of an M x K by K x N product.
bool tc_fits(const TcGemm* g, int M, int N, int K);

}  // namespace eamps
