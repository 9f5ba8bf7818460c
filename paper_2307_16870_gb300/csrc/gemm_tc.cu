// Tensor-core complex GEMM (tcgen05): interface placeholder until the kernel lands.
#include "gemm_tc.h"

namespace eamps {

struct TcGemm { int unused; };

TcGemm* tc_create(size_t) { return nullptr; }
void tc_destroy(TcGemm*) {}
cudaError_t tc_gemm(TcGemm*, int, int, int, float, const float2*, long long, long long, int, const float2*, long long,
                    long long, int, float2*, long long, long long, cudaStream_t, int*) {
  return cudaErrorNotSupported;
}

}  // namespace eamps
