// Complex64 GEMM on the tcgen05 tensor cores (sm_103a), 3xTF32 split.
//
// The complex product C = op(A) op(B) (M x K times K x N) is one real GEMM on
// interleaved operands: A' (M x 2K) holds (Re, Im) pairs of each row of
// op(A); B' (2N x 2K, K-major) holds for complex column j the two real rows
//   2j  : ( Re b, -Im b ) per k     -> real part of c_ij
//   2j+1: ( Im b,  Re b ) per k     -> imaginary part of c_ij
// so that D = A' B'^T (M x 2N) interleaves (Re, Im) of C.  Each FP32 operand
// is split x = hi + lo with hi = x rounded to TF32 and lo = x - hi (exact),
// and D = Ahi Bhi + Ahi Blo + Alo Bhi accumulates in FP32 in tensor memory:
// FP32-level accuracy from kind::tf32 MMAs.
//
// Kernel: one CTA per 128 x 128 tile of D, six warps.  Warp 0 (one lane)
// drives TMA loads of 32-wide K blocks (128-byte swizzled, K-major) into a
// three-stage shared-memory ring; warp 1 (one lane) issues 12 tcgen05.mma per
// block (3 products x 4 K-steps of 8) into one of two 128-column TMEM
// accumulators and releases the stage and the accumulator with
// tcgen05.commit; warps 2-5 (warp w owns TMEM lanes 32*(w%4)..+31) read each
// block's partial product with tcgen05.ld and add it into FP32 registers.
// The tensor core's own accumulation truncates (a bias of about -1e-8 K
// relative, measured); summing one K block at a time on the CUDA cores keeps
// the product at FP32 accuracy.  Every mbarrier wait is bounded; a timeout
// sets the status bit and the CTA drains its copies and MMAs and returns.
#include <cooperative_groups.h>
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstdio>

#include "common.cuh"
#include "gemm_tc.h"

namespace eamps {

namespace {

constexpr int BM = 128, BN = 128, BKR = 32;      // BKR: real K elements per block (128 bytes)
constexpr int STAGES = 3;
constexpr int TILE_BYTES = BM * BKR * 4;          // 16 KB, same for A and B tiles (BN == BM)
constexpr int STAGE_BYTES = 4 * TILE_BYTES;       // A_hi, A_lo, B_hi, B_lo
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024;
constexpr int kMaxSplit = 4;          // split-K factor limit
constexpr int kSplitTarget = 128;     // CTAs a split-K launch aims for (152 SMs)

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(su32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait on an mbarrier phase; on timeout sets ST_TIMEOUT and returns false.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* status, unsigned long long wait_ns) {
  const unsigned long long end = global_ns() + wait_ns;
  for (int i = 0;; ++i) {
    if (mbar_test(bar, parity)) return true;
    if (i > 64) __nanosleep(20);
    if (global_ns() > end) break;
  }
  atomicOr(status, ST_TIMEOUT);
  return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
      ::"r"(su32(dst)), "l"((uint64_t)map), "r"(su32(bar)), "r"(x), "r"(y)
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row
// groups 1024 bytes apart (the layout TMA writes with SWIZZLE_128B).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;              // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;    // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;              // descriptor version of this architecture
  d |= (uint64_t)2 << 61;              // 128-byte swizzle
  return d;
}

// Instruction descriptor of kind::tf32: D = F32, A = B = TF32, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(int m, int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n"
      ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(bar)) : "memory");
}

// Bounded wait that also gives up as soon as another role of the CTA aborted.
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t* bar, uint32_t parity, int* status,
                                                   volatile int* abort_flag, unsigned long long wait_ns) {
  const unsigned long long end = global_ns() + wait_ns;
  for (int i = 0;; ++i) {
    if (mbar_test(bar, parity)) return true;
    if ((i & 255) == 255 && *abort_flag) return false;
    if (i > 64) __nanosleep(20);
    if (global_ns() > end) break;
  }
  atomicOr(status, ST_TIMEOUT);
  *abort_flag = 1;
  return false;
}

constexpr int NTHREADS = 192;          // warp 0: TMA, warp 1: MMA, warps 2-5: accumulation + epilogue
constexpr uint32_t TMEM_COLS = 256;    // two 128-column FP32 accumulators (ping-pong)

__global__ void __launch_bounds__(NTHREADS, 1) tc_gemm_kernel(const __grid_constant__ CUtensorMap mAh,
                                                              const __grid_constant__ CUtensorMap mAl,
                                                              const __grid_constant__ CUtensorMap mBh,
                                                              const __grid_constant__ CUtensorMap mBl,
                                                              int M, int N, int nkb, int kb_per, float alpha,
                                                              float2* __restrict__ C, long long c_rs, long long c_cs,
                                                              int nsplit, int* status, int fault,
                                                              unsigned long long wait_ns) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[STAGES];
  __shared__ __align__(8) uint64_t empty_bar[STAGES];
  __shared__ __align__(8) uint64_t acc_full[2];
  __shared__ __align__(8) uint64_t acc_empty[2];
  __shared__ __align__(8) uint64_t done_bar;
  __shared__ uint32_t tmem_base_s;
  __shared__ int abort_s;
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * BM;
  const int n0 = blockIdx.x * BN;   // real columns of D
  // split K (nsplit > 1): the CTAs of a cluster along z take K blocks [kb0, kb0 + nloc) each and
  // sum their partial products through distributed shared memory in z order (deterministic)
  const int kb0 = blockIdx.z * kb_per;
  const int nloc = min(kb_per, nkb - kb0);
  volatile int* abortp = &abort_s;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) { mbar_init(&full_bar[s], 1); mbar_init(&empty_bar[s], 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(&acc_full[b], 1); mbar_init(&acc_empty[b], 4); }
    mbar_init(&done_bar, 1);
    abort_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base_s)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_s;
  constexpr uint32_t IDESC = idesc_tf32(BM, BN);

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer (failure self-test: CTA (0, 0) issues nothing, so that its
      // MMA issuer's wait on the first stage runs out)
      int issued = 0;
      const int nload = (fault && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0) ? 0 : nloc;
      for (int kb = 0; kb < nload; ++kb) {
        const int s = kb % STAGES;
        if (kb >= STAGES && !mbar_wait_or_abort(&empty_bar[s], ((kb / STAGES) - 1) & 1, status, abortp, wait_ns)) break;
        unsigned char* st = smem + s * STAGE_BYTES;
        mbar_expect_tx(&full_bar[s], STAGE_BYTES);
        const int kx = (kb0 + kb) * BKR;
        tma_load_2d(st + 0 * TILE_BYTES, &mAh, &full_bar[s], kx, m0);
        tma_load_2d(st + 1 * TILE_BYTES, &mAl, &full_bar[s], kx, m0);
        tma_load_2d(st + 2 * TILE_BYTES, &mBh, &full_bar[s], kx, n0);
        tma_load_2d(st + 3 * TILE_BYTES, &mBl, &full_bar[s], kx, n0);
        issued = kb + 1;
      }
      // every issued copy must land before the CTA may exit
      for (int kb = (issued > STAGES ? issued - STAGES : 0); kb < issued; ++kb)
        mbar_wait(&full_bar[kb % STAGES], (kb / STAGES) & 1, status, wait_ns);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer: one K block per accumulator, buffers alternate
      for (int kb = 0; kb < nloc; ++kb) {
        const int s = kb % STAGES, b = kb & 1;
        if (!mbar_wait_or_abort(&full_bar[s], (kb / STAGES) & 1, status, abortp, wait_ns)) break;
        if (kb >= 2 && !mbar_wait_or_abort(&acc_empty[b], ((kb >> 1) - 1) & 1, status, abortp, wait_ns)) break;
        tc_fence_after();
        const uint32_t base = su32(smem + s * STAGE_BYTES);
        const uint64_t dAh = sdesc(base), dAl = sdesc(base + TILE_BYTES);
        const uint64_t dBh = sdesc(base + 2 * TILE_BYTES), dBl = sdesc(base + 3 * TILE_BYTES);
        const uint32_t d = tmem + (uint32_t)(b * BN);
#pragma unroll
        for (int kk = 0; kk < BKR / 8; ++kk) {
          const uint64_t adv = (uint64_t)((kk * 32) >> 4);   // 8 TF32 = 32 bytes along K
          mma_tf32(d, dAl + adv, dBh + adv, IDESC, kk > 0 ? 1u : 0u);
          mma_tf32(d, dAh + adv, dBl + adv, IDESC, 1u);
          mma_tf32(d, dAh + adv, dBh + adv, IDESC, 1u);
        }
        mma_commit(&empty_bar[s]);
        mma_commit(&acc_full[b]);
      }
      mma_commit(&done_bar);   // arrives once every MMA issued above has completed
    }
  } else {
    // ---------------- accumulation (promotion) and epilogue: warp w reads TMEM lanes 32*(w%4)..
    // Each K block's partial product is added into FP32 registers with round-to-nearest adds,
    // so the tensor core accumulates over one block only.
    const int qd = warp & 3;
    float acc[BN];
#pragma unroll
    for (int i = 0; i < BN; ++i) acc[i] = 0.f;
    bool ok = true;
    for (int kb = 0; kb < nloc; ++kb) {
      const int b = kb & 1;
      if (!mbar_wait_or_abort(&acc_full[b], (kb >> 1) & 1, status, abortp, wait_ns)) { ok = false; break; }
      tc_fence_after();
#pragma unroll
      for (int ch = 0; ch < BN / 32; ++ch) {
        uint32_t v[32];
        tmem_ld32(tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)(b * BN + ch * 32), v);
#pragma unroll
        for (int i = 0; i < 32; ++i) acc[ch * 32 + i] += __uint_as_float(v[i]);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[b]);
    }
    if (nsplit > 1) {
      // the partial product to shared memory (the operand stages are free: every MMA and every
      // load of this CTA has completed), column-major by epilogue thread
      float* pbuf = reinterpret_cast<float*>(smem);
      const int te = threadIdx.x - 64;
#pragma unroll
      for (int c = 0; c < BN; ++c) pbuf[c * 128 + te] = acc[c];
    } else if (ok && !*abortp) {
      const int row = m0 + qd * 32 + lane;
      if (row < M) {
#pragma unroll
        for (int c = 0; c < BN / 2; ++c) {
          const int j = n0 / 2 + c;
          if (j < N) {
            float2 z;
            z.x = alpha * acc[2 * c];
            z.y = alpha * acc[2 * c + 1];
            C[(long long)row * c_rs + (long long)j * c_cs] = z;
          }
        }
      }
    }
  }
  __syncthreads();
  if (nsplit > 1) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    cl.sync();   // every partial product of the cluster is in shared memory
    if (warp >= 2) {
      // rank r sums columns [r, r + 1, ...) / nsplit of the tile over the cluster, in z order
      const int te = threadIdx.x - 64, qd = warp & 3;
      const int row = m0 + qd * 32 + lane;
      const int rank = (int)cl.block_rank();
      const float* src[kMaxSplit];
#pragma unroll
      for (int z = 0; z < kMaxSplit; ++z) src[z] = cl.map_shared_rank(reinterpret_cast<float*>(smem), z < nsplit ? z : 0);
      const int per = (BN / 2 + nsplit - 1) / nsplit;   // complex columns per rank (nsplit need not divide)
      if (row < M) {
#pragma unroll 4
        for (int c2 = 0; c2 < per; ++c2) {
          const int c = min(rank * per + c2, BN / 2 - 1);
          const int j = (rank * per + c2 < BN / 2) ? n0 / 2 + c : N;   // j = N: nothing to write
          float v[kMaxSplit][2];
#pragma unroll
          for (int z = 0; z < kMaxSplit; ++z) {
            v[z][0] = (z < nsplit) ? src[z][(2 * c) * 128 + te] : 0.f;
            v[z][1] = (z < nsplit) ? src[z][(2 * c + 1) * 128 + te] : 0.f;
          }
          float sx = v[0][0], sy = v[0][1];
#pragma unroll
          for (int z = 1; z < kMaxSplit; ++z) {
            if (z < nsplit) { sx += v[z][0]; sy += v[z][1]; }
          }
          if (j < N) C[(long long)row * c_rs + (long long)j * c_cs] = make_float2(alpha * sx, alpha * sy);
        }
      }
    }
    cl.sync();   // every partial has been read: no CTA leaves before
  }
  // no MMA may still write TMEM when it is released
  mbar_wait(&done_bar, 0, status, wait_ns);
  tc_fence_after();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
}

// Pack op(A) (M x K complex) into interleaved real rows, split hi/lo: ld = kpad reals.
__global__ void pack_a_kernel(const float2* __restrict__ A, long long a_rs, long long a_cs, int conj, int M, int K,
                              int kpad, float* __restrict__ hi, float* __restrict__ lo) {
  const long long total = (long long)M * (kpad / 2);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / (kpad / 2)), k = (int)(e % (kpad / 2));
    float2 v = make_float2(0.f, 0.f);
    if (k < K) { v = A[i * a_rs + k * a_cs]; if (conj) v.y = -v.y; }
    float h0, h1;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=f"(h0) : "f"(v.x));
    asm("cvt.rna.tf32.f32 %0, %1;" : "=f"(h1) : "f"(v.y));
    const long long o = (long long)i * kpad + 2 * k;
    reinterpret_cast<float2*>(hi)[o / 2] = make_float2(h0, h1);
    reinterpret_cast<float2*>(lo)[o / 2] = make_float2(v.x - h0, v.y - h1);
  }
}

// Pack op(B) (K x N complex) into B' rows 2j = (Re, -Im), 2j+1 = (Im, Re), split hi/lo.
__global__ void pack_b_kernel(const float2* __restrict__ B, long long b_rs, long long b_cs, int conj, int N, int K,
                              int kpad, float* __restrict__ hi, float* __restrict__ lo) {
  const long long total = (long long)N * (kpad / 2);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e / (kpad / 2)), k = (int)(e % (kpad / 2));
    float2 v = make_float2(0.f, 0.f);
    if (k < K) { v = B[k * b_rs + j * b_cs]; if (conj) v.y = -v.y; }
    float hr, hi_;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=f"(hr) : "f"(v.x));
    asm("cvt.rna.tf32.f32 %0, %1;" : "=f"(hi_) : "f"(v.y));
    const float lr = v.x - hr, li = v.y - hi_;
    const long long r0 = (long long)(2 * j) * kpad + 2 * k, r1 = r0 + kpad;
    reinterpret_cast<float2*>(hi)[r0 / 2] = make_float2(hr, -hi_);
    reinterpret_cast<float2*>(lo)[r0 / 2] = make_float2(lr, -li);
    reinterpret_cast<float2*>(hi)[r1 / 2] = make_float2(hi_, hr);
    reinterpret_cast<float2*>(lo)[r1 / 2] = make_float2(li, lr);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  // function-local static: initialised once, thread-safe
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return (PFN_cuTensorMapEncodeTiled_v12000)p;
    return nullptr;
  }();
  return fn;
}

bool make_map(CUtensorMap* map, float* base, int rows, int kpad) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)kpad, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)kpad * 4};
  cuuint32_t box[2] = {BKR, BM};
  cuuint32_t es[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

inline int grid_for(long long work) {
  long long g = (work + 255) / 256;
  return (int)std::max<long long>(1, std::min<long long>(g, 8192));
}

}  // namespace

struct TcGemm {
  float *ah = nullptr, *al = nullptr, *bh = nullptr, *bl = nullptr;
  size_t cap = 0;   // floats per buffer
};

TcGemm* tc_create(size_t max_elems) {
  TcGemm* g = new TcGemm();
  // a packed operand holds 2 floats per complex entry, K padded to a multiple of 16 complex
  g->cap = 4 * max_elems + 64 * 1024;
  if (cudaMalloc(&g->ah, g->cap * 4) != cudaSuccess || cudaMalloc(&g->al, g->cap * 4) != cudaSuccess ||
      cudaMalloc(&g->bh, g->cap * 4) != cudaSuccess || cudaMalloc(&g->bl, g->cap * 4) != cudaSuccess ||
      !encode_fn()) {
    tc_destroy(g);
    return nullptr;
  }
  if (cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES) != cudaSuccess) {
    tc_destroy(g);
    return nullptr;
  }
  return g;
}

void tc_destroy(TcGemm* g) {
  if (!g) return;
  if (g->ah) cudaFree(g->ah);
  if (g->al) cudaFree(g->al);
  if (g->bh) cudaFree(g->bh);
  if (g->bl) cudaFree(g->bl);
  delete g;
}

bool tc_fits(const TcGemm* g, int M, int N, int K) {
  const size_t kpad = (size_t)((2 * K + BKR - 1) / BKR) * BKR;
  return g && (size_t)M * kpad <= g->cap && (size_t)2 * N * kpad <= g->cap;
}

namespace {

// Pack both operands into (ah, al, bh, bl) and launch the tensor-core kernel.
cudaError_t tc_gemm_on(float* ah, float* al, float* bh, float* bl, int M, int N, int K, float alpha, const float2* A,
                       long long a_rs, long long a_cs, int conjA, const float2* B, long long b_rs, long long b_cs,
                       int conjB, float2* C, long long c_rs, long long c_cs, cudaStream_t st, int* launched,
                       int* status, int fault = 0, unsigned long long wait_ns = kWaitNs, bool allow_split = false) {
  *launched = 0;
  const int kpad = ((2 * K + BKR - 1) / BKR) * BKR;
  pack_a_kernel<<<grid_for((long long)M * kpad / 2), 256, 0, st>>>(A, a_rs, a_cs, conjA, M, K, kpad, ah, al);
  pack_b_kernel<<<grid_for((long long)N * kpad / 2), 256, 0, st>>>(B, b_rs, b_cs, conjB, N, K, kpad, bh, bl);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  CUtensorMap mAh, mAl, mBh, mBl;
  if (!make_map(&mAh, ah, M, kpad) || !make_map(&mAl, al, M, kpad) || !make_map(&mBh, bh, 2 * N, kpad) ||
      !make_map(&mBl, bl, 2 * N, kpad))
    return cudaErrorInvalidValue;
  const int nkb = kpad / BKR;
  dim3 grid((2 * N + BN - 1) / BN, (M + BM - 1) / BM);
  // split K over a cluster along z until the grid fills the GPU (at least two K blocks a CTA)
  int split = 1;
  while (allow_split && split < kMaxSplit && (int)(grid.x * grid.y) * split < kSplitTarget && nkb >= 4 * split)
    split *= 2;
  const int kb_per = (nkb + split - 1) / split;
  split = (nkb + kb_per - 1) / kb_per;
  grid.z = split;
  if (split == 1) {
    tc_gemm_kernel<<<grid, NTHREADS, SMEM_BYTES, st>>>(mAh, mAl, mBh, mBl, M, N, nkb, kb_per, alpha, C, c_rs, c_cs,
                                                       1, status, fault, wait_ns);
  } else {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(NTHREADS);
    cfg.dynamicSmemBytes = SMEM_BYTES;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 1;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = split;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e2 = cudaLaunchKernelEx(&cfg, tc_gemm_kernel, mAh, mAl, mBh, mBl, M, N, nkb, kb_per, alpha, C, c_rs,
                                        c_cs, split, status, fault, wait_ns);
    if (e2 != cudaSuccess) return e2;
  }
  *launched = 3;
  return cudaGetLastError();
}

}  // namespace

cudaError_t tc_gemm_raw(float* ah, float* al, float* bh, float* bl, int M, int N, int K, float alpha,
                        const float2* A, long long a_rs, long long a_cs, int conjA, const float2* B, long long b_rs,
                        long long b_cs, int conjB, float2* C, long long c_rs, long long c_cs, cudaStream_t st,
                        int* launched, int* status) {
  return tc_gemm_on(ah, al, bh, bl, M, N, K, alpha, A, a_rs, a_cs, conjA, B, b_rs, b_cs, conjB, C, c_rs, c_cs, st,
                    launched, status);
}

cudaError_t tc_gemm_selftest(TcGemm* g, int M, int N, int K, const float2* A, const float2* B, float2* C,
                             cudaStream_t st, int* status, unsigned long long wait_ns) {
  if (!tc_fits(g, M, N, K) || M <= 0 || N <= 0 || K <= 0) return cudaErrorInvalidValue;
  int launched = 0;
  return tc_gemm_on(g->ah, g->al, g->bh, g->bl, M, N, K, 1.f, A, K, 1, 0, B, N, 1, 0, C, N, 1, st, &launched, status,
                    1, wait_ns);
}

const void* tc_gemm_kernel_entry() { return (const void*)tc_gemm_kernel; }
int tc_gemm_smem_bytes() { return SMEM_BYTES; }

cudaError_t tc_gemm(TcGemm* g, int M, int N, int K, float alpha, const float2* A, long long a_rs, long long a_cs,
                    int conjA, const float2* B, long long b_rs, long long b_cs, int conjB, float2* C, long long c_rs,
                    long long c_cs, cudaStream_t st, int* launched, int* status) {
  *launched = 0;
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (!tc_fits(g, M, N, K) || K <= 0) return cudaErrorInvalidValue;
  return tc_gemm_on(g->ah, g->al, g->bh, g->bl, M, N, K, alpha, A, a_rs, a_cs, conjA, B, b_rs, b_cs, conjB, C, c_rs,
                    c_cs, st, launched, status, 0, kWaitNs, true);
}

}  // namespace eamps

// ======================================================================
// Allocation-free variant of mps_cgemm_c64 (tensor-core path).
//
// Its packing workspace (the hi/lo split copies of both operands) and its
// status word live in one fixed-size array in device memory that is part of
// the loaded library: every GPU that loads the library holds it until the
// process exits, and every call shares it.
#include <mutex>

#include "eamps.h"

namespace {

constexpr size_t kNoAllocPackFloats = size_t(1) << 19;            // floats per packed operand buffer (2 MiB)
constexpr size_t kNoAllocFloats = 4 * kNoAllocPackFloats + 64;   // four buffers + status word (8 MiB + 256 B)
constexpr int kMaxDevices = 64;

static __device__ __align__(256) float g_noalloc_scratch[kNoAllocFloats];

std::mutex g_noalloc_mutex;
float* g_noalloc_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device; resolved once per
// device with that device current (in host code the array's name is only a
// host-side stand-in, never a usable device address).
float* noalloc_scratch(int dev) {
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return nullptr;
    if (cudaFuncSetAttribute(eamps::tc_gemm_kernel_entry(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             eamps::tc_gemm_smem_bytes()) != cudaSuccess)
      return nullptr;
    g_noalloc_ptr[dev] = static_cast<float*>(p);
  }
  return g_noalloc_ptr[dev];
}

}  // namespace

extern "C" mps_status mps_cgemm_c64_noalloc(int M, int N, int K, float alpha, const void* A, long long a_rs,
                                            long long a_cs, int conjA, const void* B, long long b_rs, long long b_cs,
                                            int conjB, void* C, long long c_rs, long long c_cs, void* cuda_stream) {
  if (M < 0 || N < 0 || K < 0 || !A || !B || !C) return MPS_ERR_ARG;
  if (M == 0 || N == 0) return MPS_OK;
  if (K == 0) return MPS_ERR_ARG;
  const size_t kpad = (2 * (size_t)K + 31) / 32 * 32;   // 64-bit: no int overflow for large K
  if ((size_t)M * kpad > kNoAllocPackFloats || (size_t)2 * N * kpad > kNoAllocPackFloats) {
    std::fprintf(stderr,
                 "eamps: mps_cgemm_c64_noalloc: shape %d x %d x %d exceeds the fixed workspace "
                 "(M*pad32(2K) and 2N*pad32(2K) must each be <= %zu)\n",
                 M, N, K, kNoAllocPackFloats);
    return MPS_ERR_ARG;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MPS_ERR_CUDA;
  float* base = noalloc_scratch(dev);
  if (!base) return MPS_ERR_CUDA;
  float* ah = base;
  float* al = base + kNoAllocPackFloats;
  float* bh = base + 2 * kNoAllocPackFloats;
  float* bl = base + 3 * kNoAllocPackFloats;
  int* status = reinterpret_cast<int*>(base + 4 * kNoAllocPackFloats);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // the array keeps the previous call's contents: the status word must start at zero
  cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), st);
  int launched = 0;
  if (e == cudaSuccess)
    e = eamps::tc_gemm_raw(ah, al, bh, bl, M, N, K, alpha, (const float2*)A, a_rs, a_cs, conjA, (const float2*)B,
                           b_rs, b_cs, conjB, (float2*)C, c_rs, c_cs, st, &launched, status);
  int hs = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    std::fprintf(stderr, "eamps: CUDA error: %s\n", cudaGetErrorString(e));
    return MPS_ERR_CUDA;
  }
  return (hs & eamps::ST_TIMEOUT) ? MPS_ERR_TIMEOUT : MPS_OK;
}
