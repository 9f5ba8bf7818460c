// Householder QR of a complex64 matrix ("Canonicalization" section: a site is
// brought into left- or right-canonical form by a QR decomposition, and the
// triangular factor is absorbed into the neighbouring site).  Also used to
// precondition the one-sided Jacobi SVD: with X = Q R, the Jacobi on R^dagger
// converges in fewer sweeps, and its rotated, normalised columns are the right
// singular vectors of X.
//
// Design (sm_103a): one persistent cooperative kernel.  Per panel of 32 columns,
// CTA 0 factors the panel in shared memory (one thread per row, 512 threads,
// rows <= 512) and forms the triangular factor T of the block reflector
// Q_panel = I - V T V^dagger; after a grid barrier every CTA applies
// Q_panel^dagger to its 16-column tiles of the trailing matrix (W1 = V^dagger A,
// W2 = T^dagger W1, A -= V W2) with register-blocked complex FMAs; a second
// barrier precedes the next panel.  Conventions follow LAPACK's complex QR:
// H_j = I - tau_j v_j v_j^dagger with v_j[j] = 1 implicit, R = H_K^dagger ...
// H_1^dagger X, X = Q R, Q = H_1 ... H_K.  Every barrier wait is bounded.
#include <algorithm>

#include <cuda_runtime.h>

#include "kernels.h"

namespace eamps {

namespace {

constexpr int kQrThreads = 512;
constexpr int kQrPanel = 32;
constexpr int kQrTile = 16;
constexpr int kQrMaxRows = 512;
constexpr int kQrPanelLd = kQrMaxRows + 1;   // padded column stride of the factored panel

__device__ __forceinline__ float2 c_mul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
// conj(a) * b
__device__ __forceinline__ float2 c_mulc(float2 a, float2 b) { return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x); }
__device__ __forceinline__ float2 c_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 c_sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 c_conj(float2 a) { return make_float2(a.x, -a.y); }

struct QrShared {
  float2 T[kQrPanel * kQrPanel];    // triangular factor of the current panel (row-major)
  float2 tau[kQrPanel];
  float2 w[kQrPanel + 1];           // column products / scale of the current reflector
  float red[1];   // beta of the current reflector
};

// Factor the panel held column-major in pan (column j at pan + j * kQrPanelLd, rows 0..nr-1,
// rows relative to the panel's first row) into jb reflectors; fills sh.tau and sh.T.
// Per column j one transposed pass gives d_c = sum_{i > j} conj(x_i) A[i][c] for every column
// c >= j at once (d_j is the squared norm below the diagonal); with v = x / (alpha - beta) the
// reflector products are w_c = A[j][c] + conj(scale) d_c, so a column costs three barriers.
// red2: 16 x 32 partial sums.  Loops are unrolled with two accumulators to keep shared-memory
// loads in flight.
__device__ void factor_panel(float2* pan, int nr, int jb, QrShared& sh, float2* red2) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  constexpr int NW = kQrThreads / 32;
  for (int j = 0; j < jb; ++j) {
    const float2* xj = pan + j * kQrPanelLd;
    // partial d_c over this warp's 32 rows (lane = column c)
    {
      float2 acc0 = make_float2(0.f, 0.f), acc1 = make_float2(0.f, 0.f);
      const int i0 = max(warp * 32, j + 1), i1 = min(nr, warp * 32 + 32);
      const float2* ac = pan + lane * kQrPanelLd;
      if (lane >= j && lane < jb) {
        int i = i0;
#pragma unroll 4
        for (; i + 1 < i1; i += 2) {
          acc0 = c_add(acc0, c_mulc(xj[i], ac[i]));
          acc1 = c_add(acc1, c_mulc(xj[i + 1], ac[i + 1]));
        }
        if (i < i1) acc0 = c_add(acc0, c_mulc(xj[i], ac[i]));
      }
      red2[warp * 32 + lane] = c_add(acc0, acc1);
    }
    __syncthreads();
    if (warp == 0) {
      float2 dc = make_float2(0.f, 0.f);
#pragma unroll
      for (int w = 0; w < NW; ++w) dc = c_add(dc, red2[w * 32 + lane]);
      const float xn2 = __shfl_sync(0xffffffffu, dc.x, j);
      const float2 alpha = xj[j];
      float2 tj = make_float2(0.f, 0.f), sc = make_float2(0.f, 0.f);
      float beta = alpha.x;
      if (!(xn2 == 0.f && alpha.y == 0.f)) {
        const float an = sqrtf(alpha.x * alpha.x + alpha.y * alpha.y + xn2);
        beta = (alpha.x >= 0.f) ? -an : an;
        tj = make_float2((beta - alpha.x) / beta, -alpha.y / beta);
        const float2 den = make_float2(alpha.x - beta, alpha.y);          // scale = 1 / (alpha - beta)
        const float dd = den.x * den.x + den.y * den.y;
        sc = make_float2(den.x / dd, -den.y / dd);
      }
      if (lane > j && lane < jb) sh.w[lane] = c_add(pan[lane * kQrPanelLd + j], c_mul(c_conj(sc), dc));
      if (lane == 0) {
        sh.tau[j] = tj;
        sh.w[kQrPanel] = sc;
        sh.red[0] = beta;
      }
    }
    __syncthreads();
    // v = x * scale below the diagonal, R[j][j] = beta, and A[i][c] -= conj(tau) v_i w_c
    if (t >= j && t < nr) {
      const float2 sc = sh.w[kQrPanel];
      const float2 ctau = c_conj(sh.tau[j]);
      float2* col = pan + j * kQrPanelLd;
      float2 v;
      if (t == j) {
        v = make_float2(1.f, 0.f);
        col[j] = make_float2(sh.red[0], 0.f);
      } else {
        v = c_mul(col[t], sc);
        col[t] = v;
      }
      const float2 ctv = c_mul(ctau, v);
#pragma unroll 4
      for (int cc = j + 1; cc < jb; ++cc) {
        float2* a = pan + cc * kQrPanelLd;
        a[t] = c_sub(a[t], c_mul(ctv, sh.w[cc]));
      }
    }
    __syncthreads();
  }
  // T (forward, columnwise): T[j][j] = tau_j, T[0:j, j] = -tau_j T[0:j, 0:j] (V[:, 0:j]^dagger v_j)
  for (int j = 0; j < jb; ++j) {
    const float2* vj = pan + j * kQrPanelLd;
    for (int p = warp; p < j; p += NW) {
      const float2* vp = pan + p * kQrPanelLd;
      float2 acc0 = (lane == 0) ? c_conj(vp[j]) : make_float2(0.f, 0.f);   // row j: v_j[j] = 1
      float2 acc1 = make_float2(0.f, 0.f);
      int i = j + 1 + lane;
#pragma unroll 4
      for (; i + 32 < nr; i += 64) {
        acc0 = c_add(acc0, c_mulc(vp[i], vj[i]));
        acc1 = c_add(acc1, c_mulc(vp[i + 32], vj[i + 32]));
      }
      if (i < nr) acc0 = c_add(acc0, c_mulc(vp[i], vj[i]));
      float2 acc = c_add(acc0, acc1);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
      }
      if (lane == 0) sh.w[p] = acc;
    }
    __syncthreads();
    if (t < j) {
      float2 acc0 = make_float2(0.f, 0.f), acc1 = make_float2(0.f, 0.f);
      int q = t;
#pragma unroll 4
      for (; q + 1 < j; q += 2) {
        acc0 = c_add(acc0, c_mul(sh.T[t * kQrPanel + q], sh.w[q]));
        acc1 = c_add(acc1, c_mul(sh.T[t * kQrPanel + q + 1], sh.w[q + 1]));
      }
      if (q < j) acc0 = c_add(acc0, c_mul(sh.T[t * kQrPanel + q], sh.w[q]));
      const float2 v = c_mul(sh.tau[j], c_add(acc0, acc1));
      sh.T[t * kQrPanel + j] = make_float2(-v.x, -v.y);
    } else if (t == j) {
      sh.T[j * kQrPanel + j] = sh.tau[j];
    } else if (t < kQrPanel) {
      sh.T[t * kQrPanel + j] = make_float2(0.f, 0.f);
    }
    __syncthreads();
  }
}

// Copy a rows x cols block (column-major) global -> shared with eight loads in flight per thread.
__device__ __forceinline__ void load2d(float2* dst, int dld, const float2* src, long long sld, int rows, int cols) {
  const int total = rows * cols;
  for (int e0 = threadIdx.x; e0 < total; e0 += 8 * kQrThreads) {
    float2 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * kQrThreads;
      if (e < total) {
        const int j = e / rows, i = e - j * rows;
        v[u] = __ldcg(src + (long long)j * sld + i);
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * kQrThreads;
      if (e < total) {
        const int j = e / rows, i = e - j * rows;
        dst[j * dld + i] = v[u];
      }
    }
  }
}

// Reflector rows in shared memory: row i holds V[i][0..31] with the column index XOR-swizzled
// by the row, so that both "lanes = columns of one row" and "lanes = rows, one column" are
// conflict-free.
__device__ __forceinline__ int vsw(int i, int p) { return i * kQrPanel + (p ^ (i & 31)); }

// Apply the block reflector of one panel to the tile A (column-major, leading dim lda, nr rows
// starting at the panel's first row, tw <= 16 columns):
//   adjoint: A <- (I - V T V^dagger)^dagger A = A - V T^dagger (V^dagger A)
//   else:    A <- (I - V T V^dagger) A         = A - V T (V^dagger A)
// Vs: swizzled reflector rows; At: the staged tile (column c at At + c * kQrMaxRows);
// As: W1 partial sums (4 row slices x 16 x 32); W: 16 x 32.
__device__ void apply_block(float2* __restrict__ A, long long lda, int nr, int tw, int jb, const float2* Vs,
                            const float2* Ts, bool adjoint, float2* At, float2* As, float2* W) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  constexpr int NW = kQrThreads / 32;
  // stage the tile, zero columns past tw
  load2d(At, kQrMaxRows, A, lda, nr, tw);
  for (int e = tw * nr + t; e < kQrTile * nr; e += kQrThreads) {
    const int c = e / nr, i = e - c * nr;
    At[c * kQrMaxRows + i] = make_float2(0.f, 0.f);
  }
  __syncthreads();
  // W1[p][c] = sum_i conj(V[i][p]) A[i][c]: lane = p; warp -> column quad cq, row slice ks
  {
    const int cq = warp & 3, ks = warp >> 2;
    const int rows_per = (nr + 3) / 4;
    const int i0 = ks * rows_per, i1 = min(nr, i0 + rows_per);
    float2 acc[4] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    for (int i = i0; i < i1; ++i) {
      const float2 v = Vs[vsw(i, lane)];
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] = c_add(acc[u], c_mulc(v, At[(cq * 4 + u) * kQrMaxRows + i]));
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) As[(ks * kQrTile + cq * 4 + u) * kQrPanel + lane] = acc[u];
  }
  __syncthreads();
  // W1 summed over the row slices, then W2 = op(T) W1 (T upper triangular)
  float2 w1 = make_float2(0.f, 0.f);
  if (t < kQrPanel * kQrTile) {
    const int p = t & 31, c = t >> 5;
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) w1 = c_add(w1, As[(ks * kQrTile + c) * kQrPanel + p]);
    W[c * kQrPanel + p] = w1;
  }
  __syncthreads();
  float2 w2 = make_float2(0.f, 0.f);
  if (t < kQrPanel * kQrTile) {
    const int p = t & 31, c = t >> 5;
    if (p < jb) {
      if (adjoint) {   // (T^dagger W1)[p] = sum_{q <= p} conj(T[q][p]) W1[q]
        for (int q = 0; q <= p; ++q) w2 = c_add(w2, c_mulc(Ts[q * kQrPanel + p], W[c * kQrPanel + q]));
      } else {         // (T W1)[p] = sum_{q >= p} T[p][q] W1[q]
        for (int q = p; q < jb; ++q) w2 = c_add(w2, c_mul(Ts[p * kQrPanel + q], W[c * kQrPanel + q]));
      }
    }
  }
  __syncthreads();
  if (t < kQrPanel * kQrTile) W[(t >> 5) * kQrPanel + (t & 31)] = w2;
  __syncthreads();
  // A[i][c] -= sum_p V[i][p] W2[p][c]: one row per thread
  for (int i = t; i < nr; i += kQrThreads) {
    float2 v[kQrPanel];
#pragma unroll
    for (int p = 0; p < kQrPanel; ++p) v[p] = Vs[vsw(i, p)];
    for (int c = 0; c < tw; ++c) {
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int p = 0; p < kQrPanel; ++p) acc = c_add(acc, c_mul(v[p], W[c * kQrPanel + p]));
      At[c * kQrMaxRows + i] = c_sub(At[c * kQrMaxRows + i], acc);
    }
  }
  __syncthreads();
  for (int c = warp; c < tw; c += NW) {
    float2* dst = A + (long long)c * lda;
    const float2* src = At + c * kQrMaxRows;
    for (int i = lane; i < nr; i += 32) __stcg(dst + i, src[i]);
  }
  __syncthreads();
}

// Explicit reflector vectors of the panel at column c0 (rows r0.., column-major in X) into Vs.
__device__ void load_v(const float2* X, long long ldx, int r0, int nr, int c0, int jb, float2* Vs) {
  const int total = nr * kQrPanel;
  for (int e0 = threadIdx.x; e0 < total; e0 += 8 * kQrThreads) {
    float2 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * kQrThreads;
      const int p = e / nr, i = e - p * nr;   // coalesced along rows of one column
      v[u] = make_float2(0.f, 0.f);
      if (e < total && p < jb) {
        if (i == p) v[u] = make_float2(1.f, 0.f);
        else if (i > p) v[u] = __ldcg(X + (long long)(c0 + p) * ldx + r0 + i);
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * kQrThreads;
      if (e < total) {
        const int p = e / nr, i = e - p * nr;
        Vs[vsw(i, p)] = v[u];
      }
    }
  }
}

struct QrArgs {
  float2* X; long long ldx; int l; int c;
  float2* tau;      // K entries
  float2* Tm;       // panels x 32 x 32
  float2* Q; long long ldq; int kq;   // qr_form_q: output
  DevCtrl* ctrl;
};

__global__ void __launch_bounds__(kQrThreads, 1) qr_factor_kernel(QrArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ QrShared sh;
  float2* big = reinterpret_cast<float2*>(smem_raw);   // panel (CTA 0, 32 x 513) or reflector rows (512 x 32)
  float2* At = big + kQrPanel * kQrPanelLd;            // staged tile, 16 x 512
  float2* As = At + kQrMaxRows * kQrTile;              // 4 x 16 x 32
  float2* W = As + 4 * kQrTile * kQrPanel;             // 16 x 32
  const int P = gridDim.x;
  const int K = min(a.l, a.c);
  const int npan = (K + kQrPanel - 1) / kQrPanel;
  for (int k = 0; k < npan; ++k) {
    const int c0 = k * kQrPanel, jb = min(kQrPanel, K - c0), r0 = c0, nr = a.l - r0;
    if (blockIdx.x == 0) {
      load2d(big, kQrPanelLd, a.X + (long long)c0 * a.ldx + r0, a.ldx, nr, jb);
      __syncthreads();
      factor_panel(big, nr, jb, sh, W);
      for (int e = threadIdx.x; e < jb * nr; e += kQrThreads) {
        const int j = e / nr, i = e % nr;
        __stcg(a.X + (long long)(c0 + j) * a.ldx + r0 + i, big[j * kQrPanelLd + i]);
      }
      for (int e = threadIdx.x; e < kQrPanel * kQrPanel; e += kQrThreads) a.Tm[(long long)k * kQrPanel * kQrPanel + e] = sh.T[e];
      if (threadIdx.x < jb) a.tau[c0 + threadIdx.x] = sh.tau[threadIdx.x];
      __threadfence();
    }
    const int first = c0 + jb;   // trailing columns
    if (first >= a.c) break;
    if (!grid_barrier(a.ctrl, P)) return;
    // every CTA: V and T of this panel, then its tiles
    load_v(a.X, a.ldx, r0, nr, c0, jb, big);
    for (int e = threadIdx.x; e < kQrPanel * kQrPanel; e += kQrThreads) sh.T[e] = __ldcg(a.Tm + (long long)k * kQrPanel * kQrPanel + e);
    __syncthreads();
    const int ntiles = (a.c - first + kQrTile - 1) / kQrTile;
    for (int tile = blockIdx.x; tile < ntiles; tile += P) {
      const int tc = first + tile * kQrTile, tw = min(kQrTile, a.c - tc);
      apply_block(a.X + (long long)tc * a.ldx + r0, a.ldx, nr, tw, jb, big, sh.T, true, At, As, W);
    }
    __threadfence();
    if (!grid_barrier(a.ctrl, P)) return;
  }
}

// Q (l x kq, column-major) = H_1 ... H_K [I; 0] by backward accumulation of the panels.
__global__ void __launch_bounds__(kQrThreads, 1) qr_form_q_kernel(QrArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ QrShared sh;
  float2* big = reinterpret_cast<float2*>(smem_raw);
  float2* At = big + kQrPanel * kQrPanelLd;
  float2* As = At + kQrMaxRows * kQrTile;
  float2* W = As + 4 * kQrTile * kQrPanel;
  const int P = gridDim.x;
  const int K = min(a.l, a.c);
  const int npan = (K + kQrPanel - 1) / kQrPanel;
  // Q = [I; 0]
  const long long total = (long long)a.kq * a.l;
  for (long long e = blockIdx.x * (long long)kQrThreads + threadIdx.x; e < total; e += (long long)P * kQrThreads) {
    const int col = (int)(e / a.l), row = (int)(e % a.l);
    a.Q[(long long)col * a.ldq + row] = make_float2(row == col ? 1.f : 0.f, 0.f);
  }
  __threadfence();
  if (!grid_barrier(a.ctrl, P)) return;
  for (int k = npan - 1; k >= 0; --k) {
    const int c0 = k * kQrPanel, jb = min(kQrPanel, K - c0), r0 = c0, nr = a.l - r0;
    load_v(a.X, a.ldx, r0, nr, c0, jb, big);
    for (int e = threadIdx.x; e < kQrPanel * kQrPanel; e += kQrThreads) sh.T[e] = __ldcg(a.Tm + (long long)k * kQrPanel * kQrPanel + e);
    __syncthreads();
    // columns < c0 of Q are still unit vectors above row c0: untouched by this panel
    const int ntiles = (a.kq - c0 + kQrTile - 1) / kQrTile;
    for (int tile = blockIdx.x; tile < ntiles; tile += P) {
      const int tc = c0 + tile * kQrTile, tw = min(kQrTile, a.kq - tc);
      apply_block(a.Q + (long long)tc * a.ldq + r0, a.ldq, nr, tw, jb, big, sh.T, false, At, As, W);
    }
    __threadfence();
    if (!grid_barrier(a.ctrl, P)) return;
  }
}

size_t qr_smem_bytes() {
  return sizeof(float2) * ((size_t)kQrPanel * kQrPanelLd + (size_t)kQrMaxRows * kQrTile + 4 * kQrTile * kQrPanel +
                            kQrTile * kQrPanel);
}

cudaError_t launch_qr(const void* fn, QrArgs& a, int ctas, cudaStream_t st) {
  cudaError_t e = allow_dynamic_smem(fn);
  if (e != cudaSuccess) return e;
  // reset the barrier counters (bar_count, bar_gen, rot[3] are contiguous)
  e = cudaMemsetAsync(&a.ctrl->bar_count, 0, 5 * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  void* args[] = {&a};
  const size_t smem = qr_smem_bytes();
  if (ctas <= 1) return cudaLaunchKernel(fn, dim3(1), dim3(kQrThreads), args, smem, st);
  return cudaLaunchCooperativeKernel(fn, dim3(ctas), dim3(kQrThreads), args, smem, st);
}

}  // namespace

int qr_max_rows() { return kQrMaxRows; }

int qr_ctas(int l, int c, int max_ctas) {
  const int tiles = (c + kQrTile - 1) / kQrTile;
  return std::max(1, std::min(tiles, max_ctas));
}

int qr_max_ctas() {
  int per_sm = 0, dev = 0, sms = 0;
  if (allow_dynamic_smem((const void*)qr_factor_kernel) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, qr_factor_kernel, kQrThreads, qr_smem_bytes()) !=
      cudaSuccess)
    return 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return per_sm * sms;
}

cudaError_t qr_factor(float2* X, long long ldx, int l, int c, float2* tau, float2* Tm, DevCtrl* ctrl, int ctas,
                      cudaStream_t st) {
  if (l <= 0 || c <= 0) return cudaSuccess;
  if (l > kQrMaxRows) return cudaErrorInvalidValue;
  QrArgs a{};
  a.X = X; a.ldx = ldx; a.l = l; a.c = c; a.tau = tau; a.Tm = Tm; a.ctrl = ctrl;
  return launch_qr((const void*)qr_factor_kernel, a, ctas, st);
}

cudaError_t qr_form_q(const float2* X, long long ldx, int l, int c, const float2* Tm, float2* Q, long long ldq,
                      DevCtrl* ctrl, int ctas, cudaStream_t st) {
  if (l <= 0 || c <= 0) return cudaSuccess;
  if (l > kQrMaxRows) return cudaErrorInvalidValue;
  QrArgs a{};
  a.X = const_cast<float2*>(X); a.ldx = ldx; a.l = l; a.c = c; a.Tm = const_cast<float2*>(Tm);
  a.Q = Q; a.ldq = ldq; a.kq = std::min(l, c); a.ctrl = ctrl;
  return launch_qr((const void*)qr_form_q_kernel, a, ctas, st);
}

}  // namespace eamps
