// Householder QR of a complex64 matrix ("Canonicalization" section: a site is
// brought into left- or right-canonical form by a QR decomposition, and the
// triangular factor is absorbed into the neighbouring site).  Also used to
// precondition the one-sided Jacobi SVD: with X = Q R, the Jacobi on R^dagger
// converges in fewer sweeps, and its rotated, normalised columns are the right
// singular vectors of X.
//
// Design (sm_103a): one persistent kernel launched as clusters of four CTAs.  Per panel of 32
// columns, the four CTAs of cluster 0 factor the panel together (each holds 128 of its rows in
// registers, four threads per row; the column sums of each step meet in distributed shared memory
// after one cluster barrier) and CTA 0 forms the triangular factor T of the block reflector
// Q_panel = I - V T V^dagger; after a grid barrier every CTA applies Q_panel^dagger to its
// 16-column tiles of the trailing matrix (W1 = V^dagger A, W2 = T^dagger W1, A -= V W2) with
// register-blocked complex FMAs; a second barrier precedes the next panel.  Conventions follow
// LAPACK's complex QR: H_j = I - tau_j v_j v_j^dagger with v_j[j] = 1 implicit,
// R = H_K^dagger ... H_1^dagger X, X = Q R, Q = H_1 ... H_K.  Every grid-barrier wait is bounded,
// and the CTAs of cluster 0 agree on leaving after each one.
#include <algorithm>

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "kernels.h"

namespace eamps {

namespace {

namespace cg = cooperative_groups;

constexpr int kQrThreads = 512;
constexpr int kQrPanel = 32;
constexpr int kQrTile = 16;
constexpr int kQrMaxRows = 512;
constexpr int kQrVs = kQrMaxRows * kQrPanel;      // reflector rows of one panel (shared memory)
constexpr int kQrCluster = 4;                      // CTAs that factor each panel together
constexpr int kQrMaxCtas = 16;                     // CTAs of one launch at most (one cluster)
constexpr int kQrPanelRows = kQrMaxRows / kQrCluster;   // rows of the panel per CTA

__device__ __forceinline__ float2 c_mul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
// conj(a) * b
__device__ __forceinline__ float2 c_mulc(float2 a, float2 b) { return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x); }
__device__ __forceinline__ float2 c_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 c_sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 c_conj(float2 a) { return make_float2(a.x, -a.y); }

struct QrShared {
  float2 T[kQrPanel * kQrPanel];    // triangular factor of the current panel (row-major)
  float2 tau[kQrPanel];
};

// The panel is factored by the kQrCluster CTAs of cluster 0: CTA r holds rows
// [r * kQrPanelRows, (r + 1) * kQrPanelRows) of the panel, and each row is spread over four
// threads of one warp (lane = 4 * row-in-warp + g), thread g holding columns [8 g, 8 g + 8) of the
// row in registers.  Scratch layout (shared memory of each CTA), each part by column parity:
// recv [2][kQrCluster][32], the 32 column sums of every panel CTA, pushed by their warp 0; red
// [2][16 warps][32], this CTA's warp sums; rowj [2][32] (row j of the panel, pushed by CTA 0);
// then CTA 0's vg [32 x 32], vg[q * 32 + j] = (V^dagger V)[q][j] for q < j, and M [32 x 32] for
// the merge of T.
constexpr int kQrWarps = kQrThreads / 32;
constexpr int kQrRecv = kQrCluster * 32;
constexpr int kQrRedOff = 2 * kQrRecv;
constexpr int kQrRowjOff = kQrRedOff + 2 * kQrWarps * 32;
constexpr int kQrVgOff = kQrRowjOff + 64;
constexpr int kQrMOff = kQrVgOff + kQrPanel * kQrPanel;
static_assert(kQrPanelRows * 4 == kQrThreads, "four threads per panel row");
static_assert(kQrMOff + kQrPanel * kQrPanel <= kQrVs, "panel scratch fits the reflector buffer");

struct PanelCtx {
  QrShared* sh;
  float2* scratch;
  int row, nr, jb, rank;
};

// Square root and reciprocal of a positive float from the hardware approximations plus one Newton
// step (Heron's step for the root, r (2 - x r) for the reciprocal): within about an ulp, without
// the out-of-line path of the IEEE operations, which sit on the panel's critical path.  Arguments
// outside [1e-30, 1e30] take the IEEE operations.
__device__ __forceinline__ float sqrt_nr(float x) {
  if (!(x > 1e-30f && x < 1e30f)) return sqrtf(x);
  const float y = rsqrtf(x), s = x * y;
  return fmaf(0.5f * y, fmaf(-s, s, x), s);
}
__device__ __forceinline__ float rcp_nr(float x) {
  const float ax = fabsf(x);
  if (!(ax > 1e-30f && ax < 1e30f)) return 1.f / x;
  const float r = __fdividef(1.f, x);
  return r * fmaf(-x, r, 2.f);
}

// One halving round of a reduce-scatter over the lanes that differ in lane bit M: the lane keeps
// the half of v[0, 2 O) selected by that bit, adds its partner's copy of it, and stores it in v[0, O).
template <int O, int M>
__device__ __forceinline__ void rs_round(float2 (&v)[8], int lane) {
  const bool up = lane & M;
#pragma unroll
  for (int k = 0; k < O; ++k) {
    const float2 send = up ? v[k] : v[k + O], keep = up ? v[k + O] : v[k];
    v[k] = make_float2(keep.x + __shfl_xor_sync(0xffffffffu, send.x, M),
                       keep.y + __shfl_xor_sync(0xffffffffu, send.y, M));
  }
}

// Column step J of the panel.
__device__ __forceinline__ void panel_step(float2 (&a)[8], const PanelCtx& p, cg::cluster_group& cl, const int J) {
  QrShared& sh = *p.sh;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5, g = lane & 3, par = J & 1;
  float2* recv = p.scratch + par * kQrRecv;
  float2* rowj = p.scratch + kQrRowjOff + par * 32;
  // x = A[row][J], held by thread J / 8 of the row
  const bool b0 = J & 1, b1 = J & 2, b2 = J & 4;   // a[J & 7] by a tree of selects
  const float2 m01 = b0 ? a[1] : a[0], m23 = b0 ? a[3] : a[2], m45 = b0 ? a[5] : a[4], m67 = b0 ? a[7] : a[6];
  const float2 m03 = b1 ? m23 : m01, m47 = b1 ? m67 : m45;
  const float2 mine = b2 ? m47 : m03;
  const int src = (lane & ~3) | (J >> 3);
  const float2 x = make_float2(__shfl_sync(0xffffffffu, mine.x, src), __shfl_sync(0xffffffffu, mine.y, src));
  if (p.rank == 0 && p.row == J) {   // row J of the panel (CTA 0) to every CTA
#pragma unroll
    for (int r = 0; r < kQrCluster; ++r) {
      float2* dst = cl.map_shared_rank(rowj, r) + 8 * g;
#pragma unroll
      for (int k = 0; k < 8; ++k) dst[k] = a[k];
    }
  }
  // slot s = 8 g + k: d_s = sum conj(x) A[.][s] for s >= J, y_s = sum conj(V[.][s]) x for s < J,
  // over the rows below J; summed over the warp's 8 rows by a reduce-scatter over lane bits 4, 3, 2
  const float2 xm = (p.row > J && p.row < p.nr) ? x : make_float2(0.f, 0.f);
  float2 v[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = (8 * g + k >= J) ? c_mulc(xm, a[k]) : c_mulc(a[k], xm);
  rs_round<4, 16>(v, lane);
  rs_round<2, 8>(v, lane);
  rs_round<1, 4>(v, lane);
  // this lane now holds the warp's sum of slot 8 g + (lane >> 2); the CTA's sums then go to every
  // panel CTA (warp 0 pushes them)
  float2* red = p.scratch + kQrRedOff + par * (kQrWarps * 32);
  red[warp * 32 + 8 * g + (lane >> 2)] = v[0];
  __syncthreads();
  if (warp == 0) {
    float2 d4[4] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
    for (int w = 0; w < kQrWarps; ++w) d4[w & 3] = c_add(d4[w & 3], red[w * 32 + lane]);
    const float2 ds = c_add(c_add(d4[0], d4[1]), c_add(d4[2], d4[3]));
#pragma unroll
    for (int r = 0; r < kQrCluster; ++r) cl.map_shared_rank(recv, r)[p.rank * 32 + lane] = ds;
  }
  cl.sync();
  // every warp of every panel CTA forms the same scalars from the same sums, in the same order
  // (lane = slot), so no broadcast and no further barrier is needed
  const float2 dc = c_add(c_add(recv[lane], recv[32 + lane]), c_add(recv[64 + lane], recv[96 + lane]));
  const float xn2 = __shfl_sync(0xffffffffu, dc.x, J);
  const float2 alpha = rowj[J];
  const float2 rl = rowj[lane];
  float2 sc = make_float2(0.f, 0.f), tj = make_float2(0.f, 0.f);
  float beta = alpha.x;
  if (!(xn2 == 0.f && alpha.y == 0.f)) {
    const float an = sqrt_nr(alpha.x * alpha.x + alpha.y * alpha.y + xn2);
    beta = (alpha.x >= 0.f) ? -an : an;
    const float ib = rcp_nr(beta);
    tj = make_float2((beta - alpha.x) * ib, -alpha.y * ib);
    const float2 den = make_float2(alpha.x - beta, alpha.y);          // scale = 1 / (alpha - beta)
    const float idd = rcp_nr(den.x * den.x + den.y * den.y);
    sc = make_float2(den.x * idd, -den.y * idd);
  }
  const float2 wl = (lane > J && lane < p.jb) ? c_add(rl, c_mul(c_conj(sc), dc)) : make_float2(0.f, 0.f);
  if (p.rank == 0 && warp == 0) {
    if (lane < J) p.scratch[kQrVgOff + lane * 32 + J] = c_add(c_mul(sc, dc), c_conj(rl));
    if (lane == 0) sh.tau[J] = tj;
  }
  float2 wk[8];   // w of this thread's columns 8 g .. 8 g + 7
#pragma unroll
  for (int k = 0; k < 8; ++k)
    wk[k] = make_float2(__shfl_sync(0xffffffffu, wl.x, 8 * g + k), __shfl_sync(0xffffffffu, wl.y, 8 * g + k));
  // v = x * scale below the diagonal, R[J][J] = beta, and A[i][c] -= conj(tau) v_i w_c (w_c = 0
  // for c <= J, so those entries keep their values; entry J then takes v or beta)
  if (p.row >= J && p.row < p.nr) {
    const bool diag = p.row == J;
    const float2 vv = diag ? make_float2(1.f, 0.f) : c_mul(x, sc);
    const float2 nj = diag ? make_float2(beta, 0.f) : vv;
    const float2 ctv = c_mul(c_conj(tj), vv);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const float2 u = c_sub(a[k], c_mul(ctv, wk[k]));
      a[k] = (8 * g + k == J) ? nj : u;
    }
  }
}

// Factor the panel of rows r0.., columns c0.. of X (nr <= 512 rows, jb <= 32 columns) in place
// into jb reflectors (LAPACK layout: R on and above the diagonal, v below it, v_j[j] = 1
// implicit), run by the CTAs of cluster 0; CTA 0 also fills sh.tau and sh.T.  The rows stay in
// registers for the whole factorisation, so a column step moves no panel data.  Step j needs,
// over the rows i > j, d_c = sum_i conj(x_i) A[i][c] for the columns c >= j (d_j = squared norm
// below the diagonal, x = column j) and, for the compact-WY factor, y_q = sum_i conj(V[i][q]) x_i
// for the earlier reflectors q < j: together exactly 32 sums, reduced within each warp, pushed to
// every CTA of the cluster through distributed shared memory and summed there after one cluster
// barrier.  With v = x / (alpha - beta) the reflector products are w_c = A[j][c] + conj(scale) d_c,
// and (V^dagger v_j)_q = scale y_q + conj(V[j][q]).  After the last column CTA 0 builds T by
// merging blocks of reflectors: for adjacent blocks 1, 2 of size b,
// T = [[T1, -T1 (V1^dagger V2) T2], [0, T2]], five levels from the single reflectors (T = tau).
// scratch: the reflector buffer of this CTA's shared memory, unused otherwise during the panel.
__device__ void factor_panel(float2* X, long long ldx, int r0, int c0, int nr, int jb, QrShared& sh, float2* scratch,
                             cg::cluster_group& cl) {
  const int t = threadIdx.x, rank = (int)cl.block_rank(), g = t & 3;
  PanelCtx p;
  p.sh = &sh;
  p.scratch = scratch;
  float2* vg = scratch + kQrVgOff;
  float2* M = scratch + kQrMOff;   // CTA 0: products of the merge
  p.row = rank * kQrPanelRows + (t >> 2);
  p.nr = nr;
  p.jb = jb;
  p.rank = rank;
  float2 a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k)
    a[k] = (p.row < nr && 8 * g + k < jb) ? __ldcg(X + (long long)(c0 + 8 * g + k) * ldx + r0 + p.row)
                                          : make_float2(0.f, 0.f);
  if (rank == 0)
    for (int e = t; e < kQrPanel * kQrPanel; e += kQrThreads) vg[e] = make_float2(0.f, 0.f);
  cl.sync();   // every CTA of the cluster is running before remote stores (and vg is clear)
#pragma unroll 1
  for (int j = 0; j < jb; ++j) panel_step(a, p, cl, j);   // (jb is the same for the whole cluster)
#pragma unroll
  for (int k = 0; k < 8; ++k)
    if (p.row < nr && 8 * g + k < jb) __stcg(X + (long long)(c0 + 8 * g + k) * ldx + r0 + p.row, a[k]);
  if (rank == 0) {
    // T by merging: leaves T[i][i] = tau_i (0 past jb), then levels b = 1, 2, 4, 8, 16
    for (int e = t; e < kQrPanel * kQrPanel; e += kQrThreads) {
      const int i = e >> 5, j = e & 31;
      sh.T[e] = (i == j && i < jb) ? sh.tau[i] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int b = 1; b < kQrPanel; b *= 2) {
      const int n = (kQrPanel / (2 * b)) * b * b;   // entries of all the blocks T12 of this level
      for (int e = t; e < n; e += kQrThreads) {     // M = V1^dagger V2 T2
        const int blk = e / (b * b), i = (e / b) % b, j = e % b, o = 2 * b * blk;
        float2 acc = make_float2(0.f, 0.f);
        for (int k = 0; k <= j; ++k)
          acc = c_add(acc, c_mul(vg[(o + i) * 32 + o + b + k], sh.T[(o + b + k) * kQrPanel + o + b + j]));
        M[(o + i) * 32 + o + b + j] = acc;
      }
      __syncthreads();
      for (int e = t; e < n; e += kQrThreads) {     // T12 = -T1 M
        const int blk = e / (b * b), i = (e / b) % b, j = e % b, o = 2 * b * blk;
        float2 acc = make_float2(0.f, 0.f);
        for (int k = i; k < b; ++k)
          acc = c_add(acc, c_mul(sh.T[(o + i) * kQrPanel + o + k], M[(o + k) * 32 + o + b + j]));
        sh.T[(o + i) * kQrPanel + o + b + j] = make_float2(-acc.x, -acc.y);
      }
      __syncthreads();
    }
  }
  __syncthreads();
}

// The cluster barriers of factor_panel, for the CTAs of the cluster that do not factor the panel.
__device__ __forceinline__ void panel_idle(cg::cluster_group& cl, int jb) {
  cl.sync();
  for (int j = 0; j < jb; ++j) cl.sync();
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

// Both kernels run as ONE thread-block cluster (the whole grid): the hardware schedules its CTAs
// together, so the steps are separated by cluster barriers and nothing spins on memory.
__global__ void __launch_bounds__(kQrThreads, 1) qr_factor_kernel(QrArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ QrShared sh;
  float2* big = reinterpret_cast<float2*>(smem_raw);   // panel scratch (ranks < kQrCluster) or reflector rows
  float2* At = big + kQrVs;                            // staged tile, 16 x 512
  float2* As = At + kQrMaxRows * kQrTile;              // 4 x 16 x 32
  float2* W = As + 4 * kQrTile * kQrPanel;             // 16 x 32
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank(), P = (int)cl.num_blocks();
  const int K = min(a.l, a.c);
  const int npan = (K + kQrPanel - 1) / kQrPanel;
  for (int k = 0; k < npan; ++k) {
    const int c0 = k * kQrPanel, jb = min(kQrPanel, K - c0), r0 = c0, nr = a.l - r0;
    if (rank < kQrCluster) {   // ranks 0..3 factor the panel
      factor_panel(a.X, a.ldx, r0, c0, nr, jb, sh, big, cl);
      if (rank == 0) {
        for (int e = threadIdx.x; e < kQrPanel * kQrPanel; e += kQrThreads) a.Tm[(long long)k * kQrPanel * kQrPanel + e] = sh.T[e];
        if (threadIdx.x < jb) a.tau[c0 + threadIdx.x] = sh.tau[threadIdx.x];
      }
      __threadfence();
    } else {
      panel_idle(cl, jb);   // the same cluster barriers as factor_panel
    }
    const int first = c0 + jb;   // trailing columns
    if (first >= a.c) break;
    cl.sync();
    // every CTA: V and T of this panel, then its tiles
    load_v(a.X, a.ldx, r0, nr, c0, jb, big);
    for (int e = threadIdx.x; e < kQrPanel * kQrPanel; e += kQrThreads) sh.T[e] = __ldcg(a.Tm + (long long)k * kQrPanel * kQrPanel + e);
    __syncthreads();
    const int ntiles = (a.c - first + kQrTile - 1) / kQrTile;
    for (int tile = rank; tile < ntiles; tile += P) {
      const int tc = first + tile * kQrTile, tw = min(kQrTile, a.c - tc);
      apply_block(a.X + (long long)tc * a.ldx + r0, a.ldx, nr, tw, jb, big, sh.T, true, At, As, W);
    }
    __threadfence();
    cl.sync();
  }
}

// Q (l x kq, column-major) = H_1 ... H_K [I; 0] by backward accumulation of the panels.
__global__ void __launch_bounds__(kQrThreads, 1) qr_form_q_kernel(QrArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ QrShared sh;
  float2* big = reinterpret_cast<float2*>(smem_raw);
  float2* At = big + kQrVs;
  float2* As = At + kQrMaxRows * kQrTile;
  float2* W = As + 4 * kQrTile * kQrPanel;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank(), P = (int)cl.num_blocks();
  const int K = min(a.l, a.c);
  const int npan = (K + kQrPanel - 1) / kQrPanel;
  // Q = [I; 0]
  const long long total = (long long)a.kq * a.l;
  for (long long e = rank * (long long)kQrThreads + threadIdx.x; e < total; e += (long long)P * kQrThreads) {
    const int col = (int)(e / a.l), row = (int)(e % a.l);
    a.Q[(long long)col * a.ldq + row] = make_float2(row == col ? 1.f : 0.f, 0.f);
  }
  __threadfence();
  cl.sync();
  for (int k = npan - 1; k >= 0; --k) {
    const int c0 = k * kQrPanel, jb = min(kQrPanel, K - c0), r0 = c0, nr = a.l - r0;
    load_v(a.X, a.ldx, r0, nr, c0, jb, big);
    for (int e = threadIdx.x; e < kQrPanel * kQrPanel; e += kQrThreads) sh.T[e] = __ldcg(a.Tm + (long long)k * kQrPanel * kQrPanel + e);
    __syncthreads();
    // columns < c0 of Q are still unit vectors above row c0: untouched by this panel
    const int ntiles = (a.kq - c0 + kQrTile - 1) / kQrTile;
    for (int tile = rank; tile < ntiles; tile += P) {
      const int tc = c0 + tile * kQrTile, tw = min(kQrTile, a.kq - tc);
      apply_block(a.Q + (long long)tc * a.ldq + r0, a.ldq, nr, tw, jb, big, sh.T, false, At, As, W);
    }
    __threadfence();
    cl.sync();
  }
}

size_t qr_smem_bytes() {
  return sizeof(float2) * ((size_t)kQrVs + (size_t)kQrMaxRows * kQrTile + 4 * kQrTile * kQrPanel +
                            kQrTile * kQrPanel);
}

cudaError_t set_qr_attrs(const void* fn) {
  cudaError_t e = allow_dynamic_smem(fn);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return e;
}

// One cluster of `ctas` CTAs (kQrCluster .. kQrMaxCtas): the whole grid.
cudaError_t launch_qr(const void* fn, QrArgs& a, int ctas, cudaStream_t st) {
  cudaError_t e = set_qr_attrs(fn);
  if (e != cudaSuccess) return e;
  ctas = std::max(kQrCluster, std::min(ctas, kQrMaxCtas));
  void* args[] = {&a};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)ctas);
  cfg.blockDim = dim3(kQrThreads);
  cfg.dynamicSmemBytes = qr_smem_bytes();
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)ctas;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, fn, args);
}

}  // namespace

int qr_max_rows() { return kQrMaxRows; }

// CTAs of one launch (one cluster): one per 16-column tile, at least kQrCluster, at most max_ctas.
int qr_ctas(int l, int c, int max_ctas) {
  (void)l;
  const int tiles = (c + kQrTile - 1) / kQrTile;
  return std::max(kQrCluster, std::min(tiles, std::min(max_ctas, kQrMaxCtas)));
}

// The largest cluster of both kernels that the device can hold (kQrMaxCtas, 8 or kQrCluster CTAs;
// 0 if none).
int qr_max_ctas() {
  const void* fns[2] = {(const void*)qr_factor_kernel, (const void*)qr_form_q_kernel};
  for (const void* fn : fns)
    if (set_qr_attrs(fn) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
  for (int n : {kQrMaxCtas, 8, kQrCluster}) {
    bool fits = true;
    for (const void* fn : fns) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)n);
      cfg.blockDim = dim3(kQrThreads);
      cfg.dynamicSmemBytes = qr_smem_bytes();
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = (unsigned)n;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      int clusters = 0;
      if (cudaOccupancyMaxActiveClusters(&clusters, fn, &cfg) != cudaSuccess || clusters < 1) {
        cudaGetLastError();
        fits = false;
      }
    }
    if (fits) return n;
  }
  return 0;
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
