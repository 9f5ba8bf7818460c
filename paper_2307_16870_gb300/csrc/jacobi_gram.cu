// Block one-sided Jacobi SVD of the two-site matrix ("Truncation fidelity" section: the bond is cut
// from the SVD of the contraction of the two tensors around it), spread over the whole GPU.
//
// Design (sm_103a, complex64):
//  * The c columns form nb blocks of 16.  A sweep is an odd-even transposition tournament over the
//    blocks: in even rounds slot i hosts the block positions (2i, 2i+1), in odd rounds (2i+1, 2i+2)
//    (the last slot idles with the two end positions), and the two hosted blocks swap positions
//    after their round.  Every pair of blocks then meets exactly once per sweep, and a slot sends
//    one block and receives one block per round, alternately to and from its two ring neighbours.
//  * A slot (32 columns) is one thread-block cluster of R CTAs; CTA r keeps rows [r MR, (r+1) MR)
//    of the slot's columns in shared memory.
//  * Per round the slot's 32 x 32 Gram matrix is formed from each CTA's rows (register-tiled
//    products from shared memory, FP32) and summed over the cluster through distributed shared
//    memory (reduce-scatter, all-gather), so that every CTA of the slot holds the same matrix.  The
//    Jacobi steps of the round then run on that matrix (four warps): each step's rotation parameters
//    come from its entries, the matrix is updated as G <- J^H G J, and the threads that produce the
//    next step's inner products also produce its rotations, so a step costs one CTA barrier.  The
//    other four warps apply each step's rotations to the rows one step behind.  Rounds take the 16
//    steps of 16 pairs that pair every column of one block with every column of the other; the
//    first round of a sweep takes the 31 steps of a 32-player round robin, which adds the pairs
//    inside each block.
//  * A Jacobi rotation updates Gram entries with the relative accuracy of freshly computed inner
//    products.  The first round of a sweep recomputes the whole matrix from the rows; the other
//    rounds recompute the block of inner products between the two blocks and the column norms, and
//    keep each block's own 16 x 16 Gram matrix from the algebra (it travels with the block).
//  * Blocks move between slots through global memory (L2) with release/acquire flags; one counter
//    barrier per sweep collects the rotation count that decides convergence.  Every wait is bounded
//    by a wall-clock deadline; a CTA that gives up records ST_TIMEOUT, and the CTAs of a cluster
//    agree on leaving at their next cluster barrier, so no CTA waits at a barrier its peers left.
#include <cooperative_groups.h>

#include <algorithm>
#include <cfloat>
#include <cmath>

#include "kernels.h"

namespace cg = cooperative_groups;

namespace eamps {

namespace {

constexpr int kBW = 16;          // columns per block
constexpr int kNE = 544;         // Gram entries summed over the cluster: 136 tiles of 2 x 2 (full
                                 // matrix) or 64 cross tiles of 2 x 2 and 32 norms (288)
constexpr int kNX = 288;
constexpr int kXLD = 34;         // row stride (complex) of the row tile in shared memory
constexpr int kGLD = 33;         // row stride (complex) of the Gram matrix in shared memory
constexpr int kThreads = 256;

struct GArgs {
  float2* X; long long ldx; int l; int c;
  float2* W; long long ldw;
  int nb; int S; int R; int mr;
  int max_sweeps; float tol;
  float tol_stop;     // a sweep whose largest pair cosine is at most this ends the iteration
  DevCtrl* ctrl;
  float2* xbuf;       // [S][2 directions][R][mr rows x 16 columns, then the block's 16 x 16 Gram]
  unsigned* flags;    // [S][2][R] release flags, then [S][2][R] block ids
};

struct __align__(8) Prm { float cs, sr, si, dp, dq, pad; };   // J = [[cs, s], [-conj(s), cs]], new norms

__device__ __forceinline__ void st_release_u32(unsigned* a, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(a), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* a) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
  return v;
}
__device__ __forceinline__ unsigned atom_add_release_u32(unsigned* a, unsigned v) {
  unsigned old;
  asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(a), "r"(v) : "memory");
  return old;
}

// One thread: wait until *a >= target or the deadline passes (false, ST_TIMEOUT recorded), or
// another waiter of the library has already given up.
__device__ bool wait_geq(const unsigned* a, unsigned target, DevCtrl* ctrl) {
  const unsigned long long end = wait_deadline(ctrl);
  int polls = 0;
  while (ld_acquire_u32(a) < target) {
    if (++polls > 32) __nanosleep(32);
    if ((*(volatile int*)&ctrl->status & ST_TIMEOUT) || global_ns() > end) {
      atomicOr(&ctrl->status, ST_TIMEOUT);
      return false;
    }
  }
  return true;
}

// Members (p, q) of pair u at step t: the 31-step round robin of 32 players (positions u and
// 31 - u; position 0 keeps player 0) or the 16-step cross sequence (column u of the first block
// with column (u + t) mod 16 of the second).
__device__ __forceinline__ void pair_members(bool rr, int t, int u, int& p, int& q) {
  if (rr) {
    p = (u == 0) ? 0 : ((u - 1 + t) % 31) + 1;
    q = ((30 - u + t) % 31) + 1;
  } else {
    p = u;
    q = kBW + ((u + t) & 15);
  }
}
// Pair index, partner and role (0: first member p, 1: second member q) of column j at step t.
__device__ __forceinline__ void column_pair(bool rr, int t, int j, int& u, int& partner, int& role) {
  if (rr) {
    const int pos = (j == 0) ? 0 : ((j - 1 + 31 - t) % 31) + 1;
    const int pp = 31 - pos;
    partner = (pp == 0) ? 0 : ((pp - 1 + t) % 31) + 1;
    if (pos < 16) { u = pos; role = 0; } else { u = pp; role = 1; }
  } else if (j < kBW) {
    u = j; role = 0; partner = kBW + ((j + t) & 15);
  } else {
    u = (j - kBW - t) & 15; role = 1; partner = u;
  }
}

// Rotation of columns with squared norms a, b and inner product g = <x_p, x_q> that makes them
// orthogonal, and the norms after it (the larger one grows by 2|g|^2 / D, the smaller one shrinks by
// as much: no cancellation).  Identity when the pair is orthogonal to the tolerance.
__device__ __forceinline__ Prm make_prm(float a, float b, float2 g, float tol, float tol_stop, int& rot, int& big) {
  Prm P;
  P.cs = 1.f; P.sr = 0.f; P.si = 0.f; P.dp = a; P.dq = b; P.pad = 0.f;
  const float g2 = g.x * g.x + g.y * g.y;
  if (!(a > 0.f) || !(b > 0.f) || !(g2 > tol * tol * a * b)) return P;
  const float u = b - a;
  const float x = fmaf(u, u, 4.f * g2);
  const float h = x * rsqrtf(x);
  const float D = fabsf(u) + h;
  const float r = rsqrtf(fmaf(D, D, 4.f * g2));
  const float s2 = (u >= 0.f) ? 2.f * r : -2.f * r;
  P.cs = D * r;
  P.sr = s2 * g.x;
  P.si = s2 * g.y;
  big += (g2 > tol_stop * tol_stop * a * b) ? 1 : 0;
  const float del = __fdividef(2.f * g2, D);
  if (u >= 0.f) { P.dp = a - del; P.dq = b + del; }
  else { P.dp = a + del; P.dq = b - del; }
  ++rot;
  return P;
}

// Row i of the stacked matrix [X; W] in column col (zero outside).
__device__ __forceinline__ float2 load_elem(const GArgs& p, int col, int v) {
  if (col >= p.c) return make_float2(0.f, 0.f);
  if (v < p.l) return __ldcg(p.X + (long long)col * p.ldx + v);
  if (p.W && v < p.l + p.c) return __ldcg(p.W + (long long)col * p.ldw + (v - p.l));
  return make_float2(0.f, 0.f);
}
__device__ __forceinline__ void store_elem(const GArgs& p, int col, int v, float2 z) {
  if (col >= p.c) return;
  if (v < p.l) __stcg(p.X + (long long)col * p.ldx + v, z);
  else if (p.W && v < p.l + p.c) __stcg(p.W + (long long)col * p.ldw + (v - p.l), z);
}

// The Gram matrix keeps entry (i, j) once, at [min][max] (the conjugate for i > j), and the norms
// on the diagonal.
__device__ __forceinline__ float2 gget(const float2* G, int i, int j) {
  const float2 v = G[min(i, j) * kGLD + max(i, j)];
  return (i <= j) ? v : make_float2(v.x, -v.y);
}
__device__ __forceinline__ void gput(float2* G, int i, int j, float2 v) {
  G[min(i, j) * kGLD + max(i, j)] = (i <= j) ? v : make_float2(v.x, -v.y);
}

// Members of 2 x 2 tile t of the upper triangle of a 16 x 16 tile grid (ti <= tj).
__device__ __forceinline__ void upper_tile(int t, int& ti, int& tj) {
  ti = 0;
  while (t >= 16 - ti) { t -= 16 - ti; ++ti; }
  tj = ti + t;
}

template <int MR>
__global__ void __launch_bounds__(kThreads) jacobi_gram_kernel(GArgs p) {
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* Xs = reinterpret_cast<float2*>(smem_raw);         // [MR][kXLD] rows of the slot's 32 columns
  float2* G = Xs + MR * kXLD;                                // [32][kGLD] Gram matrix
  float2* part = G + 32 * kGLD;                              // [4 row groups][kNE] partial sums
  float2* pbuf = part + 4 * kNE;                             // [kNE] this CTA's partial (cluster-read)
  float2* rbuf = pbuf + kNE;                                 // [kNE] reduce-scattered sums (cluster-read)
  Prm* ring = reinterpret_cast<Prm*>(rbuf + kNE);            // [3][16] rotations of consecutive steps
  __shared__ int hdr[4];                                     // [2] abort words, [2] sweep decisions
  __shared__ unsigned rot_s, big_s;
  __shared__ int ok_s, blk_s;

  const int R = p.R, S = p.S, nb = p.nb;
  const int rank = (int)cl.block_rank();
  const int slot = (int)blockIdx.x / R;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int rowbase = rank * MR;
  const int lrows = max(0, min(MR, p.l - rowbase));   // rows of X (inner products); the rest is W or zero
  const int nctas = S * R;
  // off-diagonal 2 x 2 block (bu < bv) of the Gram update owned by algebra thread tid < 120
  int bu = 0, bv = 1;
  {
    int t = tid;
    while (bu < 15 && t >= 15 - bu) { t -= 15 - bu; ++bu; }
    bv = bu + 1 + t;
  }

  int pos0 = 2 * slot, pos1 = 2 * slot + 1;   // tournament positions of the blocks in columns 0-15, 16-31
  int blk0 = 2 * slot, blk1 = 2 * slot + 1;   // block ids in columns 0-15, 16-31
  for (int e = tid; e < MR * 32; e += kThreads) {
    const int r = e >> 5, j = e & 31;
    Xs[r * kXLD + j] = load_elem(p, ((j < kBW) ? blk0 : blk1) * kBW + (j & 15), rowbase + r);
  }

  int my_rot = 0, my_big = 0;   // rotations decided by this thread, those above tol_stop
  // failure self-test: slot 0's first CTA withholds its releases, so its neighbour's wait runs out
  const bool withhold = blockIdx.x == 0 && *(volatile const int*)&p.ctrl->test_fault == 2;
  int local_abort = 0;
  unsigned long long rot_total = 0;
  bool converged = false, aborted = false;
  unsigned gr = 0;
  int sweep = 0;
  if (tid == 0) { rot_s = 0; big_s = 0; }
  __syncthreads();

  for (sweep = 0; sweep < p.max_sweeps && !aborted; ++sweep) {
    for (int r = 0; r < nb; ++r, ++gr) {
      const int typ = r & 1;
      const bool active = (typ == 0) || (slot < S - 1);
      if (active) {
        const bool rr = (r == 0);
        const int E = rr ? kNE : kNX;
        // ---- (1) this CTA's inner products, four row groups of MR / 4 rows
        {
          constexpr int Q4 = MR / 4;
          const int ntask = rr ? 4 * 136 : 4 * 64;
          for (int task = tid; task < ntask; task += kThreads) {
            const int tile = rr ? task % 136 : task & 63, grp = rr ? task / 136 : task >> 6;
            int ci, cj;
            if (rr) {
              int ti, tj;
              upper_tile(tile, ti, tj);
              ci = 2 * ti; cj = 2 * tj;
            } else {
              ci = 2 * (tile >> 3); cj = kBW + 2 * (tile & 7);
            }
            float2 a00 = make_float2(0.f, 0.f), a01 = a00, a10 = a00, a11 = a00;
            const int r0 = grp * Q4, r1 = min(r0 + Q4, lrows);
            for (int row = r0; row < r1; ++row) {
              const float4 xa = *reinterpret_cast<const float4*>(Xs + row * kXLD + ci);
              const float4 xb = *reinterpret_cast<const float4*>(Xs + row * kXLD + cj);
              // conj(a) b
              a00.x = fmaf(xa.x, xb.x, fmaf(xa.y, xb.y, a00.x)); a00.y = fmaf(xa.x, xb.y, fmaf(-xa.y, xb.x, a00.y));
              a01.x = fmaf(xa.x, xb.z, fmaf(xa.y, xb.w, a01.x)); a01.y = fmaf(xa.x, xb.w, fmaf(-xa.y, xb.z, a01.y));
              a10.x = fmaf(xa.z, xb.x, fmaf(xa.w, xb.y, a10.x)); a10.y = fmaf(xa.z, xb.y, fmaf(-xa.w, xb.x, a10.y));
              a11.x = fmaf(xa.z, xb.z, fmaf(xa.w, xb.w, a11.x)); a11.y = fmaf(xa.z, xb.w, fmaf(-xa.w, xb.z, a11.y));
            }
            float2* o = part + grp * kNE + tile * 4;
            o[0] = a00; o[1] = a01; o[2] = a10; o[3] = a11;
          }
          if (!rr && tid < 128) {   // squared column norms
            const int j = tid & 31, grp = tid >> 5;
            const int r0 = grp * Q4, r1 = min(r0 + Q4, lrows);
            float s = 0.f;
            for (int row = r0; row < r1; ++row) {
              const float2 v = Xs[row * kXLD + j];
              s = fmaf(v.x, v.x, fmaf(v.y, v.y, s));
            }
            part[grp * kNE + 256 + j] = make_float2(s, 0.f);
          }
        }
        __syncthreads();
        for (int e = tid; e < E; e += kThreads) {
          const float2 v0 = part[e], v1 = part[kNE + e], v2 = part[2 * kNE + e], v3 = part[3 * kNE + e];
          pbuf[e] = make_float2((v0.x + v1.x) + (v2.x + v3.x), (v0.y + v1.y) + (v2.y + v3.y));
        }
        if (tid == 0) hdr[gr & 1] = local_abort;
        cl.sync();   // (barrier 1) every partial of the round is written
        {
          int ab = 0;
          if (tid < R) ab = *cl.map_shared_rank(&hdr[gr & 1], tid);
          if (__syncthreads_or(ab)) { aborted = true; break; }   // the same decision in every CTA
        }
        // ---- (2) reduce-scatter: this CTA sums its share of the entries over the cluster
        const int chunk = (E + R - 1) / R;
        {
          const int e0 = rank * chunk, e1 = min(E, e0 + chunk);
          for (int e = e0 + tid; e < e1; e += kThreads) {
            float2 v[16];
#pragma unroll
            for (int q = 0; q < 16; ++q)
              if (q < R) v[q] = cl.map_shared_rank(pbuf, q)[e];
            float2 s = v[0];
#pragma unroll
            for (int q = 1; q < 16; ++q)
              if (q < R) { s.x += v[q].x; s.y += v[q].y; }
            rbuf[e] = s;
          }
        }
        cl.sync();   // (barrier 2) every share is summed
        // ---- (3) all-gather into the Gram matrix
        for (int e = tid; e < E; e += kThreads) {
          const float2 v = cl.map_shared_rank(rbuf, e / chunk)[e];
          if (!rr && e >= 256) {
            const int j = e - 256;
            G[j * kGLD + j] = v;
          } else {
            const int tile = e >> 2, loc = e & 3;
            int i, j;
            if (rr) {
              int ti, tj;
              upper_tile(tile, ti, tj);
              i = 2 * ti + (loc >> 1); j = 2 * tj + (loc & 1);
            } else {
              i = 2 * (tile >> 3) + (loc >> 1); j = kBW + 2 * (tile & 7) + (loc & 1);
            }
            if (i == j) G[i * kGLD + i] = make_float2(v.x, 0.f);
            else if (i < j) G[i * kGLD + j] = v;
          }
        }
        __syncthreads();
        if (rank == 0 && tid < 32 && !isfinite(G[tid * kGLD + tid].x)) atomicOr(&p.ctrl->status, ST_NONFINITE);
        // ---- (4) Jacobi steps: algebra (warps 0-3) on step t, rows (warps 4-7) on step t - 1
        const int nsteps = rr ? 31 : 16;
        if (tid < 16) {
          int pp, qq;
          pair_members(rr, 0, tid, pp, qq);
          ring[tid] = make_prm(G[pp * kGLD + pp].x, G[qq * kGLD + qq].x, gget(G, pp, qq), p.tol, p.tol_stop, my_rot,
                               my_big);
        }
        __syncthreads();
        for (int t = 0; t <= nsteps; ++t) {
          if (warp < 4) {
            if (t < nsteps) {
              const Prm* cur = ring + (t % 3) * 16;
              Prm* nxt = ring + ((t + 1) % 3) * 16;
              if (tid < 16) {   // diagonal blocks: the new norms, the pair's inner product annihilated
                int a, b;
                pair_members(rr, t, tid, a, b);
                const Prm P = cur[tid];
                G[a * kGLD + a] = make_float2(P.dp, 0.f);
                G[b * kGLD + b] = make_float2(P.dq, 0.f);
                gput(G, a, b, make_float2(0.f, 0.f));
              }
              if (tid < 120) {
                int a, b, c, d;
                pair_members(rr, t, bu, a, b);
                pair_members(rr, t, bv, c, d);
                const Prm Pu = cur[bu], Pv = cur[bv];
                const float2 ac = gget(G, a, c), ad = gget(G, a, d), bc = gget(G, b, c), bd = gget(G, b, d);
                // right factor J_v: (x, y) -> (cs x - conj(s) y, s x + cs y) on each row
                float2 r0c, r0d, r1c, r1d;
                r0c.x = Pv.cs * ac.x - (Pv.sr * ad.x + Pv.si * ad.y);
                r0c.y = Pv.cs * ac.y - (Pv.sr * ad.y - Pv.si * ad.x);
                r0d.x = (Pv.sr * ac.x - Pv.si * ac.y) + Pv.cs * ad.x;
                r0d.y = (Pv.sr * ac.y + Pv.si * ac.x) + Pv.cs * ad.y;
                r1c.x = Pv.cs * bc.x - (Pv.sr * bd.x + Pv.si * bd.y);
                r1c.y = Pv.cs * bc.y - (Pv.sr * bd.y - Pv.si * bd.x);
                r1d.x = (Pv.sr * bc.x - Pv.si * bc.y) + Pv.cs * bd.x;
                r1d.y = (Pv.sr * bc.y + Pv.si * bc.x) + Pv.cs * bd.y;
                // left factor J_u^H: rows (r0, r1) -> (cs r0 - s r1, conj(s) r0 + cs r1)
                float2 nac, nad, nbc, nbd;
                nac.x = Pu.cs * r0c.x - (Pu.sr * r1c.x - Pu.si * r1c.y);
                nac.y = Pu.cs * r0c.y - (Pu.sr * r1c.y + Pu.si * r1c.x);
                nad.x = Pu.cs * r0d.x - (Pu.sr * r1d.x - Pu.si * r1d.y);
                nad.y = Pu.cs * r0d.y - (Pu.sr * r1d.y + Pu.si * r1d.x);
                nbc.x = (Pu.sr * r0c.x + Pu.si * r0c.y) + Pu.cs * r1c.x;
                nbc.y = (Pu.sr * r0c.y - Pu.si * r0c.x) + Pu.cs * r1c.y;
                nbd.x = (Pu.sr * r0d.x + Pu.si * r0d.y) + Pu.cs * r1d.x;
                nbd.y = (Pu.sr * r0d.y - Pu.si * r0d.x) + Pu.cs * r1d.y;
                // rotations of the next step whose inner product lies in this block
                if (t + 1 < nsteps) {
#pragma unroll
                  for (int h = 0; h < 2; ++h) {
                    const int i = h ? b : a;
                    int u2, pt, role2;
                    column_pair(rr, t + 1, i, u2, pt, role2);
                    if (pt == c || pt == d) {
                      const float di = h ? Pu.dq : Pu.dp;
                      const float dj = (pt == c) ? Pv.dp : Pv.dq;
                      const float2 gij = h ? ((pt == c) ? nbc : nbd) : ((pt == c) ? nac : nad);
                      nxt[u2] = role2 == 0
                                    ? make_prm(di, dj, gij, p.tol, p.tol_stop, my_rot, my_big)
                                    : make_prm(dj, di, make_float2(gij.x, -gij.y), p.tol, p.tol_stop, my_rot, my_big);
                    }
                  }
                }
                gput(G, a, c, nac);
                gput(G, a, d, nad);
                gput(G, b, c, nbc);
                gput(G, b, d, nbd);
              }
            }
          } else if (t >= 1) {   // rows: x_p' = cs x_p - conj(s) x_q, x_q' = s x_p + cs x_q
            const int u = (tid - 128) & 15, r0 = (tid - 128) >> 4;
            int pp, qq;
            pair_members(rr, t - 1, u, pp, qq);
            const Prm P = ring[((t - 1) % 3) * 16 + u];
            constexpr int NR = MR / 8;             // rows r0, r0 + 8, ... of this thread
            constexpr int NC = NR < 8 ? NR : 8;    // rows in flight
#pragma unroll 1
            for (int k0 = 0; k0 < NR; k0 += NC) {
              float2 xp[NC], xq[NC];
#pragma unroll
              for (int k = 0; k < NC; ++k) {
                xp[k] = Xs[(r0 + 8 * (k0 + k)) * kXLD + pp];
                xq[k] = Xs[(r0 + 8 * (k0 + k)) * kXLD + qq];
              }
#pragma unroll
              for (int k = 0; k < NC; ++k) {
                float2 np, nq;
                np.x = P.cs * xp[k].x - (P.sr * xq[k].x + P.si * xq[k].y);
                np.y = P.cs * xp[k].y - (P.sr * xq[k].y - P.si * xq[k].x);
                nq.x = (P.sr * xp[k].x - P.si * xp[k].y) + P.cs * xq[k].x;
                nq.y = (P.sr * xp[k].y + P.si * xp[k].x) + P.cs * xq[k].y;
                Xs[(r0 + 8 * (k0 + k)) * kXLD + pp] = np;
                Xs[(r0 + 8 * (k0 + k)) * kXLD + qq] = nq;
              }
            }
          }
          __syncthreads();
        }
        // the two hosted blocks swap tournament positions
        const int tp = pos0; pos0 = pos1; pos1 = tp;
      }
      // ---- (5) exchange: one block (its rows and its own Gram matrix) leaves for a ring neighbour
      if (S > 1) {
        int h, dir, from, inpos;
        if (typ == 0) {
          h = (pos0 == 2 * slot) ? 0 : 1;
          dir = 0;
          from = (slot + 1) % S;
          inpos = (slot < S - 1) ? 2 * slot + 2 : 0;
        } else {
          const int outpos = (slot < S - 1) ? 2 * slot + 2 : 0;
          h = (pos0 == outpos) ? 0 : 1;
          dir = 1;
          from = (slot + S - 1) % S;
          inpos = 2 * slot;
        }
        const long long blk_elems = (long long)MR * kBW + 256;
        float2* out = p.xbuf + (long long)((slot * 2 + dir) * R + rank) * blk_elems;
        const int c0 = h * kBW;
        for (int e = tid; e < MR * kBW; e += kThreads) __stcg(out + e, Xs[(e >> 4) * kXLD + c0 + (e & 15)]);
        __stcg(out + MR * kBW + tid, G[(c0 + (tid >> 4)) * kGLD + c0 + (tid & 15)]);
        unsigned* fl = p.flags;
        unsigned* ids = p.flags + 2 * nctas;
        if (tid == 0) __stcg(ids + (slot * 2 + dir) * R + rank, (unsigned)(h ? blk1 : blk0));
        __syncthreads();
        if (tid == 0) {
          __threadfence();
          if (!withhold) st_release_u32(fl + (slot * 2 + dir) * R + rank, gr + 1);
          int ok = 1;
          if (!local_abort) ok = wait_geq(fl + (from * 2 + dir) * R + rank, gr + 1, p.ctrl);
          ok_s = ok && !local_abort;
          blk_s = ok_s ? (int)__ldcg(ids + (from * 2 + dir) * R + rank) : (h ? blk1 : blk0);
        }
        __syncthreads();
        if (ok_s) {
          const float2* in = p.xbuf + (long long)((from * 2 + dir) * R + rank) * blk_elems;
          for (int e = tid; e < MR * kBW; e += kThreads) Xs[(e >> 4) * kXLD + c0 + (e & 15)] = __ldcg(in + e);
          G[(c0 + (tid >> 4)) * kGLD + c0 + (tid & 15)] = __ldcg(in + MR * kBW + tid);
        } else {
          local_abort = 1;
        }
        if (h) { blk1 = blk_s; pos1 = inpos; } else { blk0 = blk_s; pos0 = inpos; }
        __syncthreads();
      }
    }
    if (aborted) break;
    // ---- convergence vote: rotation count of every slot (rank 0 of each cluster), one counter barrier
    if (my_rot) atomicAdd(&rot_s, (unsigned)my_rot);
    if (my_big) atomicAdd(&big_s, (unsigned)my_big);
    my_rot = 0;
    my_big = 0;
    __syncthreads();
    if (tid == 0) {
      int decision = 0;   // 0: continue, 1: converged, 2: leave
      const unsigned mine = big_s;
      rot_total += rot_s;
      rot_s = 0;
      big_s = 0;
      if (nctas > 1) {
        if (rank == 0) atomicAdd(&p.ctrl->rot[sweep % 3], mine);
        const unsigned old = atom_add_release_u32(&p.ctrl->bar_count, 1u);
        const unsigned target = (old / (unsigned)nctas + 1u) * (unsigned)nctas;
        if (local_abort || !wait_geq(&p.ctrl->bar_count, target, p.ctrl)) {
          decision = 2;
        } else {
          const unsigned total = ld_acquire_u32(&p.ctrl->rot[sweep % 3]);
          if (blockIdx.x == 0) p.ctrl->rot[(sweep + 2) % 3] = 0u;
          decision = (total == 0u) ? 1 : 0;
        }
      } else {
        decision = (mine == 0u) ? 1 : 0;
      }
      hdr[2 + (sweep & 1)] = decision;
    }
    cl.sync();   // every CTA of the cluster has its decision
    {
      int dmax = 0;
      if (tid < R) dmax = *cl.map_shared_rank(&hdr[2 + (sweep & 1)], tid);
      // any CTA leaving makes the cluster leave; otherwise every CTA read the same total
      const int leave = __syncthreads_or(dmax == 2);
      const int conv = __syncthreads_or(dmax == 1);
      if (leave) { aborted = true; break; }
      if (conv) { converged = true; break; }
    }
  }
  if (!aborted) {
    for (int e = tid; e < MR * 32; e += kThreads) {
      const int r = e >> 5, j = e & 31;
      store_elem(p, ((j < kBW) ? blk0 : blk1) * kBW + (j & 15), rowbase + r, Xs[r * kXLD + j]);
    }
  }
  if (tid == 0 && rank == 0) {
    // algorithmic flops of the one-sided iteration: 24 L per rotation (two complex column
    // updates of length L), 16 l per visited pair (three complex inner products)
    const double L = (double)p.l + (p.W ? (double)p.c : 0.0);
    atomicAdd(&p.ctrl->jac_flops, 24.0 * L * (double)rot_total);
    if (blockIdx.x == 0) {
      const int used = converged ? sweep + 1 : sweep;
      p.ctrl->sweeps = used;
      atomicAdd(&p.ctrl->jac_sweeps, (unsigned long long)used);
      atomicAdd(&p.ctrl->jac_flops, 16.0 * (double)p.l * 0.5 * (double)p.c * (double)(p.c - 1) * (double)used);
      if (!converged && !aborted) atomicOr(&p.ctrl->status, ST_NOT_CONVERGED);
    }
  }
  cl.sync();   // no CTA leaves while its peers may still read its shared memory
}

struct GVariant { int mr; const void* fn; };
#define EAMPS_G(MR) {MR, (const void*)jacobi_gram_kernel<MR>}
const GVariant kGramVariants[] = {EAMPS_G(16), EAMPS_G(32), EAMPS_G(64), EAMPS_G(128), EAMPS_G(256)};
#undef EAMPS_G

// Dynamic shared memory of a CTA: at least 116 KB, so that no two CTAs of the launch share an SM
// (a CTA that shares its SM would set the pace of the whole tournament).
size_t gram_smem(int mr) {
  const size_t need = sizeof(float2) * ((size_t)mr * kXLD + 32 * kGLD + 6 * (size_t)kNE) + sizeof(Prm) * 48;
  return std::max<size_t>(need, 116 * 1024);
}

// Clusters of `R` CTAs of kernel `fn` that can be resident at once (0 on error).
int gram_max_clusters(const void* fn, int R, int mr) {
  if (allow_dynamic_smem(fn) != cudaSuccess) return 0;
  if (R > 8 && cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) return 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(R);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = gram_smem(mr);
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = R;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

}  // namespace

bool jacobi_gram_plan(int l, int c, bool accumulate, int max_ctas, JacobiPlan& plan) {
  const int L = l + (accumulate ? c : 0);
  int nb = (c + kBW - 1) / kBW;
  nb += nb & 1;
  const int S = nb / 2;
  if (S < 2) return false;
  for (int R : {16, 8, 4, 2}) {
    if (S * R > max_ctas) continue;
    const int need = (L + R - 1) / R;
    const GVariant* v = nullptr;
    for (const GVariant& g : kGramVariants)
      if (g.mr >= need) { v = &g; break; }
    if (!v) continue;
    const int fit = gram_max_clusters(v->fn, R, v->mr);
    if (fit < S) continue;
    plan = JacobiPlan();
    plan.w = kBW;
    plan.nb = nb;
    plan.smem = gram_smem(v->mr);
    plan.fn = v->fn;
    plan.threads = kThreads;
    plan.gram_R = R;
    plan.gram_mr = v->mr;
    plan.ld = 0;
    return true;
  }
  return false;
}

cudaError_t jacobi_gram_launch(const JacobiPlan& plan, float2* X, long long ldx, int l, int c, float2* W,
                               long long ldw, int max_sweeps, DevCtrl* ctrl, float2* xch, size_t xch_cap,
                               unsigned* flags, int flags_cap, cudaStream_t st) {
  const int S = plan.nb / 2, R = plan.gram_R;
  if ((size_t)S * 2 * R * ((size_t)plan.gram_mr * kBW + 256) > xch_cap || 4 * S * R > flags_cap)
    return cudaErrorInvalidValue;
  cudaError_t e = allow_dynamic_smem(plan.fn);
  if (e != cudaSuccess) return e;
  if (R > 8) {
    e = cudaFuncSetAttribute(plan.fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  e = cudaMemsetAsync(&ctrl->bar_count, 0, 5 * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(flags, 0, sizeof(unsigned) * 4 * S * R, st);
  if (e != cudaSuccess) return e;
  GArgs a;
  a.X = X; a.ldx = ldx; a.l = l; a.c = c; a.W = W; a.ldw = ldw;
  a.nb = plan.nb; a.S = S; a.R = R; a.mr = plan.gram_mr;
  a.max_sweeps = max_sweeps;
  a.tol = 4.f * std::sqrt((float)std::max(l, 1)) * FLT_EPSILON;
  a.tol_stop = plan.early_stop ? std::sqrt(a.tol) : a.tol;   // as the tournament kernels
  a.ctrl = ctrl;
  a.xbuf = xch;
  a.flags = flags;
  void* args[] = {&a};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(S * R);
  cfg.blockDim = dim3(plan.threads);
  cfg.dynamicSmemBytes = plan.smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = R;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  // every CTA waits on others: ask for a cooperative (co-resident) launch where the runtime
  // accepts one together with clusters; the plan has already checked residency
  attr[1].id = cudaLaunchAttributeCooperative;
  attr[1].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  e = cudaLaunchKernelExC(&cfg, plan.fn, args);
  if (e == cudaErrorInvalidValue || e == cudaErrorNotSupported || e == cudaErrorCooperativeLaunchTooLarge) {
    cudaGetLastError();
    cfg.numAttrs = 1;
    e = cudaLaunchKernelExC(&cfg, plan.fn, args);
  }
  return e;
}

}  // namespace eamps
