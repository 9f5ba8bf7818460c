// C ABI of the entanglement-aware MPS / MPO library and the host-side
// orchestration of the two-site update.  Every numerical step runs in the
// device kernels of this directory; the host plans launches, tracks the bond
// sizes it reads back after each truncation, and marshals arguments.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstddef>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <numeric>
#include <thread>
#include <type_traits>
#include <vector>

#include "eamps.h"
#include "gemm_tc.h"
#include "kernels.h"

using namespace eamps;

namespace {

constexpr int kDefaultCap = 1024;

// Co-resident CTAs of multi-CTA Jacobi launches (cooperative grids whose CTAs wait on one
// another, and clusters) on one device, shared by every handle that runs in a batch.  A
// handle holds CTAs from before such a launch until its next stream synchronisation; a
// handle that needs more than it holds first synchronises and returns what it holds, so a
// waiting handle never holds any and concurrent grids never exceed the device.
struct CoopBudget {
  std::mutex m;
  std::condition_variable cv;
  int free_ctas = -1;
  void acquire(int n, int capacity) {
    std::unique_lock<std::mutex> lk(m);
    if (free_ctas < 0) free_ctas = capacity;
    n = std::min(n, capacity);
    cv.wait(lk, [&] { return free_ctas >= n; });
    free_ctas -= n;
  }
  void release(int n) {
    {
      std::lock_guard<std::mutex> lk(m);
      free_ctas += n;
    }
    cv.notify_all();
  }
};

CoopBudget& coop_budget(int device) {
  static CoopBudget budgets[64];
  return budgets[device & 63];
}

// Per-truncation target of the schedule (Eq. uniform, Fig. 1) before the truncation that follows
// n_done truncations with running product `product`; the formula of the selection kernel.
double schedule_target(int strategy, double f_min, long long n_2q, long long n_done, double product) {
  if (f_min >= 1.0 || product < f_min) return 1.0;
  const long long rem = std::max<long long>(n_2q - n_done, 1);
  const double f0 = (f_min < 1.0 && n_2q > 0) ? std::pow(f_min, 1.0 / (double)n_2q) : 1.0;
  double ft;
  if (strategy == MPS_NAIVE) ft = f0;
  else if (strategy == MPS_GLOBAL) ft = std::pow(f_min / product, 1.0 / (double)rem);
  else ft = f_min / (product * std::pow(f0, (double)(rem - 1)));
  return std::min(ft, 1.0);
}

// ---------------------------------------------------------------- Jacobi layout autotuner
// The first time a handle meets a shape class (rows and columns rounded up to kTuneGrain,
// accumulation) with at least kTuneMinCols columns under MPS_SVD_AUTO, it times the layouts of the
// one-sided Jacobi (the tournament kernels with and without the row split, and the Gram-matrix
// block kernel) on copies of the matrix it is about to decompose and keeps the fastest for the
// process (the block kernel only when at least 10 % faster, so that near ties do not flip between
// runs).  Every later SVD of that class runs the chosen layout.  The classes keep the number of
// timing runs small on circuits whose bonds take many values.  (A synthetic matrix, the first
// form of this tuner, picked the unsplit tournament at 512 columns, 12-21 % faster there, while
// the split form is about 3 % faster on the benchmark's own matrices.)
constexpr int kTuneMinCols = 256;
// The QR-preconditioned gate SVD from this many columns of the Jacobi's matrix on (below it the
// QR's fixed latency outweighs the sweeps it saves).
constexpr int kPrecondMinCols = 256;
constexpr int kTuneGrain = 64;
struct TuneKey {
  int dev, l, c, acc;   // l, c: upper bounds of the class
  bool operator<(const TuneKey& o) const {
    if (dev != o.dev) return dev < o.dev;
    if (l != o.l) return l < o.l;
    if (c != o.c) return c < o.c;
    return acc < o.acc;
  }
};
struct TuneEntry {
  int kind;
  double ms_tournament, ms_gram, ms_unsplit;
};
std::mutex& tune_mutex() {
  static std::mutex m;
  return m;
}
std::map<TuneKey, TuneEntry>& tune_table() {
  static std::map<TuneKey, TuneEntry> t;
  return t;
}

// Deterministic synthetic matrix for the timing runs: entries uniform in [-1, 1) from a hash of
// the index (the values only set the Jacobi's sweep count, as a random matrix does).
__global__ void synthetic_fill_kernel(float2* __restrict__ x, long long n, unsigned seed) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    unsigned long long h = (unsigned long long)i * 0x9E3779B97F4A7C15ull + seed;
    h ^= h >> 31; h *= 0xBF58476D1CE4E5B9ull; h ^= h >> 29; h *= 0x94D049BB133111EBull; h ^= h >> 32;
    x[i] = make_float2((float)(h & 0xFFFFFF) / 8388608.f - 1.f, (float)((h >> 24) & 0xFFFFFF) / 8388608.f - 1.f);
  }
}

mps_status from_bits(int bits) {
  if (bits & ST_TIMEOUT) return MPS_ERR_TIMEOUT;
  if (bits & ST_NONFINITE) return MPS_ERR_NONFINITE;
  if (bits & ST_NOT_CONVERGED) return MPS_ERR_NOT_CONVERGED;
  if (bits & ST_BAD_ARG) return MPS_ERR_ARG;
  return MPS_OK;
}

// Superoperator of the channel {K} in the vectorisation t = 2 s + s' per qubit, qubit 0 major:
// S[(t..),(u..)] = sum_K K[(s..),(r..)] conj(K[(s'..),(r'..)]).
void superop_from_kraus_host(const double* kraus, int n_kraus, int nq, double* out) {
  const int dim = 1 << nq;
  const int D = dim * dim;
  std::memset(out, 0, sizeof(double) * 2 * D * D);
  for (int kk = 0; kk < n_kraus; ++kk) {
    const double* K = kraus + (size_t)kk * 2 * dim * dim;
    for (int s = 0; s < dim; ++s)
      for (int sp = 0; sp < dim; ++sp)
        for (int r = 0; r < dim; ++r)
          for (int rp = 0; rp < dim; ++rp) {
            const double ar = K[2 * (s * dim + r)], ai = K[2 * (s * dim + r) + 1];
            const double br = K[2 * (sp * dim + rp)], bi = -K[2 * (sp * dim + rp) + 1];
            const double vr = ar * br - ai * bi, vi = ar * bi + ai * br;
            int t = 0, u = 0;
            for (int qb = 0; qb < nq; ++qb) {
              const int sh = nq - 1 - qb;
              t = t * 4 + 2 * ((s >> sh) & 1) + ((sp >> sh) & 1);
              u = u * 4 + 2 * ((r >> sh) & 1) + ((rp >> sh) & 1);
            }
            out[2 * (t * D + u)] += vr;
            out[2 * (t * D + u) + 1] += vi;
          }
  }
}

}  // namespace

struct mps_state {
  virtual ~mps_state() {}
  virtual mps_status apply_1q(int q, const double* op, int op_dim) = 0;
  virtual mps_status apply_2q(int q, const double* op, bool on_device, int op_dim, double target) = 0;
  virtual mps_status fidelity(double* out) = 0;
  virtual mps_status expect(int q, int support, const double* op, double* out) = 0;
  virtual mps_status amplitude(const unsigned char* bits, double* out) = 0;
  virtual mps_status get_site(int i, double* out, long long cap, int* dims3) = 0;
  virtual mps_status set_site(int i, const double* data, const int* dims3) = 0;
  virtual mps_status lognorm(double* out) = 0;
  virtual mps_status last_svals(double* out, int cap, int* count) = 0;
  virtual mps_status sync() = 0;
  virtual mps_status reset() = 0;
  virtual mps_status profile(int on) = 0;
  virtual mps_status stats(mps_stats_t* out) = 0;
  virtual mps_status stats_reset() = 0;
  // site i (bonds[i] x d x bonds[i+1], row-major) converted to FP64 into dst, ordered on st
  virtual mps_status site_to_double(int i, double2* dst, cudaStream_t st) = 0;
  virtual bool is_vidal() const = 0;
  virtual mps_status apply_layer(int n, const int* qs, const double* ops_dev, int op_dim, double target,
                                 int concurrency) = 0;
  virtual mps_status gemm_device(int M, int Nn, int K, const void* A, long long a_rs, long long a_cs, int cA,
                                 const void* B, long long b_rs, long long b_cs, int cB, void* C, long long c_rs,
                                 long long c_cs) = 0;
  virtual mps_status tsvd_device(int m, int n, const void* A, long long lda, double target, int max_k,
                                 double rank_tol, void* U, double* S, void* V, void* Aq, void* Ap, double* out4) = 0;
  virtual mps_status tsvd_backward_device(int m, int n, int k, const void* U, const double* S, const void* V,
                                          const void* Aq_bar, const void* Ap_bar, double eps, void* A_bar) = 0;
  virtual mps_status selftest_timeout(int site, long long wait_ns) = 0;
  virtual mps_status svd_tune(int l, int c, int acc, int* layout) = 0;
  int N = 0;
  int d = 2;
  int centre = 0;
  std::vector<int> bonds;   // bonds[i] = left bond of site i; bonds[0] = bonds[N] = 1
  std::vector<mps_trunc_record> log;
  bool log_on = true;
  int sticky = 0;
  cudaStream_t stream = nullptr;
  bool owns_stream = false;   // stream created for this handle (batch runs); destroyed with it
  bool shared_gpu = false;    // runs beside other handles: multi-CTA launches go through the budget
  int device = 0;
  int coop_held = 0;          // CTAs held in the device budget
};

namespace {

template <class R>
struct Engine final : mps_state {
  using Z = cplx<R>;
  // Centre moves by QR: forming the explicit Q and writing the site from it run on a second
  // stream, beside the next gate (which does not touch that site; a handle that runs alone only).
  // Every later user of the QR buffers or of the sites first makes the handle's stream wait for
  // that work (join_side).
  cudaStream_t side = nullptr;
  cudaEvent_t ev_main = nullptr, ev_side = nullptr;
  Z* Xq = nullptr;      // the move's matrix, factored in place (R above the diagonal, reflectors below)
  Z* Qq = nullptr;      // its explicit Q
  Z* Tq = nullptr;      // its block-reflector factors and tau (the gate's QR has its own)
  Z* tauq = nullptr;
  bool side_pending = false;
  mps_options opt{};
  int sm_count = 1;
  int chi_cap = kDefaultCap;
  std::vector<int> cap;     // capacity of every bond
  Z* arena = nullptr;
  std::vector<Z*> site;
  Z** site_dev = nullptr;
  int* bonds_dev = nullptr;
  Z *T = nullptr, *X = nullptr, *theta = nullptr, *Wacc = nullptr, *tmp = nullptr, *tmp2 = nullptr;
  Z *G = nullptr, *O = nullptr;
  double *s_sorted = nullptr, *norms = nullptr;
  int* perm = nullptr;
  int c_max = 0;
  size_t big_cap = 0;   // elements of each two-site scratch buffer
  int last_c = 0;
  DevCtrl* ctrl = nullptr;
  DevCtrl* hctrl = nullptr;
  double2 *wdev = nullptr, *w2dev = nullptr, *work = nullptr, *outdev = nullptr, *hout = nullptr;
  double2* stage = nullptr;   // complex128 staging of one site (mps_get_site)
  Z* xch = nullptr;           // Jacobi exchange slots
  size_t xch_cap = 0;
  unsigned* jflags = nullptr; // Jacobi position flags
  static constexpr int kFlagsCap = 4096;
  size_t site_cap = 0;
  TcGemm* tc = nullptr;
  // Householder QR (complex64): centre moves and SVD preconditioning for <= qr_max_rows() rows
  Z* qr_tau = nullptr;
  Z* qr_T = nullptr;
  int qr_fit = 0;
  bool qr_on = false;
  // Vidal / Hastings form: Schmidt vector of every bond (FP64), bond b at lam + b * lam_stride
  bool vidal = false;
  double* lam = nullptr;
  int lam_stride = 0;
  bool lam_owned = true;
  // helper handles of a Vidal layer run: own scratch and stream, the sites and Schmidt vectors of
  // this handle
  std::vector<Engine*> helpers;
  int qr_mode = 2;
  // statistics
  long long n_launch = 0, n_jac = 0, n_gemm = 0, n_gates = 0, n_jac_move = 0, n_qr = 0;
  double gemm_flops = 0.0, jac_ms = 0.0, gemm_ms = 0.0, jac_move_ms = 0.0, qr_ms_sum = 0.0;
  bool in_move = false;
  bool prof = false;
  struct Timed { cudaEvent_t a, b; int kind; };
  std::vector<Timed> pending;
  std::vector<cudaEvent_t> ev_pool;

  ~Engine() override {
    for (Engine* h : helpers) delete h;
    if (side) cudaStreamSynchronize(side);
    if (stream) cudaStreamSynchronize(stream);
    coop_release();
    if (!lam_owned) lam = nullptr;
    void* bufs[] = {arena, site_dev, bonds_dev, T, X, theta, Wacc, tmp, tmp2, G, O, s_sorted, norms, perm,
                    ctrl, wdev, w2dev, work, outdev, stage, xch, jflags, qr_tau, qr_T, lam, Xq, Qq, Tq, tauq};
    for (void* b : bufs) if (b) cudaFree(b);
    if (hctrl) cudaFreeHost(hctrl);
    if (hout) cudaFreeHost(hout);
    if (tc) tc_destroy(tc);
    for (auto& t : pending) { ev_pool.push_back(t.a); ev_pool.push_back(t.b); }
    for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
    if (ev_main) cudaEventDestroy(ev_main);
    if (ev_side) cudaEventDestroy(ev_side);
    if (side) cudaStreamDestroy(side);
    if (owns_stream && stream) cudaStreamDestroy(stream);
  }

  // ------------------------------------------------------------- device budget (batch runs)
  mps_status coop_ensure(int ctas) {
    if (!shared_gpu || ctas <= 1 || ctas <= coop_held) return MPS_OK;
    if (coop_held > 0) {
      // this handle's earlier multi-CTA launches must finish before it returns their CTAs
      if (mps_status s = cu(cudaStreamSynchronize(stream))) return s;
      coop_release();
    }
    coop_budget(device).acquire(ctas, sm_count);
    coop_held = std::min(ctas, sm_count);
    return MPS_OK;
  }
  void coop_release() {
    if (coop_held > 0) coop_budget(device).release(coop_held);
    coop_held = 0;
  }

  cudaEvent_t ev_get() {
    if (!ev_pool.empty()) { cudaEvent_t e = ev_pool.back(); ev_pool.pop_back(); return e; }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  // start an event-timed region (kind 0 = Jacobi, 1 = contraction, 2 = Jacobi of a move, 3 = QR)
  // on the handle's stream (or on `on`)
  int tbegin(cudaStream_t on = nullptr) {
    if (!prof) return -1;
    Timed t{ev_get(), ev_get(), 0};
    cudaEventRecord(t.a, on ? on : stream);
    pending.push_back(t);
    return (int)pending.size() - 1;
  }
  void tend(int id, int kind, cudaStream_t on = nullptr) {
    if (id < 0) return;
    pending[id].kind = kind;
    cudaEventRecord(pending[id].b, on ? on : stream);
  }
  // the handle's stream waits for the work of the move's second stream
  mps_status join_side() {
    if (!side_pending) return MPS_OK;
    side_pending = false;
    return cu(cudaStreamWaitEvent(stream, ev_side, 0));
  }
  // after a stream synchronisation: harvest the event durations
  void harvest() {
    for (auto& t : pending) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) {
        if (t.kind == 1) gemm_ms += ms;
        else if (t.kind == 3) qr_ms_sum += ms;
        else {
          jac_ms += ms;
          if (t.kind == 2) jac_move_ms += ms;
        }
      }
      ev_pool.push_back(t.a);
      ev_pool.push_back(t.b);
    }
    pending.clear();
  }
  mps_status kl(cudaError_t e) { ++n_launch; return cu(e); }

  template <class P> bool dalloc(P** p, size_t count) {
    return cudaMalloc((void**)p, sizeof(P) * (count ? count : 1)) == cudaSuccess;
  }

  mps_status cu(cudaError_t e) {
    if (e == cudaSuccess) return MPS_OK;
    std::fprintf(stderr, "eamps: CUDA error: %s\n", cudaGetErrorString(e));
    cudaGetLastError();
    return MPS_ERR_CUDA;
  }

  // share != nullptr: a helper of a Vidal layer run, on the sites and Schmidt vectors of share
  mps_status init(int n, const mps_options& o, cudaStream_t st, const Engine* share = nullptr) {
    N = n;
    opt = o;
    stream = st;
    d = (o.kind == MPS_MIXED) ? 4 : 2;
    log_on = o.log_truncations != 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MPS_ERR_CUDA;
    device = dev;
    cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev);
    chi_cap = o.chi_max > 0 ? o.chi_max : kDefaultCap;
    if (o.fixed_chi > 0) chi_cap = std::min(chi_cap, o.fixed_chi);
    cap.assign(N + 1, 1);
    for (int b = 1; b < N; ++b) {
      const int e = std::min(b, N - b);
      long long v = 1;
      for (int i = 0; i < e && v < chi_cap; ++i) v *= d;
      cap[b] = (int)std::min<long long>(v, chi_cap);
    }
    bonds.assign(N + 1, 1);
    std::vector<size_t> off(N + 1);
    size_t total = 0, site_max = 0, pair_max = 0;
    for (int i = 0; i < N; ++i) {
      off[i] = total;
      const size_t sz = (size_t)cap[i] * d * cap[i + 1];
      site_max = std::max(site_max, sz);
      total += (sz + 31) & ~size_t(31);
    }
    for (int q = 0; q + 1 < N; ++q) {
      const size_t m = (size_t)d * cap[q], nn = (size_t)d * cap[q + 2];
      pair_max = std::max(pair_max, m * nn);
      c_max = std::max<int>(c_max, (int)std::max(m, nn));
    }
    const size_t big = std::max(pair_max, site_max);
    big_cap = big;
    if (!(share || dalloc(&arena, total)) || !dalloc(&T, big) || !dalloc(&X, big) || !dalloc(&theta, big) ||
        !dalloc(&Wacc, big) || !dalloc(&tmp, big) || !dalloc(&tmp2, big) || !dalloc(&G, 256) ||
        !dalloc(&O, 256) || !dalloc(&s_sorted, c_max) || !dalloc(&norms, c_max) || !dalloc(&perm, c_max) ||
        !dalloc(&site_dev, N) || !dalloc(&bonds_dev, N + 1) || !dalloc(&ctrl, 1) ||
        !dalloc(&wdev, (size_t)N * d) || !dalloc(&w2dev, 16) || !dalloc(&work, (size_t)(2 + d) * (chi_cap + 8)) ||
        !dalloc(&outdev, 4) || !dalloc(&stage, site_max))
      return MPS_ERR_OOM;
    // exchange slots: 2 parities x (columns + padding of one block per CTA) x column stride; the
    // stride is the longer side plus accumulated rotations, padded to 32 * (rows per lane) <= 1024
    // rows by the register-resident kernels
    xch_cap = (size_t)2 * ((size_t)c_max + 2 * 64) * (size_t)std::max(1024, 2 * c_max + 32);
    if (!dalloc(&xch, xch_cap) || !dalloc(&jflags, kFlagsCap)) return MPS_ERR_OOM;
    site_cap = site_max;
    if (cudaMallocHost((void**)&hctrl, sizeof(DevCtrl)) != cudaSuccess) return MPS_ERR_OOM;
    if (cudaMallocHost((void**)&hout, sizeof(double2) * 4) != cudaSuccess) return MPS_ERR_OOM;
    site.resize(N);
    for (int i = 0; i < N; ++i) site[i] = share ? share->site[i] : arena + off[i];
    if (!share)
      if (mps_status s = cu(cudaMemsetAsync(arena, 0, sizeof(Z) * total, stream))) return s;
    // |0> (PURE) or vec(|0><0|) (MIXED, t = 0): entry [0, 0, 0] = 1 on every site.  Every copy
    // is ordered on the handle's stream behind the memset above (a copy on the legacy default
    // stream is not ordered after work on a non-blocking stream); the final synchronisation
    // keeps the host sources alive until the copies have run.
    std::vector<Z> ones(1, mk<R>(1, 0));
    for (int i = 0; i < N && !share; ++i)
      if (mps_status s = cu(cudaMemcpyAsync(site[i], ones.data(), sizeof(Z), cudaMemcpyHostToDevice, stream)))
        return s;
    if (mps_status s = cu(cudaMemcpyAsync(site_dev, site.data(), sizeof(Z*) * N, cudaMemcpyHostToDevice, stream)))
      return s;
    if (mps_status s = cu(cudaStreamSynchronize(stream))) return s;
    std::memset(hctrl, 0, sizeof(DevCtrl));
    hctrl->product = 1.0;
    hctrl->f_min = o.f_min;
    hctrl->n_2q = o.n_2q;
    hctrl->f0 = (o.f_min < 1.0 && o.n_2q > 0) ? std::pow(o.f_min, 1.0 / (double)o.n_2q) : 1.0;
    hctrl->strategy = o.strategy;
    hctrl->fixed_chi = o.fixed_chi;
    hctrl->chi_max = chi_cap;
    hctrl->mixed_fid = o.mixed_fid;
    hctrl->kind = o.kind;
    if (mps_status s = cu(cudaMemcpyAsync(ctrl, hctrl, sizeof(DevCtrl), cudaMemcpyHostToDevice, stream))) return s;
    if (mps_status s = cu(cudaStreamSynchronize(stream))) return s;
    if (o.precision == MPS_TF32X3 && std::is_same<R, float>::value) {
      tc = tc_create(big);
      if (!tc) return MPS_ERR_OOM;
    }
    vidal = o.vidal != 0;
    if (vidal && share) {
      lam = share->lam;
      lam_stride = share->lam_stride;
      lam_owned = false;
    } else if (vidal) {
      for (int b = 0; b <= N; ++b) lam_stride = std::max(lam_stride, cap[b]);
      if (!dalloc(&lam, (size_t)(N + 1) * lam_stride)) return MPS_ERR_OOM;
      if (mps_status s = reset_lambda()) return s;
    }
    if (std::is_same<R, float>::value) {
      // mps_options.qr bits: MPS_QR_PRECONDITION the QR-preconditioned gate SVD, MPS_QR_MOVES the
      // centre moves by QR (default both: measured on the 100-qubit benchmark, the preconditioned
      // Jacobi takes 7.2 sweeps instead of 9.1, which pays for the extra QR)
      qr_mode = o.qr;
      qr_on = (qr_mode & 3) != 0;
      qr_fit = qr_on ? qr_max_ctas() : 0;
      if (qr_fit <= 0) qr_on = false;
      if (qr_on && (!dalloc(&qr_tau, (size_t)c_max) || !dalloc(&qr_T, (size_t)1024 * ((c_max + 31) / 32))))
        return MPS_ERR_OOM;
      if (qr_on && (qr_mode & 2)) {
        if (!dalloc(&Xq, (size_t)qr_max_rows() * c_max) || !dalloc(&Qq, (size_t)qr_max_rows() * qr_max_rows()) ||
            !dalloc(&Tq, (size_t)1024 * ((c_max + 31) / 32)) || !dalloc(&tauq, (size_t)c_max))
          return MPS_ERR_OOM;
        if (cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ev_main, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&ev_side, cudaEventDisableTiming) != cudaSuccess)
          return MPS_ERR_CUDA;
      }
    }
    return MPS_OK;
  }

  // ------------------------------------------------------------- building blocks
  mps_status gemm(int M, int Nn, int K, R alpha, const Z* A, long long a_rs, long long a_cs, int cA,
                  const Z* B, long long b_rs, long long b_cs, int cB, Z* C, long long c_rs, long long c_cs) {
    if (M <= 0 || Nn <= 0) return MPS_OK;
    ++n_gemm;
    gemm_flops += 8.0 * M * (double)Nn * K;
    const int id = tbegin();
    mps_status s;
    if (tc && K >= 8 && (long long)M * Nn * K >= 32768LL && tc_fits(tc, M, Nn, K)) {
      int launched = 0;
      s = cu(tc_gemm(tc, M, Nn, K, (float)alpha, (const float2*)A, a_rs, a_cs, cA, (const float2*)B, b_rs, b_cs,
                     cB, (float2*)C, c_rs, c_cs, stream, &launched, &ctrl->status));
      n_launch += launched;
    } else {
      s = kl(cgemm_simt<R>(M, Nn, K, alpha, A, a_rs, a_cs, cA, B, b_rs, b_cs, cB, C, c_rs, c_cs, stream));
    }
    tend(id, 1);
    return s;
  }

  // out[j*o_js + r*o_rs] = scale_j * op(src[col(j)*s_js + r*s_rs])
  mps_status extract(Z* out, long long o_js, long long o_rs, int kout, int rows, const Z* src, long long s_js,
                     long long s_rs, const int* pm, int conj, const double* sv, int wk) {
    if (kout <= 0 || rows <= 0) return MPS_OK;
    return kl(extract_columns<R>(out, o_js, o_rs, kout, rows, src, s_js, s_rs, pm, conj, sv, wk, ctrl, stream));
  }

  mps_status copy(Z* dst, const Z* src, size_t count) {
    return cu(cudaMemcpyAsync(dst, src, sizeof(Z) * count, cudaMemcpyDeviceToDevice, stream));
  }

  // Launch plan of one Jacobi SVD for a layout kind, with the co-residency check of the
  // tournament kernels (the Gram layout is checked when it is planned).
  mps_status make_plan(int l, int c, bool acc, int kind, JacobiPlan& plan) {
    const int ns = shared_gpu ? kJacobiNoSplit : 0;   // beside other handles: no 512-thread CTAs
    plan = jacobi_plan<R>(l, c, acc, sm_count, sm_count, kind | ns);
    if (plan.gram_R == 0) {
      const int fit = plan.cluster > 0 ? plan.cluster : jacobi_max_ctas<R>(plan);
      if (fit <= 0) return MPS_ERR_CUDA;
      if (plan.nb / 2 > fit) {
        plan = jacobi_plan<R>(l, c, acc, sm_count, fit,
                              (kind == MPS_SVD_TOURNAMENT_UNSPLIT ? MPS_SVD_TOURNAMENT_UNSPLIT : MPS_SVD_TOURNAMENT) | ns);
        if (plan.nb / 2 > fit) return MPS_ERR_ARG;
      }
    }
    return MPS_OK;
  }

  // The layout kind for a shape: the option, or under MPS_SVD_AUTO the tuned choice (measured on
  // first use of the shape when this handle runs alone on the GPU; the fixed rule otherwise).  The
  // timing runs take copies of src (l x c, column-major, ld lds: the matrix about to be
  // decomposed) when given, else a synthetic matrix.
  int layout_for(int l, int c, bool acc, bool force = false, const Z* src = nullptr, long long lds = 0) {
    if (!std::is_same<R, float>::value || opt.svd_kernel != MPS_SVD_AUTO || c < kTuneMinCols) return opt.svd_kernel;
    // a handle that runs beside others keeps the fixed rule: the table was measured alone, and a
    // layout that spans the GPU (the block kernel) would serialise the concurrent handles
    if (shared_gpu && !force) return MPS_SVD_AUTO;
    const auto up = [](int v) { return (v + kTuneGrain - 1) / kTuneGrain * kTuneGrain; };
    const TuneKey key{device, up(l), up(c), acc ? 1 : 0};
    {
      std::lock_guard<std::mutex> lk(tune_mutex());
      auto it = tune_table().find(key);
      if (it != tune_table().end()) return it->second.kind;
    }
    double ms[3] = {-1.0, -1.0, -1.0};
    const int kinds[3] = {MPS_SVD_TOURNAMENT, MPS_SVD_GRAM, MPS_SVD_TOURNAMENT_UNSPLIT};
    const void* split_fn = nullptr;
    const long long nx = (long long)l * c, nw = acc ? (long long)c * c : 0;
    Z* xt = nullptr;
    DevCtrl* tc = nullptr;
    cudaEvent_t e0 = ev_get(), e1 = ev_get();
    if (cudaMalloc(&xt, sizeof(Z) * (nx + nw + 1)) == cudaSuccess && cudaMalloc(&tc, sizeof(DevCtrl)) == cudaSuccess) {
      for (int v = 0; v < 3; ++v) {
        JacobiPlan plan;
        if (make_plan(l, c, acc, kinds[v], plan) != MPS_OK) continue;
        if (kinds[v] == MPS_SVD_GRAM && plan.gram_R == 0) continue;
        if (v == 0) split_fn = plan.fn;
        if (v == 2 && plan.fn == split_fn) continue;   // no split variant for this shape: the same launch
        double best = -1.0;
        for (int rep = 0; rep < 2; ++rep) {
          if (src)
            cudaMemcpy2DAsync(xt, sizeof(Z) * l, src, sizeof(Z) * lds, sizeof(Z) * l, c, cudaMemcpyDeviceToDevice, stream);
          else
            synthetic_fill_kernel<<<256, 256, 0, stream>>>(reinterpret_cast<float2*>(xt), nx, 12345u);
          if (acc) set_identity<R>(xt + nx, c, c, stream);
          cudaMemsetAsync(tc, 0, sizeof(DevCtrl), stream);
          cudaEventRecord(e0, stream);
          cudaError_t e = jacobi_launch<R>(plan, xt, l, l, c, acc ? xt + nx : nullptr, c, opt.max_sweeps, tc, xch,
                                           xch_cap, jflags, kFlagsCap, stream);
          cudaEventRecord(e1, stream);
          int st = 1;
          if (e == cudaSuccess && cudaStreamSynchronize(stream) == cudaSuccess)
            cudaMemcpy(&st, &tc->status, sizeof(int), cudaMemcpyDeviceToHost);
          float t = 0.f;
          if (st == 0 && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess) best = (best < 0.0) ? t : std::min(best, (double)t);
          cudaGetLastError();
        }
        ms[v] = best;
      }
    }
    cudaGetLastError();
    if (xt) cudaFree(xt);
    if (tc) cudaFree(tc);
    ev_pool.push_back(e0);
    ev_pool.push_back(e1);
    // the faster tournament form, then the block layout only when at least 10 % faster than it
    int kind = MPS_SVD_TOURNAMENT;
    double tbest = ms[0];
    if (ms[2] > 0.0 && (tbest < 0.0 || ms[2] < tbest)) { kind = MPS_SVD_TOURNAMENT_UNSPLIT; tbest = ms[2]; }
    if (ms[1] > 0.0 && (tbest < 0.0 || ms[1] < 0.9 * tbest)) kind = MPS_SVD_GRAM;
    if (ms[0] < 0.0 && ms[1] < 0.0 && ms[2] < 0.0) kind = MPS_SVD_AUTO;   // no measurement: the fixed rule
    std::lock_guard<std::mutex> lk(tune_mutex());
    auto ins = tune_table().emplace(key, TuneEntry{kind, ms[0], ms[1], ms[2]});
    return ins.first->second.kind;
  }

  mps_status svd_tune(int l, int c, int acc, int* layout) override {
    if (mps_status js = join_side()) return js;
    if (l < 1 || c < 1 || l > c_max || c > c_max) return MPS_ERR_ARG;
    if (mps_status s = sync()) return s;
    const int kind = layout_for(l, c, acc != 0, true);
    if (layout) *layout = kind;
    return cu(cudaStreamSynchronize(stream));
  }

  // early_stop: the sweep after which the rotations are below sqrt(tol) is the last (a gate SVD,
  // whose singular values are recomputed from theta); false where the rotated columns themselves
  // must be orthonormal to the full tolerance (the Jacobi orthogonalisation of a centre move).
  mps_status run_jacobi(int l, int c, bool acc, Z* Xp, long long ldx, bool early_stop = true) {
    last_c = c;
    if (acc)
      if (mps_status s = kl(set_identity<R>(Wacc, c, c, stream))) return s;
    if (c <= 1) return MPS_OK;
    JacobiPlan plan;
    if (mps_status s = make_plan(l, c, acc, layout_for(l, c, acc, false, Xp, ldx), plan)) return s;
    plan.early_stop = early_stop;
    if (mps_status s = coop_ensure(jacobi_plan_ctas(plan))) return s;
    ++n_jac;
    if (in_move) ++n_jac_move;
    const int id = tbegin();
    mps_status s = kl(jacobi_launch<R>(plan, Xp, ldx, l, c, acc ? Wacc : nullptr, c, opt.max_sweeps, ctrl, xch,
                                       xch_cap, jflags, kFlagsCap, stream));
    tend(id, in_move ? 2 : 0);
    return s;
  }

  // ------------------------------------------------------------- Householder QR
  bool qr_ok(int rows, int cols) const { return qr_on && rows <= qr_max_rows() && rows >= 1 && cols >= 1; }

  // X (l x c, column-major, ld ldx) = Q R in place; with Q != nullptr also the explicit Q
  // (l x min(l, c), column-major, ld ldq).
  // tmat, tvec: the block-reflector factors and tau (qr_T / qr_tau by default; a centre move whose
  // Q is formed on the second stream passes its own, so the gate's QR need not wait for it)
  mps_status qr_run(int l, int c, Z* Xp, long long ldx, Z* Q, long long ldq, Z* tmat = nullptr, Z* tvec = nullptr) {
    if (!tmat) tmat = qr_T;
    if (!tvec) tvec = qr_tau;
    if constexpr (std::is_same<R, float>::value) {
      const int ctas = qr_ctas(l, c, qr_fit);   // one cluster: no co-residency budget needed
      ++n_qr;
      const int id = tbegin();
      mps_status s = kl(qr_factor(Xp, ldx, l, c, tvec, tmat, ctrl, ctas, stream));
      if (s == MPS_OK && Q) s = kl(qr_form_q(Xp, ldx, l, c, tmat, Q, ldq, ctrl, qr_ctas(l, std::min(l, c), qr_fit), stream));
      tend(id, 3);
      return s;
    } else {
      (void)l; (void)c; (void)Xp; (void)ldx; (void)Q; (void)ldq;
      return MPS_ERR_ARG;
    }
  }

  // The explicit Q (l x min(l, c), ld l, into Qq) of the move's matrix QX just factored on the
  // handle's stream, then the site write-back out <- Qq (the extract of the plain path), both on
  // the second stream; the handle's stream goes on with the next steps.
  mps_status side_q(int l, int c, const Z* QX, Z* out, long long o_js, long long o_rs, int kout, int rows,
                    int conj) {
    if constexpr (std::is_same<R, float>::value) {
      if (mps_status s = cu(cudaEventRecord(ev_main, stream))) return s;
      if (mps_status s = cu(cudaStreamWaitEvent(side, ev_main, 0))) return s;
      const int id = tbegin(side);
      mps_status s = kl(qr_form_q(QX, l, l, c, Tq, Qq, l, ctrl, qr_ctas(l, std::min(l, c), qr_fit), side));
      tend(id, 3, side);
      if (s == MPS_OK)
        s = kl(extract_columns<R>(out, o_js, o_rs, kout, rows, Qq, l, 1, nullptr, conj, nullptr, 0, ctrl, side));
      if (s == MPS_OK) s = cu(cudaEventRecord(ev_side, side));
      if (s == MPS_OK) side_pending = true;
      return s;
    } else {
      (void)l; (void)c; (void)QX; (void)out; (void)o_js; (void)o_rs; (void)kout; (void)rows; (void)conj;
      return MPS_ERR_ARG;
    }
  }

  // Vidal form of a product state: every bond of dimension 1 with Schmidt value 1
  mps_status reset_lambda() {
    std::vector<double> h((size_t)(N + 1) * lam_stride, 0.0);
    for (int b = 0; b <= N; ++b) h[(size_t)b * lam_stride] = 1.0;
    if (mps_status s = cu(cudaMemcpyAsync(lam, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice, stream)))
      return s;
    return cu(cudaStreamSynchronize(stream));
  }

  mps_status read_ctrl() {
    if (mps_status s = join_side()) return s;
    if (mps_status s = cu(cudaMemcpyAsync(hctrl, ctrl, sizeof(DevCtrl), cudaMemcpyDeviceToHost, stream))) return s;
    if (mps_status s = cu(cudaStreamSynchronize(stream))) return s;
    coop_release();   // every launch of this handle has finished
    harvest();
    sticky |= hctrl->status & (ST_TIMEOUT | ST_NONFINITE | ST_NOT_CONVERGED | ST_BAD_ARG);
    return from_bits(sticky);
  }

  // ------------------------------------------------------------- centre moves
  // Moving the orthogonality centre by one site replaces the QR step of the
  // canonical form ("Canonicalization" section) by a one-sided Jacobi
  // orthogonalisation: any isometry Q with C = Q R serves, and the bond
  // becomes the rank bound min(rows, cols) exactly as with a reduced QR.
  mps_status move_right(int c) {
    const int m = bonds[c] * d, n = bonds[c + 1], n2 = d * bonds[c + 2];
    Z* C = site[c];
    Z* Nx = site[c + 1];
    mps_status s;
    if ((qr_mode & 2) && qr_ok(m, n)) {
      // C (m x n) = Q R: A_c <- Q (m x K), A_{c+1} <- R A_{c+1} (K x n2), bond K = min(m, n)
      const int K = std::min(m, n);
      const bool ovl = side && !shared_gpu;   // Q and the write-back of A_c beside the next steps
      Z* QX = ovl ? Xq : X;
      if ((s = join_side())) return s;
      if ((s = extract(QX, m, 1, n, m, C, 1, n, nullptr, 0, nullptr, 0))) return s;      // QX = C column-major
      if ((s = qr_run(m, n, QX, m, ovl ? nullptr : Wacc, m, ovl ? Tq : nullptr, ovl ? tauq : nullptr))) return s;
      if (ovl && (s = side_q(m, n, QX, C, 1, K, K, m, 0))) return s;                      // A_c = Q row-major
      if ((s = kl(triu_extract<R>(tmp2, n, 1, QX, m, K, n, 0, stream)))) return s;         // R row-major K x n
      if ((s = gemm(K, n2, n, R(1), tmp2, n, 1, 0, Nx, n2, 1, 0, T, n2, 1))) return s;     // R A_{c+1}
      if ((s = copy(Nx, T, (size_t)K * n2))) return s;
      if (!ovl && (s = extract(C, 1, K, K, m, Wacc, m, 1, nullptr, 0, nullptr, 0))) return s;   // A_c = Q row-major
      bonds[c + 1] = K;
    } else if (n <= m) {
      // X = C column-major; C W = Y; Q = Y/|Y| (m x n), R = Q^dagger C, A_{c+1} <- R A_{c+1}
      if ((s = extract(X, m, 1, n, m, C, 1, n, nullptr, 0, nullptr, 0))) return s;
      if ((s = run_jacobi(m, n, false, X, m, false))) return s;
      if ((s = kl(column_norms<R>(X, m, m, n, norms, stream)))) return s;
      if ((s = extract(tmp, 1, n, n, m, X, m, 1, nullptr, 0, norms, 0))) return s;       // Q, row-major m x n
      if ((s = gemm(n, n, m, R(1), tmp, 1, n, 1, C, n, 1, 0, tmp2, n, 1))) return s;       // R = Q^dagger C
      if ((s = gemm(n, n2, n, R(1), tmp2, n, 1, 0, Nx, n2, 1, 0, T, n2, 1))) return s;     // R A_{c+1}
      if ((s = copy(Nx, T, (size_t)n * n2))) return s;
      if ((s = copy(C, tmp, (size_t)m * n))) return s;
    } else {
      // X = C^dagger (column i = conj of row i of C), accumulate W (m x m):
      // C^dagger W = Y  ->  C = W Y^dagger: Q = W with unit columns, R = Q^dagger C
      if ((s = extract(X, n, 1, m, n, C, n, 1, nullptr, 1, nullptr, 0))) return s;
      if ((s = run_jacobi(n, m, true, X, n, false))) return s;
      if ((s = kl(column_norms<R>(Wacc, m, m, m, norms, stream)))) return s;
      if ((s = extract(tmp, 1, m, m, m, Wacc, m, 1, nullptr, 0, norms, 0))) return s;      // Q row-major m x m
      if ((s = gemm(m, n, m, R(1), tmp, 1, m, 1, C, n, 1, 0, tmp2, n, 1))) return s;       // R = Q^dagger C
      if ((s = gemm(m, n2, n, R(1), tmp2, n, 1, 0, Nx, n2, 1, 0, T, n2, 1))) return s;     // R A_{c+1}
      if ((s = copy(Nx, T, (size_t)m * n2))) return s;
      if ((s = copy(C, tmp, (size_t)m * m))) return s;
      bonds[c + 1] = m;
    }
    centre = c + 1;
    return MPS_OK;
  }

  mps_status move_left(int c) {
    const int m = bonds[c], n = d * bonds[c + 1], m2 = bonds[c - 1] * d;
    Z* C = site[c];
    Z* Pv = site[c - 1];
    mps_status s;
    if ((qr_mode & 2) && qr_ok(n, m)) {
      // C^dagger (n x m) = Q R, so C = R^dagger Q^dagger: A_c <- Q^dagger (K x n),
      // A_{c-1} <- A_{c-1} R^dagger (m2 x K), bond K = min(m, n)
      const int K = std::min(m, n);
      const bool ovl = side && !shared_gpu;   // Q and the write-back of A_c beside the next steps
      Z* QX = ovl ? Xq : X;
      if ((s = join_side())) return s;
      if ((s = extract(QX, n, 1, m, n, C, n, 1, nullptr, 1, nullptr, 0))) return s;       // QX = C^dagger
      if ((s = qr_run(n, m, QX, n, ovl ? nullptr : Wacc, n, ovl ? Tq : nullptr, ovl ? tauq : nullptr))) return s;
      // Q^dagger row-major (K x n): element (r, j) = conj(Q(j, r)) sits where Q(j, r) sits
      if (ovl && (s = side_q(n, m, QX, C, n, 1, K, n, 1))) return s;
      if ((s = kl(triu_extract<R>(tmp2, m, 1, QX, n, K, m, 0, stream)))) return s;         // R row-major K x m
      if ((s = gemm(m2, K, m, R(1), Pv, m, 1, 0, tmp2, 1, m, 1, T, K, 1))) return s;       // A_{c-1} R^dagger
      if ((s = copy(Pv, T, (size_t)m2 * K))) return s;
      if (!ovl && (s = extract(C, n, 1, K, n, Wacc, n, 1, nullptr, 1, nullptr, 0))) return s;
      bonds[c] = K;
    } else if (m <= n) {
      // X = C^dagger; C^dagger W = Y -> C = (W S) Yn^dagger: Q' = Yn^dagger (m x n), L = C Q'^dagger
      if ((s = extract(X, n, 1, m, n, C, n, 1, nullptr, 1, nullptr, 0))) return s;
      if ((s = run_jacobi(n, m, false, X, n, false))) return s;
      if ((s = kl(column_norms<R>(X, n, n, m, norms, stream)))) return s;
      if ((s = extract(tmp, n, 1, m, n, X, n, 1, nullptr, 1, norms, 0))) return s;        // Q' row-major m x n
      if ((s = gemm(m, m, n, R(1), C, n, 1, 0, tmp, 1, n, 1, tmp2, m, 1))) return s;       // L = C Q'^dagger
      if ((s = gemm(m2, m, m, R(1), Pv, m, 1, 0, tmp2, m, 1, 0, T, m, 1))) return s;       // A_{c-1} L
      if ((s = copy(Pv, T, (size_t)m2 * m))) return s;
      if ((s = copy(C, tmp, (size_t)m * n))) return s;
    } else {
      // X = C column-major, accumulate W (n x n): C W = Y -> C = Y W^dagger:
      // Q' = W^dagger with unit rows, L = C Q'^dagger
      if ((s = extract(X, m, 1, n, m, C, 1, n, nullptr, 0, nullptr, 0))) return s;
      if ((s = run_jacobi(m, n, true, X, m, false))) return s;
      if ((s = kl(column_norms<R>(Wacc, n, n, n, norms, stream)))) return s;
      if ((s = extract(tmp, n, 1, n, n, Wacc, n, 1, nullptr, 1, norms, 0))) return s;      // Q' row-major n x n
      if ((s = gemm(m, n, n, R(1), C, n, 1, 0, tmp, 1, n, 1, tmp2, n, 1))) return s;       // L = C Q'^dagger
      if ((s = gemm(m2, n, m, R(1), Pv, m, 1, 0, tmp2, n, 1, 0, T, n, 1))) return s;       // A_{c-1} L
      if ((s = copy(Pv, T, (size_t)m2 * n))) return s;
      if ((s = copy(C, tmp, (size_t)n * n))) return s;
      bonds[c] = n;
    }
    centre = c - 1;
    return MPS_OK;
  }

  mps_status move_to(int to) {
    in_move = true;
    mps_status s = MPS_OK;
    while (!s && centre < to) s = move_right(centre);
    while (!s && centre > to) s = move_left(centre);
    in_move = false;
    return s;
  }

  // ------------------------------------------------------------- operators
  // Host copy of an operator lifted to the local index: PURE: as given; MIXED: a unitary U becomes
  // the superoperator of U rho U^dagger, a superoperator is taken as given.
  bool lift(const double* op, int op_dim, int nq, std::vector<double>& out) {
    const int dloc = 1 << nq;                // qubit-space dimension
    const int D = (d == 2) ? dloc : dloc * dloc;
    if (d == 2) {
      if (op_dim != dloc) return false;
      out.assign(op, op + 2 * D * D);
      return true;
    }
    if (op_dim == dloc) {
      out.resize(2 * D * D);
      superop_from_kraus_host(op, 1, nq, out.data());
      return true;
    }
    if (op_dim != D) return false;
    out.assign(op, op + 2 * D * D);
    return true;
  }

  mps_status apply_1q(int q, const double* op, int op_dim) override {
    if (mps_status js = join_side()) return js;
    if (sticky) return from_bits(sticky);
    if (q < 0 || q >= N || !op) return MPS_ERR_ARG;
    std::vector<double> g;
    if (!lift(op, op_dim, 1, g)) return MPS_ERR_ARG;
    mps_status s;
    if ((s = kl(load_gate_param<R>(g.data(), d, G, stream)))) return s;
    if (d == 4)
      if ((s = move_to(q))) return s;
    if ((s = kl(apply_local<R>(site[q], bonds[q], d, bonds[q + 1], G, stream)))) return s;
    if (d == 4)
      if ((s = kl(renormalise_site<R>(site[q], (long long)bonds[q] * d * bonds[q + 1], ctrl, stream)))) return s;
    return MPS_OK;
  }

  // The hot path of the entanglement-aware algorithm for one two-qubit gate.
  mps_status apply_2q(int q, const double* op, bool on_device, int op_dim, double target) override {
    if (mps_status js = join_side()) return js;
    if (sticky) return from_bits(sticky);
    if (q < 0 || q + 1 >= N || !op) return MPS_ERR_ARG;
    const int D2 = d * d;
    mps_status s;
    if (on_device) {
      if (!(op_dim == D2 && (d == 4 ? true : op_dim == 4))) return MPS_ERR_ARG;   // device operators: d^2 x d^2
      if ((s = kl(load_gate_device<R>(op, D2, G, stream)))) return s;
    } else {
      std::vector<double> g;
      if (!lift(op, op_dim, 2, g)) return MPS_ERR_ARG;
      if ((s = kl(load_gate_param<R>(g.data(), D2, G, stream)))) return s;
    }
    // (a0) centre onto the pair: to q when it sits at or left of q (leaves at q+1), else to q+1.
    // Vidal form: no centre; every update is a leftward one (V^dagger becomes B_{q+1})
    const bool right = vidal ? false : centre <= q;
    if (!vidal)
      if ((s = move_to(right ? q : q + 1))) return s;
    const int cl = bonds[q], chi = bonds[q + 1], cr = bonds[q + 2];
    const int m = d * cl, n = d * cr;
    // (a1) theta = A_q A_{q+1} (m x n as (cl, d, d, cr)), then the gate on the physical pair
    if ((s = gemm(m, n, chi, R(1), site[q], chi, 1, 0, site[q + 1], n, 1, 0, T, n, 1))) return s;
    // Jacobi on the short side; the orthonormal factor lands on the side the centre leaves
    enum { R_COLS, R_ROWS_ACC, L_ROWS, L_COLS_ACC } mode;
    if (right) mode = (n <= m) ? R_COLS : R_ROWS_ACC;
    else mode = (m <= n) ? L_ROWS : L_COLS_ACC;
    // QR preconditioning when the wanted directions are the right singular vectors of a tall X:
    // X = theta^dagger (n >= m) for a rightward update, X = theta (m >= n) for a leftward one
    const bool use_qr = (qr_mode & 1) && std::min(m, n) >= kPrecondMinCols && (right ? n >= m : m >= n) &&
                        qr_ok(std::max(m, n), std::min(m, n));
    const bool cols = use_qr ? !right : (mode == R_COLS || mode == L_COLS_ACC);   // X = theta (else theta^dagger)
    const int l = cols ? m : n, c = cols ? n : m;
    if ((s = kl(gate_theta<R>(T, cl, d, cr, G, X, cols ? 0 : 1, theta, stream)))) return s;
    // Vidal form: the SVD is of lambda_{q-1} theta (rows of theta scaled by the Schmidt values of
    // bond q); theta itself stays unscaled for B_q = theta V below
    if (vidal && q > 0)
      if ((s = kl(scale_by_lambda<R>(X, l, l, c, lam + (size_t)q * lam_stride, d, cols ? 1 : 0, stream)))) return s;
    // (a2) SVD: one-sided Jacobi gives the singular directions D with unit columns (FP64
    // norms): left vectors U (m x c) for a rightward update, right vectors V (n x c) for a
    // leftward one.  X (l x c, l >= c) is theta or theta^dagger.
    const bool acc = (mode == R_ROWS_ACC || mode == L_COLS_ACC);
    const bool u_type = right;
    if (use_qr) {
      // Preconditioned: X = Q R, one-sided Jacobi on Y = R^dagger (c x c, column-major in Wacc);
      // the rotated, normalised columns of Y are the right singular vectors of X: U when X is
      // theta^dagger (rightward, c = m), V when X is theta (leftward, c = n).  They are
      // orthonormal to the Jacobi tolerance whatever their singular values.
      if ((s = qr_run(l, c, X, l, nullptr, 0))) return s;
      if ((s = kl(triu_extract<R>(Wacc, c, 1, X, l, c, c, 1, stream)))) return s;
      if ((s = run_jacobi(c, c, false, Wacc, c))) return s;
      if ((s = kl(column_norms<R>(Wacc, c, c, c, norms, stream)))) return s;
      if (u_type) s = extract(tmp, 1, c, c, m, Wacc, c, 1, nullptr, 0, norms, 0);   // U row-major (m x c)
      else s = extract(tmp, n, 1, c, n, Wacc, c, 1, nullptr, 0, norms, 0);          // V column-major (n x c)
      if (s) return s;
    } else {
      // from the rotated columns, or from the accumulated rotations when the Jacobi ran on the
      // other side
      if ((s = run_jacobi(l, c, acc, X, l))) return s;
      const Z* src = acc ? Wacc : X;
      const int len = acc ? c : l;
      if ((s = kl(column_norms<R>(src, len, len, c, norms, stream)))) return s;
      if (u_type)   // U row-major (m x c)
        s = extract(tmp, 1, c, c, m, src, len, 1, nullptr, 0, norms, 0);
      else          // V column-major (n x c)
        s = extract(tmp, n, 1, c, n, src, len, 1, nullptr, 0, norms, 0);
      if (s) return s;
    }
    // Refinement: singular values from the original theta, P = U^dagger theta (c x n, row-major;
    // row j = s_j v_j^dagger) or P = theta V (m x c, column-major; column j = s_j u_j), FP64 norms.
    // The rotations' rounding drift in FP32 column norms does not reach these values.
    if (u_type) { if ((s = gemm(c, n, m, R(1), tmp, 1, c, 1, theta, n, 1, 0, tmp2, n, 1))) return s; }
    else { if ((s = gemm(m, c, n, R(1), theta, n, 1, 0, tmp, 1, n, 0, tmp2, 1, m))) return s; }
    const long long pld = u_type ? n : m;
    const int plen = u_type ? n : m;
    // (a3) selection and FP64 bookkeeping
    const Z* psel = tmp2;
    if (vidal && q > 0) {   // singular values of lambda_{q-1} theta: the scaled copy of P = theta V
      if ((s = copy(Wacc, tmp2, (size_t)m * c))) return s;
      if ((s = kl(scale_by_lambda<R>(Wacc, m, m, c, lam + (size_t)q * lam_stride, d, 1, stream)))) return s;
      psel = Wacc;
    }
    ++n_launch;   // select_bond launches two kernels (FP64 norms, then the selection)
    if ((s = kl(select_bond<R>(psel, pld, plen, c, ctrl, target, s_sorted, perm, stream)))) return s;
    if ((s = read_ctrl())) return s;
    const int k = hctrl->k;
    Z* Aq = site[q];
    Z* Ap = site[q + 1];
    // (a4) write-back: A_q (cl, d, k) row-major, A_{q+1} (k, d, cr) row-major; the kept
    // singular values are renormalised by 1/sqrt(W_k)
    if (u_type) {   // A_q = U[:, perm], A_{q+1} = P[perm, :] / sqrt(W_k)
      if ((s = extract(Aq, 1, k, k, m, tmp, 1, c, perm, 0, nullptr, 0))) return s;
      if ((s = extract(Ap, n, 1, k, n, tmp2, n, 1, perm, 0, nullptr, 1))) return s;
    } else {        // A_q = P[:, perm] / sqrt(W_k), A_{q+1} = V[:, perm]^dagger
      if ((s = extract(Aq, 1, k, k, m, tmp2, m, 1, perm, 0, nullptr, 1))) return s;
      if ((s = extract(Ap, n, 1, k, n, tmp, n, 1, perm, 1, nullptr, 0))) return s;
    }
    bonds[q + 1] = k;
    if (vidal) {
      if ((s = kl(store_lambda(lam + (size_t)(q + 1) * lam_stride, s_sorted, ctrl, lam_stride, stream)))) return s;
    } else {
      centre = right ? q + 1 : q;
    }
    ++n_gates;
    if (log_on) {
      mps_trunc_record r;
      r.q = q; r.k = k; r.rank_bound = c; r.cap_hit = hctrl->cap_hit;
      r.f = hctrl->f; r.f_t = hctrl->f_t; r.W = hctrl->W; r.W_k = hctrl->Wk;
      log.push_back(r);
    }
    return hctrl->cap_hit ? MPS_WARN_CHI_CAP : MPS_OK;
  }

  // One layer of gates on disjoint pairs in Vidal form, up to `concurrency` at a time on helper
  // handles (own scratch and stream, this handle's sites and Schmidt vectors).  Every gate of the
  // layer is truncated against the same per-truncation target: `target` when >= 0, else the
  // schedule's value for the product at the layer's start.
  mps_status apply_layer(int n, const int* qs, const double* ops_dev, int op_dim, double target,
                         int concurrency) override {
    if (mps_status js = join_side()) return js;
    if (sticky) return from_bits(sticky);
    if (!vidal) return MPS_ERR_STATE;
    if (n < 0 || (n > 0 && (!qs || !ops_dev)) || concurrency < 1 || op_dim != 4) return MPS_ERR_ARG;
    if (n == 0) return MPS_OK;
    std::vector<char> used(N, 0);
    for (int i = 0; i < n; ++i) {
      const int q = qs[i];
      if (q < 0 || q + 1 >= N || used[q] || used[q + 1]) return MPS_ERR_ARG;
      used[q] = used[q + 1] = 1;
    }
    mps_status s = read_ctrl();   // everything of this handle done; product and gate count current
    if (s != MPS_OK && s != MPS_WARN_CHI_CAP) return s;
    double ft = target;
    if (ft < 0.0) ft = schedule_target(opt.strategy, opt.f_min, opt.n_2q, hctrl->n_done, hctrl->product);
    const int nh = std::min(concurrency, n);
    while ((int)helpers.size() < nh) {
      cudaStream_t hs = nullptr;
      if (cudaStreamCreateWithFlags(&hs, cudaStreamNonBlocking) != cudaSuccess) return MPS_ERR_CUDA;
      Engine* h = new (std::nothrow) Engine<R>();
      if (!h) { cudaStreamDestroy(hs); return MPS_ERR_OOM; }
      mps_options ho = opt;
      ho.log_truncations = 1;
      if ((s = h->init(N, ho, hs, this)) != MPS_OK) { delete h; cudaStreamDestroy(hs); return s; }
      h->owns_stream = true;
      helpers.push_back(h);
    }
    for (int w = 0; w < nh; ++w) {
      Engine* h = helpers[w];
      h->bonds = bonds;
      h->log.clear();
      h->shared_gpu = nh > 1;
    }
    std::vector<mps_status> st(n, MPS_OK);
    const size_t ostride = (size_t)2 * op_dim * op_dim;
    auto worker = [&](int w) {
      cudaSetDevice(device);
      for (int i = w; i < n; i += nh) st[i] = helpers[w]->apply_2q(qs[i], ops_dev + i * ostride, true, op_dim, ft);
    };
    if (nh == 1) {
      worker(0);
    } else {
      std::vector<std::thread> pool;
      for (int w = 0; w < nh; ++w) pool.emplace_back(worker, w);
      for (std::thread& t : pool) t.join();
    }
    mps_status worst = MPS_OK;
    for (int i = 0; i < n; ++i) {
      if (st[i] == MPS_WARN_CHI_CAP) {
        worst = st[i];
      } else if (st[i] != MPS_OK) {   // the shared sites may be half-updated: this handle fails too
        for (int w = 0; w < nh; ++w) sticky |= helpers[w]->sticky;
        if (!sticky) sticky = ST_BAD_ARG;
        return st[i];
      }
    }
    for (int w = 0; w < nh; ++w)   // the write-back kernels of every helper have finished
      if ((s = helpers[w]->read_ctrl())) {
        sticky |= helpers[w]->sticky ? helpers[w]->sticky : ST_BAD_ARG;
        return s;
      }
    // merge: the bonds the layer changed, the truncation records and the product, in gate order
    // (the same multiplications as gate after gate, whatever the concurrency)
    for (int i = 0; i < n; ++i) {
      Engine* h = helpers[i % nh];
      const mps_trunc_record& r = h->log[i / nh];
      bonds[qs[i] + 1] = h->bonds[qs[i] + 1];
      hctrl->product *= r.f;
      if (log_on) log.push_back(r);
    }
    n_gates += n;
    hctrl->n_done += n;
    if ((s = cu(cudaMemcpyAsync(&ctrl->product, &hctrl->product, sizeof(double), cudaMemcpyHostToDevice, stream))))
      return s;
    if ((s = cu(cudaMemcpyAsync(&ctrl->n_done, &hctrl->n_done, sizeof(hctrl->n_done), cudaMemcpyHostToDevice,
                                stream))))
      return s;
    if ((s = cu(cudaStreamSynchronize(stream)))) return s;
    return worst;
  }

  // ---------------------------------------------- differentiable two-site update (stateless)
  // The handle's scratch and stream serve; its state is not touched.

  mps_status gemm_device(int M, int Nn, int K, const void* A, long long a_rs, long long a_cs, int cA, const void* B,
                         long long b_rs, long long b_cs, int cB, void* C, long long c_rs, long long c_cs) override {
    if (mps_status js = join_side()) return js;
    if (sticky) return from_bits(sticky);
    if (M < 1 || Nn < 1 || K < 1 || !A || !B || !C) return MPS_ERR_ARG;
    return gemm(M, Nn, K, R(1), (const Z*)A, a_rs, a_cs, cA, (const Z*)B, b_rs, b_cs, cB, (Z*)C, c_rs, c_cs);
  }

  // Full thin SVD of A (m x n, row-major, ld lda): U (m x c), S (c, FP64, descending), V (n x c),
  // row-major, c = min(m, n); then the cut and the write-back of a rightward update:
  // Aq = U_k (m x k), Ap = U_k^H A / sqrt(W_k) (k x n).  out4 (host) = {k, W_k/W, W, W_k}.
  mps_status tsvd_device(int m, int n, const void* Av, long long lda, double target, int max_k, double rank_tol,
                         void* Uv, double* S, void* Vv, void* Aqv, void* Apv, double* out4) override {
    if (mps_status js = join_side()) return js;
    if (sticky) return from_bits(sticky);
    if (m < 1 || n < 1 || !Av || lda < n || !Uv || !S || !Vv || !Aqv || !Apv || !out4 || !(target >= 0.0) ||
        !(rank_tol >= 0.0))
      return MPS_ERR_ARG;
    if (std::max(m, n) > c_max || (size_t)m * n > big_cap) return MPS_ERR_ARG;
    const Z* A = (const Z*)Av;
    Z *U = (Z*)Uv, *V = (Z*)Vv;
    const bool tall = m >= n;   // X = A (tall) or A^H: l x c column-major, l >= c
    const int l = tall ? m : n, c = tall ? n : m;
    mps_status s;
    if (tall) s = extract(X, l, 1, c, l, A, 1, lda, nullptr, 0, nullptr, 0);
    else s = extract(X, l, 1, c, l, A, lda, 1, nullptr, 1, nullptr, 0);
    if (s) return s;
    if ((s = run_jacobi(l, c, true, X, l))) return s;
    // Vx: the accumulated rotations with unit columns (c x c, column-major, in tmp)
    if ((s = kl(column_norms<R>(Wacc, c, c, c, norms, stream)))) return s;
    if ((s = extract(tmp, c, 1, c, c, Wacc, c, 1, nullptr, 0, norms, 0))) return s;
    // the other factor from the rotated columns of X, each scaled to unit norm (tmp2): the
    // Jacobi leaves them orthogonal relative to their own norms, so small values keep
    // orthonormal vectors (X V recomputed from A would not)
    if ((s = kl(column_norms<R>(X, l, l, c, norms, stream)))) return s;
    if ((s = extract(tmp2, l, 1, c, l, X, l, 1, nullptr, 0, norms, 0))) return s;
    // the values: FP64 norms of P = X Vx (l x c, column-major, in T) from the original A
    if (tall) s = gemm(l, c, c, R(1), A, lda, 1, 0, tmp, 1, c, 0, T, 1, l);
    else s = gemm(l, c, c, R(1), A, 1, lda, 1, tmp, 1, c, 0, T, 1, l);
    if (s) return s;
    if ((s = kl(column_norms<R>(T, l, l, c, norms, stream)))) return s;
    if ((s = kl(rank_sort(norms, c, perm, s_sorted, stream)))) return s;
    // A = X: U = the unit rotated columns, V = Vx;  A = X^H: U = Vx, V = the unit rotated
    // columns (columns in descending order of the values)
    if (tall) {
      if ((s = extract(U, 1, c, c, m, tmp2, l, 1, perm, 0, nullptr, 0))) return s;
      if ((s = extract(V, 1, c, c, n, tmp, c, 1, perm, 0, nullptr, 0))) return s;
    } else {
      if ((s = extract(U, 1, c, c, m, tmp, c, 1, perm, 0, nullptr, 0))) return s;
      if ((s = extract(V, 1, c, c, n, tmp2, l, 1, perm, 0, nullptr, 0))) return s;
    }
    double* od = (double*)outdev;
    if ((s = kl(select_values(s_sorted, c, target, max_k, rank_tol, od, stream)))) return s;
    if ((s = cu(cudaMemcpyAsync(S, s_sorted, sizeof(double) * c, cudaMemcpyDeviceToDevice, stream)))) return s;
    if ((s = cu(cudaMemcpyAsync(hout, od, sizeof(double) * 4, cudaMemcpyDeviceToHost, stream)))) return s;
    if ((s = read_ctrl())) return s;
    const double* ho = (const double*)hout;
    const int k = (int)ho[0];
    const double Wk = ho[3];
    if (!(Wk > 0.0) || !std::isfinite(Wk) || k < 1 || k > c) return MPS_ERR_NONFINITE;
    if ((s = extract((Z*)Aqv, 1, k, k, m, U, 1, c, nullptr, 0, nullptr, 0))) return s;
    if ((s = gemm(k, n, m, R(1.0 / std::sqrt(Wk)), U, 1, c, 1, A, lda, 1, 0, (Z*)Apv, n, 1))) return s;
    for (int i = 0; i < 4; ++i) out4[i] = ho[i];
    return cu(cudaStreamSynchronize(stream));
  }

  // Reverse-mode derivative of tsvd_device's (Aq, Ap) with respect to A (see tsvd_grad.cu)
  mps_status tsvd_backward_device(int m, int n, int k, const void* Uv, const double* S, const void* Vv,
                                  const void* Aq_bar, const void* Ap_bar, double eps, void* A_bar) override {
    if (mps_status js = join_side()) return js;
    if (sticky) return from_bits(sticky);
    const int c = std::min(m, n);
    if (m < 1 || n < 1 || k < 1 || k > c || !Uv || !S || !Vv || !A_bar || !(eps >= 0.0)) return MPS_ERR_ARG;
    if (std::max(m, n) > c_max || (size_t)m * n > big_cap) return MPS_ERR_ARG;
    const Z *U = (const Z*)Uv, *V = (const Z*)Vv;
    Z* out = (Z*)A_bar;
    double* wk = (double*)outdev + 4;
    mps_status s;
    // Ubar (tmp, m x c), Vbar (tmp2, n x c), sbar (norms)
    if ((s = kl(tsvd_cotangents<R>(m, n, c, k, V, S, (const Z*)Aq_bar, (const Z*)Ap_bar, tmp, tmp2, norms, wk,
                                   stream))))
      return s;
    // Ju = U^H Ubar (X), Jv = V^H Vbar (theta), c x c row-major
    if ((s = gemm(c, c, m, R(1), U, 1, c, 1, tmp, c, 1, 0, X, c, 1))) return s;
    if ((s = gemm(c, c, n, R(1), V, 1, c, 1, tmp2, c, 1, 0, theta, c, 1))) return s;
    const bool tall = m >= n;
    if (tall) {   // complement on the U side: Yu = Ubar S^-1 (tmp), Zu = U^H Yu (T)
      if ((s = kl(tsvd_scale<R>(tmp, m, c, k, S, stream)))) return s;
      if ((s = gemm(c, c, m, R(1), U, 1, c, 1, tmp, c, 1, 0, T, c, 1))) return s;
    } else {      // on the V side: Yv = Vbar S^-1 (tmp2), Zv = V^H Yv (T)
      if ((s = kl(tsvd_scale<R>(tmp2, n, c, k, S, stream)))) return s;
      if ((s = gemm(c, c, n, R(1), V, 1, c, 1, tmp2, c, 1, 0, T, c, 1))) return s;
    }
    if ((s = kl(tsvd_core<R>(c, X, theta, S, norms, eps, T, tall ? 0 : 1, Wacc, stream)))) return s;
    if (tall) {   // Abar = (U G + Yu) V^H
      if ((s = gemm(m, c, c, R(1), U, c, 1, 0, Wacc, c, 1, 0, X, c, 1))) return s;
      if ((s = kl(cadd_strided<R>(X, c, m, c, tmp, c, 1, 0, stream)))) return s;
      if ((s = gemm(m, n, c, R(1), X, c, 1, 0, V, 1, c, 1, out, n, 1))) return s;
    } else {      // Abar = U (G V^H + Yv^H)
      if ((s = gemm(c, n, c, R(1), Wacc, c, 1, 0, V, 1, c, 1, X, n, 1))) return s;
      if ((s = kl(cadd_strided<R>(X, n, c, n, tmp2, 1, c, 1, stream)))) return s;
      if ((s = gemm(m, n, c, R(1), U, c, 1, 0, X, n, 1, 0, out, n, 1))) return s;
    }
    return read_ctrl();
  }

  // failure detection: a bounded wait whose signal never comes gives up at the handle's deadline,
  // and the status word carries the timeout to the host (see mps_selftest_timeout)
  mps_status selftest_timeout(int site, long long wait_ns) override {
    if (mps_status js = join_side()) return js;
    if (sticky) return from_bits(sticky);
    if (site < MPS_SELFTEST_FLAG || site > MPS_SELFTEST_GEMM || wait_ns < 1000 || wait_ns > 20000000000LL)
      return MPS_ERR_ARG;
    if (site != MPS_SELFTEST_FLAG && !std::is_same<R, float>::value) return MPS_ERR_ARG;
    if (site == MPS_SELFTEST_GEMM && !tc) return MPS_ERR_ARG;
    mps_status s;
    // the limit and the knob go to the device control block; mps_reset restores both
    hctrl->wait_ns = (unsigned long long)wait_ns;
    hctrl->test_fault = site;
    if ((s = cu(cudaMemcpyAsync(&ctrl->wait_ns, &hctrl->wait_ns, sizeof(hctrl->wait_ns), cudaMemcpyHostToDevice,
                                stream))))
      return s;
    if ((s = cu(cudaMemcpyAsync(&ctrl->test_fault, &hctrl->test_fault, sizeof(int), cudaMemcpyHostToDevice,
                                stream))))
      return s;
    if (site == MPS_SELFTEST_FLAG) {
      unsigned* flag = (unsigned*)((double*)outdev + 6);   // the selection output slot 6, zeroed here
      if ((s = cu(cudaMemsetAsync(flag, 0, sizeof(unsigned), stream)))) return s;
      if ((s = kl(wait_probe(flag, 1u, ctrl, stream)))) return s;
      return read_ctrl();
    }
    if constexpr (std::is_same<R, float>::value) {
      // a small problem of the kernel under test, on buffers of its own (zero data: the exchange
      // protocol runs in every round whatever the values)
      const int l = 64, c = (site == MPS_SELFTEST_JACOBI) ? 288 : 128;
      float2 *x = nullptr, *xb = nullptr, *bb = nullptr, *cb = nullptr;
      unsigned* fl = nullptr;
      const size_t xcap = (size_t)1 << 21;
      auto release = [&]() {
        cudaStreamSynchronize(stream);
        for (void* b : {(void*)x, (void*)xb, (void*)bb, (void*)cb, (void*)fl}) if (b) cudaFree(b);
      };
      if (cudaMalloc(&x, sizeof(float2) * l * c) != cudaSuccess || cudaMalloc(&xb, sizeof(float2) * xcap) != cudaSuccess ||
          cudaMalloc(&bb, sizeof(float2) * 128 * 128) != cudaSuccess ||
          cudaMalloc(&cb, sizeof(float2) * 128 * 128) != cudaSuccess || cudaMalloc(&fl, sizeof(unsigned) * 4096) != cudaSuccess) {
        release();
        return MPS_ERR_OOM;
      }
      s = cu(cudaMemsetAsync(x, 0, sizeof(float2) * l * c, stream));
      if (!s) s = cu(cudaMemsetAsync(bb, 0, sizeof(float2) * 128 * 128, stream));
      if (!s && site == MPS_SELFTEST_GEMM) {
        s = cu(tc_gemm_selftest(tc, 128, 128, 64, x, bb, cb, stream, &ctrl->status, (unsigned long long)wait_ns));
        ++n_launch;
      } else if (!s) {
        JacobiPlan plan = jacobi_plan<R>(l, c, false, sm_count, sm_count,
                                         site == MPS_SELFTEST_GRAM ? MPS_SVD_GRAM : MPS_SVD_TOURNAMENT);
        const bool right_kind = (site == MPS_SELFTEST_GRAM) ? plan.gram_R > 0 : (plan.gram_R == 0 && plan.cluster == 0 &&
                                                                                  plan.nb / 2 > 1);
        if (!right_kind) {
          release();
          return MPS_ERR_ARG;
        }
        s = kl(jacobi_launch<R>(plan, x, l, l, c, nullptr, 0, 4, ctrl, xb, xcap, fl, 4096, stream));
      }
      mps_status r = s ? s : read_ctrl();
      release();
      return r;
    }
    return MPS_ERR_ARG;
  }

  mps_status fidelity(double* out) override {
    mps_status s = read_ctrl();
    *out = hctrl->product;
    return s;
  }

  bool is_vidal() const override { return vidal; }

  mps_status site_to_double(int i, double2* dst, cudaStream_t st) override {
    if (mps_status js = join_side()) return js;
    if (i < 0 || i >= N || !dst) return MPS_ERR_ARG;
    return kl(to_double<R>(site[i], dst, (long long)bonds[i] * d * bonds[i + 1], st));
  }

  mps_status lognorm(double* out) override {
    mps_status s = read_ctrl();
    *out = hctrl->lognorm;
    return s;
  }

  mps_status sync() override { return read_ctrl(); }

  mps_status reset() override {
    if (mps_status js = join_side()) return js;
    mps_status s;
    if ((s = cu(cudaStreamSynchronize(stream)))) return s;
    fold_helper_stats();
    harvest();
    if ((s = kl(product_state<R>(site_dev, N, d, stream)))) return s;
    std::fill(bonds.begin(), bonds.end(), 1);
    centre = 0;
    log.clear();
    sticky = 0;
    // statistics survive a state reset: take the device's current counters
    if ((s = cu(cudaMemcpyAsync(hctrl, ctrl, sizeof(DevCtrl), cudaMemcpyDeviceToHost, stream)))) return s;
    if ((s = cu(cudaStreamSynchronize(stream)))) return s;
    const double jf = hctrl->jac_flops;
    const unsigned long long js = hctrl->jac_sweeps;
    std::memset(hctrl, 0, sizeof(DevCtrl));
    hctrl->product = 1.0;
    hctrl->f_min = opt.f_min;
    hctrl->n_2q = opt.n_2q;
    hctrl->f0 = (opt.f_min < 1.0 && opt.n_2q > 0) ? std::pow(opt.f_min, 1.0 / (double)opt.n_2q) : 1.0;
    hctrl->strategy = opt.strategy;
    hctrl->fixed_chi = opt.fixed_chi;
    hctrl->chi_max = chi_cap;
    hctrl->mixed_fid = opt.mixed_fid;
    hctrl->kind = opt.kind;
    hctrl->jac_flops = jf;
    hctrl->jac_sweeps = js;
    if ((s = cu(cudaMemcpyAsync(ctrl, hctrl, sizeof(DevCtrl), cudaMemcpyHostToDevice, stream)))) return s;
    if ((s = cu(cudaStreamSynchronize(stream)))) return s;
    return vidal ? reset_lambda() : MPS_OK;
  }

  mps_status profile(int on) override {
    if (mps_status js = join_side()) return js;
    prof = on != 0;
    return MPS_OK;
  }

  // the layer runs' helper handles are dropped on a state reset; their counters stay in the
  // handle's statistics
  mps_stats_t folded{};
  void fold_helper_stats() {
    for (Engine* h : helpers) {
      mps_stats_t t{};
      h->stats(&t);
      add_stats(folded, t);
      delete h;
    }
    helpers.clear();
  }
  static void add_stats(mps_stats_t& a, const mps_stats_t& b) {
    a.kernel_launches += b.kernel_launches;
    a.jacobi_launches += b.jacobi_launches;
    a.jacobi_sweeps += b.jacobi_sweeps;
    a.jacobi_ms += b.jacobi_ms;
    a.jacobi_flops += b.jacobi_flops;
    a.gemm_launches += b.gemm_launches;
    a.gemm_ms += b.gemm_ms;
    a.gemm_flops += b.gemm_flops;
    a.move_jacobi_launches += b.move_jacobi_launches;
    a.move_jacobi_ms += b.move_jacobi_ms;
    a.qr_launches += b.qr_launches;
    a.qr_ms += b.qr_ms;
  }

  // gates run on helper handles count once, as gates of this handle
  mps_status stats(mps_stats_t* out) override {
    if (mps_status js = join_side()) return js;
    mps_status s = read_ctrl();
    out->kernel_launches = n_launch;
    out->jacobi_launches = n_jac;
    out->jacobi_sweeps = (long long)hctrl->jac_sweeps;
    out->jacobi_ms = jac_ms;
    out->jacobi_flops = hctrl->jac_flops;
    out->gemm_launches = n_gemm;
    out->gemm_ms = gemm_ms;
    out->gemm_flops = gemm_flops;
    out->gates = n_gates;
    out->move_jacobi_launches = n_jac_move;
    out->move_jacobi_ms = jac_move_ms;
    out->qr_launches = n_qr;
    out->qr_ms = qr_ms_sum;
    add_stats(*out, folded);
    for (Engine* h : helpers) {
      mps_stats_t t{};
      h->stats(&t);
      add_stats(*out, t);
    }
    return s;
  }

  mps_status stats_reset() override {
    if (mps_status js = join_side()) return js;
    mps_status s;
    if ((s = cu(cudaStreamSynchronize(stream)))) return s;
    harvest();
    for (Engine* h : helpers)
      if ((s = h->stats_reset())) return s;
    folded = mps_stats_t{};
    n_launch = n_jac = n_gemm = n_gates = n_jac_move = n_qr = 0;
    gemm_flops = jac_ms = gemm_ms = jac_move_ms = qr_ms_sum = 0.0;
    const size_t off = offsetof(DevCtrl, jac_sweeps);
    if ((s = cu(cudaMemsetAsync((char*)ctrl + off, 0, sizeof(DevCtrl) - off, stream)))) return s;
    // the host copy too: reset() carries the statistics over from it
    hctrl->jac_sweeps = 0;
    hctrl->jac_flops = 0.0;
    return cu(cudaStreamSynchronize(stream));
  }

  // v <- v * sum_t w_i[t] A_i[:, t, :] along the chain (optional two-site weight at q2)
  mps_status chain(const std::vector<double2>& w, int q2, const double2* w2, double2* result) {
    mps_status s;
    if ((s = cu(cudaMemcpyAsync(bonds_dev, bonds.data(), sizeof(int) * (N + 1), cudaMemcpyHostToDevice, stream)))) return s;
    if ((s = cu(cudaMemcpyAsync(wdev, w.data(), sizeof(double2) * w.size(), cudaMemcpyHostToDevice, stream)))) return s;
    if (w2)
      if ((s = cu(cudaMemcpyAsync(w2dev, w2, sizeof(double2) * 16, cudaMemcpyHostToDevice, stream)))) return s;
    if ((s = kl(chain_contract<R>(N, (const Z* const*)site_dev, bonds_dev, d, wdev, q2, w2dev, work, chi_cap + 8,
                                  outdev, stream))))
      return s;
    if ((s = cu(cudaMemcpyAsync(hout, outdev, sizeof(double2), cudaMemcpyDeviceToHost, stream)))) return s;
    if ((s = cu(cudaStreamSynchronize(stream)))) return s;
    *result = hout[0];
    return MPS_OK;
  }

  mps_status trace_stored(double2* tr) {
    std::vector<double2> w((size_t)N * d, make_double2(0, 0));
    for (int i = 0; i < N; ++i) { w[(size_t)i * d + 0] = make_double2(1, 0); w[(size_t)i * d + 3] = make_double2(1, 0); }
    return chain(w, -1, nullptr, tr);
  }

  mps_status expect(int q, int support, const double* op, double* out) override {
    if (mps_status js = join_side()) return js;
    if (sticky) return from_bits(sticky);
    if (vidal) return MPS_ERR_STATE;   // the local formula needs a canonical centre on the support
    if (!op || !out || (support != 1 && support != 2) || q < 0 || q + support > N) return MPS_ERR_ARG;
    mps_status s;
    if (d == 2) {
      const int D = support == 1 ? 2 : 4;
      if ((s = kl(load_gate_param<R>(op, D, O, stream)))) return s;
      if (support == 1) {
        if ((s = move_to(q))) return s;
        if ((s = kl(local_expect<R>(site[q], bonds[q], 2, bonds[q + 1], O, outdev, stream)))) return s;
      } else {
        if (centre > q + 1) { if ((s = move_to(q + 1))) return s; }
        else if (centre < q) { if ((s = move_to(q))) return s; }
        const int cl = bonds[q], chi = bonds[q + 1], cr = bonds[q + 2];
        if ((s = gemm(2 * cl, 2 * cr, chi, R(1), site[q], chi, 1, 0, site[q + 1], 2 * cr, 1, 0, T, 2 * cr, 1))) return s;
        if ((s = kl(local_expect<R>(T, cl, 4, cr, O, outdev, stream)))) return s;
      }
      if ((s = cu(cudaMemcpyAsync(hout, outdev, sizeof(double2), cudaMemcpyDeviceToHost, stream)))) return s;
      if ((s = cu(cudaStreamSynchronize(stream)))) return s;
      out[0] = hout[0].x;
      out[1] = hout[0].y;
      return MPS_OK;
    }
    // MIXED: Tr(O rho) / Tr(rho), weights over t = 2 s + s': Tr(O rho) = sum O[s', s] rho[s, s']
    std::vector<double2> w((size_t)N * d, make_double2(0, 0));
    for (int i = 0; i < N; ++i) { w[(size_t)i * d + 0] = make_double2(1, 0); w[(size_t)i * d + 3] = make_double2(1, 0); }
    double2 w2[16];
    int q2 = -1;
    if (support == 1) {
      for (int sg = 0; sg < 2; ++sg)
        for (int sp = 0; sp < 2; ++sp)
          w[(size_t)q * d + 2 * sg + sp] = make_double2(op[2 * (sp * 2 + sg)], op[2 * (sp * 2 + sg) + 1]);
    } else {
      q2 = q;
      for (int s1 = 0; s1 < 2; ++s1)
        for (int s1p = 0; s1p < 2; ++s1p)
          for (int s2 = 0; s2 < 2; ++s2)
            for (int s2p = 0; s2p < 2; ++s2p) {
              const int row = 2 * s1p + s2p, colx = 2 * s1 + s2;
              w2[(2 * s1 + s1p) * 4 + (2 * s2 + s2p)] = make_double2(op[2 * (row * 4 + colx)], op[2 * (row * 4 + colx) + 1]);
            }
    }
    double2 num, tr;
    if ((s = chain(w, q2, q2 >= 0 ? w2 : nullptr, &num))) return s;
    if ((s = trace_stored(&tr))) return s;
    const double den = tr.x * tr.x + tr.y * tr.y;
    out[0] = (num.x * tr.x + num.y * tr.y) / den;
    out[1] = (num.y * tr.x - num.x * tr.y) / den;
    return MPS_OK;
  }

  mps_status amplitude(const unsigned char* bits, double* out) override {
    if (mps_status js = join_side()) return js;
    if (sticky) return from_bits(sticky);
    if (!bits || !out) return MPS_ERR_ARG;
    std::vector<double2> w((size_t)N * d, make_double2(0, 0));
    for (int i = 0; i < N; ++i) {
      if (bits[i] > 1) return MPS_ERR_ARG;
      const int t = (d == 2) ? bits[i] : 3 * bits[i];
      w[(size_t)i * d + t] = make_double2(1, 0);
    }
    double2 v;
    mps_status s;
    if ((s = chain(w, -1, nullptr, &v))) return s;
    if (d == 4) {
      double2 tr;
      if ((s = trace_stored(&tr))) return s;
      const double den = tr.x * tr.x + tr.y * tr.y;
      const double2 r = make_double2((v.x * tr.x + v.y * tr.y) / den, (v.y * tr.x - v.x * tr.y) / den);
      v = r;
    }
    out[0] = v.x;
    out[1] = v.y;
    return MPS_OK;
  }

  mps_status get_site(int i, double* out, long long capd, int* dims3) override {
    if (mps_status js = join_side()) return js;
    if (i < 0 || i >= N || !out || !dims3) return MPS_ERR_ARG;
    const long long count = (long long)bonds[i] * d * bonds[i + 1];
    dims3[0] = bonds[i]; dims3[1] = d; dims3[2] = bonds[i + 1];
    if (capd < 2 * count || (size_t)count > site_cap) return MPS_ERR_ARG;
    mps_status s;
    if ((s = kl(to_double<R>(site[i], stage, count, stream)))) return s;
    if ((s = cu(cudaMemcpyAsync(out, stage, sizeof(double2) * count, cudaMemcpyDeviceToHost, stream)))) return s;
    return cu(cudaStreamSynchronize(stream));
  }

  mps_status set_site(int i, const double* data, const int* dims3) override {
    if (mps_status js = join_side()) return js;
    if (sticky) return from_bits(sticky);
    if (vidal) return MPS_ERR_STATE;   // the Schmidt vectors would no longer match the sites
    if (i < 0 || i >= N || !data || !dims3) return MPS_ERR_ARG;
    const int cl = dims3[0], dd = dims3[1], cr = dims3[2];
    if (dd != d || cl < 1 || cr < 1 || cl > cap[i] || cr > cap[i + 1]) return MPS_ERR_ARG;
    if ((i == 0 && cl != 1) || (i == N - 1 && cr != 1)) return MPS_ERR_ARG;
    const long long count = (long long)cl * d * cr;
    mps_status s;
    if ((s = cu(cudaMemcpyAsync(stage, data, sizeof(double2) * count, cudaMemcpyHostToDevice, stream)))) return s;
    if ((s = kl(from_double<R>(stage, site[i], count, stream)))) return s;
    if ((s = cu(cudaStreamSynchronize(stream)))) return s;
    bonds[i] = cl;
    bonds[i + 1] = cr;
    return MPS_OK;
  }

  mps_status last_svals(double* out, int capn, int* count) override {
    if (mps_status js = join_side()) return js;
    if (!out || !count) return MPS_ERR_ARG;
    const int nwr = std::min(capn, last_c);
    *count = nwr;
    if (nwr <= 0) return MPS_OK;
    mps_status s;
    if ((s = cu(cudaMemcpyAsync(out, s_sorted, sizeof(double) * nwr, cudaMemcpyDeviceToHost, stream)))) return s;
    return cu(cudaStreamSynchronize(stream));
  }
};

template <class R>
mps_status make_engine(mps_handle* out, int n, const mps_options& o, cudaStream_t st) {
  Engine<R>* e = new (std::nothrow) Engine<R>();
  if (!e) return MPS_ERR_OOM;
  mps_status s = e->init(n, o, st);
  if (s != MPS_OK) { delete e; return s; }
  *out = e;
  return MPS_OK;
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

void mps_default_options(mps_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->kind = MPS_PURE;
  o->f_min = 1.0;
  o->n_2q = 0;
  o->strategy = MPS_GLOBAL;
  o->chi_max = 0;
  o->fixed_chi = 0;
  o->precision = MPS_TF32X3;
  o->mixed_fid = MPS_KEPT_RATIO;
  o->max_sweeps = 40;
  o->log_truncations = 1;
  o->vidal = 0;
  o->svd_kernel = MPS_SVD_AUTO;
  o->qr = MPS_QR_MOVES | MPS_QR_PRECONDITION;
}

const char* mps_status_string(mps_status s) {
  switch (s) {
    case MPS_OK: return "ok";
    case MPS_ERR_ARG: return "invalid argument";
    case MPS_ERR_NONADJACENT: return "gate on non-neighbouring qubits";
    case MPS_ERR_OOM: return "out of memory";
    case MPS_ERR_CUDA: return "CUDA error";
    case MPS_ERR_NOT_CONVERGED: return "Jacobi SVD did not converge within max_sweeps";
    case MPS_ERR_NONFINITE: return "non-finite singular value or weight";
    case MPS_WARN_CHI_CAP: return "bond cap reached: fidelity target no longer guaranteed";
    case MPS_ERR_TIMEOUT: return "device-side wait timed out";
    case MPS_ERR_STATE: return "invalid state";
  }
  return "unknown status";
}

mps_status mps_create(mps_handle* out, int n_qubits, const mps_options* opt, void* cuda_stream) {
  if (!out) return MPS_ERR_ARG;
  *out = nullptr;
  if (!opt || n_qubits < 2 || n_qubits > 100000) return MPS_ERR_ARG;
  if (opt->kind != MPS_PURE && opt->kind != MPS_MIXED) return MPS_ERR_ARG;
  if (!(opt->f_min > 0.0) || opt->strategy < 0 || opt->strategy > 2 || opt->chi_max < 0 || opt->fixed_chi < 0 ||
      opt->precision < 0 || opt->precision > 2 || opt->mixed_fid < 0 || opt->mixed_fid > 1 || opt->max_sweeps < 1 ||
      opt->n_2q < 0 || opt->chi_max > 4096 || opt->vidal < 0 || opt->vidal > 1 || opt->svd_kernel < 0 ||
      opt->svd_kernel > 3 || opt->qr < 0 || opt->qr > 3 ||
      (opt->vidal && opt->kind != MPS_PURE))
    return MPS_ERR_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (opt->precision == MPS_FP64) return make_engine<double>(out, n_qubits, *opt, st);
  return make_engine<float>(out, n_qubits, *opt, st);
}

mps_status mps_destroy(mps_handle h) {
  delete h;
  return MPS_OK;
}

mps_status mps_apply_1q(mps_handle h, int q, const double* op, int op_dim) {
  if (!h) return MPS_ERR_ARG;
  return h->apply_1q(q, op, op_dim);
}

mps_status mps_apply_2q(mps_handle h, int q, const double* op, int op_dim, double target) {
  if (!h) return MPS_ERR_ARG;
  return h->apply_2q(q, op, false, op_dim, target);
}

mps_status mps_apply_2q_device(mps_handle h, int q, const double* op_dev, int op_dim, double target) {
  if (!h) return MPS_ERR_ARG;
  return h->apply_2q(q, op_dev, true, op_dim, target);
}

mps_status mps_apply_circuit_device(mps_handle h, int n_gates, const int* qs, const double* ops_dev, int op_dim,
                                    double target) {
  if (!h || n_gates < 0 || (n_gates > 0 && (!qs || !ops_dev))) return MPS_ERR_ARG;
  mps_status worst = MPS_OK;
  for (int g = 0; g < n_gates; ++g) {
    mps_status s = h->apply_2q(qs[g], ops_dev + (size_t)g * 2 * op_dim * op_dim, true, op_dim, target);
    if (s == MPS_WARN_CHI_CAP) { worst = s; continue; }
    if (s != MPS_OK) return s;
  }
  return worst;
}

mps_status mps_batch_run(mps_batch_item* items, int count, int concurrency, mps_handle* keep) {
  if (count < 0 || (count > 0 && !items) || concurrency < 1) return MPS_ERR_ARG;
  if (count == 0) return MPS_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MPS_ERR_CUDA;
  for (int i = 0; i < count; ++i) {
    items[i].status = MPS_ERR_STATE;
    items[i].fidelity = 0.0;
    items[i].max_bond = 0;
    if (keep) keep[i] = nullptr;
  }
  // longest circuits first (gates x qubits), so the tail of the batch is short work
  std::vector<int> order(count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return (long long)items[a].n_gates * items[a].n_qubits > (long long)items[b].n_gates * items[b].n_qubits;
  });
  std::atomic<int> next{0};
  auto worker = [&]() {
    cudaSetDevice(dev);
    for (;;) {
      const int i = next.fetch_add(1);
      if (i >= count) break;
      mps_batch_item& it = items[order[i]];
      cudaStream_t st = nullptr;
      if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) { it.status = MPS_ERR_CUDA; continue; }
      mps_handle h = nullptr;
      mps_status s = mps_create(&h, it.n_qubits, &it.opt, st);
      if (s != MPS_OK) {
        cudaStreamDestroy(st);
        it.status = s;
        continue;
      }
      h->owns_stream = true;
      h->shared_gpu = concurrency > 1;
      s = mps_apply_circuit_device(h, it.n_gates, it.qs, it.ops_dev, it.op_dim, it.target);
      if (s == MPS_OK || s == MPS_WARN_CHI_CAP) {
        mps_status f = mps_fidelity(h, &it.fidelity);
        if (f != MPS_OK) s = f;
        int mx = 1;
        for (int b = 1; b < h->N; ++b) mx = std::max(mx, h->bonds[b]);
        it.max_bond = mx;
      }
      it.status = s;
      if (keep) keep[order[i]] = h;
      else mps_destroy(h);
    }
  };
  const int nthreads = std::min(concurrency, count);
  if (nthreads == 1) {
    worker();
  } else {
    std::vector<std::thread> pool;
    pool.reserve(nthreads);
    for (int t = 0; t < nthreads; ++t) pool.emplace_back(worker);
    for (std::thread& t : pool) t.join();
  }
  mps_status worst = MPS_OK;
  for (int i = 0; i < count; ++i) {
    const mps_status s = (mps_status)items[i].status;
    if (s == MPS_OK) continue;
    if (s == MPS_WARN_CHI_CAP) { if (worst == MPS_OK) worst = s; continue; }
    if (worst == MPS_OK || worst == MPS_WARN_CHI_CAP) worst = s;
  }
  return worst;
}

mps_status mps_qr_c64(int l, int c, void* X, long long ldx, void* Q, long long ldq, void* stream) {
  if (l < 1 || c < 1 || !X || ldx < l || l > qr_max_rows() || (Q && ldq < l)) return MPS_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int K = std::min(l, c), npan = (K + 31) / 32;
  float2 *tau = nullptr, *Tm = nullptr;
  DevCtrl* ctrl = nullptr;
  auto release = [&]() {
    if (tau) cudaFree(tau);
    if (Tm) cudaFree(Tm);
    if (ctrl) cudaFree(ctrl);
  };
  if (cudaMalloc(&tau, sizeof(float2) * K) != cudaSuccess || cudaMalloc(&Tm, sizeof(float2) * 1024 * npan) != cudaSuccess ||
      cudaMalloc(&ctrl, sizeof(DevCtrl)) != cudaSuccess) {
    release();
    return MPS_ERR_OOM;
  }
  const int fit = qr_max_ctas();
  const int ctas = qr_ctas(l, c, std::max(1, fit));
  cudaError_t err = cudaMemsetAsync(ctrl, 0, sizeof(DevCtrl), st);
  if (err == cudaSuccess) err = qr_factor((float2*)X, ldx, l, c, tau, Tm, ctrl, ctas, st);
  if (err == cudaSuccess && Q) err = qr_form_q((const float2*)X, ldx, l, c, Tm, (float2*)Q, ldq, ctrl, qr_ctas(l, K, std::max(1, fit)), st);
  int status = 0;
  if (err == cudaSuccess) err = cudaMemcpyAsync(&status, &ctrl->status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (err == cudaSuccess) err = cudaStreamSynchronize(st);
  release();
  if (err != cudaSuccess) return MPS_ERR_CUDA;
  return from_bits(status);
}

mps_status mps_overlap(mps_handle a, mps_handle b, double* out_re_im) {
  if (!a || !b || !out_re_im || a->N != b->N || a->d != b->d) return MPS_ERR_ARG;
  // finish and check the pending work of both handles (and read their log-norms)
  double la = 0.0, lb = 0.0;
  if (mps_status s = a->lognorm(&la)) return s;
  if (mps_status s = b->lognorm(&lb)) return s;
  const int N = a->N, d = a->d;
  int xa = 1, xb = 1;
  size_t sa = 1, sb = 1;
  for (int i = 0; i < N; ++i) {
    xa = std::max(xa, a->bonds[i + 1]);
    xb = std::max(xb, b->bonds[i + 1]);
    sa = std::max(sa, (size_t)a->bonds[i] * d * a->bonds[i + 1]);
    sb = std::max(sb, (size_t)b->bonds[i] * d * b->bonds[i + 1]);
  }
  cudaStream_t st = a->stream;
  double2 *E = nullptr, *T = nullptr, *SA = nullptr, *SB = nullptr;
  auto release = [&]() {
    cudaStreamSynchronize(st);
    for (double2* p : {E, T, SA, SB}) if (p) cudaFree(p);
  };
  if (cudaMalloc(&E, sizeof(double2) * (size_t)xa * xb) != cudaSuccess ||
      cudaMalloc(&T, sizeof(double2) * (size_t)xa * d * xb) != cudaSuccess ||
      cudaMalloc(&SA, sizeof(double2) * sa) != cudaSuccess || cudaMalloc(&SB, sizeof(double2) * sb) != cudaSuccess) {
    release();
    return MPS_ERR_OOM;
  }
  const double2 one = make_double2(1.0, 0.0);
  mps_status s = MPS_OK;
  auto ck = [&](cudaError_t e) { if (e != cudaSuccess && s == MPS_OK) s = MPS_ERR_CUDA; return s == MPS_OK; };
  ck(cudaMemcpyAsync(E, &one, sizeof(double2), cudaMemcpyHostToDevice, st));
  // transfer contraction: E (cla x clb) -> E' (cra x crb) = sum_s A_s^dagger E B_s
  for (int i = 0; i < N && s == MPS_OK; ++i) {
    const int cla = a->bonds[i], cra = a->bonds[i + 1], clb = b->bonds[i], crb = b->bonds[i + 1];
    if ((s = a->site_to_double(i, SA, st)) != MPS_OK) break;
    if ((s = b->site_to_double(i, SB, st)) != MPS_OK) break;
    // T[(alpha, s), beta'] = sum_beta E[alpha, beta] B[beta, s, beta']
    for (int t = 0; t < d && s == MPS_OK; ++t)
      ck(cgemm_simt<double>(cla, crb, clb, 1.0, E, clb, 1, 0, SB + (size_t)t * crb, (long long)d * crb, 1, 0,
                            T + (size_t)t * crb, (long long)d * crb, 1, st));
    // E'[alpha', beta'] = sum_{(alpha, s)} conj(A[(alpha, s), alpha']) T[(alpha, s), beta']
    if (s == MPS_OK)
      ck(cgemm_simt<double>(cra, crb, cla * d, 1.0, SA, 1, cra, 1, T, crb, 1, 0, E, crb, 1, st));
  }
  double2 r = make_double2(0.0, 0.0);
  if (s == MPS_OK) ck(cudaMemcpyAsync(&r, E, sizeof(double2), cudaMemcpyDeviceToHost, st));
  if (s == MPS_OK) ck(cudaStreamSynchronize(st));
  release();
  if (s != MPS_OK) return s;
  const double scale = std::exp(la + lb);
  out_re_im[0] = r.x * scale;
  out_re_im[1] = r.y * scale;
  return MPS_OK;
}

mps_status mps_apply_layer_device(mps_handle h, int n_gates, const int* qs, const double* ops_dev, int op_dim,
                                  double target, int concurrency) {
  if (!h) return MPS_ERR_ARG;
  return h->apply_layer(n_gates, qs, ops_dev, op_dim, target, concurrency);
}

mps_status mps_gemm_device(mps_handle h, int M, int N, int K, const void* A, long long a_rs, long long a_cs, int conjA,
                           const void* B, long long b_rs, long long b_cs, int conjB, void* C, long long c_rs,
                           long long c_cs) {
  if (!h) return MPS_ERR_ARG;
  return h->gemm_device(M, N, K, A, a_rs, a_cs, conjA, B, b_rs, b_cs, conjB, C, c_rs, c_cs);
}

mps_status mps_tsvd_device(mps_handle h, int m, int n, const void* A, long long lda, double target, int max_k,
                           double rank_tol, void* U, double* S, void* V, void* Aq, void* Ap, double* out4) {
  if (!h) return MPS_ERR_ARG;
  return h->tsvd_device(m, n, A, lda, target, max_k, rank_tol, U, S, V, Aq, Ap, out4);
}

mps_status mps_tsvd_backward_device(mps_handle h, int m, int n, int k, const void* U, const double* S, const void* V,
                                    const void* Aq_bar, const void* Ap_bar, double eps, void* A_bar) {
  if (!h) return MPS_ERR_ARG;
  return h->tsvd_backward_device(m, n, k, U, S, V, Aq_bar, Ap_bar, eps, A_bar);
}

int mps_svd_tuning(int cap, int* rows, int* cols, int* accumulate, int* layout, double* ms_tournament,
                   double* ms_gram, double* ms_unsplit) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  std::lock_guard<std::mutex> lk(tune_mutex());
  int n = 0;
  for (const auto& kv : tune_table()) {
    if (kv.first.dev != dev) continue;
    if (n < cap && rows && cols && accumulate && layout && ms_tournament && ms_gram && ms_unsplit) {
      rows[n] = kv.first.l;
      cols[n] = kv.first.c;
      accumulate[n] = kv.first.acc;
      layout[n] = kv.second.kind;
      ms_tournament[n] = kv.second.ms_tournament;
      ms_gram[n] = kv.second.ms_gram;
      ms_unsplit[n] = kv.second.ms_unsplit;
    }
    ++n;
  }
  return n;
}

mps_status mps_schedule_target(int strategy, double f_min, long long n_2q, long long n_done, double product,
                               double* f_t) {
  if (!f_t || strategy < MPS_NAIVE || strategy > MPS_NEAREST || !(f_min > 0.0) || n_2q < 0 || n_done < 0 ||
      !(product >= 0.0))
    return MPS_ERR_ARG;
  *f_t = schedule_target(strategy, f_min, n_2q, n_done, product);
  return MPS_OK;
}

mps_status mps_selftest_timeout(mps_handle h, int site, long long wait_ns) {
  if (!h) return MPS_ERR_ARG;
  return h->selftest_timeout(site, wait_ns);
}

mps_status mps_svd_tune(mps_handle h, int rows, int cols, int accumulate, int* layout) {
  if (!h) return MPS_ERR_ARG;
  return h->svd_tune(rows, cols, accumulate, layout);
}

mps_status mps_fidelity(mps_handle h, double* inferred) {
  if (!h || !inferred) return MPS_ERR_ARG;
  return h->fidelity(inferred);
}

mps_status mps_expect(mps_handle h, int q, int support, const double* op, double* out_re_im) {
  if (!h) return MPS_ERR_ARG;
  return h->expect(q, support, op, out_re_im);
}

mps_status mps_amplitude(mps_handle h, const unsigned char* bits, double* out_re_im) {
  if (!h) return MPS_ERR_ARG;
  return h->amplitude(bits, out_re_im);
}

mps_status mps_bond_dims(mps_handle h, int* out) {
  if (!h || !out) return MPS_ERR_ARG;
  for (int i = 0; i + 1 < h->N; ++i) out[i] = h->bonds[i + 1];
  return MPS_OK;
}

mps_status mps_centre(mps_handle h, int* out) {
  if (!h || !out) return MPS_ERR_ARG;
  *out = h->centre;
  return MPS_OK;
}

mps_status mps_get_site(mps_handle h, int i, double* out, long long cap, int* dims3) {
  if (!h) return MPS_ERR_ARG;
  return h->get_site(i, out, cap, dims3);
}

mps_status mps_set_site(mps_handle h, int i, const double* data, const int* dims3) {
  if (!h) return MPS_ERR_ARG;
  return h->set_site(i, data, dims3);
}

mps_status mps_set_centre(mps_handle h, int c) {
  if (!h || c < 0 || c >= h->N) return MPS_ERR_ARG;
  if (h->is_vidal()) return MPS_ERR_STATE;
  h->centre = c;
  return MPS_OK;
}

mps_status mps_lognorm(mps_handle h, double* out) {
  if (!h || !out) return MPS_ERR_ARG;
  return h->lognorm(out);
}

mps_status mps_last_singular_values(mps_handle h, double* out, int cap, int* count) {
  if (!h) return MPS_ERR_ARG;
  return h->last_svals(out, cap, count);
}

mps_status mps_truncation_log(mps_handle h, mps_trunc_record* out, int cap, int* count) {
  if (!h || !count || (cap > 0 && !out)) return MPS_ERR_ARG;
  const int n = std::min<int>(cap, (int)h->log.size());
  for (int i = 0; i < n; ++i) out[i] = h->log[i];
  *count = n;
  return MPS_OK;
}

mps_status mps_sync(mps_handle h) {
  if (!h) return MPS_ERR_ARG;
  return h->sync();
}

mps_status mps_reset(mps_handle h) {
  if (!h) return MPS_ERR_ARG;
  return h->reset();
}

mps_status mps_profile(mps_handle h, int on) {
  if (!h) return MPS_ERR_ARG;
  return h->profile(on);
}

mps_status mps_stats(mps_handle h, mps_stats_t* out) {
  if (!h || !out) return MPS_ERR_ARG;
  return h->stats(out);
}

mps_status mps_stats_reset(mps_handle h) {
  if (!h) return MPS_ERR_ARG;
  return h->stats_reset();
}

mps_status mps_cgemm_c64(int precision, int M, int N, int K, float alpha, const void* A, long long a_rs,
                         long long a_cs, int conjA, const void* B, long long b_rs, long long b_cs, int conjB, void* C,
                         long long c_rs, long long c_cs, void* cuda_stream) {
  if (M < 0 || N < 0 || K < 0 || !A || !B || !C) return MPS_ERR_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  cudaError_t e;
  if (precision == MPS_FP32) {
    e = cgemm_simt<float>(M, N, K, alpha, (const float2*)A, a_rs, a_cs, conjA, (const float2*)B, b_rs, b_cs, conjB,
                          (float2*)C, c_rs, c_cs, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? MPS_OK : MPS_ERR_CUDA;
  }
  if (precision != MPS_TF32X3) return MPS_ERR_ARG;
  const size_t need = (size_t)std::max<long long>((long long)M * (K + 16), (long long)N * (K + 16));
  TcGemm* g = tc_create(need);
  if (!g) return MPS_ERR_OOM;
  int* status = nullptr;
  if (cudaMalloc(&status, sizeof(int)) != cudaSuccess) { tc_destroy(g); return MPS_ERR_OOM; }
  cudaMemsetAsync(status, 0, sizeof(int), st);
  int launched = 0;
  e = tc_gemm(g, M, N, K, alpha, (const float2*)A, a_rs, a_cs, conjA, (const float2*)B, b_rs, b_cs, conjB,
              (float2*)C, c_rs, c_cs, st, &launched, status);
  int hs = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(status);
  tc_destroy(g);
  if (e != cudaSuccess) { std::fprintf(stderr, "eamps: CUDA error: %s\n", cudaGetErrorString(e)); return MPS_ERR_CUDA; }
  return (hs & ST_TIMEOUT) ? MPS_ERR_TIMEOUT : MPS_OK;
}

mps_status mps_superop_from_kraus(const double* kraus, int n_kraus, int nq, double* out) {
  if (!kraus || !out || n_kraus < 1 || (nq != 1 && nq != 2)) return MPS_ERR_ARG;
  superop_from_kraus_host(kraus, n_kraus, nq, out);
  return MPS_OK;
}

}  // extern "C"
