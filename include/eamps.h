/*
 * eamps.h -- C ABI of the GB300 entanglement-aware MPS / MPO two-site update.
 *
 * The library simulates a quantum circuit of nearest-neighbour gates on a
 * matrix product state (pure states, local dimension 2, Eq. (mps) of the
 * paper) or on a vectorised matrix product operator (mixed states, local
 * dimension 4, Eq. (mpo)).  Every two-qubit gate runs the hot path of the
 * entanglement-aware algorithm ("Entanglement-aware simulations" section):
 *   move the orthogonality centre onto the gate pair (canonical form,
 *   "Canonicalization" section), contract the two site tensors with the
 *   gate into theta, take the SVD of theta, keep the smallest bond whose
 *   truncation fidelity (Eq. fT-pure / Eq. fT-mixed) is not lower than the
 *   target, and multiply the running product of truncation fidelities
 *   (Eq. prod), which is the inferred state fidelity.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Operators on the API are row-major complex matrices of doubles stored as
 *    interleaved (re, im) pairs: a d x d matrix is 2*d*d doubles.
 *  - Qubits are numbered 0..N-1 along the chain.  A two-qubit operator acts on
 *    (q, q+1) in the basis |s_q s_{q+1}>, s_q the more significant index.
 *  - Mixed states: the local index of an MPO site is t = 2 s + s' for the
 *    operator |s><s'|.  A superoperator of a channel {K} on n_q qubits is the
 *    4^n_q x 4^n_q matrix S[(t_1..), (u_1..)] = sum_K K[(s..),(r..)] conj(K[(s'..),(r'..)])
 *    with t_i = 2 s_i + s'_i, u_i = 2 r_i + r'_i (see mps_superop_from_kraus).
 *  - Ownership: host buffers passed in are borrowed and fully read (or
 *    written) before the call returns.  All device memory is owned by the
 *    handle and released by mps_destroy.  Pointers documented as "device"
 *    must point to memory of the handle's device.
 *  - Streams: all GPU work of a handle is ordered on the CUDA stream given to
 *    mps_create (NULL = the legacy default stream).
 *  - Errors: no exception crosses the ABI.  Every call returns an mps_status.
 *    GPU-side failures (non-convergence, non-finite values, a wait that timed
 *    out) are recorded in a sticky status word and returned by this and every
 *    later call of the handle.  One handle must not be used by two host
 *    threads at once.
 */
#ifndef EAMPS_H
#define EAMPS_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mps_state* mps_handle;

typedef enum {
  MPS_OK = 0,
  MPS_ERR_ARG = 1,            /* invalid argument (sizes, qubit index, operator dimension) */
  MPS_ERR_NONADJACENT = 2,    /* a two-qubit gate on non-neighbouring qubits (linear nearest-neighbour only) */
  MPS_ERR_OOM = 3,            /* device or host allocation failed */
  MPS_ERR_CUDA = 4,           /* a CUDA runtime call failed */
  MPS_ERR_NOT_CONVERGED = 5,  /* the Jacobi SVD reached max_sweeps */
  MPS_ERR_NONFINITE = 6,      /* a singular value or a weight was NaN / Inf */
  MPS_WARN_CHI_CAP = 7,       /* the bond cap bound a truncation: the fidelity target is no longer guaranteed */
  MPS_ERR_TIMEOUT = 8,        /* a device-side wait gave up (bounded spin); the handle is unusable */
  MPS_ERR_STATE = 9           /* call not valid in the current state (e.g. after a sticky error) */
} mps_status;

enum { MPS_PURE = 0, MPS_MIXED = 1 };                          /* mps_options.kind */
enum { MPS_NAIVE = 0, MPS_GLOBAL = 1, MPS_NEAREST = 2 };       /* mps_options.strategy */
enum { MPS_FP64 = 0, MPS_TF32X3 = 1, MPS_FP32 = 2 };           /* mps_options.precision */
enum { MPS_KEPT_RATIO = 0, MPS_WANG_SQRT = 1 };                /* mps_options.mixed_fid */
enum { MPS_SVD_AUTO = 0, MPS_SVD_TOURNAMENT = 1, MPS_SVD_GRAM = 2,
       MPS_SVD_TOURNAMENT_UNSPLIT = 3 };                              /* mps_options.svd_kernel */
enum { MPS_QR_PRECONDITION = 1, MPS_QR_MOVES = 2 };             /* mps_options.qr (bit flags) */

typedef struct {
  int kind;             /* MPS_PURE (d = 2) or MPS_MIXED (d = 4) */
  double f_min;         /* final fidelity to reach, F_min of Eq. (uniform); >= 1 disables truncation */
  long long n_2q;       /* number of two-qubit gates of the circuit, known in advance (Eq. uniform) */
  int strategy;         /* target schedule: MPS_NAIVE, MPS_GLOBAL (default), MPS_NEAREST (Fig. 1) */
  int chi_max;          /* cap on every bond (0 = no cap beyond 1024); the paper's advised cap */
  int fixed_chi;        /* > 0: standard fixed-maximum truncation k = min(fixed_chi, rank bound) */
  int precision;        /* MPS_TF32X3 (complex64, tensor-core 3xTF32 contractions, default),
                           MPS_FP32 (complex64, CUDA-core contractions), MPS_FP64 (complex128 throughout) */
  int mixed_fid;        /* MPO truncation fidelity: MPS_KEPT_RATIO f = W_k/W (default), MPS_WANG_SQRT f = sqrt(W_k/W) */
  int max_sweeps;       /* Jacobi sweep limit (default 40) */
  int log_truncations;  /* keep a host-side record of every truncation (default 1) */
  int vidal;            /* 1: Vidal/Hastings form (PURE only): every site right-canonical, a Schmidt vector
                           lambda kept on every bond, no centre moves; a gate on (q, q+1) is truncated from
                           the SVD of lambda_{q-1} B_q B_{q+1} ("The matrix product formalism": the
                           canonical form of Vidal), so the gates of a layer are independent.  The
                           truncation fidelity is exact only while the form stays canonical.  Default 0. */
  int svd_kernel;       /* layout of the one-sided Jacobi SVD (complex64; every layout computes the same
                           rotations up to rounding): MPS_SVD_AUTO (default) the layout measured faster for the
                           matrix's shape class (see mps_svd_tuning); where no timing was made, and always in a
                           handle that runs beside others (batch, Vidal layers), the fixed rule: the block kernel
                           with Gram-matrix inner sweeps, one thread-block cluster per pair of 16-column blocks
                           across the GPU, from 1024 columns on, else the tournament kernels (beside others
                           without the row split); MPS_SVD_TOURNAMENT the
                           cluster-resident / point-to-point tournament kernels only (the point-to-point
                           kernel at 256 and 512 rows with the rows of each column pair split over two warps);
                           MPS_SVD_TOURNAMENT_UNSPLIT the same with one warp per column pair; MPS_SVD_GRAM the
                           Gram block kernel wherever a layout fits (64 columns and more). */
  int qr;               /* Householder QR in the update (complex64), bit flags (default both): MPS_QR_MOVES
                           moves the orthogonality centre by QR ("Canonicalization" section; otherwise by a
                           Jacobi orthogonalisation), MPS_QR_PRECONDITION runs the gate SVD on the triangular
                           factor of theta (fewer sweeps, one QR more) when its shorter side has at least
                           256 columns.  Both apply to matrices of at most 512 rows. */
} mps_options;

/* One record per two-qubit gate: bond size kept, truncation fidelity f, the
 * target f_t it was chosen against, total weight W = sum s_i^2 and kept
 * weight W_k (both FP64), and the rank bound min(rows, cols) of theta. */
typedef struct {
  int q;
  int k;
  int rank_bound;
  int cap_hit;
  double f;
  double f_t;
  double W;
  double W_k;
} mps_trunc_record;

/* Fill *opt with the defaults listed above.  Never fails. */
void mps_default_options(mps_options* opt);

/* Human-readable name of a status code (static string; never NULL). */
const char* mps_status_string(mps_status s);

/* Create the product state |0...0> (PURE) or |0...0><0...0| (MIXED) on
 * n_qubits >= 2 qubits, on the current CUDA device, ordered on cuda_stream
 * (a cudaStream_t; NULL = default stream).  Allocates the site arena for the
 * largest bonds the options allow (min(cap, d^min(i, N-i)) per bond i) and
 * the scratch of the two-site update.  The uniform target f0 = F_min^(1/n_2q)
 * of Eq. (uniform) is set here.  *out receives the handle, or NULL on error.
 * Errors: MPS_ERR_ARG (n_qubits < 2, bad option values, NULL out/opt),
 * MPS_ERR_OOM, MPS_ERR_CUDA. */
mps_status mps_create(mps_handle* out, int n_qubits, const mps_options* opt, void* cuda_stream);

/* Release all device and host memory of the handle (waits for its stream).
 * NULL is accepted and ignored. */
mps_status mps_destroy(mps_handle h);

/* Apply a single-qubit operator to qubit q ("The matrix product formalism":
 * single-qubit gates do not change any bond).  op: host, 2*op_dim*op_dim
 * doubles.  PURE: op_dim = 2, a unitary; applied in place on site q.
 * MIXED: op_dim = 2 (a unitary U, applied as U rho U^dagger) or 4 (a
 * superoperator); the centre is moved to q first so that the canonical form
 * survives a non-unitary channel, and the norm change is folded into the
 * FP64 log-norm.  Errors: MPS_ERR_ARG. */
mps_status mps_apply_1q(mps_handle h, int q, const double* op, int op_dim);

/* The hot path: apply a two-qubit operator to (q, q+1) and truncate the bond
 * between them ("Truncation fidelity" and "Entanglement-aware simulations"
 * sections).  op: host, 2*op_dim*op_dim doubles; PURE: op_dim = 4 (unitary);
 * MIXED: op_dim = 4 (unitary, applied as U rho U^dagger) or 16
 * (superoperator, e.g. a gate followed by noise).
 * target < 0: use the schedule of mps_options (Eq. uniform and Fig. 1);
 * target >= 1: keep every singular value (no cut); otherwise the
 * per-truncation target f_t for this gate.  The schedule counter advances in
 * every case.  The call returns after the truncation is decided (the chosen
 * bond is read back); kernels of later calls overlap nothing of this one.
 * Errors: MPS_ERR_ARG, MPS_ERR_NONADJACENT is not possible by construction
 * (the pair is always (q, q+1)); q must satisfy 0 <= q < N-1. */
mps_status mps_apply_2q(mps_handle h, int q, const double* op, int op_dim, double target);

/* As mps_apply_2q, but op_dev points to the operator in DEVICE memory
 * (2*op_dim*op_dim doubles, same layout), e.g. a whole circuit uploaded
 * once.  The pointer must stay valid until the call returns. */
mps_status mps_apply_2q_device(mps_handle h, int q, const double* op_dev, int op_dim, double target);

/* Apply n_gates two-qubit gates: gate g acts on (qs[g], qs[g]+1) (qs: host)
 * with the operator at ops_dev + g*2*op_dim*op_dim (DEVICE doubles).  Same
 * target semantics as mps_apply_2q for every gate.  Stops at the first error. */
mps_status mps_apply_circuit_device(mps_handle h, int n_gates, const int* qs, const double* ops_dev,
                                    int op_dim, double target);

/* One layer of two-qubit gates on DISJOINT pairs of a Vidal handle
 * (mps_options.vidal = 1), run concurrently: gate g acts on (qs[g], qs[g]+1)
 * (qs: host) with the operator at ops_dev + g*32 (DEVICE doubles, op_dim 4).
 * In the canonical form of Vidal ("The matrix product formalism") a gate
 * reads the Schmidt vector of its left bond and writes its own sites and
 * middle bond only, so the gates of a layer are independent.  Up to
 * `concurrency` of them run at once, each on a helper with its own scratch
 * and stream (created on first use, kept with the handle) and the handle's
 * sites and Schmidt vectors; multi-CTA kernels share the SM count.
 * Every gate of the layer is truncated against ONE per-truncation target:
 * `target` when >= 0, else the schedule's value (mps_options.strategy) for the
 * product of fidelities at the layer's start, so the result does not depend
 * on `concurrency` or on which helper ran which gate.  Afterwards the product
 * holds all n_gates fidelities and the truncation records are in gate order.
 * Errors: MPS_ERR_STATE (not a Vidal handle); MPS_ERR_ARG (n_gates < 0, null
 * pointers with n_gates > 0, op_dim != 4, concurrency < 1, a pair out of
 * range or two pairs sharing a qubit; nothing has run then).  A failure inside
 * a gate leaves the handle in the failed state until mps_reset. */
mps_status mps_apply_layer_device(mps_handle h, int n_gates, const int* qs, const double* ops_dev, int op_dim,
                                  double target, int concurrency);

/* The Jacobi layout autotuner's table for the current device (this process).
 * Under MPS_SVD_AUTO, the first time a handle that runs alone meets a shape
 * class of the SVD's matrix (rows and columns rounded up to multiples of 64,
 * whether rotations are accumulated) with at least 256 columns, the layouts
 * of the one-sided Jacobi are timed:
 * the tournament kernels with and without the row split (the faster is kept)
 * and the Gram block layout, kept when it is at least 10 % faster still, each
 * on a copy of the matrix about to be decomposed (mps_svd_tune: on a
 * synthetic matrix).
 * Fills up to `cap` entries (class rows and columns, accumulated rotations
 * 0/1, chosen layout MPS_SVD_TOURNAMENT / MPS_SVD_TOURNAMENT_UNSPLIT /
 * MPS_SVD_GRAM, or MPS_SVD_AUTO when nothing could be timed and the fixed size
 * rule applies, and the three times in ms, -1 where a layout does not apply or
 * is the same launch as another) and returns the number of entries (-1 on a
 * CUDA error).  With cap 0 and null pointers it only counts.  Host only. */
int mps_svd_tuning(int cap, int* rows, int* cols, int* accumulate, int* layout, double* ms_tournament,
                   double* ms_gram, double* ms_unsplit);

/* Tune the Jacobi layout of one shape class ahead of use (the timing runs the
 * autotuner would otherwise make inside the first SVD of that class, see
 * mps_svd_tuning); also runs for a handle built for concurrent use, on its own
 * stream.  rows, cols: 1..the handle's largest matrix side; accumulate: 0/1.
 * *layout (may be null) receives the layout the class now uses (the handle's
 * own svd_kernel when that is not MPS_SVD_AUTO, or below 256 columns).  Blocks
 * until the timing runs end.  MPS_ERR_ARG on bad sizes. */
mps_status mps_svd_tune(mps_handle h, int rows, int cols, int accumulate, int* layout);

/* The per-truncation target f_t of the schedule (Eq. uniform and the strategies
 * of Fig. 1) before the truncation that follows n_done truncations whose
 * fidelities multiply to `product`: NAIVE f_t = F_min^(1/n_2q); GLOBAL
 * f_t = (F_min / product)^(1/m); NEAREST f_t = F_min / (product f0^(m-1)),
 * m = max(n_2q - n_done, 1); clamped to at most 1, and 1 once product < F_min
 * or F_min >= 1.  The formula the selection kernel evaluates on the device
 * (there in CUDA's pow), for callers that drive the stateless update calls.
 * Host only, no handle.  Errors: MPS_ERR_ARG (strategy out of range, f_min <= 0,
 * n_2q or n_done < 0, product < 0 or NaN, NULL f_t). */
mps_status mps_schedule_target(int strategy, double f_min, long long n_2q, long long n_done, double product,
                               double* f_t);

/* Failure-detection self-test (no trap, no fault: a signal is withheld and a
 * bounded wait runs out).  Every device-side wait of the library gives up at a
 * wall-clock deadline (2 s by default); this call sets the handle's limit to
 * wait_ns (10^3 <= wait_ns <= 2*10^10) and runs one of:
 *   MPS_SELFTEST_FLAG        one thread waits for a flag that nothing sets;
 *   MPS_SELFTEST_JACOBI      the point-to-point tournament Jacobi kernel (18
 *                            CTAs on a 64 x 288 matrix), CTA 0 withholding its
 *                            block releases, so its neighbours' waits run out
 *                            and every CTA returns;
 *   MPS_SELFTEST_GRAM        the Gram-matrix block Jacobi kernel (64 x 128,
 *                            clusters of CTAs), slot 0 withholding its block
 *                            releases: the clusters agree on leaving at their
 *                            next cluster barrier;
 *   MPS_SELFTEST_GEMM        the tensor-core contraction (128 x 128 x 64) with
 *                            CTA (0, 0)'s operand loads withheld: its MMA
 *                            issuer's wait runs out, every role returns and the
 *                            tensor memory is released.
 * The kernel records the timeout in the handle's status word and returns.
 * Returns MPS_ERR_TIMEOUT; the handle then stays in the failed state until
 * mps_reset (which also restores the default limit), like after any
 * device-side timeout.  Other handles are not affected.  The multi-CTA forms
 * need a complex64 handle (MPS_SELFTEST_GEMM: MPS_TF32X3).
 * Errors: MPS_ERR_ARG (site or wait_ns out of range, wrong precision),
 * MPS_ERR_OOM, MPS_ERR_CUDA. */
enum { MPS_SELFTEST_FLAG = 0, MPS_SELFTEST_JACOBI = 1, MPS_SELFTEST_GRAM = 2, MPS_SELFTEST_GEMM = 3 };
mps_status mps_selftest_timeout(mps_handle h, int site, long long wait_ns);

/* ---- Differentiable two-site update (stateless; the paper differentiates nothing) ----
 * These three calls run the steps of one two-site update (Eq. svd and the cut
 * of the "Entanglement-aware" section) on caller-owned DEVICE buffers, so that
 * an autograd layer can chain them and run their derivatives.  They use the
 * scratch, stream and precision of handle h: complex64 elements (float2) for
 * MPS_TF32X3 and MPS_FP32 handles, complex128 (double2) for MPS_FP64 handles.
 * The handle's state, schedule and statistics other than launch counts are
 * not touched.  Sizes are limited by the handle's scratch: max(m, n) at most
 * d * (the largest bond cap) and m * n at most its largest two-site block.
 * All matrices are row-major unless strides say otherwise. */

/* C (M x N) = op(A) op(B), element (r, t) of A at A + r*a_rs + t*a_cs, op =
 * conjugation when conjA / conjB; C(r, j) at C + r*c_rs + j*c_cs.  M, N, K >= 1.
 * Asynchronous on the handle's stream.  Errors: MPS_ERR_ARG. */
mps_status mps_gemm_device(mps_handle h, int M, int N, int K, const void* A, long long a_rs, long long a_cs, int conjA,
                           const void* B, long long b_rs, long long b_cs, int conjB, void* C, long long c_rs,
                           long long c_cs);

/* Full thin SVD A = U diag(S) V^H of A (m x n, ld lda >= n) with c = min(m, n):
 * U (m x c), S (c doubles, descending), V (n x c); one-sided Jacobi on the
 * short side with FP64 column norms, as in the gate update.  Then the cut:
 * k = the smallest count with W_k >= target * W (target >= 1 keeps all c),
 * at most the number of values above rank_tol * S[0], at most max_k when
 * max_k > 0, at least 1.  Then the write-back of a rightward update:
 * Aq = U[:, :k] (m x k) and Ap = U_k^H A / sqrt(W_k) = diag(S_k/sqrt(W_k)) V_k^H
 * (k x n).  Aq and Ap need room for m*c and c*n elements.  out4 (HOST, 4
 * doubles) receives {k, W_k/W, W, W_k}.  Synchronises the handle's stream.
 * Errors: MPS_ERR_ARG (sizes, null pointers, target < 0 or NaN, rank_tol < 0),
 * MPS_ERR_NONFINITE (W_k = 0 or not finite), MPS_ERR_NOT_CONVERGED,
 * MPS_ERR_TIMEOUT, MPS_ERR_CUDA. */
mps_status mps_tsvd_device(mps_handle h, int m, int n, const void* A, long long lda, double target, int max_k,
                           double rank_tol, void* U, double* S, void* V, void* Aq, void* Ap, double* out4);

/* Reverse-mode derivative of mps_tsvd_device: from the factors it returned (U,
 * S, V) and the cotangents Aq_bar (m x k) and Ap_bar (k x n) of its outputs
 * (either may be NULL for zero), A_bar (m x n) = dL/dRe A + i dL/dIm A for a
 * real loss L.  This is the complex SVD adjoint with the gauge term and the
 * coupling to the discarded values (the exact derivative of the truncated
 * outputs when the values are distinct).  The factor 1/(s_j^2 - s_i^2) is
 * broadened to (s_j^2 - s_i^2)/((s_j^2 - s_i^2)^2 + eps), eps >= 0 (0 = exact).
 * Kept values must be > 0.  Synchronises the handle's stream.
 * Errors: MPS_ERR_ARG, MPS_ERR_TIMEOUT, MPS_ERR_CUDA. */
mps_status mps_tsvd_backward_device(mps_handle h, int m, int n, int k, const void* U, const double* S, const void* V,
                                    const void* Aq_bar, const void* Ap_bar, double eps, void* A_bar);

/* One circuit of a batch (mps_batch_run).  The inputs are read and the
 * outputs written by the call; the item array is owned by the caller. */
typedef struct {
  int n_qubits;            /* chain length, >= 2 */
  int n_gates;             /* two-qubit gates in the circuit */
  const int* qs;           /* HOST, n_gates entries: gate g acts on (qs[g], qs[g]+1) */
  const double* ops_dev;   /* DEVICE, n_gates operators of 2*op_dim*op_dim doubles (row-major complex) */
  int op_dim;              /* 4 (PURE: unitary) or 16 (MIXED: superoperator) */
  double target;           /* as for mps_apply_2q: < 0 schedule, >= 1 no truncation, else per-truncation */
  mps_options opt;         /* options of this circuit's handle */
  double fidelity;         /* out: running product of truncation fidelities (Eq. prod) */
  int max_bond;            /* out: largest bond dimension after the circuit */
  int status;              /* out: mps_status of this circuit */
} mps_batch_item;

/* Run many independent circuits, each one the gate-by-gate algorithm of
 * the "Entanglement-aware" section (as mps_apply_circuit_device from
 * |0...0>), up to `concurrency` at a time: every circuit has its own handle
 * and CUDA stream, driven by its own host thread; the longest circuits
 * (gates x qubits) start first.  With concurrency > 1 the multi-CTA Jacobi
 * launches of all running circuits share one budget of co-resident CTAs per
 * device, so no grid waits on CTAs that cannot become resident.  Each
 * circuit's results are those of running it alone.
 * keep: NULL (each handle is destroyed when its circuit ends) or an array of
 * `count` handles that receives every circuit's handle (it owns its stream;
 * release with mps_destroy).  The device operators must stay valid until
 * the call returns.
 * Returns MPS_OK; MPS_WARN_CHI_CAP when some circuit reached its bond cap;
 * else the error of the first failing item (each item's status is in
 * items[i].status).  MPS_ERR_ARG: count < 0, items == NULL with count > 0,
 * or concurrency < 1. */
mps_status mps_batch_run(mps_batch_item* items, int count, int concurrency, mps_handle* keep);

/* *inferred = running product of truncation fidelities (Eq. prod), FP64. */
mps_status mps_fidelity(mps_handle h, double* inferred);

/* Householder QR of an l x c complex64 matrix in DEVICE memory, the
 * factorisation that brings a site into canonical form ("Canonicalization"
 * section): X = Q R.  X: column-major, leading dimension ldx >= l, factored
 * in place (R, min(l, c) x c upper trapezoid with a real diagonal, in the
 * upper part; the Householder vectors, unit leading entry implicit, below).
 * Q: NULL, or DEVICE column-major l x min(l, c) (ldq >= l) receiving the
 * factor with orthonormal columns.  l <= 512.  Runs on `stream` (NULL: the
 * default stream) and synchronises it; allocates its workspace for the call.
 * Errors: MPS_ERR_ARG (sizes, NULL X), MPS_ERR_OOM, MPS_ERR_CUDA,
 * MPS_ERR_TIMEOUT (a bounded device barrier gave up). */
mps_status mps_qr_c64(int l, int c, void* X, long long ldx, void* Q, long long ldq, void* stream);

/* <a|b>: the inner product of two handles of the same length and kind
 * ("The matrix product formalism" section: the overlap of two MPS is the
 * chain of transfer contractions E <- sum_s A_s^dagger E B_s).  PURE: the
 * state overlap (|<a|b>|^2 is the true fidelity of Eq. F-pure when one
 * handle holds the exact state).  MIXED: the Hilbert-Schmidt inner product
 * Tr(rho_a^dagger rho_b) of the vectorised operators.  Both handles' norm
 * factors (the FP64 log-norms) are included.  Computed in FP64 on a's
 * stream after the pending work of both handles; the bonds and precisions of
 * a and b may differ.  Allocates its FP64 workspace for the call.
 * out_re_im: host, 2 doubles.  Errors: MPS_ERR_ARG (NULL, different lengths
 * or kinds), MPS_ERR_OOM, MPS_ERR_CUDA, or a sticky error of either handle. */
mps_status mps_overlap(mps_handle a, mps_handle b, double* out_re_im);

/* PURE: <psi|O|psi>, computed from the canonical form with only the tensors
 * on the support ("Canonicalization" section; the centre is moved onto the
 * support).  MIXED: Tr(O rho)/Tr(rho) by a transfer contraction along the
 * chain.  support = 1 (O on q, op_dim 2) or 2 (O on (q, q+1), op_dim 4).
 * op: host row-major complex; out_re_im: host, 2 doubles. */
mps_status mps_expect(mps_handle h, int q, int support, const double* op, double* out_re_im);

/* PURE: <b|psi>.  MIXED: <b|rho|b> / Tr(rho).  bits: host, N bytes (0/1),
 * qubit 0 first.  out_re_im: host, 2 doubles. */
mps_status mps_amplitude(mps_handle h, const unsigned char* bits, double* out_re_im);

/* Current bonds (N-1 ints, bond i between qubits i and i+1). */
mps_status mps_bond_dims(mps_handle h, int* out);

/* Orthogonality centre (site index). */
mps_status mps_centre(mps_handle h, int* out);

/* Copy site tensor i to the host as complex128, shape (chi_L, d, chi_R)
 * row-major, 2*chi_L*d*chi_R doubles; dims3 (host, 3 ints) receives the
 * shape.  Errors: MPS_ERR_ARG if cap (in doubles) is too small. */
mps_status mps_get_site(mps_handle h, int i, double* out, long long cap, int* dims3);

/* Load site tensor i from the host: complex128 (2*chi_L*d*chi_R doubles,
 * row-major (chi_L, d, chi_R)), dims3 = {chi_L, d, chi_R}; converted to the
 * handle's working precision.  Sets bonds i and i+1 to chi_L and chi_R.  The
 * caller loads every site it changes with consistent bonds and then declares
 * the orthogonality centre with mps_set_centre; the state must be in
 * canonical form around that centre ("Canonicalization" section) for the
 * truncation fidelities to hold.  Together with mps_get_site this saves and
 * restores a state.  Errors: MPS_ERR_ARG (index, d, bonds above the handle's
 * capacity min(cap, d^min(i, N-i)) or zero). */
mps_status mps_set_site(mps_handle h, int i, const double* data, const int* dims3);

/* Declare site c the orthogonality centre (no computation). */
mps_status mps_set_centre(mps_handle h, int c);

/* FP64 log of the norm factor of an MPO (rho = exp(lognorm) * stored rho). */
mps_status mps_lognorm(mps_handle h, double* out);

/* Singular values of the last two-qubit gate, in decreasing order (FP64),
 * all rank_bound of them.  *count receives how many were written (at most cap). */
mps_status mps_last_singular_values(mps_handle h, double* out, int cap, int* count);

/* Copy up to cap truncation records (oldest first); *count receives the number copied. */
mps_status mps_truncation_log(mps_handle h, mps_trunc_record* out, int cap, int* count);

/* Wait for all queued work of the handle and return its sticky status. */
mps_status mps_sync(mps_handle h);

/* Return the handle to its initial product state and reset the fidelity
 * product, the schedule counter, the log-norm, the truncation log and the
 * sticky status, keeping every allocation (so that repeated runs allocate
 * nothing).  Errors: MPS_ERR_CUDA. */
mps_status mps_reset(mps_handle h);

/* Kernel statistics of a handle, accumulated since the last mps_stats_reset.
 * Durations come from CUDA events recorded on the handle's stream around the
 * launches of the Jacobi SVD and of the contractions when profiling is on
 * (mps_profile); counts are always kept. */
typedef struct {
  long long kernel_launches;   /* every kernel this library launched */
  long long jacobi_launches;
  long long jacobi_sweeps;     /* sweeps summed over launches */
  double jacobi_ms;            /* summed event durations (profiling on) */
  double jacobi_flops;         /* algorithmic flops of the Jacobi launches: 16 l per visited pair
                                  (three complex inner products over l rows) + 24 L per applied
                                  rotation (two complex column updates of L rows) */
  long long gemm_launches;
  double gemm_ms;
  double gemm_flops;           /* 8 M N K per complex GEMM */
  long long gates;             /* two-qubit updates applied */
  long long move_jacobi_launches;  /* Jacobi launches of centre moves (included in jacobi_*) */
  double move_jacobi_ms;           /* their summed event durations (profiling on) */
  long long qr_launches;           /* Householder QR launches (centre moves and SVD preconditioning) */
  double qr_ms;                    /* their summed event durations (profiling on) */
} mps_stats_t;

/* Switch event timing of the Jacobi and contraction launches on (1) or off (0). */
mps_status mps_profile(mps_handle h, int on);
mps_status mps_stats(mps_handle h, mps_stats_t* out);
mps_status mps_stats_reset(mps_handle h);

/* Complex64 GEMM on device buffers with the library's contraction kernels:
 * C = alpha * op(A) * op(B), op(A)[i,k] = A[i*a_rs + k*a_cs] (conjugated if
 * conjA), likewise for B; C[i,j] at C + i*c_rs + j*c_cs.  A, B, C: DEVICE
 * float2 (interleaved complex64).  precision = MPS_TF32X3 (tcgen05 tensor
 * cores, 3xTF32 split, FP32 accumulation) or MPS_FP32 (CUDA cores).  This is
 * the contraction used for theta (the product of the two site tensors,
 * "Truncation fidelity" section); it is exported so that callers and tests
 * can run it alone.  Allocates (and frees) its packing workspace per call;
 * ordered on cuda_stream and synchronised before return.
 * Errors: MPS_ERR_ARG (sizes, precision), MPS_ERR_OOM, MPS_ERR_CUDA,
 * MPS_ERR_TIMEOUT. */
mps_status mps_cgemm_c64(int precision, int M, int N, int K, float alpha,
                         const void* A, long long a_rs, long long a_cs, int conjA,
                         const void* B, long long b_rs, long long b_cs, int conjB,
                         void* C, long long c_rs, long long c_cs, void* cuda_stream);

/* Allocation-free form of mps_cgemm_c64 with precision MPS_TF32X3 (the
 * paper has no counterpart: this is a deployment convenience).  Some callers
 * cannot call cudaMalloc or cudaFree: a host framework that owns all device
 * memory through its own pool, or a loop that must not stall, since cudaFree
 * synchronises the device.  This entry point allocates nothing: the packing
 * workspace and the status word live in one fixed array of 8 MiB + 256 bytes
 * of device memory that belongs to the loaded library, and every GPU that
 * loads the library holds it until the process exits.
 * Limits: with kp = 2K rounded up to a multiple of 32, both M*kp and 2*N*kp
 * must be <= 524288; larger shapes are rejected with MPS_ERR_ARG and a message
 * on stderr.  Arguments, layouts and results are those of mps_cgemm_c64 (A, B,
 * C in DEVICE memory, owned by the caller); the call is ordered on cuda_stream
 * and synchronised before it returns.
 * The first call on each device resolves the device address of the array
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  Every call on a device shares the same array,
 * so calls that overlap on the GPU (other host threads, other streams) race
 * and must be serialised by the caller.
 * Errors: MPS_ERR_ARG, MPS_ERR_CUDA, MPS_ERR_TIMEOUT. */
mps_status mps_cgemm_c64_noalloc(int M, int N, int K, float alpha,
                                 const void* A, long long a_rs, long long a_cs, int conjA,
                                 const void* B, long long b_rs, long long b_cs, int conjB,
                                 void* C, long long c_rs, long long c_cs, void* cuda_stream);

/* Host helper: the superoperator of the channel {K} (n_kraus operators of
 * dimension 2^nq, host, 2*4^nq doubles each, concatenated) in the library's
 * vectorisation convention (see the top of this file).  out: host,
 * 2*16^nq doubles.  nq = 1 or 2.  Errors: MPS_ERR_ARG. */
mps_status mps_superop_from_kraus(const double* kraus, int n_kraus, int nq, double* out);

#ifdef __cplusplus
}
#endif
#endif /* EAMPS_H */
