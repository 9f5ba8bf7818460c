"""GB300-native entanglement-aware MPS / MPO simulation (arXiv:2307.16870 hot path).

Thin ctypes binding of ``libeamps.so`` (C ABI declared in ``include/eamps.h``).
Every step of the two-site update runs in the library's CUDA kernels; this
module only marshals arguments.  Importing it loads the library; when the
library is missing or cannot be loaded, the import fails loudly (there is no
CPU fallback).

Functions carry the C names (``mps_create``, ``mps_apply_2q``, ...).  The
class :class:`MPS` is a convenience wrapper over the same calls.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import LIB, _stale, build

__all__ = [
    "PURE", "MIXED", "NAIVE", "GLOBAL", "NEAREST", "FP64", "TF32X3", "FP32", "KEPT_RATIO", "WANG_SQRT",
    "MpsError", "MpsOptions", "TruncRecord", "load", "lib", "MPS",
    "mps_default_options", "mps_create", "mps_destroy", "mps_apply_1q", "mps_apply_2q",
    "mps_apply_2q_device", "mps_apply_circuit_device", "mps_fidelity", "mps_expect", "mps_amplitude",
    "mps_bond_dims", "mps_centre", "mps_get_site", "mps_lognorm", "mps_last_singular_values",
    "mps_truncation_log", "mps_sync", "mps_superop_from_kraus", "mps_status_string",
    "mps_reset", "mps_profile", "mps_stats", "mps_stats_reset", "MpsStats", "mps_cgemm_c64",
    "mps_set_site", "mps_set_centre", "mps_cgemm_c64_noalloc", "BatchItem", "mps_batch_run", "mps_overlap", "mps_qr_c64",
    "mps_apply_layer_device", "mps_gemm_device", "mps_tsvd_device", "mps_tsvd_backward_device",
    "mps_selftest_timeout", "mps_schedule_target", "mps_svd_tuning", "mps_svd_tune",
]

PURE, MIXED = 0, 1
NAIVE, GLOBAL, NEAREST = 0, 1, 2
FP64, TF32X3, FP32 = 0, 1, 2
KEPT_RATIO, WANG_SQRT = 0, 1
SVD_AUTO, SVD_TOURNAMENT, SVD_GRAM, SVD_TOURNAMENT_UNSPLIT = 0, 1, 2, 3
QR_PRECONDITION, QR_MOVES = 1, 2
SELFTEST_FLAG, SELFTEST_JACOBI, SELFTEST_GRAM, SELFTEST_GEMM = 0, 1, 2, 3

OK, WARN_CHI_CAP = 0, 7

# The tensor-core (tcgen05) contraction path of precision TF32X3.
TC_AVAILABLE = True


class MpsOptions(C.Structure):
    _fields_ = [("kind", C.c_int), ("f_min", C.c_double), ("n_2q", C.c_longlong), ("strategy", C.c_int),
                ("chi_max", C.c_int), ("fixed_chi", C.c_int), ("precision", C.c_int), ("mixed_fid", C.c_int),
                ("max_sweeps", C.c_int), ("log_truncations", C.c_int), ("vidal", C.c_int),
                ("svd_kernel", C.c_int), ("qr", C.c_int)]


class BatchItem(C.Structure):
    """One circuit of mps_batch_run (same layout as the C struct)."""
    _fields_ = [("n_qubits", C.c_int), ("n_gates", C.c_int), ("qs", C.POINTER(C.c_int)), ("ops_dev", C.c_void_p),
                ("op_dim", C.c_int), ("target", C.c_double), ("opt", MpsOptions), ("fidelity", C.c_double),
                ("max_bond", C.c_int), ("status", C.c_int)]


class TruncRecord(C.Structure):
    _fields_ = [("q", C.c_int), ("k", C.c_int), ("rank_bound", C.c_int), ("cap_hit", C.c_int),
                ("f", C.c_double), ("f_t", C.c_double), ("W", C.c_double), ("W_k", C.c_double)]


class MpsStats(C.Structure):
    _fields_ = [("kernel_launches", C.c_longlong), ("jacobi_launches", C.c_longlong),
                ("jacobi_sweeps", C.c_longlong), ("jacobi_ms", C.c_double), ("jacobi_flops", C.c_double),
                ("gemm_launches", C.c_longlong), ("gemm_ms", C.c_double), ("gemm_flops", C.c_double),
                ("gates", C.c_longlong), ("move_jacobi_launches", C.c_longlong), ("move_jacobi_ms", C.c_double),
                ("qr_launches", C.c_longlong), ("qr_ms", C.c_double)]


class MpsError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {mps_status_string(code)} (status {code})")


_lib = None


def load(path: str | None = None):
    """Load libeamps.so (building it first if it is missing or older than its sources)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB
    if not os.path.exists(path) or (path == LIB and _stale([])):
        build()     # missing, or older than a source or header
    lib = C.CDLL(path)
    H = C.c_void_p
    D = C.POINTER(C.c_double)
    sig = {
        "mps_default_options": (None, [C.POINTER(MpsOptions)]),
        "mps_status_string": (C.c_char_p, [C.c_int]),
        "mps_create": (C.c_int, [C.POINTER(H), C.c_int, C.POINTER(MpsOptions), C.c_void_p]),
        "mps_destroy": (C.c_int, [H]),
        "mps_apply_1q": (C.c_int, [H, C.c_int, D, C.c_int]),
        "mps_apply_2q": (C.c_int, [H, C.c_int, D, C.c_int, C.c_double]),
        "mps_apply_2q_device": (C.c_int, [H, C.c_int, C.c_void_p, C.c_int, C.c_double]),
        "mps_apply_circuit_device": (C.c_int, [H, C.c_int, C.POINTER(C.c_int), C.c_void_p, C.c_int, C.c_double]),
        "mps_apply_layer_device": (C.c_int, [H, C.c_int, C.POINTER(C.c_int), C.c_void_p, C.c_int, C.c_double,
                                             C.c_int]),
        "mps_fidelity": (C.c_int, [H, D]),
        "mps_expect": (C.c_int, [H, C.c_int, C.c_int, D, D]),
        "mps_amplitude": (C.c_int, [H, C.POINTER(C.c_ubyte), D]),
        "mps_bond_dims": (C.c_int, [H, C.POINTER(C.c_int)]),
        "mps_centre": (C.c_int, [H, C.POINTER(C.c_int)]),
        "mps_get_site": (C.c_int, [H, C.c_int, D, C.c_longlong, C.POINTER(C.c_int)]),
        "mps_lognorm": (C.c_int, [H, D]),
        "mps_set_site": (C.c_int, [H, C.c_int, D, C.POINTER(C.c_int)]),
        "mps_cgemm_c64_noalloc": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_float, C.c_void_p, C.c_longlong,
                                            C.c_longlong, C.c_int, C.c_void_p, C.c_longlong, C.c_longlong, C.c_int,
                                            C.c_void_p, C.c_longlong, C.c_longlong, C.c_void_p]),
        "mps_set_centre": (C.c_int, [H, C.c_int]),
        "mps_last_singular_values": (C.c_int, [H, D, C.c_int, C.POINTER(C.c_int)]),
        "mps_truncation_log": (C.c_int, [H, C.POINTER(TruncRecord), C.c_int, C.POINTER(C.c_int)]),
        "mps_sync": (C.c_int, [H]),
        "mps_superop_from_kraus": (C.c_int, [D, C.c_int, C.c_int, D]),
        "mps_reset": (C.c_int, [H]),
        "mps_cgemm_c64": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_float, C.c_void_p, C.c_longlong,
                                    C.c_longlong, C.c_int, C.c_void_p, C.c_longlong, C.c_longlong, C.c_int,
                                    C.c_void_p, C.c_longlong, C.c_longlong, C.c_void_p]),
        "mps_profile": (C.c_int, [H, C.c_int]),
        "mps_stats": (C.c_int, [H, C.POINTER(MpsStats)]),
        "mps_stats_reset": (C.c_int, [H]),
        "mps_batch_run": (C.c_int, [C.POINTER(BatchItem), C.c_int, C.c_int, C.POINTER(H)]),
        "mps_overlap": (C.c_int, [H, H, D]),
        "mps_qr_c64": (C.c_int, [C.c_int, C.c_int, C.c_void_p, C.c_longlong, C.c_void_p, C.c_longlong, C.c_void_p]),
        "mps_gemm_device": (C.c_int, [H, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_longlong, C.c_longlong, C.c_int,
                                      C.c_void_p, C.c_longlong, C.c_longlong, C.c_int, C.c_void_p, C.c_longlong,
                                      C.c_longlong]),
        "mps_tsvd_device": (C.c_int, [H, C.c_int, C.c_int, C.c_void_p, C.c_longlong, C.c_double, C.c_int, C.c_double,
                                      C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.POINTER(C.c_double)]),
        "mps_tsvd_backward_device": (C.c_int, [H, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                               C.c_void_p, C.c_void_p, C.c_double, C.c_void_p]),
        "mps_selftest_timeout": (C.c_int, [H, C.c_int, C.c_longlong]),
        "mps_svd_tune": (C.c_int, [H, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int)]),
        "mps_svd_tuning": (C.c_int, [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                     C.POINTER(C.c_int), C.POINTER(C.c_double), C.POINTER(C.c_double),
                                     C.POINTER(C.c_double)]),
        "mps_schedule_target": (C.c_int, [C.c_int, C.c_double, C.c_longlong, C.c_longlong, C.c_double,
                                          C.POINTER(C.c_double)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def lib():
    return load()


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _cplx(op) -> np.ndarray:
    """Row-major complex matrix -> contiguous interleaved doubles (kept alive by the caller)."""
    return np.ascontiguousarray(np.asarray(op, dtype=np.complex128)).view(np.float64).reshape(-1)


def _check(code: int, where: str, allow_warn: bool = True) -> int:
    if code == OK or (allow_warn and code == WARN_CHI_CAP):
        return code
    raise MpsError(code, where)


# ---------------------------------------------------------------- C-named wrappers
def mps_status_string(code: int) -> str:
    return load().mps_status_string(int(code)).decode()


def mps_default_options() -> MpsOptions:
    o = MpsOptions()
    load().mps_default_options(C.byref(o))
    return o


def mps_create(n_qubits: int, opt: MpsOptions, stream: int = 0) -> int:
    h = C.c_void_p()
    _check(load().mps_create(C.byref(h), int(n_qubits), C.byref(opt), C.c_void_p(stream or None)), "mps_create")
    return h.value


def mps_destroy(h: int) -> None:
    load().mps_destroy(C.c_void_p(h))


def mps_apply_1q(h: int, q: int, op) -> int:
    a = _cplx(op)
    dim = int(round((a.size // 2) ** 0.5))
    return _check(load().mps_apply_1q(C.c_void_p(h), int(q), _dptr(a), dim), "mps_apply_1q")


def mps_apply_2q(h: int, q: int, op, target: float = -1.0) -> int:
    a = _cplx(op)
    dim = int(round((a.size // 2) ** 0.5))
    return _check(load().mps_apply_2q(C.c_void_p(h), int(q), _dptr(a), dim, float(target)), "mps_apply_2q")


def mps_apply_2q_device(h: int, q: int, op_dev_ptr: int, op_dim: int, target: float = -1.0) -> int:
    return _check(load().mps_apply_2q_device(C.c_void_p(h), int(q), C.c_void_p(op_dev_ptr), int(op_dim),
                                             float(target)), "mps_apply_2q_device")


def mps_apply_circuit_device(h: int, qs, ops_dev_ptr: int, op_dim: int, target: float = -1.0) -> int:
    q = np.ascontiguousarray(np.asarray(qs, dtype=np.int32))
    return _check(load().mps_apply_circuit_device(C.c_void_p(h), int(q.size), q.ctypes.data_as(C.POINTER(C.c_int)),
                                                  C.c_void_p(ops_dev_ptr), int(op_dim), float(target)),
                  "mps_apply_circuit_device")


def mps_apply_layer_device(h: int, qs, ops_dev_ptr: int, op_dim: int = 4, target: float = -1.0,
                           concurrency: int = 8) -> int:
    """One layer of gates on disjoint pairs of a Vidal handle, run concurrently (see include/eamps.h)."""
    q = np.ascontiguousarray(np.asarray(qs, dtype=np.int32))
    return _check(load().mps_apply_layer_device(C.c_void_p(h), int(q.size), q.ctypes.data_as(C.POINTER(C.c_int)),
                                                C.c_void_p(ops_dev_ptr), int(op_dim), float(target),
                                                int(concurrency)), "mps_apply_layer_device")


def mps_gemm_device(h: int, M: int, N: int, K: int, a: int, a_rs: int, a_cs: int, conj_a: int, b: int, b_rs: int,
                    b_cs: int, conj_b: int, c: int, c_rs: int, c_cs: int) -> int:
    """C = op(A) op(B) on device buffers with the handle's scratch and stream (see include/eamps.h)."""
    return _check(load().mps_gemm_device(C.c_void_p(h), int(M), int(N), int(K), C.c_void_p(a), int(a_rs), int(a_cs),
                                         int(conj_a), C.c_void_p(b), int(b_rs), int(b_cs), int(conj_b), C.c_void_p(c),
                                         int(c_rs), int(c_cs)), "mps_gemm_device")


def mps_tsvd_device(h: int, m: int, n: int, a: int, lda: int, target: float, max_k: int, rank_tol: float, u: int,
                    s: int, v: int, aq: int, ap: int) -> tuple:
    """Truncated SVD and rightward write-back on device buffers; returns (k, W_k/W, W, W_k)."""
    out = (C.c_double * 4)()
    _check(load().mps_tsvd_device(C.c_void_p(h), int(m), int(n), C.c_void_p(a), int(lda), float(target), int(max_k),
                                  float(rank_tol), C.c_void_p(u), C.c_void_p(s), C.c_void_p(v), C.c_void_p(aq),
                                  C.c_void_p(ap), out), "mps_tsvd_device")
    return int(out[0]), out[1], out[2], out[3]


def mps_tsvd_backward_device(h: int, m: int, n: int, k: int, u: int, s: int, v: int, aq_bar: int, ap_bar: int,
                             eps: float, a_bar: int) -> int:
    """Reverse-mode derivative of mps_tsvd_device's outputs (see include/eamps.h)."""
    return _check(load().mps_tsvd_backward_device(C.c_void_p(h), int(m), int(n), int(k), C.c_void_p(u), C.c_void_p(s),
                                                  C.c_void_p(v), C.c_void_p(aq_bar or None),
                                                  C.c_void_p(ap_bar or None), float(eps), C.c_void_p(a_bar)),
                  "mps_tsvd_backward_device")


def mps_svd_tuning() -> list[dict]:
    """The Jacobi layout autotuner's table for the current device (see include/eamps.h)."""
    lib = load()
    n = lib.mps_svd_tuning(0, None, None, None, None, None, None, None)
    if n <= 0:
        return []
    ib = [(C.c_int * n)() for _ in range(4)]
    db = [(C.c_double * n)() for _ in range(3)]
    lib.mps_svd_tuning(n, *ib, *db)
    names = {SVD_TOURNAMENT: "tournament", SVD_GRAM: "gram", SVD_TOURNAMENT_UNSPLIT: "tournament_unsplit",
             SVD_AUTO: "rule"}
    return [{"rows": ib[0][i], "cols": ib[1][i], "accumulate": bool(ib[2][i]), "layout": names.get(ib[3][i], "?"),
             "ms_tournament": db[0][i], "ms_gram": db[1][i], "ms_unsplit": db[2][i]} for i in range(n)]


def mps_schedule_target(strategy: int, f_min: float, n_2q: int, n_done: int, product: float) -> float:
    """The schedule's per-truncation target (see include/eamps.h)."""
    out = C.c_double()
    _check(load().mps_schedule_target(int(strategy), float(f_min), int(n_2q), int(n_done), float(product),
                                      C.byref(out)), "mps_schedule_target")
    return out.value


def mps_svd_tune(h: int, rows: int, cols: int, accumulate: bool = False) -> int:
    """Tune the Jacobi layout of one shape class ahead of use; returns the layout it now uses."""
    out = C.c_int(0)
    _check(load().mps_svd_tune(C.c_void_p(h), int(rows), int(cols), int(bool(accumulate)), C.byref(out)),
           "mps_svd_tune")
    return out.value


def mps_selftest_timeout(h: int, site: int = 0, wait_ns: int = 50_000_000) -> int:
    """Failure-detection self-test: a withheld signal makes a bounded device wait run out
    (site: SELFTEST_FLAG, SELFTEST_JACOBI, SELFTEST_GRAM, SELFTEST_GEMM; see include/eamps.h)."""
    return _check(load().mps_selftest_timeout(C.c_void_p(h), int(site), int(wait_ns)), "mps_selftest_timeout")


def mps_qr_c64(l: int, c: int, x_ptr: int, ldx: int, q_ptr: int = 0, ldq: int = 0, stream: int = 0) -> int:
    """In-place Householder QR of a device complex64 matrix (see include/eamps.h)."""
    return _check(load().mps_qr_c64(int(l), int(c), C.c_void_p(x_ptr), int(ldx), C.c_void_p(q_ptr or None),
                                    int(ldq), C.c_void_p(stream or None)), "mps_qr_c64")


def mps_overlap(a: int, b: int) -> complex:
    out = np.zeros(2)
    _check(load().mps_overlap(C.c_void_p(a), C.c_void_p(b), _dptr(out)), "mps_overlap")
    return complex(out[0], out[1])


def mps_fidelity(h: int) -> float:
    v = C.c_double()
    _check(load().mps_fidelity(C.c_void_p(h), C.byref(v)), "mps_fidelity")
    return v.value


def mps_expect(h: int, q: int, op) -> complex:
    a = _cplx(op)
    dim = int(round((a.size // 2) ** 0.5))
    out = np.zeros(2)
    _check(load().mps_expect(C.c_void_p(h), int(q), 1 if dim == 2 else 2, _dptr(a), _dptr(out)), "mps_expect")
    return complex(out[0], out[1])


def mps_amplitude(h: int, bits) -> complex:
    b = np.ascontiguousarray(np.asarray(bits, dtype=np.uint8))
    out = np.zeros(2)
    _check(load().mps_amplitude(C.c_void_p(h), b.ctypes.data_as(C.POINTER(C.c_ubyte)), _dptr(out)), "mps_amplitude")
    return complex(out[0], out[1])


def mps_bond_dims(h: int, n_qubits: int) -> list[int]:
    out = (C.c_int * max(n_qubits - 1, 1))()
    _check(load().mps_bond_dims(C.c_void_p(h), out), "mps_bond_dims")
    return list(out)[: n_qubits - 1]


def mps_centre(h: int) -> int:
    v = C.c_int()
    _check(load().mps_centre(C.c_void_p(h), C.byref(v)), "mps_centre")
    return v.value


def mps_get_site(h: int, i: int, max_elems: int) -> np.ndarray:
    buf = np.zeros(2 * max_elems)
    dims = (C.c_int * 3)()
    _check(load().mps_get_site(C.c_void_p(h), int(i), _dptr(buf), buf.size, dims), "mps_get_site")
    n = dims[0] * dims[1] * dims[2]
    return buf[: 2 * n].view(np.complex128).reshape(dims[0], dims[1], dims[2]).copy()


def mps_set_site(h: int, i: int, tensor) -> int:
    t = np.ascontiguousarray(np.asarray(tensor, dtype=np.complex128))
    if t.ndim != 3:
        raise ValueError("site tensor must be (chi_L, d, chi_R)")
    dims = (C.c_int * 3)(*t.shape)
    return _check(load().mps_set_site(C.c_void_p(h), int(i), _dptr(t.view(np.float64).reshape(-1)), dims),
                  "mps_set_site")


def mps_set_centre(h: int, c: int) -> int:
    return _check(load().mps_set_centre(C.c_void_p(h), int(c)), "mps_set_centre")


def mps_lognorm(h: int) -> float:
    v = C.c_double()
    _check(load().mps_lognorm(C.c_void_p(h), C.byref(v)), "mps_lognorm")
    return v.value


def mps_last_singular_values(h: int, cap: int = 1 << 14) -> np.ndarray:
    buf = np.zeros(cap)
    cnt = C.c_int()
    _check(load().mps_last_singular_values(C.c_void_p(h), _dptr(buf), cap, C.byref(cnt)), "mps_last_singular_values")
    return buf[: cnt.value].copy()


def mps_truncation_log(h: int, cap: int = 1 << 20) -> list[dict]:
    arr = (TruncRecord * cap)()
    cnt = C.c_int()
    _check(load().mps_truncation_log(C.c_void_p(h), arr, cap, C.byref(cnt)), "mps_truncation_log")
    return [{"q": r.q, "k": r.k, "rank_bound": r.rank_bound, "cap_hit": r.cap_hit, "f": r.f, "f_t": r.f_t,
             "W": r.W, "W_k": r.W_k} for r in arr[: cnt.value]]


def mps_sync(h: int) -> int:
    return _check(load().mps_sync(C.c_void_p(h)), "mps_sync")


def mps_reset(h: int) -> int:
    return _check(load().mps_reset(C.c_void_p(h)), "mps_reset")


def mps_profile(h: int, on: bool) -> int:
    return _check(load().mps_profile(C.c_void_p(h), int(bool(on))), "mps_profile")


def mps_stats(h: int) -> dict:
    st = MpsStats()
    _check(load().mps_stats(C.c_void_p(h), C.byref(st)), "mps_stats")
    return {name: getattr(st, name) for name, _ in MpsStats._fields_}


def mps_stats_reset(h: int) -> int:
    return _check(load().mps_stats_reset(C.c_void_p(h)), "mps_stats_reset")


def mps_cgemm_c64(precision: int, M: int, N: int, K: int, alpha: float, A: int, a_rs: int, a_cs: int, conjA: bool,
                  B: int, b_rs: int, b_cs: int, conjB: bool, Cp: int, c_rs: int, c_cs: int, stream: int = 0) -> int:
    """C = alpha op(A) op(B) on device complex64 buffers (pointers as ints)."""
    return _check(load().mps_cgemm_c64(int(precision), M, N, K, float(alpha), C.c_void_p(A), a_rs, a_cs, int(conjA),
                                       C.c_void_p(B), b_rs, b_cs, int(conjB), C.c_void_p(Cp), c_rs, c_cs,
                                       C.c_void_p(stream or None)), "mps_cgemm_c64")


def mps_cgemm_c64_noalloc(M: int, N: int, K: int, alpha: float, A: int, a_rs: int, a_cs: int, conjA: bool,
                          B: int, b_rs: int, b_cs: int, conjB: bool, Cp: int, c_rs: int, c_cs: int,
                          stream: int = 0) -> int:
    """Allocation-free tensor-core C = alpha op(A) op(B) on device complex64 buffers (pointers as ints)."""
    return _check(load().mps_cgemm_c64_noalloc(M, N, K, float(alpha), C.c_void_p(A), a_rs, a_cs, int(conjA),
                                               C.c_void_p(B), b_rs, b_cs, int(conjB), C.c_void_p(Cp), c_rs, c_cs,
                                               C.c_void_p(stream or None)), "mps_cgemm_c64_noalloc")


def mps_batch_run(circuits: list, concurrency: int = 4, keep: bool = False):
    """Run independent circuits concurrently (see mps_batch_run in include/eamps.h).

    circuits: dicts with n_qubits, qs (gate left qubits), ops_dev (device pointer to the
    gates, 2*op_dim*op_dim doubles each), op_dim, and optionally target and the MPS option
    names (kind, f_min, n_2q, strategy, chi_max, fixed_chi, precision, mixed_fid, max_sweeps).
    Returns (status, results) with one dict per circuit (fidelity, max_bond, status and, with
    keep, an MPS object adopting the circuit's handle)."""
    n = len(circuits)
    items = (BatchItem * max(n, 1))()
    qs_keep = []
    for i, c in enumerate(circuits):
        q = np.ascontiguousarray(np.asarray(c["qs"], dtype=np.int32))
        qs_keep.append(q)
        it = items[i]
        it.n_qubits, it.n_gates = int(c["n_qubits"]), int(q.size)
        it.qs = q.ctypes.data_as(C.POINTER(C.c_int))
        it.ops_dev = C.c_void_p(int(c["ops_dev"]))
        it.op_dim = int(c.get("op_dim", 4))
        it.target = float(c.get("target", -1.0))
        o = mps_default_options()
        for name in ("kind", "f_min", "n_2q", "strategy", "chi_max", "fixed_chi", "precision", "mixed_fid",
                     "max_sweeps", "vidal", "svd_kernel", "qr"):
            if name in c:
                setattr(o, name, c[name])
        o.log_truncations = int(c.get("log_truncations", 0))
        it.opt = o
    handles = (C.c_void_p * max(n, 1))() if keep else None
    code = load().mps_batch_run(items, n, int(concurrency), handles)
    results = []
    for i, c in enumerate(circuits):
        r = {"fidelity": items[i].fidelity, "max_bond": items[i].max_bond, "status": items[i].status}
        if keep and handles[i]:
            r["mps"] = MPS.adopt(handles[i], int(c["n_qubits"]), int(c.get("kind", PURE)))
        results.append(r)
    del qs_keep
    return code, results


def mps_superop_from_kraus(kraus: list, nq: int) -> np.ndarray:
    ks = np.concatenate([_cplx(k) for k in kraus])
    out = np.zeros(2 * 16 ** nq)
    _check(load().mps_superop_from_kraus(_dptr(ks), len(kraus), int(nq), _dptr(out)), "mps_superop_from_kraus")
    d = 4 ** nq
    return out.view(np.complex128).reshape(d, d).copy()


# ---------------------------------------------------------------- convenience class
class MPS:
    """One EA-MPS (kind=PURE) or EA-MPO (kind=MIXED) handle on the current CUDA device."""

    def __init__(self, n_qubits: int, kind: int = PURE, f_min: float = 1.0, n_2q: int = 0,
                 strategy: int = GLOBAL, chi_max: int = 0, fixed_chi: int = 0, precision: int = TF32X3,
                 mixed_fid: int = KEPT_RATIO, max_sweeps: int = 40, log_truncations: bool = True,
                 stream: int = 0, vidal: bool = False, svd_kernel: int | None = None, qr: int | None = None):
        o = mps_default_options()
        o.kind, o.f_min, o.n_2q, o.strategy = kind, f_min, n_2q, strategy
        o.chi_max, o.fixed_chi, o.precision, o.mixed_fid = chi_max, fixed_chi, precision, mixed_fid
        o.max_sweeps, o.log_truncations = max_sweeps, int(log_truncations)
        o.vidal = int(vidal)
        if svd_kernel is not None:
            o.svd_kernel = int(svd_kernel)
        if qr is not None:
            o.qr = int(qr)
        self.n = n_qubits
        self.kind = kind
        self.d = 2 if kind == PURE else 4
        self.h = mps_create(n_qubits, o, stream)

    @classmethod
    def adopt(cls, handle: int, n_qubits: int, kind: int = PURE) -> "MPS":
        """Wrap an existing handle (e.g. one kept by mps_batch_run); the object destroys it."""
        obj = cls.__new__(cls)
        obj.n, obj.kind, obj.d, obj.h = n_qubits, kind, 2 if kind == PURE else 4, handle
        return obj

    def svd_tune(self, rows: int, cols: int, accumulate: bool = False) -> int:
        return mps_svd_tune(self.h, rows, cols, accumulate)

    def close(self):
        if getattr(self, "h", None):
            mps_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def apply_1q(self, q, op):
        return mps_apply_1q(self.h, q, op)

    def apply_2q(self, q, op, target=-1.0):
        return mps_apply_2q(self.h, q, op, target)

    def run(self, gates, target=-1.0):
        for q, u in gates:
            mps_apply_2q(self.h, q, u, target)
        return self

    def apply_layer(self, qs, ops_dev_ptr: int, target=-1.0, concurrency: int = 8):
        """Gates on disjoint pairs (qs[g], qs[g]+1) with device operators ops_dev_ptr + g*256 bytes,
        concurrently; Vidal handles only.  Returns the status (OK or WARN_CHI_CAP)."""
        return mps_apply_layer_device(self.h, qs, ops_dev_ptr, 4, target, concurrency)

    def fidelity(self):
        return mps_fidelity(self.h)

    def overlap(self, other: "MPS") -> complex:
        """<self|other> (MIXED: Tr(rho_self^dagger rho_other)), FP64."""
        return mps_overlap(self.h, other.h)

    def expect(self, q, op):
        return mps_expect(self.h, q, op)

    def amplitude(self, bits):
        return mps_amplitude(self.h, bits)

    def bond_dims(self):
        return mps_bond_dims(self.h, self.n)

    def centre(self):
        return mps_centre(self.h)

    def site(self, i):
        b = [1] + self.bond_dims() + [1]
        return mps_get_site(self.h, i, b[i] * self.d * b[i + 1])

    def lognorm(self):
        return mps_lognorm(self.h)

    def load_sites(self, sites, centre: int):
        """Load every site tensor (list of (chi_L, d, chi_R) arrays) and declare the centre."""
        for i, a in enumerate(sites):
            mps_set_site(self.h, i, a)
        mps_set_centre(self.h, centre)

    def last_singular_values(self):
        return mps_last_singular_values(self.h)

    def truncation_log(self):
        return mps_truncation_log(self.h)

    def sync(self):
        return mps_sync(self.h)

    def reset(self):
        return mps_reset(self.h)

    def profile(self, on=True):
        return mps_profile(self.h, on)

    def stats(self):
        return mps_stats(self.h)

    def stats_reset(self):
        return mps_stats_reset(self.h)


load()
