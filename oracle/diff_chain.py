"""The differentiable two-site update and the chain built from it (test infrastructure: CPU,
FP64, plain NumPy/LAPACK).

Only tests, the smoke check and the benchmark's CPU leg use this module.

The paper differentiates nothing.  Its update is the two-site SVD with a cut (Eq. svd and the
"Entanglement-aware" section: keep the smallest k with W_k >= f_t W, renormalise the kept
values).  This module states that update as a function of the two-site block and gives

* ``tsvd``: full thin SVD, the cut, and the outputs of a rightward update
  A_q = U_k and A_p = diag(s_k / sqrt(W_k)) V_k^H;
* ``tsvd_backward``: the reverse-mode derivative of (A_q, A_p) with respect to the block,
  derived from first-order perturbation of the SVD (steps in the function body);
* ``DiffChain``: an MPS in mixed canonical form that moves its centre by the same update with
  no cut and applies every gate as a rightward update at (q, q+1), with the energy
  sum_i <Z_i Z_{i+1}>.

Pins (tests/test_oracle_diff.py): ``tsvd_backward`` against central finite differences of
phase-invariant losses (truncated and untruncated, tall and wide blocks); ``DiffChain`` without a
cut against the exact state vector; its energy gradient against the parameter-shift rule on the
exact state vector.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["tsvd", "tsvd_backward", "DiffChain", "zz_energy_dense"]


def _select(s: np.ndarray, target: float, max_k: int, rank_tol: float) -> tuple[int, float, float, float]:
    """The cut of the "Entanglement-aware" section on descending values s: the smallest k with
    W_k >= target * W (all values when target >= 1), never keeping values at or below
    rank_tol * s_0, at most max_k (> 0), at least 1.  Returns (k, W_k/W, W, W_k)."""
    c = len(s)
    w = float(np.sum(s * s))
    k = c
    if target < 1.0:
        cum = np.cumsum(s * s)
        k = int(np.argmax(cum >= target * w)) + 1
    nz = int(np.sum(s > rank_tol * s[0]))
    k = min(k, nz)
    if max_k > 0:
        k = min(k, max_k)
    k = max(k, 1)
    wk = float(np.sum(s[:k] ** 2))
    return k, (wk / w if w > 0 else 1.0), w, wk


def tsvd(a: np.ndarray, target: float = 1.0, max_k: int = 0, rank_tol: float = 0.0) -> dict:
    """Full thin SVD of a (m x n) and the outputs of a rightward update with the cut."""
    u, s, vh = np.linalg.svd(a, full_matrices=False)
    v = vh.conj().T
    k, f, w, wk = _select(s, target, max_k, rank_tol)
    aq = u[:, :k].copy()
    ap = (s[:k] / math.sqrt(wk))[:, None] * vh[:k]
    return {"U": u, "S": s, "V": v, "k": k, "f": f, "W": w, "W_k": wk, "Aq": aq, "Ap": ap}


def tsvd_backward(u: np.ndarray, s: np.ndarray, v: np.ndarray, k: int, aq_bar, ap_bar,
                  eps: float = 0.0) -> np.ndarray:
    """dL/dRe(A) + i dL/dIm(A) from the cotangents of A_q = U_k and A_p = diag(s_k/sqrt(W_k)) V_k^H.

    Cotangent convention: for a real loss L and complex X, Xbar = dL/dRe X + i dL/dIm X, so that
    dL = Re sum(conj(Xbar) * dX).  u (m x c), s (c), v (n x c) are the full thin SVD.
    """
    m, c = u.shape
    n = v.shape[0]
    aq_bar = np.zeros((m, k), complex) if aq_bar is None else aq_bar
    ap_bar = np.zeros((k, n), complex) if ap_bar is None else ap_bar
    wk = float(np.sum(s[:k] ** 2))
    sig = s[:k] / math.sqrt(wk)
    # 1. A_p = diag(sigma) V_k^H: sigmabar_i = Re (Abar_p V)_ii, Vbar_k = Abar_p^H diag(sigma)
    sig_bar = np.real(np.einsum("ij,ji->i", ap_bar, v[:, :k]))
    # 2. sigma_i = s_i / sqrt(W_k): sbar_l = sigmabar_l / sqrt(W_k) - s_l (sigmabar . s) / W_k^(3/2)
    s_bar = np.zeros(c)
    s_bar[:k] = sig_bar / math.sqrt(wk) - s[:k] * float(sig_bar @ s[:k]) / wk ** 1.5
    u_bar = np.zeros((m, c), complex)
    u_bar[:, :k] = aq_bar
    v_bar = np.zeros((n, c), complex)
    v_bar[:, :k] = ap_bar.conj().T * sig[None, :]
    # 3. first-order SVD perturbation: U^H dA V = dP S + dS - S dQ with dP = U^H dU and
    #    dQ = V^H dV anti-Hermitian; off-diagonal dP_ij, dQ_ij solve a 2x2 system with
    #    determinant s_j^2 - s_i^2, the diagonal gives ds_i and the phase difference.
    ju = u.conj().T @ u_bar
    jv = v.conj().T @ v_bar
    dd = s[None, :] ** 2 - s[:, None] ** 2          # s_j^2 - s_i^2 at (i, j)
    den = dd * dd + eps
    f = np.where(den > 0, dd / np.where(den > 0, den, 1.0), 0.0)
    np.fill_diagonal(f, 0.0)
    g = (f * (ju - ju.conj().T)) * s[None, :] + s[:, None] * (f * (jv - jv.conj().T))
    gauge = np.where(s > 0, (np.imag(np.diag(ju)) - np.imag(np.diag(jv))) / (2 * np.where(s > 0, s, 1.0)), 0.0)
    g = g + np.diag(s_bar + 1j * gauge)
    a_bar = u @ g @ v.conj().T
    # 4. the parts of dU, dV outside span(U), span(V): (1 - U U^H) dA V S^-1 and its V analogue
    inv = np.where(s > 0, 1.0 / np.where(s > 0, s, 1.0), 0.0)
    yu = u_bar * inv[None, :]
    yv = v_bar * inv[None, :]
    a_bar = a_bar + (yu - u @ (u.conj().T @ yu)) @ v.conj().T
    a_bar = a_bar + u @ (yv.conj().T - (yv.conj().T @ v) @ v.conj().T)
    return a_bar


_Z = np.array([1.0, -1.0, -1.0, 1.0])


def zz_energy_dense(psi: np.ndarray, n: int) -> float:
    """sum_i <Z_i Z_{i+1}> of a dense state (qubit 0 most significant)."""
    x = np.arange(2 ** n)
    z = [1 - 2 * ((x >> (n - 1 - i)) & 1) for i in range(n)]
    p = np.abs(psi) ** 2
    return float(sum(np.sum(p * z[i] * z[i + 1]) for i in range(n - 1)))


class DiffChain:
    """Pure-state MPS driven only by the update above (FP64).

    Centre moves: rightward by tsvd of the centre site (rows (a, s), no cut), leftward by tsvd of
    the site's adjoint.  A gate on (q, q+1) moves the centre to q, contracts theta, applies the
    gate on the physical pair and takes the rightward update with the cut at target f_t; the
    centre ends at q+1.  Values at or below rank_tol * s_0 are never kept (moves and gates).
    ``k_fixed`` (a list consumed in order, one entry per tsvd call) freezes every k, for finite
    differences that must not cross a change of bond.
    """

    def __init__(self, n: int, f_min: float = 1.0, n_2q: int = 0, rank_tol: float = 1e-10, k_fixed=None):
        self.n = n
        self.sites = [np.array([1.0, 0.0], complex).reshape(1, 2, 1) for _ in range(n)]
        self.centre = 0
        self.f_min = f_min
        self.n_2q = n_2q
        self.n_done = 0
        self.product = 1.0
        self.rank_tol = rank_tol
        self.k_fixed = list(k_fixed) if k_fixed is not None else None
        self.k_log = []

    def _tsvd(self, a, target):
        if self.k_fixed is not None:
            k = self.k_fixed.pop(0)
            r = tsvd(a, 1.0, k, 0.0)
            assert r["k"] == k
        else:
            r = tsvd(a, target, 0, self.rank_tol)
        self.k_log.append(r["k"])
        return r

    def target(self) -> float:
        """The global schedule (before truncation j+1): (F_min / P_j)^(1/(n - j)), clamped to 1."""
        if self.f_min >= 1.0 or self.product < self.f_min:
            return 1.0
        rem = max(self.n_2q - self.n_done, 1)
        return min((self.f_min / self.product) ** (1.0 / rem), 1.0)

    def move_right(self) -> None:
        c = self.centre
        a = self.sites[c]
        cl, _, cr = a.shape
        r = self._tsvd(a.reshape(cl * 2, cr), 1.0)
        k = r["k"]
        self.sites[c] = r["Aq"].reshape(cl, 2, k)
        b = self.sites[c + 1]
        self.sites[c + 1] = (r["Ap"] @ b.reshape(cr, -1)).reshape(k, 2, b.shape[2])
        self.centre = c + 1

    def move_left(self) -> None:
        c = self.centre
        a = self.sites[c]
        cl, _, cr = a.shape
        r = self._tsvd(a.reshape(cl, 2 * cr).conj().T, 1.0)     # M^H = Aq Ap, so M = Ap^H Aq^H
        k = r["k"]
        self.sites[c] = r["Aq"].conj().T.reshape(k, 2, cr)
        b = self.sites[c - 1]
        self.sites[c - 1] = (b.reshape(-1, cl) @ r["Ap"].conj().T).reshape(b.shape[0], 2, k)
        self.centre = c - 1

    def move_to(self, q: int) -> None:
        while self.centre < q:
            self.move_right()
        while self.centre > q:
            self.move_left()

    def apply_2q(self, q: int, g: np.ndarray) -> dict:
        self.move_to(q)
        a, b = self.sites[q], self.sites[q + 1]
        cl, cr = a.shape[0], b.shape[2]
        theta = (a.reshape(cl * 2, -1) @ b.reshape(b.shape[0], -1)).reshape(cl, 4, cr)
        theta = np.einsum("st,atb->asb", g, theta).reshape(cl * 2, 2 * cr)
        f_t = self.target()
        r = self._tsvd(theta, f_t)
        k = r["k"]
        self.sites[q] = r["Aq"].reshape(cl, 2, k)
        self.sites[q + 1] = r["Ap"].reshape(k, 2, cr)
        self.centre = q + 1
        self.product *= r["f"]
        self.n_done += 1
        return r

    def energy_zz(self) -> float:
        """sum_i <Z_i Z_{i+1}>, each term from theta at the centre (the centre sweeps left to right
        from site 0)."""
        self.move_to(0)
        e = 0.0
        for i in range(self.n - 1):
            self.move_to(i)
            a, b = self.sites[i], self.sites[i + 1]
            t = (a.reshape(-1, a.shape[2]) @ b.reshape(b.shape[0], -1)).reshape(a.shape[0], 4, b.shape[2])
            e += float(np.sum((np.abs(t) ** 2) * _Z[None, :, None]))
        return e

    def to_statevector(self) -> np.ndarray:
        v = self.sites[0].reshape(2, -1)
        for a in self.sites[1:]:
            v = (v @ a.reshape(a.shape[0], -1)).reshape(-1, a.shape[2])
        return v.reshape(-1)
