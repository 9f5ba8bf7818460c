"""Textbook entanglement-aware MPS / MPO (oracle; test infrastructure only).

Follows the paper step by step, in FP64 / complex128, with NumPy QR and SVD:

* State (Eq. mps / Eq. mpo): N site tensors A[i] of shape (chi_L, d, chi_R),
  d = 2 for a pure state and d = 4 for a vectorised density matrix (local
  index t = 2 s + s').  Sites are numbered from 0.
* Canonical form ("Canonicalization" section): one orthogonality centre c;
  sites left of c are left-normalised (sum_s A_s^dagger A_s = I), sites right
  of c are right-normalised (sum_s A_s A_s^dagger = I).  The centre moves by
  one site with a QR decomposition (reduced; the bond becomes the rank bound
  min(rows, cols)), the triangular factor being absorbed by the neighbour.
* Two-qubit gate on (q, q+1) ("Truncation fidelity" section): move the centre
  onto the pair (to q when it is at or left of q, continuing to the right; to
  q+1 when it is right of q, continuing to the left), contract both tensors
  neighbouring the bond with the gate into theta, reshape theta to a
  (d chi_L) x (d chi_R) matrix, take its SVD (singular values in decreasing
  order), keep the leading k of them, and leave the centre on the far site of
  the pair (q+1 when continuing to the right, q otherwise).
* Truncation fidelity.  Pure states, Eq. (fT-pure), read as the squared
  overlap of the state with its renormalised truncation:
  f = (sum_i L_ii Lt_ii)^2 with unit-norm L and Lt, i.e. f = W_k / W where
  W = sum_i s_i^2 and W_k = sum_{i<k} s_i^2.  (The printed form sum L^2 Lt^2
  is not 1 without truncation, so it cannot be meant literally.)  Mixed
  states, Eq. (fT-mixed), read the same way: f = W_k / W, the square of the
  Wang fidelity (Eq. Wang) between the state and its truncation; the strict
  Wang value sqrt(W_k / W) is available as ``mixed_fid=WANG_SQRT``.
* Bond size (entanglement-aware rule): the smallest k >= 1 whose truncation
  fidelity is not lower than the target f_t, compared as W_k >= f_t W in
  FP64 (W_k >= f_t^2 W for WANG_SQRT); f_t >= 1 keeps every value (no cut,
  also none on zero values).  An optional cap chi_max bounds k and sets a
  flag when it binds (the paper's advice to cap adaptive bonds, after which
  the fidelity is no longer guaranteed).  ``fixed_chi`` > 0 gives the
  standard fixed-maximum truncation k = min(fixed_chi, rank bound).
* Normalisation after a cut: the kept singular values are divided by
  sqrt(W_k), so the represented vector keeps unit norm.  For an MPO the
  factor is accumulated in ``lognorm`` (rho = exp(lognorm) * stored rho).
* Inferred fidelity (Eq. prod): running product of the truncation fidelities.
* Target schedule: n (the number of two-qubit gates) is known in advance; the
  uniform target is f0 = F_min^(1/n) (Eq. uniform).  Before truncation j+1,
  with product P_j and m = n - j truncations left (at least 1):
  NAIVE   f_t = f0;
  GLOBAL  f_t = (F_min / P_j)^(1/m)   (all upcoming targets updated evenly);
  NEAREST f_t = F_min / (P_j f0^(m-1)) (only the upcoming target updated);
  clamped to at most 1, and 1 once P_j < F_min.
"""
from __future__ import annotations

import math

import numpy as np

from . import superop as _superop

PURE, MIXED = 0, 1
NAIVE, GLOBAL, NEAREST = 0, 1, 2
KEPT_RATIO, WANG_SQRT = 0, 1


def select_bond(s: np.ndarray, f_t: float, fixed_chi: int = 0, chi_max: int = 0,
                mixed_fid: int = KEPT_RATIO):
    """Pick the kept bond size from singular values in decreasing order.

    Returns (k, f, W, W_k, cap_hit).  Entanglement-aware rule of the
    "Entanglement-aware simulations" section: the smallest k whose truncation
    fidelity is not lower than f_t.
    """
    r = len(s)
    w = s.astype(np.float64) ** 2
    cum = np.cumsum(w)
    big_w = float(cum[-1]) if r else 0.0
    cap_hit = False
    if r == 0 or big_w <= 0.0:
        return max(r, 1) if r else 0, 1.0, big_w, big_w, False
    if fixed_chi > 0:
        k = min(fixed_chi, r)
    elif f_t >= 1.0:
        k = r
    else:
        thr = (f_t * f_t if mixed_fid == WANG_SQRT else f_t) * big_w
        k = int(np.searchsorted(cum, thr, side="left")) + 1   # first index with cum >= thr
        k = min(max(k, 1), r)
    if chi_max > 0 and k > chi_max:
        k = chi_max
        cap_hit = True
    wk = float(cum[k - 1])
    f = wk / big_w
    if mixed_fid == WANG_SQRT:
        f = math.sqrt(f)
    return k, f, big_w, wk, cap_hit


class TextbookMPS:
    """FP64 entanglement-aware MPS (kind=PURE) or MPO (kind=MIXED)."""

    def __init__(self, n_qubits: int, kind: int = PURE, f_min: float = 1.0, n_2q: int = 0,
                 strategy: int = GLOBAL, chi_max: int = 0, fixed_chi: int = 0,
                 mixed_fid: int = KEPT_RATIO, record_svals: bool = False):
        self.n = n_qubits
        self.kind = kind
        self.d = 2 if kind == PURE else 4
        site = np.zeros((1, self.d, 1), np.complex128)
        site[0, 0, 0] = 1.0          # |0> ; for an MPO vec(|0><0|) has t = 0
        self.sites = [site.copy() for _ in range(n_qubits)]
        self.centre = 0
        self.f_min = f_min
        self.n_2q = n_2q
        self.strategy = strategy
        self.chi_max = chi_max
        self.fixed_chi = fixed_chi
        self.mixed_fid = mixed_fid
        self.product = 1.0
        self.lognorm = 0.0
        self.n_done = 0
        self.f0 = f_min ** (1.0 / n_2q) if (n_2q > 0 and f_min < 1.0) else 1.0
        self.cap_hit = False
        self.record_svals = record_svals
        self.log: list[dict] = []

    # ---------------------------------------------------------------- schedule
    def scheduled_target(self) -> float:
        if self.f_min >= 1.0:
            return 1.0
        if self.product < self.f_min:
            return 1.0
        m = max(self.n_2q - self.n_done, 1)
        if self.strategy == NAIVE:
            ft = self.f0
        elif self.strategy == GLOBAL:
            ft = (self.f_min / self.product) ** (1.0 / m)
        else:
            ft = self.f_min / (self.product * self.f0 ** (m - 1))
        return min(ft, 1.0)

    # ------------------------------------------------------------ canonical
    def move_centre(self, to: int) -> None:
        while self.centre < to:
            c = self.centre
            a = self.sites[c]
            cl, d, cr = a.shape
            q, r = np.linalg.qr(a.reshape(cl * d, cr))
            k = q.shape[1]
            self.sites[c] = q.reshape(cl, d, k)
            nxt = self.sites[c + 1]
            self.sites[c + 1] = (r @ nxt.reshape(nxt.shape[0], -1)).reshape(k, nxt.shape[1], nxt.shape[2])
            self.centre += 1
        while self.centre > to:
            c = self.centre
            a = self.sites[c]
            cl, d, cr = a.shape
            q, r = np.linalg.qr(a.reshape(cl, d * cr).conj().T)   # M^dagger = Q R  ->  M = R^dagger Q^dagger
            k = q.shape[1]
            self.sites[c] = q.conj().T.reshape(k, d, cr)
            prv = self.sites[c - 1]
            self.sites[c - 1] = (prv.reshape(-1, prv.shape[2]) @ r.conj().T).reshape(prv.shape[0], prv.shape[1], k)
            self.centre -= 1

    def bond_dims(self) -> list[int]:
        return [self.sites[i].shape[2] for i in range(self.n - 1)]

    # ------------------------------------------------------------ operators
    def _lift(self, op: np.ndarray, nq: int) -> np.ndarray:
        """Operator acting on the local index: unitary for PURE, superoperator for MIXED."""
        op = np.asarray(op, np.complex128)
        if self.kind == PURE:
            return op
        if op.shape[0] == 2 ** nq:           # a unitary: U rho U^dagger
            return _superop.from_unitary(op)
        return op

    def apply_1q(self, q: int, op: np.ndarray) -> None:
        g = self._lift(op, 1)
        if self.kind == MIXED:
            self.move_centre(q)
        self.sites[q] = np.einsum("st,atb->asb", g, self.sites[q])
        if self.kind == MIXED:
            w = float(np.vdot(self.sites[q], self.sites[q]).real)
            self.sites[q] = self.sites[q] / math.sqrt(w)
            self.lognorm += 0.5 * math.log(w)

    def theta(self, q: int, op: np.ndarray) -> np.ndarray:
        """Two-site tensor of sites q, q+1 with the gate applied, as a (d chi_L) x (d chi_R) matrix."""
        d = self.d
        g = self._lift(op, 2).reshape(d, d, d, d)
        a, b = self.sites[q], self.sites[q + 1]
        cl, cr = a.shape[0], b.shape[2]
        t = np.tensordot(a, b, axes=([2], [0]))              # (cl, d, d, cr)
        t = np.einsum("stuv,auvb->astb", g, t)
        return t.reshape(cl * d, d * cr)

    def apply_2q(self, q: int, op: np.ndarray, target: float | None = None) -> dict:
        if q < 0 or q + 1 >= self.n:
            raise ValueError("gate outside the chain")
        rightward = self.centre <= q
        self.move_centre(q if rightward else q + 1)
        d = self.d
        cl, cr = self.sites[q].shape[0], self.sites[q + 1].shape[2]
        m = self.theta(q, op)
        u, s, vh = np.linalg.svd(m, full_matrices=False)
        if target is None or target < 0:
            f_t = self.scheduled_target()
        else:
            f_t = min(float(target), 1.0)
        k, f, big_w, wk, cap = select_bond(s, f_t, self.fixed_chi, self.chi_max, self.mixed_fid)
        self.cap_hit |= cap
        sk = s[:k] / math.sqrt(wk)
        if self.kind == MIXED:
            self.lognorm += 0.5 * math.log(wk)
        if rightward:
            self.sites[q] = u[:, :k].reshape(cl, d, k)
            self.sites[q + 1] = (sk[:, None] * vh[:k]).reshape(k, d, cr)
            self.centre = q + 1
        else:
            self.sites[q] = (u[:, :k] * sk[None, :]).reshape(cl, d, k)
            self.sites[q + 1] = vh[:k].reshape(k, d, cr)
            self.centre = q
        self.product *= f
        self.n_done += 1
        rec = {"q": q, "k": k, "f": f, "f_t": f_t, "W": big_w, "W_k": wk, "rank_bound": len(s)}
        if self.record_svals:
            rec["s"] = s.copy()
        self.log.append(rec)
        return rec

    def run(self, gates, target: float | None = None) -> "TextbookMPS":
        for q, u in gates:
            self.apply_2q(q, u, target)
        return self

    # ------------------------------------------------------------- readout
    def contract(self) -> np.ndarray:
        """All site tensors contracted into the flat coefficient tensor (d^N entries)."""
        t = self.sites[0].reshape(self.d, -1)
        for i in range(1, self.n):
            b = self.sites[i]
            t = (t @ b.reshape(b.shape[0], -1)).reshape(-1, b.shape[2])
        return t.reshape(-1)

    def to_statevector(self) -> np.ndarray:
        assert self.kind == PURE
        return self.contract()

    def to_density_matrix(self) -> np.ndarray:
        """Dense rho (including exp(lognorm)) from the MPO; t_i = 2 s_i + s'_i."""
        assert self.kind == MIXED
        n = self.n
        c = self.contract().reshape((2, 2) * n)
        perm = list(range(0, 2 * n, 2)) + list(range(1, 2 * n, 2))
        rho = c.transpose(perm).reshape(2 ** n, 2 ** n)
        return rho * math.exp(self.lognorm)

    def amplitude(self, bits) -> complex:
        """PURE: <b|psi>.  MIXED: <b|rho|b> / Tr(rho)."""
        v = np.ones((1,), np.complex128)
        for i, b in enumerate(bits):
            t = int(b) if self.kind == PURE else 3 * int(b)
            v = v @ self.sites[i][:, t, :]
        val = complex(v[0])
        if self.kind == MIXED:
            val /= self.trace_stored()
        return val

    def trace_stored(self) -> complex:
        """Tr of the stored (unit-Frobenius-norm) operator."""
        v = np.ones((1,), np.complex128)
        for a in self.sites:
            v = v @ (a[:, 0, :] + a[:, 3, :])
        return complex(v[0])

    def expect(self, q: int, op: np.ndarray) -> complex:
        """PURE: <psi|O|psi> from the canonical form, using only the tensors on the
        support (Section "Canonicalization").  MIXED: Tr(O rho)/Tr(rho) by a
        transfer-vector contraction along the chain."""
        op = np.asarray(op, np.complex128)
        nq = 1 if op.shape[0] == 2 else 2
        if self.kind == PURE:
            if nq == 1:
                self.move_centre(q)
                a = self.sites[q]
                return complex(np.einsum("asb,st,atb->", a.conj(), op, a))
            if self.centre > q + 1:
                self.move_centre(q + 1)
            elif self.centre < q:
                self.move_centre(q)
            t = np.tensordot(self.sites[q], self.sites[q + 1], axes=([2], [0]))   # (cl, 2, 2, cr)
            tt = t.reshape(t.shape[0], 4, t.shape[3])
            return complex(np.einsum("aib,ij,ajb->", tt.conj(), op, tt))
        # MIXED: weights over the local index t = 2 s + s' (Tr(O rho) = sum O[s', s] rho[s, s'])
        v = np.ones((1,), np.complex128)
        i = 0
        while i < self.n:
            if i == q:
                if nq == 1:
                    w = np.array([op[s2, s1] for s1 in range(2) for s2 in range(2)])
                    v = v @ np.einsum("t,atb->ab", w, self.sites[i])
                    i += 1
                else:
                    t = np.tensordot(self.sites[i], self.sites[i + 1], axes=([2], [0]))  # (cl, 4, 4, cr)
                    w = np.zeros((4, 4), np.complex128)
                    for s1 in range(2):
                        for s1p in range(2):
                            for s2 in range(2):
                                for s2p in range(2):
                                    w[2 * s1 + s1p, 2 * s2 + s2p] = op[2 * s1p + s2p, 2 * s1 + s2]
                    v = v @ np.einsum("tu,atub->ab", w, t)
                    i += 2
            else:
                a = self.sites[i]
                v = v @ (a[:, 0, :] + a[:, 3, :])
                i += 1
        return complex(v[0] / self.trace_stored())

    # ------------------------------------------------------------- checks
    def canonical_error(self) -> float:
        """max over sites of the deviation from left/right normalisation around the centre."""
        err = 0.0
        for i, a in enumerate(self.sites):
            cl, d, cr = a.shape
            if i < self.centre:
                m = a.reshape(cl * d, cr)
                err = max(err, float(np.abs(m.conj().T @ m - np.eye(cr)).max()))
            elif i > self.centre:
                m = a.reshape(cl, d * cr)
                err = max(err, float(np.abs(m @ m.conj().T - np.eye(cl)).max()))
        return err


def mps_from_statevector(psi: np.ndarray, n: int) -> TextbookMPS:
    """Decompose a state vector into an MPS by successive SVDs (Eq. mps), centre at the last site."""
    out = TextbookMPS(n)
    rest = psi.reshape(1, -1)
    chi = 1
    for i in range(n - 1):
        m = rest.reshape(chi * 2, -1)
        u, s, vh = np.linalg.svd(m, full_matrices=False)
        k = len(s)
        out.sites[i] = u.reshape(chi, 2, k)
        rest = s[:, None] * vh
        chi = k
    out.sites[n - 1] = rest.reshape(chi, 2, 1)
    out.centre = n - 1
    return out
