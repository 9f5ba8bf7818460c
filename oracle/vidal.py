"""Vidal / Hastings form of an MPS (test infrastructure: CPU, FP64, plain NumPy/LAPACK).

Only tests, the smoke check and the benchmark's CPU leg use this module.

The paper builds its MPS by successive SVDs following Vidal ("The matrix product
formalism" section, Eq. mps_repr).  This variant keeps that form throughout: every
site is a right-isometry B_i = Gamma_i lambda_i, and the Schmidt vector lambda_b of
every bond b (between sites b-1 and b) is stored.  A gate on (q, q+1) is then
truncated without moving a canonical centre (Hastings' update, which needs no
division by Schmidt values):

    theta~ = B_q B_{q+1} with the gate applied        (rows (a, s_q), columns (s_{q+1}, b))
    theta  = diag(lambda_q (x) 1_d) theta~            (the two-site wave function of the cut)
    theta  = U S V^dagger,  k kept by the same rule as the canonical method
    B_q <- theta~ V_k / sqrt(W_k),  B_{q+1} <- V_k^dagger,  lambda_{q+1} <- S_k / sqrt(W_k)

The truncation fidelity W_k / W is exact only while the whole chain is in this
canonical form; truncations break it slightly (the canonicality error).  Gates of
a layer act on disjoint pairs and are independent in this form.
"""
from __future__ import annotations

import math

import numpy as np

from .textbook_mps import GLOBAL, PURE, TextbookMPS, select_bond

__all__ = ["VidalMPS"]


class VidalMPS(TextbookMPS):
    """Pure-state MPS in Vidal / Hastings form with the entanglement-aware truncation rule."""

    def __init__(self, n_qubits: int, f_min: float = 1.0, n_2q: int = 0, strategy: int = GLOBAL,
                 chi_max: int = 0, fixed_chi: int = 0, record_svals: bool = False):
        super().__init__(n_qubits, kind=PURE, f_min=f_min, n_2q=n_2q, strategy=strategy, chi_max=chi_max,
                         fixed_chi=fixed_chi, record_svals=record_svals)
        self.lam = [np.ones(1) for _ in range(n_qubits + 1)]   # lam[b]: bond b, left of site b

    def apply_2q(self, q: int, op: np.ndarray, target: float | None = None) -> dict:
        if q < 0 or q + 1 >= self.n:
            raise ValueError("gate outside the chain")
        d = self.d
        cl, cr = self.sites[q].shape[0], self.sites[q + 1].shape[2]
        theta_t = self.theta(q, op)                               # (cl d) x (d cr)
        theta = np.repeat(self.lam[q], d)[:, None] * theta_t
        _, s, vh = np.linalg.svd(theta, full_matrices=False)
        f_t = self.scheduled_target() if (target is None or target < 0) else min(float(target), 1.0)
        k, f, big_w, wk, cap = select_bond(s, f_t, self.fixed_chi, self.chi_max)
        self.cap_hit |= cap
        vk = vh[:k]
        self.sites[q] = ((theta_t @ vk.conj().T) / math.sqrt(wk)).reshape(cl, d, k)
        self.sites[q + 1] = vk.reshape(k, d, cr)
        self.lam[q + 1] = s[:k] / math.sqrt(wk)
        self.product *= f
        self.n_done += 1
        rec = {"q": q, "k": k, "f": f, "f_t": f_t, "W": big_w, "W_k": wk, "rank_bound": len(s)}
        if self.record_svals:
            rec["s"] = s.copy()
        self.log.append(rec)
        return rec

    def apply_layer(self, gates, target: float | None = None) -> list:
        """Gates [(q, op), ...] on disjoint pairs, all truncated against one target: `target` when
        given (>= 0), else the schedule's value for the product at the layer's start.  In this form
        every gate reads only its own sites and the Schmidt vector of its left bond, so the order
        within the layer does not change the result."""
        used = set()
        for q, _ in gates:
            if q in used or q + 1 in used:
                raise ValueError("gates of a layer must act on disjoint pairs")
            used.update((q, q + 1))
        f_t = self.scheduled_target() if (target is None or target < 0) else min(float(target), 1.0)
        return [self.apply_2q(q, op, f_t) for q, op in gates]

    def right_canonical_error(self) -> float:
        """max_i || sum_{s,b} B_i[:, s, b] B_i[:, s, b]^dagger - I ||_max over all sites."""
        err = 0.0
        for b in self.sites:
            m = b.reshape(b.shape[0], -1)
            err = max(err, float(np.abs(m @ m.conj().T - np.eye(b.shape[0])).max()))
        return err
