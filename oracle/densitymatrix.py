"""Dense density-matrix simulator (oracle; test infrastructure only).

rho is a 2^N x 2^N matrix with qubit 0 the most significant index of both the
row (ket) and the column (bra), matching the density-matrix expansion of the
"matrix product formalism" section.  Channels act through Kraus operators,
rho -> sum_K K rho K^dagger.  The mixed-state fidelity is the one of Wang et
al. (Eq. Wang), which the paper adopts for MPOs because it needs neither
positivity nor normalisation.
"""
from __future__ import annotations

import numpy as np


def zero_rho(n: int) -> np.ndarray:
    rho = np.zeros((2 ** n, 2 ** n), np.complex128)
    rho[0, 0] = 1.0
    return rho


def from_statevector(psi: np.ndarray) -> np.ndarray:
    return np.outer(psi, psi.conj())


def apply_kraus(rho: np.ndarray, n: int, q: int, kraus, nq: int) -> np.ndarray:
    """Apply the channel {K} on qubits q..q+nq-1 (K is 2^nq x 2^nq)."""
    k = 2 ** nq
    left, right = 2 ** q, 2 ** (n - q - nq)
    r = rho.reshape(left, k, right, left, k, right)
    out = np.zeros_like(r)
    for kop in kraus:
        out += np.einsum("ij,ajbckd,lk->aibcld", kop, r, kop.conj())
    return out.reshape(2 ** n, 2 ** n)


def apply_unitary(rho: np.ndarray, n: int, q: int, u: np.ndarray) -> np.ndarray:
    nq = 1 if u.shape[0] == 2 else 2
    return apply_kraus(rho, n, q, [u], nq)


def trace(rho: np.ndarray) -> complex:
    return complex(np.trace(rho))


def tr_product(rho: np.ndarray, sigma: np.ndarray) -> complex:
    """Tr(rho sigma) = sum_ij rho_ij sigma_ji."""
    return complex(np.sum(rho * sigma.T))


def wang_fidelity(rho: np.ndarray, sigma: np.ndarray) -> float:
    """|Tr(rho sigma)| / sqrt(Tr(rho^2) Tr(sigma^2))  (Eq. Wang)."""
    num = abs(tr_product(rho, sigma))
    den = np.sqrt(tr_product(rho, rho).real * tr_product(sigma, sigma).real)
    return float(num / den)


def expect(rho: np.ndarray, n: int, q: int, op: np.ndarray) -> complex:
    """Tr(O rho) / Tr(rho) for O on qubit q (2x2) or on (q, q+1) (4x4)."""
    nq = 1 if op.shape[0] == 2 else 2
    full = np.kron(np.kron(np.eye(2 ** q), op), np.eye(2 ** (n - q - nq)))
    return complex(np.trace(full @ rho) / np.trace(rho))
