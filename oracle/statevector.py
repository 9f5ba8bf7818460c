"""Dense state-vector simulator (oracle; test infrastructure only).

The state is the 2^N tensor C_{s_1..s_N} of Eq. (qstate), stored flat with
s_1 (qubit 0) the most significant index, so that contracting the MPS of
Eq. (mps) from left to right gives the same order.
"""
from __future__ import annotations

import numpy as np


def zero_state(n: int) -> np.ndarray:
    """|0...0> on n qubits."""
    psi = np.zeros(2 ** n, np.complex128)
    psi[0] = 1.0
    return psi


def apply_1q(psi: np.ndarray, n: int, q: int, u: np.ndarray) -> np.ndarray:
    """Apply a 2x2 operator to qubit q."""
    t = psi.reshape(2 ** q, 2, 2 ** (n - q - 1))
    return np.einsum("ij,ajb->aib", u, t).reshape(-1)


def apply_2q(psi: np.ndarray, n: int, q: int, u: np.ndarray) -> np.ndarray:
    """Apply a 4x4 operator to the neighbouring qubits (q, q+1); |s_q s_q+1>, s_q major."""
    t = psi.reshape(2 ** q, 4, 2 ** (n - q - 2))
    return np.einsum("ij,ajb->aib", u, t).reshape(-1)


def run_circuit(n: int, gates, psi: np.ndarray | None = None) -> np.ndarray:
    """Apply a list of (q, U4) two-qubit gates in order."""
    psi = zero_state(n) if psi is None else psi.copy()
    for q, u in gates:
        psi = apply_2q(psi, n, q, u)
    return psi


def overlap(a: np.ndarray, b: np.ndarray) -> complex:
    """<a|b>."""
    return complex(np.vdot(a, b))


def fidelity(a: np.ndarray, b: np.ndarray) -> float:
    """Pure-state fidelity |<a|b>|^2 of Eq. (pureF); a and b must be normalised."""
    return abs(np.vdot(a, b)) ** 2


def expect(psi: np.ndarray, n: int, q: int, op: np.ndarray) -> complex:
    """<psi| O |psi> for O acting on qubit q (2x2) or on (q, q+1) (4x4)."""
    if op.shape == (2, 2):
        phi = apply_1q(psi, n, q, op)
    else:
        phi = apply_2q(psi, n, q, op)
    return complex(np.vdot(psi, phi))


def full_operator_2q(n: int, q: int, u: np.ndarray) -> np.ndarray:
    """The 2^n x 2^n matrix I (x) U (x) I of a gate on (q, q+1), built with Kronecker products."""
    return np.kron(np.kron(np.eye(2 ** q), u), np.eye(2 ** (n - q - 2)))
