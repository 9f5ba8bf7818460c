"""Superoperators in the vectorised-MPO convention (oracle; test infrastructure only).

An MPO site carries the local index t = 2*s + s' for the operator |s><s'|
(row-major vectorisation of the 2x2 local block), so local dimension 4, as in
the MPO of the "matrix product formalism" section.  A channel with Kraus
operators {K} on n_q qubits maps rho -> sum_K K rho K^dagger; in vectorised
form it is the matrix

    S[(t_1..t_nq), (u_1..u_nq)] = sum_K K[(s_1..s_nq), (r_1..r_nq)]
                                       * conj(K[(s'_1..s'_nq), (r'_1..r'_nq)])

with t_i = 2 s_i + s'_i and u_i = 2 r_i + r'_i, qubit 1 most significant.
Composition of channels is the matrix product of their superoperators.
"""
from __future__ import annotations

import numpy as np


def from_kraus(kraus, nq: int) -> np.ndarray:
    """Superoperator (4^nq x 4^nq) of the channel {K} on nq (1 or 2) qubits."""
    dim = 2 ** nq
    acc = np.zeros((dim,) * 4, np.complex128)   # [s, r, s', r'] with multi-qubit s, r
    for k in kraus:
        acc += np.einsum("sr,tu->srtu", k, k.conj())
    if nq == 1:
        # t = 2 s + s', u = 2 r + r'
        out = acc.transpose(0, 2, 1, 3).reshape(4, 4)
        return np.ascontiguousarray(out)
    # nq == 2: s=(s1,s2), r=(r1,r2), s'=(s1',s2'), r'=(r1',r2')
    a = acc.reshape(2, 2, 2, 2, 2, 2, 2, 2)            # s1 s2 r1 r2 s1' s2' r1' r2'
    a = a.transpose(0, 4, 1, 5, 2, 6, 3, 7)            # s1 s1' s2 s2' r1 r1' r2 r2'
    return np.ascontiguousarray(a.reshape(16, 16))


def from_unitary(u: np.ndarray) -> np.ndarray:
    nq = 1 if u.shape[0] == 2 else 2
    return from_kraus([u], nq)


def kron_1q(s_a: np.ndarray, s_b: np.ndarray) -> np.ndarray:
    """Two single-qubit superoperators side by side, as one two-qubit superoperator."""
    return np.kron(s_a, s_b)
