"""Pins of the dense oracle simulators against closed forms and independent constructions."""
import json
import math
import os

import numpy as np

import workloads as W
from oracle import densitymatrix as DM
from oracle import statevector as SV
from oracle import superop as SO

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))

H = np.array([[1, 1], [1, -1]], np.complex128) / math.sqrt(2)
I2 = np.eye(2, dtype=np.complex128)
CNOT = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], np.complex128)


def _rand_state(n, seed):
    g = W.normals(seed, 0, 2 * 2 ** n).reshape(2, -1)
    psi = g[0] + 1j * g[1]
    return psi / np.linalg.norm(psi)


def test_bell_and_ghz_closed_form():
    psi = SV.zero_state(2)
    psi = SV.apply_2q(psi, 2, 0, CNOT @ np.kron(H, I2))
    assert np.allclose(psi, np.array([1, 0, 0, 1]) / math.sqrt(2), atol=1e-15)
    g = GOLDEN["ghz5_amplitudes"]
    n = g["n"]
    psi = SV.apply_1q(SV.zero_state(n), n, 0, H)
    for q in range(n - 1):
        psi = SV.apply_2q(psi, n, q, CNOT)
    expect = np.zeros(2 ** n)
    expect[0] = expect[-1] = g["amp"]
    assert np.allclose(psi, expect, atol=1e-15)


def test_apply_2q_matches_kronecker_operator():
    n = 6
    psi = _rand_state(n, 1)
    for q in range(n - 1):
        u = W.haar_unitary(4, 2, q)
        a = SV.apply_2q(psi, n, q, u)
        b = SV.full_operator_2q(n, q, u) @ psi
        assert np.abs(a - b).max() < 1e-13


def test_apply_1q_matches_kronecker_operator():
    n = 5
    psi = _rand_state(n, 4)
    u = W.haar_unitary(2, 5, 0)
    for q in range(n):
        full = np.kron(np.kron(np.eye(2 ** q), u), np.eye(2 ** (n - q - 1)))
        assert np.abs(SV.apply_1q(psi, n, q, u) - full @ psi).max() < 1e-13


def test_pure_fidelity_values():
    a = _rand_state(4, 7)
    assert abs(SV.fidelity(a, a) - 1.0) < 1e-14
    b = SV.zero_state(4)
    c = np.zeros(16, np.complex128)
    c[1] = 1
    assert SV.fidelity(b, c) == 0.0


def test_density_matrix_unitary_matches_state_vector():
    n = 5
    psi = _rand_state(n, 9)
    rho = DM.from_statevector(psi)
    for q in range(n - 1):
        u = W.haar_unitary(4, 10, q)
        psi = SV.apply_2q(psi, n, q, u)
        rho = DM.apply_unitary(rho, n, q, u)
    assert np.abs(rho - np.outer(psi, psi.conj())).max() < 1e-13


def test_channels_trace_preserving_and_closed_forms():
    n = 4
    rho = DM.from_statevector(_rand_state(n, 12))
    rho = DM.apply_kraus(rho, n, 1, W.depolarizing_2q_kraus(0.2), 2)
    rho = DM.apply_kraus(rho, n, 3, W.amplitude_damping_kraus(0.4), 1)
    assert abs(DM.trace(rho) - 1.0) < 1e-13
    assert np.abs(rho - rho.conj().T).max() < 1e-14
    # full depolarisation of a pair -> I/4
    g = GOLDEN["depolarizing_full"]
    r2 = DM.from_statevector(_rand_state(2, 13))
    r2 = DM.apply_kraus(r2, 2, 0, W.depolarizing_2q_kraus(g["p"]), 2)
    assert np.abs(r2 - g["rho_diag"] * np.eye(4)).max() < 1e-14
    # full amplitude damping -> |0><0|
    r1 = DM.from_statevector(_rand_state(1, 14))
    r1 = DM.apply_kraus(r1, 1, 0, W.amplitude_damping_kraus(GOLDEN["amplitude_damping_full"]["gamma"]), 1)
    assert np.abs(r1 - np.diag([1.0, 0.0])).max() < 1e-15


def test_wang_fidelity_reduces_to_pure_overlap():
    a, b = _rand_state(3, 15), _rand_state(3, 16)
    f = DM.wang_fidelity(DM.from_statevector(a), DM.from_statevector(b))
    assert abs(f - SV.fidelity(a, b)) < 1e-14
    r = DM.apply_kraus(DM.from_statevector(a), 3, 0, W.depolarizing_2q_kraus(0.3), 2)
    assert abs(DM.wang_fidelity(r, r) - 1.0) < 1e-14
    assert abs(DM.wang_fidelity(r, 3.7 * r) - 1.0) < 1e-14    # scale free (unnormalised input)


def _vec_mpo_order(rho, n):
    """rho -> flat tensor over (t_1..t_n), t_i = 2 s_i + s'_i, qubit 0 most significant."""
    r = rho.reshape((2,) * (2 * n))
    perm = []
    for i in range(n):
        perm += [i, n + i]
    return r.transpose(perm).reshape(-1)


def test_superop_matches_kraus_channel():
    n = 2
    rho = DM.from_statevector(_rand_state(n, 17))
    rho = DM.apply_kraus(rho, n, 0, W.amplitude_damping_kraus(0.3), 1)   # make it mixed
    ks = [W.haar_unitary(4, 18, 0) @ k for k in W.depolarizing_2q_kraus(0.1)]
    s = SO.from_kraus(ks, 2)
    out = DM.apply_kraus(rho, n, 0, ks, 2)
    assert np.abs(s @ _vec_mpo_order(rho, n) - _vec_mpo_order(out, n)).max() < 1e-14
    # single-qubit superoperators side by side equal the channel on both qubits
    ad = W.amplitude_damping_kraus(0.2)
    s1 = SO.kron_1q(SO.from_kraus(ad, 1), SO.from_kraus(ad, 1))
    out2 = DM.apply_kraus(DM.apply_kraus(rho, n, 0, ad, 1), n, 1, ad, 1)
    assert np.abs(s1 @ _vec_mpo_order(rho, n) - _vec_mpo_order(out2, n)).max() < 1e-14
