"""Pins of the textbook entanglement-aware MPS/MPO oracle.

Each pin comes from something other than the oracle itself: the dense
simulators (brute force), closed forms, exact identities of the canonical
form, or invariants the paper states (adjoint circuit returns to bond 1).
"""
import json
import math
import os

import numpy as np
import pytest

import workloads as W
from oracle import densitymatrix as DM
from oracle import statevector as SV
from oracle import superop as SO
from oracle import textbook_mps as T

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))

H = np.array([[1, 1], [1, -1]], np.complex128) / math.sqrt(2)
I2 = np.eye(2, dtype=np.complex128)
CNOT = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], np.complex128)


def _rand_state(n, seed):
    g = W.normals(seed, 0, 2 * 2 ** n).reshape(2, -1)
    psi = g[0] + 1j * g[1]
    return psi / np.linalg.norm(psi)


# ---------------------------------------------------------------- pure, exact
def test_untruncated_mps_equals_state_vector():
    circ = W.brickwork_circuit(10, 8, 1001)
    m = T.TextbookMPS(10, n_2q=circ.n_2q).run(circ.gates(), target=1.0)
    psi = SV.run_circuit(10, circ.gates())
    assert 1.0 - SV.fidelity(psi, m.to_statevector()) < 1e-12
    assert m.product == 1.0
    bound = [min(2 ** (i + 1), 2 ** (10 - 1 - i)) for i in range(9)]
    assert all(b <= c for b, c in zip(m.bond_dims(), bound))


def test_successive_svd_roundtrip():
    psi = _rand_state(7, 2)
    m = T.mps_from_statevector(psi, 7)
    assert np.abs(m.contract() - psi).max() < 1e-13
    assert m.canonical_error() < 1e-13


def test_canonical_form_kept_after_every_gate():
    circ = W.brickwork_circuit(8, 6, 3)
    m = T.TextbookMPS(8, f_min=0.95, n_2q=circ.n_2q)
    for q, u in circ.gates():
        m.apply_2q(q, u)
        assert m.canonical_error() < 1e-12


def qr_built_mps(psi, n):
    """MPS by successive QR (not SVD), so the bonds are not Schmidt bases and
    every centre move has a non-diagonal triangular factor."""
    m = T.TextbookMPS(n)
    rest = psi.reshape(1, -1)
    chi = 1
    for i in range(n - 1):
        q, r = np.linalg.qr(rest.reshape(chi * 2, -1))
        k = q.shape[1]
        m.sites[i] = q.reshape(chi, 2, k)
        rest, chi = r, k
    m.sites[n - 1] = rest.reshape(chi, 2, 1)
    m.centre = n - 1
    return m


def test_centre_moves_preserve_state():
    psi = _rand_state(6, 5)
    m = qr_built_mps(psi, 6)
    assert np.abs(m.contract() - psi).max() < 1e-13
    for c in (0, 4, 1, 5, 2):
        m.move_centre(c)
        assert m.centre == c
        assert np.abs(m.contract() - psi).max() < 1e-13
        assert m.canonical_error() < 1e-13


def test_bell_single_cut_closed_form():
    g = GOLDEN["bell_single_cut"]
    m = T.TextbookMPS(2, record_svals=True)
    rec = m.apply_2q(0, CNOT @ np.kron(H, I2), target=0.4)
    assert rec["k"] == g["k"]
    assert abs(rec["f"] - g["f"]) < 1e-15
    assert np.allclose(rec["s"], [1 / math.sqrt(2)] * 2, atol=1e-15)


def test_ghz_bonds():
    g = GOLDEN["ghz5_amplitudes"]
    n = g["n"]
    m = T.TextbookMPS(n, n_2q=n - 1)
    m.apply_2q(0, CNOT @ np.kron(H, I2), target=1.0)
    for q in range(1, n - 1):
        m.apply_2q(q, CNOT, target=1.0)
    psi = m.to_statevector()
    assert abs(psi[0] - g["amp"]) < 1e-15 and abs(psi[-1] - g["amp"]) < 1e-15
    assert abs(m.amplitude([1] * n) - g["amp"]) < 1e-15


@pytest.mark.parametrize("target", [0.999, 0.99, 0.9, 0.6])
def test_single_cut_fidelity_is_overlap(target):
    """Eq. (fT-pure): f from singular values equals |<psi|psi_trunc>|^2 by brute force."""
    n = 9
    psi = _rand_state(n, 20)
    for q in (0, 3, 7):
        m = T.mps_from_statevector(psi, n)
        u = W.haar_unitary(4, 21, q)
        exact = SV.apply_2q(psi, n, q, u)
        rec = m.apply_2q(q, u, target=target)
        trunc = m.to_statevector()
        assert abs(np.linalg.norm(trunc) - 1.0) < 1e-13
        f_true = SV.fidelity(exact, trunc)
        assert abs(rec["f"] - f_true) < 1e-12
        assert rec["f"] >= target
        assert rec["k"] == 1 or rec["W_k"] - (rec["W_k"] - 0) >= 0   # k is minimal: checked below
        s = np.linalg.svd(exact.reshape(2 ** (q + 1), -1), compute_uv=False)
        cum = np.cumsum(s ** 2)
        assert rec["k"] == 1 or cum[rec["k"] - 2] < target * cum[-1]


def test_singular_values_properties():
    circ = W.brickwork_circuit(8, 6, 7)
    m = T.TextbookMPS(8, n_2q=circ.n_2q, record_svals=True)
    for q, u in circ.gates():
        m.sites_before = [a.copy() for a in m.sites]
        rec = m.apply_2q(q, u, target=1.0)
        s = rec["s"]
        assert np.all(s >= 0) and np.all(np.diff(s) <= 1e-15)
        assert abs(np.sum(s ** 2) - 1.0) < 1e-12      # sum s^2 = ||theta||_F^2 = 1 for a unit state


def test_adjoint_circuit_returns_to_product_state():
    """Fig. 2a: a circuit followed by its adjoint comes back to bond 1 everywhere."""
    circ = W.brickwork_circuit(10, 6, 8)
    full = circ.gates() + circ.adjoint().gates()
    for f_min in (1.0, 0.999):
        m = T.TextbookMPS(10, f_min=f_min, n_2q=len(full))
        m.run(full)
        amp2 = abs(m.amplitude([0] * 10)) ** 2       # true fidelity with |0...0>
        assert m.product >= f_min
        if f_min >= 1.0:
            assert abs(amp2 - 1.0) < 1e-10
        else:
            assert amp2 >= f_min
            # the untruncated mode keeps zero singular values (no cutoff), so
            # only the entanglement-aware run drops back to bond 1
            assert m.bond_dims() == [1] * 9


@pytest.mark.parametrize("strategy", [T.NAIVE, T.GLOBAL, T.NEAREST])
def test_schedule_final_product_at_least_f_min(strategy):
    circ = W.brickwork_circuit(12, 8, 1000)
    m = T.TextbookMPS(12, f_min=0.99, n_2q=circ.n_2q, strategy=strategy).run(circ.gates())
    assert m.product >= 0.99
    ft = [r["f_t"] for r in m.log]
    f0 = 0.99 ** (1 / circ.n_2q)
    assert abs(ft[0] - f0) < 1e-13
    if strategy == T.NAIVE:
        assert max(abs(x - f0) for x in ft) < 1e-15
    p = 1.0
    for j, r in enumerate(m.log):
        rem = circ.n_2q - j
        if strategy == T.GLOBAL:
            assert abs(r["f_t"] - min(1.0, (0.99 / p) ** (1 / rem))) < 1e-14
        if strategy == T.NEAREST:
            assert abs(r["f_t"] - min(1.0, 0.99 / (p * f0 ** (rem - 1)))) < 1e-14
        assert r["f"] >= r["f_t"] - 1e-15
        p *= r["f"]
    # the adaptive strategies use the budget at least as well as the naive one
    naive = T.TextbookMPS(12, f_min=0.99, n_2q=circ.n_2q, strategy=T.NAIVE).run(circ.gates())
    assert m.product <= naive.product + 1e-12 or strategy == T.NAIVE


def test_inferred_fidelity_vs_true_overlap_reported():
    """Eq. (prod) is an approximation for many cuts (parity unpinned): report the gap, bound it loosely."""
    circ = W.brickwork_circuit(12, 8, 1000)
    m = T.TextbookMPS(12, f_min=0.99, n_2q=circ.n_2q).run(circ.gates())
    f_true = SV.fidelity(SV.run_circuit(12, circ.gates()), m.to_statevector())
    assert abs(m.product - f_true) < 0.01
    assert f_true > 0.98


def test_fixed_chi_and_cap():
    circ = W.brickwork_circuit(12, 8, 4)
    m = T.TextbookMPS(12, fixed_chi=8, n_2q=circ.n_2q).run(circ.gates())
    assert max(m.bond_dims()) <= 8
    m2 = T.TextbookMPS(12, f_min=0.999999, n_2q=circ.n_2q, chi_max=4).run(circ.gates())
    assert max(m2.bond_dims()) <= 4 and m2.cap_hit


def test_expect_and_amplitude_match_state_vector():
    n = 8
    circ = W.brickwork_circuit(n, 5, 6)
    m = T.TextbookMPS(n, n_2q=circ.n_2q).run(circ.gates(), target=1.0)
    psi = SV.run_circuit(n, circ.gates())
    z = np.diag([1.0, -1.0]).astype(np.complex128)
    for q in range(n):
        assert abs(m.expect(q, z) - SV.expect(psi, n, q, z)) < 1e-12
    for q in range(n - 1):
        o = W.haar_unitary(4, 30, q)
        o = o + o.conj().T
        assert abs(m.expect(q, o) - SV.expect(psi, n, q, o)) < 1e-12
    rng = np.random.default_rng(0)
    for _ in range(10):
        bits = rng.integers(0, 2, n)
        idx = int("".join(map(str, bits)), 2)
        assert abs(m.amplitude(bits) - psi[idx]) < 1e-13


# ---------------------------------------------------------------- mixed (MPO)
def _noisy_superop(u, p, gamma):
    ad = W.amplitude_damping_kraus(gamma)
    s_ad = SO.kron_1q(SO.from_kraus(ad, 1), SO.from_kraus(ad, 1))
    return s_ad @ SO.from_kraus(W.depolarizing_2q_kraus(p), 2) @ SO.from_unitary(u)


def _dm_run(n, circ, p, gamma):
    rho = DM.zero_rho(n)
    for q, u in circ.gates():
        rho = DM.apply_unitary(rho, n, q, u)
        rho = DM.apply_kraus(rho, n, q, W.depolarizing_2q_kraus(p), 2)
        rho = DM.apply_kraus(rho, n, q, W.amplitude_damping_kraus(gamma), 1)
        rho = DM.apply_kraus(rho, n, q + 1, W.amplitude_damping_kraus(gamma), 1)
    return rho


def test_untruncated_mpo_equals_density_matrix():
    n = 6
    circ = W.brickwork_circuit(n, 5, 40)
    m = T.TextbookMPS(n, kind=T.MIXED, n_2q=circ.n_2q)
    for q, u in circ.gates():
        m.apply_2q(q, _noisy_superop(u, 0.05, 0.03), target=1.0)
    rho = _dm_run(n, circ, 0.05, 0.03)
    assert np.abs(m.to_density_matrix() - rho).max() < 1e-13
    assert abs(DM.trace(m.to_density_matrix()) - 1.0) < 1e-12
    assert m.canonical_error() < 1e-12
    z = np.diag([1.0, -1.0]).astype(np.complex128)
    for q in range(n):
        assert abs(m.expect(q, z) - DM.expect(rho, n, q, z)) < 1e-12
    zz = np.kron(z, z)
    for q in range(n - 1):
        assert abs(m.expect(q, zz) - DM.expect(rho, n, q, zz)) < 1e-12
    for b in ([0] * n, [1, 0, 1, 1, 0, 0]):
        idx = int("".join(map(str, b)), 2)
        assert abs(m.amplitude(b) - rho[idx, idx] / np.trace(rho)) < 1e-13


def test_pure_mpo_bond_is_square_of_mps_bond():
    n = 6
    circ = W.brickwork_circuit(n, 4, 41)
    mps = T.TextbookMPS(n, n_2q=circ.n_2q, record_svals=True).run(circ.gates(), target=1.0)
    mpo = T.TextbookMPS(n, kind=T.MIXED, n_2q=circ.n_2q, record_svals=True).run(circ.gates(), target=1.0)
    for a, b in zip(mps.log, mpo.log):
        s_mps = a["s"]
        s_mpo = np.sort(np.outer(s_mps, s_mps).reshape(-1))[::-1]
        r = len(b["s"])
        assert np.abs(b["s"] - s_mpo[:r]).max() < 1e-12
    rho = mpo.to_density_matrix()
    assert abs(DM.tr_product(rho, rho) - GOLDEN["pure_mpo_bond"]["purity"]) < 1e-12
    psi = mps.to_statevector()
    assert np.abs(rho - np.outer(psi, psi.conj())).max() < 1e-13


@pytest.mark.parametrize("target", [0.999, 0.99, 0.9])
def test_mpo_single_cut_fidelity_is_wang(target):
    """Eq. (fT-mixed) against the Wang fidelity (Eq. Wang) computed by brute force."""
    n = 5
    circ = W.brickwork_circuit(n, 4, 42)
    base = T.TextbookMPS(n, kind=T.MIXED, n_2q=circ.n_2q)
    for q, u in circ.gates():
        base.apply_2q(q, _noisy_superop(u, 0.05, 0.02), target=1.0)
    for q in (0, 2, 3):
        for mode in (T.KEPT_RATIO, T.WANG_SQRT):
            m = T.TextbookMPS(n, kind=T.MIXED, mixed_fid=mode)
            m.sites = [a.copy() for a in base.sites]
            m.centre, m.lognorm = base.centre, base.lognorm
            u = W.haar_unitary(4, 43, q)
            s = SO.from_unitary(u)
            ref = T.TextbookMPS(n, kind=T.MIXED)
            ref.sites = [a.copy() for a in base.sites]
            ref.centre, ref.lognorm = base.centre, base.lognorm
            ref.apply_2q(q, s, target=1.0)
            rec = m.apply_2q(q, s, target=target)
            fw = DM.wang_fidelity(ref.to_density_matrix(), m.to_density_matrix())
            want = fw * fw if mode == T.KEPT_RATIO else fw
            assert abs(rec["f"] - want) < 1e-12
            assert rec["f"] >= target


def test_noisy_product_is_lower_bound():
    """Eq. (lower): with noise the product of truncation fidelities does not exceed the true fidelity."""
    n = 7
    circ = W.brickwork_circuit(n, 8, 44)
    m = T.TextbookMPS(n, kind=T.MIXED, f_min=0.95, n_2q=circ.n_2q, mixed_fid=T.WANG_SQRT)
    for q, u in circ.gates():
        m.apply_2q(q, _noisy_superop(u, 0.05, 0.05))
    rho = _dm_run(n, circ, 0.05, 0.05)
    fw = DM.wang_fidelity(rho, m.to_density_matrix())
    assert fw >= m.product - 1e-3
    assert m.product >= 0.95


def test_mpo_noise_shrinks_bonds():
    """Fig. 2b: strong noise reduces the bonds an EA-MPO needs."""
    n = 8
    circ = W.brickwork_circuit(n, 12, 45)
    clean = T.TextbookMPS(n, kind=T.MIXED, f_min=0.99, n_2q=circ.n_2q)
    noisy = T.TextbookMPS(n, kind=T.MIXED, f_min=0.99, n_2q=circ.n_2q)
    for q, u in circ.gates():
        clean.apply_2q(q, SO.from_unitary(u))
        noisy.apply_2q(q, _noisy_superop(u, 0.3, 0.1))
    assert sum(noisy.bond_dims()) < sum(clean.bond_dims())
