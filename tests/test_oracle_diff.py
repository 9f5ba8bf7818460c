"""Pins of the differentiable-update oracle: its backward against central finite differences of
phase-invariant losses, its chain against the exact state vector, and the chain's energy
gradient against the parameter-shift rule on the exact state vector."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import statevector as SV
from oracle.diff_chain import DiffChain, tsvd, tsvd_backward, zz_energy_dense


def _rand(rng, m, n):
    return rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))


def _loss_and_cotangents(r, m1, w1, w2, m2):
    """A loss of (A_q, A_p) that is invariant under A_q -> A_q D, A_p -> D^* A_p for every diagonal
    phase D (the SVD's gauge): a linear term in A_q A_p, weighted squared moduli of both outputs
    and a quadratic term in the projector A_q A_q^H.  Returns (L, Abar_q, Abar_p)."""
    aq, ap = r["Aq"], r["Ap"]
    prod = aq @ ap
    proj = aq @ aq.conj().T
    lin = float(np.real(np.sum(np.conj(m1) * prod)))
    sq = float(np.sum(w1[:, :aq.shape[1]] * np.abs(aq) ** 2) + np.sum(w2[:ap.shape[0]] * np.abs(ap) ** 2))
    quad = float(np.real(np.sum(np.conj(m2) * proj)))
    loss = lin + sq + quad ** 2
    # gradients (dL/dRe + i dL/dIm): d lin = Re<m1, dAq Ap + Aq dAp>, d|x|^2 = 2 Re(conj x dx),
    # d quad = Re<m2, dAq Aq^H + Aq dAq^H> = Re<(m2 + m2^H) Aq, dAq>
    aq_bar = m1 @ ap.conj().T + 2 * w1[:, :aq.shape[1]] * aq + 2 * quad * ((m2 + m2.conj().T) @ aq)
    ap_bar = aq.conj().T @ m1 + 2 * w2[:ap.shape[0]] * ap
    return loss, aq_bar, ap_bar


@pytest.mark.parametrize("m,n,target", [(12, 8, 0.9), (8, 12, 0.9), (10, 10, 0.8), (12, 8, 1.0), (6, 14, 1.0)])
def test_tsvd_backward_matches_finite_differences(m, n, target):
    rng = np.random.default_rng(1000 + 10 * m + n)
    a = _rand(rng, m, n)
    r = tsvd(a, target)
    k = r["k"]
    if target < 1.0:
        assert k < min(m, n)
    c = min(m, n)
    m1, m2 = _rand(rng, m, n), _rand(rng, m, m)
    w1, w2 = rng.random((m, c)), rng.random((c, n))
    _, aq_bar, ap_bar = _loss_and_cotangents(r, m1, w1, w2, m2)
    a_bar = tsvd_backward(r["U"], r["S"], r["V"], k, aq_bar, ap_bar)

    def loss(x):
        rr = tsvd(x, 1.0, k, 0.0)
        return _loss_and_cotangents(rr, m1, w1, w2, m2)[0]

    h = 1e-6
    for _ in range(4):
        e = _rand(rng, m, n)
        fd = (loss(a + h * e) - loss(a - h * e)) / (2 * h)
        an = float(np.real(np.sum(np.conj(a_bar) * e)))
        assert abs(fd - an) < 1e-6 * max(1.0, abs(fd))


def test_tsvd_backward_without_the_coupling_terms_is_wrong():
    """The pins see a dropped term: the same check with F = 0 (no kept/discarded coupling) fails."""
    rng = np.random.default_rng(7)
    a = _rand(rng, 9, 7)
    r = tsvd(a, 0.85)
    k = r["k"]
    m1 = _rand(rng, 9, 7)
    z = np.zeros((9, 7))
    _, aq_bar, ap_bar = _loss_and_cotangents(r, m1, np.zeros((9, 7)), np.zeros((7, 7)), np.zeros((9, 9)))
    good = tsvd_backward(r["U"], r["S"], r["V"], k, aq_bar, ap_bar)
    broad = tsvd_backward(r["U"], r["S"], r["V"], k, aq_bar, ap_bar, eps=1e30)   # F -> 0
    e = _rand(rng, 9, 7)
    h = 1e-6

    def loss(x):
        return _loss_and_cotangents(tsvd(x, 1.0, k, 0.0), m1, z, np.zeros((7, 7)), np.zeros((9, 9)))[0]

    fd = (loss(a + h * e) - loss(a - h * e)) / (2 * h)
    assert abs(fd - np.real(np.sum(np.conj(good) * e))) < 1e-6 * max(1.0, abs(fd))
    assert abs(fd - np.real(np.sum(np.conj(broad) * e))) > 1e-3 * max(1.0, abs(fd))


def test_tsvd_cut_and_outputs():
    rng = np.random.default_rng(3)
    a = _rand(rng, 6, 5)
    r = tsvd(a, 0.7)
    s = r["S"]
    cum = np.cumsum(s ** 2) / np.sum(s ** 2)
    assert r["k"] == int(np.argmax(cum >= 0.7)) + 1
    assert abs(r["f"] - cum[r["k"] - 1]) < 1e-14
    # A_q A_p is the rank-k truncation renormalised to unit Frobenius norm
    u, sv, vh = np.linalg.svd(a)
    k = r["k"]
    best = (u[:, :k] * sv[:k]) @ vh[:k]
    assert np.allclose(r["Aq"] @ r["Ap"], best / np.linalg.norm(best), atol=1e-12)
    assert np.allclose(r["Aq"].conj().T @ r["Aq"], np.eye(k), atol=1e-12)


def test_untruncated_chain_is_the_exact_state():
    n = 8
    circ = W.brickwork_circuit(n, 6, 41)
    ch = DiffChain(n)
    for q, u in circ.gates():
        ch.apply_2q(q, u)
    psi = SV.run_circuit(n, circ.gates())
    assert abs(abs(np.vdot(psi, ch.to_statevector())) - 1.0) < 1e-12
    assert abs(ch.energy_zz() - zz_energy_dense(psi, n)) < 1e-12
    # the energy sweep keeps the state
    assert abs(abs(np.vdot(psi, ch.to_statevector())) - 1.0) < 1e-12


def test_zz_energy_of_basis_states():
    n = 5
    psi = np.zeros(2 ** n, complex)
    psi[0b01100] = 1.0   # Z eigenvalues +1 -1 -1 +1 +1: ZZ terms -1, +1, -1, +1
    assert zz_energy_dense(psi, n) == 0.0
    psi[:] = 0
    psi[0] = 1.0
    assert zz_energy_dense(psi, n) == n - 1


def test_chain_energy_gradient_is_the_parameter_shift_gradient():
    """Reverse mode through the chain's updates (oracle backward chained by hand for one gate
    parameter) is not needed here: the chain without a cut is the exact state, so its
    finite-difference gradient must equal the exact parameter-shift gradient."""
    n, layers = 6, 2
    p = W.ansatz_params(n, layers, 17)

    def e_chain(pp):
        c = W.ansatz_circuit(n, layers, pp)
        ch = DiffChain(n, n_2q=c.n_2q)
        for q, u in c.gates():
            ch.apply_2q(q, u)
        return ch.energy_zz()

    def e_exact(pp):
        c = W.ansatz_circuit(n, layers, pp)
        return zz_energy_dense(SV.run_circuit(n, c.gates()), n)

    for j in (0, 5, 2 * n + 1, 3 * n + 2):
        sh = np.zeros_like(p)
        sh[j] = math.pi / 2
        ps = 0.5 * (e_exact(p + sh) - e_exact(p - sh))
        h = np.zeros_like(p)
        h[j] = 1e-5
        fd = (e_chain(p + h) - e_chain(p - h)) / 2e-5
        assert abs(ps - fd) < 1e-7


@pytest.mark.parametrize("m,n", [(11, 6), (6, 11)])
def test_planted_mistakes_in_the_backward_are_caught(m, n):
    """The finite-difference pin sees each term of the adjoint: flipping the sign of the phase
    (gauge) term, or dropping the complement term of the non-square side, fails it."""
    rng = np.random.default_rng(100 + m)
    a = _rand(rng, m, n)
    r = tsvd(a, 0.9)
    k, u, s, v = r["k"], r["U"], r["S"], r["V"]
    c = min(m, n)
    m1, m2 = _rand(rng, m, n), _rand(rng, m, m)
    w1, w2 = rng.random((m, c)), rng.random((c, n))
    _, aq_bar, ap_bar = _loss_and_cotangents(r, m1, w1, w2, m2)
    good = tsvd_backward(u, s, v, k, aq_bar, ap_bar)
    # the two pieces, recomputed here only to plant the mistakes
    u_bar = np.zeros((m, c), complex)
    u_bar[:, :k] = aq_bar
    sig = s[:k] / math.sqrt(float(np.sum(s[:k] ** 2)))
    v_bar = np.zeros((n, c), complex)
    v_bar[:, :k] = ap_bar.conj().T * sig[None, :]
    ju, jv = u.conj().T @ u_bar, v.conj().T @ v_bar
    gauge = u @ np.diag(1j * (np.imag(np.diag(ju)) - np.imag(np.diag(jv))) / (2 * s)) @ v.conj().T
    if m > n:
        yu = u_bar / s[None, :]
        comp = (yu - u @ (u.conj().T @ yu)) @ v.conj().T
    else:
        yv = v_bar / s[None, :]
        comp = u @ (yv.conj().T - (yv.conj().T @ v) @ v.conj().T)
    assert np.linalg.norm(gauge) > 1e-3 and np.linalg.norm(comp) > 1e-3

    def loss(x):
        return _loss_and_cotangents(tsvd(x, 1.0, k, 0.0), m1, w1, w2, m2)[0]

    h = 1e-6
    e = _rand(rng, m, n)
    fd = (loss(a + h * e) - loss(a - h * e)) / (2 * h)

    def dl(g):
        return float(np.real(np.sum(np.conj(g) * e)))

    assert abs(fd - dl(good)) < 1e-6 * max(1.0, abs(fd))
    for wrong in (good - 2 * gauge, good - comp):
        assert abs(fd - dl(wrong)) > 1e-4 * max(1.0, abs(fd))
