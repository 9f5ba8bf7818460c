"""Planted mistakes: each test breaks the oracle on purpose (CPU only) and checks
that one of the pins catches it, so the pins are known to bite."""
import math

import numpy as np

import workloads as W
from oracle import densitymatrix as DM
from oracle import statevector as SV
from oracle import superop as SO
from oracle import textbook_mps as T


def _untruncated_overlap_defect(n=8, depth=6, seed=1001):
    circ = W.brickwork_circuit(n, depth, seed)
    m = T.TextbookMPS(n, n_2q=circ.n_2q).run(circ.gates(), target=1.0)
    return 1.0 - SV.fidelity(SV.run_circuit(n, circ.gates()), m.to_statevector())


def _single_cut_defect(target=0.9):
    n = 8
    g = W.normals(20, 0, 2 * 2 ** n).reshape(2, -1)
    psi = (g[0] + 1j * g[1]) / np.linalg.norm(g[0] + 1j * g[1])
    m = T.mps_from_statevector(psi, n)
    u = W.haar_unitary(4, 21, 3)
    rec = m.apply_2q(3, u, target=target)
    return abs(rec["f"] - SV.fidelity(SV.apply_2q(psi, n, 3, u), m.to_statevector()))


def test_pins_hold_unplanted():
    assert _untruncated_overlap_defect() < 1e-12
    assert _single_cut_defect() < 1e-12


def test_transposed_gate_is_caught(monkeypatch):
    orig = T.TextbookMPS._lift

    def bad(self, op, nq):
        return orig(self, op, nq).T
    monkeypatch.setattr(T.TextbookMPS, "_lift", bad)
    assert _untruncated_overlap_defect() > 1e-3


def test_wrong_absorbed_factor_in_left_move_is_caught(monkeypatch):
    """Absorbing R instead of R^dagger into the left neighbour changes the state."""
    orig = T.TextbookMPS.move_centre

    def bad(self, to):
        while self.centre > to:
            c = self.centre
            a = self.sites[c]
            cl, d, cr = a.shape
            q, r = np.linalg.qr(a.reshape(cl, d * cr).conj().T)
            k = q.shape[1]
            self.sites[c] = q.conj().T.reshape(k, d, cr)
            prv = self.sites[c - 1]
            self.sites[c - 1] = (prv.reshape(-1, prv.shape[2]) @ r).reshape(prv.shape[0], prv.shape[1], k)
            self.centre -= 1
        orig(self, to)
    monkeypatch.setattr(T.TextbookMPS, "move_centre", bad)
    from tests.test_oracle_mps import qr_built_mps
    g = W.normals(5, 0, 2 * 2 ** 6).reshape(2, -1)
    psi = (g[0] + 1j * g[1]) / np.linalg.norm(g[0] + 1j * g[1])
    m = qr_built_mps(psi, 6)
    m.move_centre(0)
    assert np.abs(m.contract() - psi).max() > 1e-3


def test_skipped_canonicalisation_is_caught(monkeypatch):
    """Without the canonical form the local renormalisation by sqrt(W_k) no longer
    matches the global norm, and the untruncated state-vector pin fails."""
    def bad(self, to):
        self.centre = to
    monkeypatch.setattr(T.TextbookMPS, "move_centre", bad)
    assert _untruncated_overlap_defect() > 1e-3


def test_literal_fidelity_formula_is_caught(monkeypatch):
    """Reading Eq. (fT-pure) literally as sum s^2 s~^2 fails the brute-force overlap pin."""
    orig = T.select_bond

    def bad(s, f_t, fixed_chi=0, chi_max=0, mixed_fid=T.KEPT_RATIO):
        k, f, w, wk, cap = orig(s, f_t, fixed_chi, chi_max, mixed_fid)
        st = s[:k] / math.sqrt(wk)
        return k, float(np.sum(s[:k] ** 2 * st ** 2)), w, wk, cap
    monkeypatch.setattr(T, "select_bond", bad)
    assert _single_cut_defect() > 1e-3


def test_unnormalised_truncation_is_caught(monkeypatch):
    """Forgetting the renormalisation by sqrt(W_k) breaks the unit norm the overlap pin assumes."""
    orig_sqrt = math.sqrt

    class FakeMath:
        def __getattr__(self, name):
            return getattr(math, name)

        @staticmethod
        def sqrt(x):
            return 1.0 if 0.0 < x < 1.0 else orig_sqrt(x)
    monkeypatch.setattr(T, "math", FakeMath())
    assert _single_cut_defect() > 1e-3


def test_wrong_superoperator_conventions_are_caught():
    """Conjugating the ket factor instead of the bra factor, or vectorising the
    input and the output with different conventions, fails the Kraus pin."""
    ks = [W.haar_unitary(2, 50, 0) @ k for k in W.amplitude_damping_kraus(0.3)]

    def conj_on_ket(kraus, nq):
        acc = sum(np.einsum("sr,tu->srtu", k.conj(), k) for k in kraus)
        return np.ascontiguousarray(acc.transpose(0, 2, 1, 3).reshape(4, 4))

    def mixed_orders(kraus, nq):
        acc = sum(np.einsum("sr,tu->srtu", k, k.conj()) for k in kraus)
        return np.ascontiguousarray(acc.transpose(0, 2, 3, 1).reshape(4, 4))   # u = 2 r' + r

    g = W.normals(51, 0, 4)
    psi = (g[:2] + 1j * g[2:]) / np.linalg.norm(g[:2] + 1j * g[2:])
    rho = DM.from_statevector(psi)
    out = DM.apply_kraus(rho, 1, 0, ks, 1)
    vec = lambda r: r.reshape(-1)          # t = 2 s + s' for one qubit
    assert np.abs(SO.from_kraus(ks, 1) @ vec(rho) - vec(out)).max() < 1e-15
    assert np.abs(conj_on_ket(ks, 1) @ vec(rho) - vec(out)).max() > 1e-3
    assert np.abs(mixed_orders(ks, 1) @ vec(rho) - vec(out)).max() > 1e-3
