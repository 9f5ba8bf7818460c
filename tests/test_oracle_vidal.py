"""Pins of the Vidal / Hastings oracle against definitions: the exact state, the exact Schmidt
values of every cut, right-canonicality, and the exact single-cut fidelity of a first truncation."""
import numpy as np
import pytest

import workloads as W
from oracle import statevector as SV
from oracle import textbook_mps as T
from oracle.vidal import VidalMPS


def _schmidt(psi, n, b):
    s = np.linalg.svd(psi.reshape(2 ** b, 2 ** (n - b)), compute_uv=False)
    return s[s > 1e-12]


def test_untruncated_vidal_is_exact_with_exact_schmidt_vectors():
    n = 8
    circ = W.brickwork_circuit(n, 6, 91)
    v = VidalMPS(n)
    psi = SV.zero_state(n)
    for q, u in circ.gates():
        v.apply_2q(q, u)
        psi = SV.apply_2q(psi, n, q, u)
        got = _schmidt(psi, n, q + 1)
        lam = v.lam[q + 1][v.lam[q + 1] > 1e-12]
        assert np.allclose(lam, got, atol=1e-12)
    assert abs(abs(np.vdot(psi, v.to_statevector())) - 1.0) < 1e-12
    assert v.right_canonical_error() < 1e-12
    assert v.product == 1.0


def test_first_truncation_fidelity_is_the_exact_single_cut_fidelity():
    n = 8
    circ = W.brickwork_circuit(n, 4, 92)
    gates = circ.gates()
    v = VidalMPS(n)
    psi = SV.zero_state(n)
    for q, u in gates[:-1]:
        v.apply_2q(q, u)
        psi = SV.apply_2q(psi, n, q, u)
    q, u = gates[-1]
    rec = v.apply_2q(q, u, target=0.9)
    psi = SV.apply_2q(psi, n, q, u)
    assert rec["k"] < rec["rank_bound"]
    f_true = abs(np.vdot(psi, v.to_statevector())) ** 2
    assert abs(rec["f"] - f_true) < 1e-12


def test_vidal_and_canonical_agree_before_any_truncation_breaks_the_form():
    """Up to the first truncation both forms hold the same state and decide the same bonds."""
    n = 10
    circ = W.brickwork_circuit(n, 8, 93)
    v = VidalMPS(n, f_min=0.95, n_2q=circ.n_2q)
    t = T.TextbookMPS(n, f_min=0.95, n_2q=circ.n_2q)
    for q, u in circ.gates():
        rv = v.apply_2q(q, u)
        rt = t.apply_2q(q, u)
        assert rv["k"] == rt["k"] and abs(rv["f"] - rt["f"]) < 1e-10
        if rv["k"] < rv["rank_bound"]:
            break
    assert abs(abs(np.vdot(v.to_statevector(), t.to_statevector())) - 1.0) < 1e-10


def _layers(circ):
    out = {}
    for q, u, layer in zip(circ.qs, circ.ops, circ.layers):
        out.setdefault(layer, []).append((q, u))
    return [out[k] for k in sorted(out)]


def test_layer_result_does_not_depend_on_the_order_within_the_layer():
    """In the Vidal form a gate touches its own sites and the Schmidt vector of its left bond only:
    running each layer forwards or backwards (same target) gives the same sites and vectors."""
    n = 12
    circ = W.brickwork_circuit(n, 8, 94)
    a = VidalMPS(n, f_min=0.9, n_2q=circ.n_2q)
    b = VidalMPS(n, f_min=0.9, n_2q=circ.n_2q)
    for layer in _layers(circ):
        ra = a.apply_layer(layer)
        rb = b.apply_layer(layer[::-1])
        assert len({r["f_t"] for r in ra}) == 1
        assert [r["k"] for r in ra] == [r["k"] for r in rb[::-1]]
    assert a.bond_dims() == b.bond_dims()
    assert max(a.bond_dims()) < 2 ** (n // 2)   # the run truncated
    for sa, sb in zip(a.sites, b.sites):
        assert np.abs(sa - sb).max() < 1e-12
    for la, lb in zip(a.lam, b.lam):
        assert np.abs(la - lb).max() < 1e-12
    assert abs(a.product - b.product) < 1e-14


def test_first_layer_target_is_the_global_per_gate_share():
    """Before any truncation the product is 1, so the global schedule's target is F_min^(1/n_2q)
    for every gate of the first layer."""
    n = 10
    circ = W.brickwork_circuit(n, 6, 95)
    v = VidalMPS(n, f_min=0.8, n_2q=circ.n_2q)
    recs = v.apply_layer(_layers(circ)[0])
    for r in recs:
        assert abs(r["f_t"] - 0.8 ** (1.0 / circ.n_2q)) < 1e-15


def test_untruncated_layers_give_the_exact_state():
    n = 9
    circ = W.brickwork_circuit(n, 7, 96)
    v = VidalMPS(n)
    for layer in _layers(circ):
        v.apply_layer(layer)
    psi = SV.run_circuit(n, circ.gates())
    assert abs(abs(np.vdot(psi, v.to_statevector())) - 1.0) < 1e-12


def test_a_layer_with_overlapping_pairs_is_refused():
    v = VidalMPS(6)
    u = W.haar_unitary(4, 1, 0)
    with pytest.raises(ValueError):
        v.apply_layer([(1, u), (2, u)])
