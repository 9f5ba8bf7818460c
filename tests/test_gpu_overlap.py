"""mps_overlap: the FP64 transfer contraction against dense inner products, the oracle's
true fidelity, mixed precisions, and the purity of an MPO."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
E = pytest.importorskip("paper_2307_16870_gb300")

import workloads as W  # noqa: E402
from oracle import densitymatrix as DM  # noqa: E402
from oracle import statevector as SV  # noqa: E402
from oracle import textbook_mps as T  # noqa: E402
from tests.helpers import contract_sites  # noqa: E402


def _run(n, circ, precision=E.TF32X3, f_min=1.0, target=-1.0, **kw):
    m = E.MPS(n, f_min=f_min, n_2q=circ.n_2q, precision=precision, **kw)
    m.run(circ.gates(), target)
    return m


def test_overlap_equals_dense_inner_product_and_oracle_true_fidelity():
    n = 10
    circ = W.brickwork_circuit(n, 8, 311)
    exact = _run(n, circ, target=1.0)
    ea = _run(n, circ, f_min=0.95)
    assert max(ea.bond_dims()) < max(exact.bond_dims())       # the EA run did truncate
    a, b = contract_sites(exact), contract_sites(ea)
    ov = exact.overlap(ea)
    assert abs(ov - np.vdot(a, b)) < 1e-12 * max(1.0, abs(ov))
    assert abs(ea.overlap(ea) - np.vdot(b, b)) < 1e-12
    assert abs(ea.overlap(ea) - 1.0) < 1e-5                    # normalised state
    assert abs(ea.overlap(exact) - np.conj(ov)) < 1e-12
    # true fidelity against the oracle: exact state vector vs the oracle's EA state
    psi = SV.run_circuit(n, circ.gates())
    o = T.TextbookMPS(n, f_min=0.95, n_2q=circ.n_2q)
    for q, u in circ.gates():
        o.apply_2q(q, u)
    f_oracle = abs(np.vdot(psi, o.to_statevector())) ** 2
    f_gpu = abs(ov) ** 2
    assert abs(f_gpu - f_oracle) < 1e-5
    assert abs(ea.fidelity() - o.product) < 1e-4
    exact.close()
    ea.close()


def test_overlap_across_precisions_and_bonds():
    n = 9
    circ = W.brickwork_circuit(n, 7, 312)
    a = _run(n, circ, precision=E.FP64, target=1.0)
    b = _run(n, circ, precision=E.TF32X3, target=1.0)
    assert abs(a.overlap(b) - 1.0) < 1e-5
    assert abs(a.overlap(a) - 1.0) < 1e-12
    # a product state against the evolved one: <0...0|psi>
    z = E.MPS(n, precision=E.FP64)
    assert abs(z.overlap(a) - a.amplitude([0] * n)) < 1e-12
    for m in (a, b, z):
        m.close()


def test_overlap_of_an_mpo_with_itself_is_its_purity():
    n = 6
    circ = W.brickwork_circuit(n, 5, 41)
    ad = E.mps_superop_from_kraus(W.amplitude_damping_kraus(0.03), 1)
    dep = E.mps_superop_from_kraus(W.depolarizing_2q_kraus(0.05), 2)
    m = E.MPS(n, kind=E.MIXED, n_2q=circ.n_2q, precision=E.FP64)
    rho = DM.zero_rho(n)
    for q, u in circ.gates():
        m.apply_2q(q, np.kron(ad, ad) @ dep @ E.mps_superop_from_kraus([u], 2), 1.0)
        rho = DM.apply_unitary(rho, n, q, u)
        rho = DM.apply_kraus(rho, n, q, W.depolarizing_2q_kraus(0.05), 2)
        rho = DM.apply_kraus(rho, n, q, W.amplitude_damping_kraus(0.03), 1)
        rho = DM.apply_kraus(rho, n, q + 1, W.amplitude_damping_kraus(0.03), 1)
    purity = np.trace(rho @ rho).real
    assert purity < 0.99                                        # the noise made it mixed
    assert abs(m.overlap(m) - purity) < 1e-10
    m.close()


def test_overlap_rejects_mismatched_handles():
    a = E.MPS(6)
    b = E.MPS(7)
    c = E.MPS(6, kind=E.MIXED)
    with pytest.raises(E.MpsError):
        a.overlap(b)
    with pytest.raises(E.MpsError):
        a.overlap(c)
    for m in (a, b, c):
        m.close()
