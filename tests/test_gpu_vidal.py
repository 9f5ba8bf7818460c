"""The Vidal / Hastings mode (mps_options.vidal) against the FP64 oracle of the same form."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
E = pytest.importorskip("paper_2307_16870_gb300")

import workloads as W  # noqa: E402
from oracle import statevector as SV  # noqa: E402
from oracle.vidal import VidalMPS  # noqa: E402
from tests.helpers import contract_sites  # noqa: E402


def _norm(v):
    return v / np.linalg.norm(v)


@pytest.mark.parametrize("prec", [E.TF32X3, E.FP64])
def test_untruncated_vidal_matches_the_state_vector(prec):
    n = 10
    circ = W.brickwork_circuit(n, 8, 501)
    m = E.MPS(n, n_2q=circ.n_2q, precision=prec, vidal=True).run(circ.gates(), 1.0)
    psi = SV.run_circuit(n, circ.gates())
    tol = 1e-12 if prec == E.FP64 else 1e-6
    assert 1.0 - abs(np.vdot(psi, _norm(contract_sites(m)))) ** 2 < tol
    assert m.centre() == 0
    m.close()


@pytest.mark.parametrize("prec", [E.TF32X3, E.FP64])
@pytest.mark.parametrize("seed,f_min", [(502, 0.95), (503, 0.8)])
def test_ea_vidal_matches_the_vidal_oracle(prec, seed, f_min):
    n = 12
    circ = W.brickwork_circuit(n, 10, seed)
    m = E.MPS(n, f_min=f_min, n_2q=circ.n_2q, precision=prec, vidal=True).run(circ.gates())
    o = VidalMPS(n, f_min=f_min, n_2q=circ.n_2q)
    for q, u in circ.gates():
        o.apply_2q(q, u)
    assert m.bond_dims() == o.bond_dims()
    assert abs(m.fidelity() - o.product) < (1e-10 if prec == E.FP64 else 1e-4)
    ov = abs(np.vdot(_norm(o.to_statevector()), _norm(contract_sites(m)))) ** 2
    assert 1.0 - ov < (1e-12 if prec == E.FP64 else 1e-5)
    # the amplitude chain works on the Vidal form (no centre move)
    bits = [0] * n
    assert abs(m.amplitude(bits) - o.to_statevector()[0]) < (1e-10 if prec == E.FP64 else 1e-4)
    m.close()


def test_vidal_handles_refuse_centre_dependent_operations():
    n = 6
    m = E.MPS(n, vidal=True)
    m.apply_2q(2, W.haar_unitary(4, 1, 0))
    z = np.diag([1.0, -1.0]).astype(np.complex128)
    with pytest.raises(E.MpsError):
        m.expect(0, z)
    with pytest.raises(E.MpsError):
        E.mps_set_centre(m.h, 2)
    ref = E.MPS(n)
    ref.apply_2q(2, W.haar_unitary(4, 1, 0))
    assert abs(abs(m.overlap(ref)) - 1.0) < 1e-5
    m.close()
    ref.close()
    with pytest.raises(E.MpsError):
        E.MPS(4, kind=E.MIXED, vidal=True)


def _layer_bounds(circ):
    n = circ.n_2q
    return [0] + [g for g in range(1, n) if circ.layers[g] != circ.layers[g - 1]] + [n]


def _ops_dev(circ):
    return torch.from_numpy(circ.ops_array().view(np.float64).reshape(circ.n_2q, 32).copy()).cuda()


def _run_layers(circ, conc, f_min, prec=E.TF32X3, chi_max=0):
    n = circ.n_qubits
    ops = _ops_dev(circ)
    qs = np.asarray(circ.qs, dtype=np.int32)
    m = E.MPS(n, f_min=f_min, n_2q=circ.n_2q, precision=prec, chi_max=chi_max, vidal=True)
    b = _layer_bounds(circ)
    for a0, a1 in zip(b[:-1], b[1:]):
        m.apply_layer(qs[a0:a1], ops.data_ptr() + a0 * 256, concurrency=conc)
    torch.cuda.synchronize()
    return m


@pytest.mark.parametrize("prec", [E.TF32X3, E.FP64])
def test_layer_runs_match_the_oracle_layer_by_layer(prec):
    n = 16
    circ = W.brickwork_circuit(n, 12, 511)
    m = _run_layers(circ, 4, 0.9, prec)
    o = VidalMPS(n, f_min=0.9, n_2q=circ.n_2q)
    b = _layer_bounds(circ)
    for a0, a1 in zip(b[:-1], b[1:]):
        o.apply_layer(list(zip(circ.qs[a0:a1], circ.ops[a0:a1])))
    assert m.bond_dims() == o.bond_dims()
    assert max(o.bond_dims()) < 2 ** (n // 2)
    assert abs(m.fidelity() - o.product) < (1e-10 if prec == E.FP64 else 1e-4)
    log = m.truncation_log()
    assert len(log) == circ.n_2q
    for r, ro in zip(log, o.log):
        assert r["q"] == ro["q"] and r["k"] == ro["k"]
        assert abs(r["f_t"] - ro["f_t"]) < (1e-12 if prec == E.FP64 else 1e-5)
    ov = abs(np.vdot(_norm(o.to_statevector()), _norm(contract_sites(m)))) ** 2
    assert 1.0 - ov < (1e-12 if prec == E.FP64 else 1e-5)
    assert m.stats()["gates"] == circ.n_2q
    m.close()


def test_layer_result_does_not_depend_on_the_concurrency():
    """One target per layer and disjoint pairs: concurrency 1 and 8 run the same kernels on the same
    data, so the bonds, fidelities and states agree exactly."""
    n = 24
    circ = W.brickwork_circuit(n, 14, 512)
    a = _run_layers(circ, 1, 0.8, chi_max=64)
    b = _run_layers(circ, 8, 0.8, chi_max=64)
    assert a.bond_dims() == b.bond_dims()
    assert a.fidelity() == b.fidelity()
    assert [r["f"] for r in a.truncation_log()] == [r["f"] for r in b.truncation_log()]
    for i in range(n):
        assert np.array_equal(a.site(i), b.site(i))
    a.close()
    b.close()


def test_layer_equals_sequential_gates_with_the_layer_targets():
    n = 14
    circ = W.brickwork_circuit(n, 10, 513)
    m = _run_layers(circ, 6, 0.85)
    targets = [r["f_t"] for r in m.truncation_log()]
    ops = _ops_dev(circ)
    s = E.MPS(n, f_min=0.85, n_2q=circ.n_2q, vidal=True)
    for g, q in enumerate(circ.qs):
        E.mps_apply_2q_device(s.h, q, ops.data_ptr() + g * 256, 4, targets[g])
    assert s.bond_dims() == m.bond_dims()
    assert abs(s.fidelity() - m.fidelity()) < 1e-12
    # truncations leave a Vidal-form state slightly off unit norm: compare the normalised overlap
    ov = abs(s.overlap(m)) / np.sqrt(s.overlap(s).real * m.overlap(m).real)
    assert abs(ov - 1.0) < 1e-6
    s.close()
    m.close()


def test_layer_call_refuses_bad_arguments():
    n = 8
    u = torch.from_numpy(np.stack([W.haar_unitary(4, 2, g) for g in range(3)]).view(np.float64)
                         .reshape(3, 32).copy()).cuda()
    m = E.MPS(n, vidal=True)
    with pytest.raises(E.MpsError):
        m.apply_layer([1, 2], u.data_ptr())          # pairs share qubit 2
    with pytest.raises(E.MpsError):
        m.apply_layer([6, 7], u.data_ptr())          # (7, 8) outside the chain
    with pytest.raises(E.MpsError):
        m.apply_layer([0, 2], u.data_ptr(), concurrency=0)
    m.apply_layer([0, 2, 4], u.data_ptr())           # nothing ran before: the handle is still usable
    assert m.stats()["gates"] == 3
    m.close()
    c = E.MPS(n)
    with pytest.raises(E.MpsError):
        c.apply_layer([0, 2], u.data_ptr())          # not a Vidal handle
    c.close()
