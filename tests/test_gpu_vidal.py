"""The Vidal / Hastings mode (mps_options.vidal) against the FP64 oracle of the same form."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
E = pytest.importorskip("paper_2307_16870_gb300")

import workloads as W  # noqa: E402
from oracle import statevector as SV  # noqa: E402
from oracle.vidal import VidalMPS  # noqa: E402


def _norm(v):
    return v / np.linalg.norm(v)


@pytest.mark.parametrize("prec", [E.TF32X3, E.FP64])
def test_untruncated_vidal_matches_the_state_vector(prec):
    n = 10
    circ = W.brickwork_circuit(n, 8, 501)
    m = E.MPS(n, n_2q=circ.n_2q, precision=prec, vidal=True).run(circ.gates(), 1.0)
    psi = SV.run_circuit(n, circ.gates())
    tol = 1e-12 if prec == E.FP64 else 1e-6
    assert 1.0 - abs(np.vdot(psi, _norm(m.contract()))) ** 2 < tol
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
    ov = abs(np.vdot(_norm(o.to_statevector()), _norm(m.contract()))) ** 2
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
