"""Parameter-shift gradients through the simulator (paper_2307_16870_gb300.grad) against the
state-vector oracle: the value, central finite differences and the oracle's own parameter shift."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
E = pytest.importorskip("paper_2307_16870_gb300")

import workloads as W  # noqa: E402
from oracle import statevector as SV  # noqa: E402

ZZ = np.diag([1.0, -1.0, -1.0, 1.0]).astype(np.complex128)


def _sv_energy(n, layers, p):
    psi = SV.run_circuit(n, W.ansatz_circuit(n, layers, p).gates())
    return sum(SV.expect(psi, n, i, ZZ).real for i in range(n - 1))


def test_energy_and_parameter_shift_gradient_match_the_oracle():
    from paper_2307_16870_gb300 import grad as G
    n, layers = 12, 2
    p = W.ansatz_params(n, layers, 21)
    fn = lambda a: W.ansatz_circuit(n, layers, a)   # noqa: E731
    e, g, info = G.energy_and_grad(fn, n, p, concurrency=8)
    assert info["circuits"] == 2 * p.size + 1
    assert abs(e - _sv_energy(n, layers, p)) < 1e-5
    # the oracle's parameter shift on a subset of the angles, and central differences
    rng = np.random.default_rng(0)
    for k in rng.choice(p.size, 8, replace=False):
        shift = np.zeros_like(p)
        shift[k] = math.pi / 2
        ps = 0.5 * (_sv_energy(n, layers, p + shift) - _sv_energy(n, layers, p - shift))
        h = np.zeros_like(p)
        h[k] = 1e-3
        fd = (_sv_energy(n, layers, p + h) - _sv_energy(n, layers, p - h)) / 2e-3
        assert abs(g[k] - ps) < 1e-5, (k, g[k], ps)
        assert abs(g[k] - fd) < 1e-4, (k, g[k], fd)


def test_autograd_function_returns_the_gradient():
    from paper_2307_16870_gb300 import grad as G
    n, layers = 8, 1
    p = torch.tensor(W.ansatz_params(n, layers, 5), dtype=torch.float64, requires_grad=True)
    fn = lambda a: W.ansatz_circuit(n, layers, a)   # noqa: E731
    val = G.CircuitEnergy.apply(p, fn, n)
    val.backward()
    _, g, _ = G.energy_and_grad(fn, n, p.detach().numpy())
    assert torch.allclose(p.grad, torch.as_tensor(g), atol=1e-12)
    assert abs(val.item() - _sv_energy(n, layers, p.detach().numpy())) < 1e-5
