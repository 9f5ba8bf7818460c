"""Gradients of circuit expectation values through the EA-MPS simulator, by the
parameter-shift rule, evaluated as one batch of circuits on the GPU.

For a gate exp(-i t P / 2) with P a Pauli product, d<H>/dt = (<H>(t + pi/2) -
<H>(t - pi/2)) / 2 exactly (for the untruncated simulation).  The gradient with
respect to all P angles of a circuit is therefore 2P + 1 independent circuit
simulations (the unshifted one gives the value), which mps_batch_run executes
concurrently, each circuit on its own handle and stream.  Every numerical step
runs in the library's kernels; this module builds the shifted gate lists and
combines the expectation values.

With truncation (F_min < 1) the shifted circuits are truncated independently,
so the result is the parameter-shift estimate of the truncated simulation.
"""
from __future__ import annotations

import math

import numpy as np

from . import GLOBAL, OK, TF32X3, WARN_CHI_CAP, MPS, MpsError, mps_batch_run

__all__ = ["zz_chain_energy", "energy_and_grad", "CircuitEnergy"]

_ZZ = np.diag([1.0, -1.0, -1.0, 1.0]).astype(np.complex128)


def zz_chain_energy(m: MPS) -> float:
    """sum_i <Z_i Z_{i+1}> of a pure-state handle."""
    return float(sum(m.expect(i, _ZZ).real for i in range(m.n - 1)))


def energy_and_grad(circuit_fn, n_qubits: int, params, observable=zz_chain_energy, f_min: float = 1.0,
                    chi_max: int = 0, precision: int = TF32X3, concurrency: int = 8, with_grad: bool = True):
    """Value of observable(final state) for the circuit circuit_fn(params) and its gradient with
    respect to every entry of params by the parameter-shift rule.

    circuit_fn(angles) -> an object with qs (left qubits), ops_array() (n_gates x 4 x 4 complex)
    and n_2q, whose every angle enters as exp(-i t P / 2) for a Pauli product P, with the same
    gate count for every angle vector.  observable(MPS) -> float.
    Returns (value, grad, info): grad has the shape of params (None without with_grad); info
    holds the number of circuits, of two-qubit updates and the inferred fidelities.
    """
    import torch

    p0 = np.asarray(params, dtype=np.float64).reshape(-1)
    shifts = [p0]
    if with_grad:
        for k in range(p0.size):
            for sgn in (1.0, -1.0):
                p = p0.copy()
                p[k] += sgn * math.pi / 2
                shifts.append(p)
    circuits = [circuit_fn(p.reshape(np.shape(params))) for p in shifts]
    n_2q = circuits[0].n_2q
    if any(c.n_2q != n_2q for c in circuits):
        raise ValueError("circuit_fn must give the same gate count for every angle vector")
    ops = np.stack([c.ops_array() for c in circuits]).view(np.float64).reshape(len(circuits), n_2q, 32)
    ops_dev = torch.from_numpy(np.ascontiguousarray(ops)).cuda()
    stride = n_2q * 32 * 8
    base = ops_dev.data_ptr()
    items = [{"n_qubits": n_qubits, "qs": c.qs, "ops_dev": base + i * stride, "op_dim": 4, "f_min": f_min,
              "n_2q": n_2q, "strategy": GLOBAL, "chi_max": chi_max, "precision": precision}
             for i, c in enumerate(circuits)]
    code, res = mps_batch_run(items, concurrency=concurrency, keep=True)
    try:
        if code not in (OK, WARN_CHI_CAP):
            raise MpsError(code, "mps_batch_run")
        values = np.array([observable(r["mps"]) for r in res])
    finally:
        for r in res:
            if "mps" in r:
                r["mps"].close()
    grad = None
    if with_grad:
        grad = (0.5 * (values[1::2] - values[2::2])).reshape(np.shape(params))
    info = {"circuits": len(circuits), "updates": len(circuits) * n_2q,
            "inferred_fidelity": [r["fidelity"] for r in res]}
    return float(values[0]), grad, info


try:
    import torch as _torch

    class CircuitEnergy(_torch.autograd.Function):
        """value = observable(final state of circuit_fn(params)) as a differentiable torch function;
        forward evaluates the value and the parameter-shift gradient as one batch on the GPU."""

        @staticmethod
        def forward(ctx, params, circuit_fn, n_qubits: int, f_min: float = 1.0, chi_max: int = 0,
                    concurrency: int = 8):
            v, g, _ = energy_and_grad(circuit_fn, n_qubits, params.detach().cpu().numpy(), f_min=f_min,
                                      chi_max=chi_max, concurrency=concurrency)
            ctx.save_for_backward(_torch.as_tensor(g, dtype=params.dtype))
            return params.new_tensor(v)

        @staticmethod
        def backward(ctx, grad_out):
            (g,) = ctx.saved_tensors
            return grad_out * g.to(grad_out.device), None, None, None, None, None
except ImportError:   # pragma: no cover
    CircuitEnergy = None
