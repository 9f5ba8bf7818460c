"""Stream ordering of a handle created on a caller's non-blocking stream that still has
work queued: the initial state must be written behind that work, not beside it."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
E = pytest.importorskip("paper_2307_16870_gb300")

import workloads as W  # noqa: E402


def test_handle_on_a_busy_nonblocking_stream_starts_from_the_product_state():
    s = torch.cuda.Stream()          # pool streams are created non-blocking
    with torch.cuda.stream(s):
        torch.cuda._sleep(100_000_000)   # a bounded spin queued ahead of the handle's initialisation
    m = E.MPS(6, stream=s.cuda_stream)
    amp = m.amplitude([0] * 6)
    assert abs(amp - 1.0) < 1e-6
    u = W.haar_unitary(4, 5, 0)
    m.apply_2q(2, u)
    assert m.fidelity() == 1.0
    # <0..0|U|0..0> on qubits (2, 3): the (0, 0) entry of the gate
    assert abs(m.amplitude([0] * 6) - u[0, 0]) < 1e-5
    m.close()


def test_statistics_after_stats_reset_and_state_reset():
    """Counters zeroed by stats_reset stay zeroed through a later state reset (the benchmark's
    warm-up runs must not leak into the timed statistics)."""
    circ = W.brickwork_circuit(10, 8, 3)
    m = E.MPS(10, f_min=0.99, n_2q=circ.n_2q, log_truncations=False)
    m.run(circ.gates())
    m.stats_reset()
    m.reset()
    st = m.stats()
    assert st["jacobi_sweeps"] == 0 and st["jacobi_flops"] == 0.0 and st["jacobi_launches"] == 0
    m.run(circ.gates())
    one = m.stats()
    m.reset()
    m.run(circ.gates())
    two = m.stats()
    assert one["jacobi_launches"] > 0
    assert two["jacobi_sweeps"] == 2 * one["jacobi_sweeps"]
    assert two["jacobi_flops"] == pytest.approx(2 * one["jacobi_flops"], rel=1e-12)
    m.close()
