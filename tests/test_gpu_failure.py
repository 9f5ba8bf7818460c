"""Failure detection without a GPU fault: a bounded device wait on a flag that nothing sets runs
out, the kernel records the timeout in the status word and returns, the host reads the error,
the handle stays failed (sticky) until mps_reset, and the context stays usable."""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
E = pytest.importorskip("paper_2307_16870_gb300")

import workloads as W  # noqa: E402
from oracle import statevector as SV  # noqa: E402


def test_a_wait_that_runs_out_is_reported_and_the_handle_recovers_after_reset():
    n = 6
    m = E.MPS(n)
    u = W.haar_unitary(4, 3, 0)
    m.apply_2q(2, u)
    t0 = time.perf_counter()
    with pytest.raises(E.MpsError) as ei:
        E.mps_selftest_wait(m.h, 1000000)
    assert ei.value.code == 8                      # MPS_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 10.0
    with pytest.raises(E.MpsError):                # sticky until reset
        m.apply_2q(0, u)
    m.reset()
    circ = W.brickwork_circuit(n, 4, 31)
    m.run(circ.gates(), 1.0)
    psi = SV.run_circuit(n, circ.gates())
    got = m.contract()
    assert 1.0 - abs(np.vdot(psi, got)) ** 2 / np.vdot(got, got).real < 1e-6
    # another handle on the same context was never affected
    other = E.MPS(n)
    other.apply_2q(1, u)
    assert abs(other.fidelity() - 1.0) < 1e-12
    other.close()
    with pytest.raises(E.MpsError):
        E.mps_selftest_wait(m.h, 0)                # out of range
    m.close()
