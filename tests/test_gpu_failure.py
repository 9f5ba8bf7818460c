"""Failure detection without a GPU fault: a signal is withheld, the bounded wait for it runs out
at the handle's wall-clock limit, the kernel records the timeout in the status word and every
CTA returns; the host reads the error, the handle stays failed (sticky) until mps_reset, the
context stays usable and other handles are unaffected.  The waits tested are the real ones: a
single-flag wait, the block exchange of the point-to-point Jacobi kernel, the exchange and
cluster agreement of the Gram-matrix block Jacobi kernel, and the mbarrier pipeline of the
tensor-core contraction."""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
E = pytest.importorskip("paper_2307_16870_gb300")

import workloads as W  # noqa: E402
from oracle import statevector as SV  # noqa: E402
from tests.helpers import contract_sites  # noqa: E402

SITES = ["flag", "jacobi", "gram", "gemm"]


@pytest.mark.parametrize("site", range(4), ids=SITES)
def test_a_wait_that_runs_out_is_reported_and_the_handle_recovers_after_reset(site):
    n = 6
    m = E.MPS(n, precision=E.TF32X3)
    u = W.haar_unitary(4, 3, 0)
    m.apply_2q(2, u)
    t0 = time.perf_counter()
    with pytest.raises(E.MpsError) as ei:
        E.mps_selftest_timeout(m.h, site, 50_000_000)   # 50 ms limit
    assert ei.value.code == 8                      # MPS_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 5.0          # every CTA returned promptly
    with pytest.raises(E.MpsError):                # sticky until reset
        m.apply_2q(0, u)
    m.reset()
    circ = W.brickwork_circuit(n, 4, 31)
    m.run(circ.gates(), 1.0)
    psi = SV.run_circuit(n, circ.gates())
    got = contract_sites(m)
    assert 1.0 - abs(np.vdot(psi, got)) ** 2 / np.vdot(got, got).real < 1e-6
    # another handle on the same context was never affected
    other = E.MPS(n)
    other.apply_2q(1, u)
    assert abs(other.fidelity() - 1.0) < 1e-12
    other.close()
    m.close()


def test_self_test_arguments():
    m = E.MPS(4, precision=E.FP64)
    for site, ns in [(4, 10**6), (-1, 10**6), (0, 10), (0, 10**12), (1, 10**6), (3, 10**6)]:
        with pytest.raises(E.MpsError) as ei:      # out of range, or a complex64 site on an FP64 handle
            E.mps_selftest_timeout(m.h, site, ns)
        assert ei.value.code == 1
    m.close()
