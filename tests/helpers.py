"""Test-only helpers shared by the GPU tests and the smoke check."""
from workloads import random_canonical_mps  # noqa: F401


def contract_sites(m):
    """Every site of a library handle (paper_2307_16870_gb300.MPS) read back and contracted on the
    host into its d^N coefficients (small chains only)."""
    t = m.site(0).reshape(m.d, -1)
    for i in range(1, m.n):
        b = m.site(i)
        t = (t @ b.reshape(b.shape[0], -1)).reshape(-1, b.shape[2])
    return t.reshape(-1)
