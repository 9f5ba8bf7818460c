"""Test-only builders shared by the GPU parity tests."""
import numpy as np

import workloads as W


def random_canonical_mps(n, chi_cap, centre, seed, d=2, round_c64=True):
    """Random MPS in canonical form around ``centre``: sites left of it are random
    left isometries, sites right of it random right isometries, the centre a random
    unit tensor.  Bonds are min(chi_cap, d^min(b, n-b)).  With ``round_c64`` every
    entry is first rounded to complex64, so a complex64 device copy is exact."""
    bonds = [1] + [min(chi_cap, d ** min(b, n - b)) for b in range(1, n)] + [1]
    sites = []
    off = 0
    for i in range(n):
        cl, cr = bonds[i], bonds[i + 1]
        cnt = cl * d * cr
        g = W.normals(seed, off, 2 * cnt).reshape(2, cnt)
        off += 2 * cnt + 2
        t = (g[0] + 1j * g[1]).reshape(cl, d, cr)
        if i < centre:
            q, _ = np.linalg.qr(t.reshape(cl * d, cr))
            t = q.reshape(cl, d, cr)
        elif i > centre:
            q, _ = np.linalg.qr(t.reshape(cl, d * cr).conj().T)
            t = q.conj().T.reshape(cl, d, cr)
        else:
            t = t / np.linalg.norm(t)
        if round_c64:
            t = t.astype(np.complex64).astype(np.complex128)
        sites.append(np.ascontiguousarray(t))
    return sites, bonds
