"""Single two-site updates on identical inputs at the benchmark's full size.

The state is a random canonical MPS on 100 qubits with every bond capped at 256
(theta is 512 x 512, the saturated regime of the benchmark circuit), rounded to
complex64 so that both sides start from the same numbers.  The oracle applies
the update in FP64 (QR centre moves, LAPACK SVD); the CUDA path runs the same
launch configuration as bench.py.  Checked: bond size, truncation fidelity and
every retained singular value to 1e-5 relative (complex64 path)."""
import numpy as np
import pytest

import workloads as W
from oracle import textbook_mps as T
from tests.helpers import random_canonical_mps

pytestmark = pytest.mark.gpu
E = pytest.importorskip("paper_2307_16870_gb300")

N, CAP = 100, 256
PRECS = [("tf32x3", 1, 1e-5), ("fp32", 2, 1e-5), ("fp64", 0, 1e-10)]


def _oracle_from(sites, centre, kind=T.PURE, cap=CAP):
    o = T.TextbookMPS(len(sites), kind=kind, record_svals=True, chi_max=cap)
    o.sites = [s.copy() for s in sites]
    o.centre = centre
    return o


@pytest.mark.parametrize("name,prec,tol", PRECS)
@pytest.mark.parametrize("centre,q", [(50, 50), (47, 50), (55, 50), (3, 1), (97, 98)])
def test_single_update_exact_input(name, prec, tol, centre, q):
    sites, bonds = random_canonical_mps(N, CAP, centre, seed=500 + centre)
    u = W.haar_unitary(4, 501, q)
    target = 0.99
    orc = _oracle_from(sites, centre)
    rec = orc.apply_2q(q, u, target=target)
    m = E.MPS(N, chi_max=CAP, precision=prec)
    m.load_sites(sites, centre)
    m.apply_2q(q, u, target)
    g = m.truncation_log()[-1]
    s_gpu = m.last_singular_values()
    s_orc = rec["s"]
    assert g["rank_bound"] == rec["rank_bound"] == len(s_orc) == len(s_gpu)
    assert g["k"] == rec["k"], (g["k"], rec["k"])
    k = rec["k"]
    rel = np.abs(s_gpu[:k] - s_orc[:k]) / s_orc[:k]
    assert rel.max() < tol, rel.max()
    assert abs(g["f"] - rec["f"]) < max(tol, 1e-9)
    assert m.bond_dims() == orc.bond_dims()
    assert m.centre() == orc.centre
    # the updated pair represents the same two-site block (gauge-invariant check)
    a = m.site(q).reshape(-1, k) @ m.site(q + 1).reshape(k, -1)
    b = orc.sites[q].reshape(-1, k) @ orc.sites[q + 1].reshape(k, -1)
    if centre == q:   # same gauge on the outer bonds only when no centre move touched them
        assert np.abs(a - b).max() < 50 * tol


@pytest.mark.parametrize("name,prec,tol", PRECS[:2])
def test_single_update_mpo_exact_input(name, prec, tol):
    """Mixed state: d = 4 sites, bonds capped at 128, theta 512 x 512, a noisy superoperator."""
    from oracle import superop as SO
    n, cap, centre, q = 30, 128, 15, 15
    sites, _ = random_canonical_mps(n, cap, centre, seed=777, d=4)
    ad = W.amplitude_damping_kraus(0.005)
    s_op = np.kron(SO.from_kraus(ad, 1), SO.from_kraus(ad, 1)) @ \
        SO.from_kraus(W.depolarizing_2q_kraus(0.01), 2) @ SO.from_unitary(W.haar_unitary(4, 778, 0))
    orc = _oracle_from(sites, centre, kind=T.MIXED, cap=cap)
    rec = orc.apply_2q(q, s_op, target=0.95)
    m = E.MPS(n, kind=E.MIXED, chi_max=cap, precision=prec)
    m.load_sites(sites, centre)
    m.apply_2q(q, s_op, 0.95)
    g = m.truncation_log()[-1]
    s_gpu = m.last_singular_values()
    assert g["k"] == rec["k"]
    k = rec["k"]
    rel = np.abs(s_gpu[:k] - rec["s"][:k]) / rec["s"][:k]
    assert rel.max() < tol, rel.max()
    assert abs(m.lognorm() - orc.lognorm) < 1e-6


@pytest.mark.parametrize("name,prec,tol", PRECS[:2])
@pytest.mark.parametrize("centre", [12, 10])
def test_single_update_theta_1024_pure_chi_512(name, prec, tol, centre):
    """The largest point of the pure-state benchmark (fixed chi = 512): bonds 512 around the pair,
    theta 1024 x 1024 (the Gram-matrix block Jacobi layout), with and without centre moves."""
    n, cap, q = 24, 512, 12
    sites, _ = random_canonical_mps(n, cap, centre, seed=610 + centre)
    u = W.haar_unitary(4, 611, q)
    orc = _oracle_from(sites, centre, cap=cap)
    rec = orc.apply_2q(q, u, target=0.999)
    m = E.MPS(n, chi_max=cap, precision=prec)
    m.load_sites(sites, centre)
    m.apply_2q(q, u, 0.999)
    g = m.truncation_log()[-1]
    assert g["rank_bound"] == rec["rank_bound"] == 1024
    assert g["k"] == rec["k"], (g["k"], rec["k"])
    k = rec["k"]
    rel = np.abs(m.last_singular_values()[:k] - rec["s"][:k]) / rec["s"][:k]
    assert rel.max() < tol, rel.max()
    assert abs(g["f"] - rec["f"]) < tol
    assert m.bond_dims() == orc.bond_dims()


@pytest.mark.parametrize("name,prec,tol", PRECS[:2])
def test_single_update_mpo_cap_256_theta_1024(name, prec, tol):
    """Mixed state at its full size: d = 4 sites with bonds capped at 256, theta 1024 x 1024, a
    noisy superoperator (gate, two-qubit depolarising, amplitude damping on both qubits)."""
    from oracle import superop as SO
    n, cap, centre, q = 12, 256, 6, 6
    sites, _ = random_canonical_mps(n, cap, centre, seed=779, d=4)
    ad = W.amplitude_damping_kraus(0.005)
    s_op = np.kron(SO.from_kraus(ad, 1), SO.from_kraus(ad, 1)) @ \
        SO.from_kraus(W.depolarizing_2q_kraus(0.01), 2) @ SO.from_unitary(W.haar_unitary(4, 780, 0))
    orc = _oracle_from(sites, centre, kind=T.MIXED, cap=cap)
    rec = orc.apply_2q(q, s_op, target=0.95)
    m = E.MPS(n, kind=E.MIXED, chi_max=cap, precision=prec)
    m.load_sites(sites, centre)
    m.apply_2q(q, s_op, 0.95)
    g = m.truncation_log()[-1]
    assert g["rank_bound"] == rec["rank_bound"] == 1024
    assert g["k"] == rec["k"]
    k = rec["k"]
    rel = np.abs(m.last_singular_values()[:k] - rec["s"][:k]) / rec["s"][:k]
    assert rel.max() < tol, rel.max()
    assert abs(m.lognorm() - orc.lognorm) < 1e-6
