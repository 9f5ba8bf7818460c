"""The two layouts of the one-sided Jacobi SVD against the FP64 oracle (LAPACK's SVD).

mps_options.svd_kernel selects the tournament kernels (MPS_SVD_TOURNAMENT) or the block kernel
with Gram-matrix inner sweeps over thread-block clusters (MPS_SVD_GRAM).  The automatic choice
times both on the first use of a shape class from 256 columns on and keeps the faster; these
tests force each layout at sizes the oracle finishes in seconds: several slots and rounds, ragged column counts (zero padding columns), both orientations,
and accumulated rotations (the rows of W below those of X).  Tolerances as everywhere for the
complex64 path: retained singular values 1e-5 relative on identical inputs, untruncated overlap
1 - 1e-6, vectors orthonormal to 1e-5."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
E = pytest.importorskip("paper_2307_16870_gb300")

import workloads as W  # noqa: E402
from oracle import statevector as SV  # noqa: E402
from oracle import textbook_mps as T  # noqa: E402
from oracle.diff_chain import tsvd as o_tsvd  # noqa: E402
from tests.helpers import contract_sites  # noqa: E402

if E is not None:
    from paper_2307_16870_gb300 import autodiff as AD  # noqa: E402

LAYOUTS = [("gram", 2), ("tournament", 1), ("tournament_unsplit", 3)]


@pytest.mark.parametrize("name,kernel", LAYOUTS)
@pytest.mark.parametrize("centre,q", [(50, 50), (47, 50)])
def test_single_update_exact_input_theta_512(name, kernel, centre, q):
    """theta 512 x 512 of a 100-qubit canonical state with bonds 256 (the benchmark's regime)."""
    n, cap = 100, 256
    sites, _ = W.random_canonical_mps(n, cap, centre, seed=900 + centre)
    u = W.haar_unitary(4, 901, q)
    orc = T.TextbookMPS(n, record_svals=True, chi_max=cap)
    orc.sites = [s.copy() for s in sites]
    orc.centre = centre
    rec = orc.apply_2q(q, u, target=0.99)
    m = E.MPS(n, chi_max=cap, precision=E.TF32X3, svd_kernel=kernel)
    m.load_sites(sites, centre)
    m.apply_2q(q, u, 0.99)
    g = m.truncation_log()[-1]
    k = rec["k"]
    assert g["k"] == k and g["rank_bound"] == rec["rank_bound"] == 512
    s_gpu = m.last_singular_values()
    rel = np.abs(s_gpu[:k] - rec["s"][:k]) / rec["s"][:k]
    assert rel.max() < 1e-5, rel.max()
    assert abs(g["f"] - rec["f"]) < 1e-5
    assert m.bond_dims() == orc.bond_dims()


def test_untruncated_circuit_through_the_gram_layout():
    """14 qubits, depth 10, no truncation: theta up to 256 x 256 (4 to 8 slots) every gate."""
    n, depth = 14, 10
    circ = W.brickwork_circuit(n, depth, 1203)
    m = E.MPS(n, n_2q=circ.n_2q, precision=E.TF32X3, svd_kernel=E.SVD_GRAM).run(circ.gates(), 1.0)
    psi = SV.run_circuit(n, circ.gates())
    got = contract_sites(m)
    ov = abs(np.vdot(psi, got)) ** 2 / np.vdot(got, got).real
    assert ov > 1 - 1e-6, ov
    assert max(m.bond_dims()) == 2 ** (n // 2)


@pytest.fixture(scope="module")
def ws_gram():
    w = AD.Workspace(20, 512, E.TF32X3, svd_kernel=E.SVD_GRAM)   # pair scratch up to 1024 x 1024
    yield w
    w.close()


@pytest.mark.parametrize("m,n", [(200, 130), (130, 200), (96, 96), (300, 257), (257, 64)])
def test_accumulated_rotations_match_the_oracle(m, n, ws_gram):
    """The stateless SVD runs the Jacobi with accumulated rotations (X rows, then W rows)."""
    rng = np.random.default_rng(7 * m + n)
    a = rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))
    r = o_tsvd(a, 1.0, 0, 1e-6)
    aq, ap, info = AD.tsvd(ws_gram, torch.from_numpy(a).to(torch.complex64).cuda(), 1.0)
    k = r["k"]
    assert info["k"] == k == min(m, n)
    aq = aq.cpu().numpy().astype(np.complex128)
    ap = ap.cpu().numpy().astype(np.complex128)
    assert np.abs(aq.conj().T @ aq - np.eye(k)).max() < 1e-5
    s_gpu = np.linalg.norm(ap, axis=1) * np.sqrt(info["W_k"])
    rel = np.abs(s_gpu - r["S"][:k]) / r["S"][:k]
    assert rel.max() < 1e-5, rel.max()
    assert np.abs(aq @ ap - r["Aq"] @ r["Ap"]).max() < 1e-5 * np.abs(r["Aq"] @ r["Ap"]).max() * 10


def test_autotuner_times_the_layouts_and_keeps_the_faster():
    """mps_svd_tune on a 512 x 512 class (with and without accumulated rotations): the table then
    holds the timings, the kept tournament form is the faster of the two (with and without the row
    split, where both exist), and the block kernel is kept exactly when it was at least 10 % faster
    than that.  A second call does not time again."""
    m = E.MPS(100, chi_max=256, precision=E.TF32X3)
    for acc in (False, True):
        layout = m.svd_tune(512, 512, acc)
        assert layout in (E.SVD_TOURNAMENT, E.SVD_TOURNAMENT_UNSPLIT, E.SVD_GRAM)
    tab = {(t["rows"], t["cols"], t["accumulate"]): t for t in E.mps_svd_tuning()}
    for acc in (False, True):
        t = tab[(512, 512, acc)]
        assert t["ms_tournament"] > 0 and t["ms_gram"] > 0
        tours = [x for x in (t["ms_tournament"], t["ms_unsplit"]) if x > 0]
        best = min(tours)
        assert (t["layout"] == "gram") == (t["ms_gram"] < 0.9 * best)
        if t["layout"] != "gram":
            want = "tournament_unsplit" if 0 < t["ms_unsplit"] < t["ms_tournament"] else "tournament"
            assert t["layout"] == want
    # the class of 500 x 470 is that of 512 x 512: no new timing run
    before = len(E.mps_svd_tuning())
    m.svd_tune(500, 470, False)
    assert len(E.mps_svd_tuning()) == before
    m.close()


def test_autotuner_respects_a_forced_layout_and_small_shapes():
    m = E.MPS(100, chi_max=256, precision=E.TF32X3, svd_kernel=E.SVD_TOURNAMENT)
    assert m.svd_tune(512, 512) == E.SVD_TOURNAMENT
    m.close()
    m = E.MPS(100, chi_max=256, precision=E.TF32X3)
    assert m.svd_tune(128, 128) == E.SVD_AUTO      # below 256 columns: the fixed rule, no timing
    with pytest.raises(Exception):
        m.svd_tune(0, 512)
    with pytest.raises(Exception):
        m.svd_tune(512, 4096)
    m.close()


def test_tuned_automatic_choice_keeps_parity_at_theta_512():
    """After tuning, the automatic choice runs whichever layout won; the update still matches the
    oracle (retained singular values 1e-5 relative, same k)."""
    n, cap, centre, q = 100, 256, 50, 50
    sites, _ = W.random_canonical_mps(n, cap, centre, seed=950)
    u = W.haar_unitary(4, 951, q)
    orc = T.TextbookMPS(n, record_svals=True, chi_max=cap)
    orc.sites = [s.copy() for s in sites]
    orc.centre = centre
    rec = orc.apply_2q(q, u, target=0.99)
    m = E.MPS(n, chi_max=cap, precision=E.TF32X3)
    m.svd_tune(512, 512, False)
    m.svd_tune(512, 512, True)
    m.load_sites(sites, centre)
    m.apply_2q(q, u, 0.99)
    k = rec["k"]
    assert m.truncation_log()[-1]["k"] == k
    rel = np.abs(m.last_singular_values()[:k] - rec["s"][:k]) / rec["s"][:k]
    assert rel.max() < 1e-5, rel.max()
    m.close()
