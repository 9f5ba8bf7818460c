"""Householder QR kernels (mps_qr_c64) against the definition X = Q R, Q^dagger Q = I,
R upper triangular, and against LAPACK's R (same real-diagonal convention)."""
import numpy as np
import pytest
from tests.helpers import contract_sites  # noqa: E402

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
E = pytest.importorskip("paper_2307_16870_gb300")


def _rand(l, c, seed, graded=False):
    g = np.random.default_rng(seed)
    x = (g.normal(size=(l, c)) + 1j * g.normal(size=(l, c))) / np.sqrt(2)
    if graded:      # singular values spanning 1 .. e^-10
        u, _ = np.linalg.qr(x)
        v, _ = np.linalg.qr(g.normal(size=(c, c)) + 1j * g.normal(size=(c, c)))
        k = min(l, c)
        x = (u[:, :k] * np.exp(-np.linspace(0, 10, k))) @ v[:k, :]
    return x.astype(np.complex64)


def _qr_gpu(x):
    l, c = x.shape
    k = min(l, c)
    xd = torch.from_numpy(np.asfortranarray(x).T.copy()).cuda()          # column-major: row j = column j
    qd = torch.zeros((k, l), dtype=torch.complex64, device="cuda")
    E.mps_qr_c64(l, c, xd.data_ptr(), l, qd.data_ptr(), l)
    f = xd.cpu().numpy().T                                               # factored, l x c
    q = qd.cpu().numpy().T                                               # l x k
    r = np.triu(f[:k, :])
    return q.astype(np.complex128), r.astype(np.complex128)


SHAPES = [(1, 1), (7, 3), (32, 32), (33, 31), (64, 96), (100, 40), (256, 256), (300, 129), (512, 256),
          (512, 512), (480, 500), (512, 37)]


@pytest.mark.parametrize("l,c", SHAPES)
def test_qr_definition(l, c):
    x = _rand(l, c, l * 1000 + c)
    q, r = _qr_gpu(x)
    x64 = x.astype(np.complex128)
    nx = np.linalg.norm(x64)
    assert np.linalg.norm(q @ r - x64) < 2e-6 * nx * np.sqrt(max(l, c) / 32)
    k = min(l, c)
    assert np.abs(q.conj().T @ q - np.eye(k)).max() < 3e-6 * np.sqrt(l / 32)
    assert np.all(np.abs(np.imag(np.diag(r))) < 1e-6 * np.abs(np.diag(r)).max())   # real diagonal
    # LAPACK's R (numpy) has the same convention: equal up to rounding
    _, r_ref = np.linalg.qr(x64, mode="reduced" if l >= c else "complete")
    r_ref = r_ref[:k, :]
    assert np.abs(r - r_ref).max() < 5e-6 * np.abs(r_ref).max() * np.sqrt(max(l, c) / 32)


def test_qr_graded_and_rank_deficient():
    x = _rand(512, 512, 5, graded=True)
    q, r = _qr_gpu(x)
    x64 = x.astype(np.complex128)
    assert np.linalg.norm(q @ r - x64) < 1e-5 * np.linalg.norm(x64)
    assert np.abs(q.conj().T @ q - np.eye(512)).max() < 1e-5
    # exact zero columns and a rank-one block
    z = np.zeros((64, 48), np.complex64)
    z[:, 5] = _rand(64, 1, 9)[:, 0]
    z[:, 20] = 2 * z[:, 5]
    q, r = _qr_gpu(z)
    assert np.linalg.norm(q @ r - z) < 1e-5 * np.linalg.norm(z)
    assert np.abs(q.conj().T @ q - np.eye(48)).max() < 1e-5


def test_qr_rejects_too_many_rows():
    x = torch.zeros((4, 513), dtype=torch.complex64, device="cuda")
    with pytest.raises(E.MpsError):
        E.mps_qr_c64(513, 4, x.data_ptr(), 513)


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_circuit_with_qr_modes_matches_oracle(mode):
    """mps_options.qr bits: QR_PRECONDITION the preconditioned gate SVD, QR_MOVES the QR centre
    moves (0: Jacobi only)."""
    import workloads as W
    from oracle import textbook_mps as T
    from oracle import statevector as SV
    n = 12
    circ = W.brickwork_circuit(n, 10, 77)
    m = E.MPS(n, f_min=0.97, n_2q=circ.n_2q, precision=E.TF32X3, log_truncations=False, qr=mode)
    m.run(circ.gates())
    o = T.TextbookMPS(n, f_min=0.97, n_2q=circ.n_2q)
    for q, u in circ.gates():
        o.apply_2q(q, u)
    assert m.bond_dims() == o.bond_dims()
    assert abs(m.fidelity() - o.product) < 1e-4
    psi = SV.run_circuit(n, circ.gates())
    got = contract_sites(m)
    f_true = abs(np.vdot(psi, got)) ** 2 / np.vdot(got, got).real
    f_orc = abs(np.vdot(psi, o.to_statevector())) ** 2
    assert abs(f_true - f_orc) < 1e-4
    st = m.stats()
    if mode & E.QR_MOVES:
        assert st["qr_launches"] > 0
    else:   # bonds <= 64 here: the gate SVD is preconditioned only from 256 columns on
        assert st["qr_launches"] == 0
    m.close()


@pytest.mark.parametrize("centre,q", [(20, 20), (20, 21)])
def test_preconditioned_update_from_256_columns(centre, q):
    """The QR-preconditioned gate SVD at its smallest size (theta 256 x 256, bonds 128) in both
    orientations, against the oracle's LAPACK SVD on identical inputs: same k, retained singular
    values to 1e-5 relative."""
    import workloads as W
    from oracle import textbook_mps as T
    n, cap = 40, 128
    sites, _ = W.random_canonical_mps(n, cap, centre, seed=600 + q)
    u = W.haar_unitary(4, 601, q)
    orc = T.TextbookMPS(n, record_svals=True, chi_max=cap)
    orc.sites = [x.copy() for x in sites]
    orc.centre = centre
    rec = orc.apply_2q(q, u, target=0.999)
    m = E.MPS(n, chi_max=cap, precision=E.TF32X3, qr=E.QR_PRECONDITION)
    m.load_sites(sites, centre)
    m.stats_reset()
    m.apply_2q(q, u, 0.999)
    k = rec["k"]
    assert m.truncation_log()[-1]["k"] == k
    rel = np.abs(m.last_singular_values()[:k] - rec["s"][:k]) / rec["s"][:k]
    assert rel.max() < 1e-5, rel.max()
    assert m.stats()["qr_launches"] >= 1
    m.close()
