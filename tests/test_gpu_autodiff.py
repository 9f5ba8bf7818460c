"""The differentiable update (mps_gemm_device, mps_tsvd_device, mps_tsvd_backward_device and
paper_2307_16870_gb300.autodiff) against the FP64 oracle of the same update."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
E = pytest.importorskip("paper_2307_16870_gb300")

import workloads as W  # noqa: E402
from oracle import statevector as SV  # noqa: E402
from oracle.diff_chain import DiffChain, tsvd as o_tsvd, tsvd_backward as o_backward, zz_energy_dense  # noqa: E402

if E is not None:
    from paper_2307_16870_gb300 import autodiff as AD  # noqa: E402


def _rand(rng, m, n):
    return rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))


def _cot(aq, ap, m1, w1, w2):
    """Cotangents of L = Re<m1, A_q A_p> + sum w1 |A_q|^2 + sum w2 |A_p|^2 (phase invariant)."""
    k = aq.shape[1]
    return m1 @ ap.conj().T + 2 * w1[:, :k] * aq, aq.conj().T @ m1 + 2 * w2[:k] * ap


def _adjoint_condition(s, k):
    """s_0^2 / min |s_i^2 - s_j^2| over the pairs i != j with i or j kept."""
    d = np.abs(s[:, None] ** 2 - s[None, :] ** 2)
    np.fill_diagonal(d, np.inf)
    d[k:, k:] = np.inf
    return float(s[0] ** 2 / d.min()) if np.isfinite(d.min()) else 0.0


@pytest.fixture(scope="module")
def ws32():
    w = AD.Workspace(16, 64, E.TF32X3)
    yield w
    w.close()


@pytest.fixture(scope="module")
def ws64():
    w = AD.Workspace(16, 64, E.FP64)
    yield w
    w.close()


SHAPES = [(96, 64, 0.9), (64, 96, 0.9), (80, 80, 0.95), (33, 17, 1.0), (17, 45, 1.0), (128, 128, 0.99), (8, 1, 1.0)]


@pytest.mark.parametrize("m,n,target", SHAPES)
@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_tsvd_matches_the_oracle(m, n, target, prec, ws32, ws64):
    ws = ws32 if prec == "c64" else ws64
    rng = np.random.default_rng(m * 1000 + n)
    a = _rand(rng, m, n)
    r = o_tsvd(a, target, 0, 1e-6)
    ta = torch.from_numpy(a).to(ws.dtype).cuda()
    aq, ap, info = AD.tsvd(ws, ta, target)
    tol = 1e-5 if prec == "c64" else 1e-12
    assert info["k"] == r["k"]
    assert abs(info["f"] - r["f"]) < tol
    aq = aq.cpu().numpy().astype(np.complex128)
    ap = ap.cpu().numpy().astype(np.complex128)
    assert np.abs(aq.conj().T @ aq - np.eye(r["k"])).max() < 10 * tol
    assert np.abs(aq @ ap - r["Aq"] @ r["Ap"]).max() < 10 * tol * np.abs(r["Aq"] @ r["Ap"]).max()


def _graded(rng, m, n, s):
    qa, _ = np.linalg.qr(_rand(rng, m, len(s)))
    qb, _ = np.linalg.qr(_rand(rng, n, len(s)))
    return (qa * s[None, :]) @ qb.conj().T


@pytest.mark.parametrize("m,n", [(64, 40), (40, 64)])
def test_tsvd_keeps_orthonormal_vectors_for_small_values(m, n, ws32):
    """Values down to 1e-5 of the largest: the vectors stay orthonormal to FP32 accuracy, the
    exact zeros beyond the rank are not kept, and A_q A_p is A / |A|."""
    rng = np.random.default_rng(m + 5 * n)
    sv = np.logspace(0, -5, 30)
    a = _graded(rng, m, n, sv)
    aq, ap, info = AD.tsvd(ws32, torch.from_numpy(a).to(torch.complex64).cuda(), 1.0)
    assert info["k"] == 30
    aq = aq.cpu().numpy().astype(np.complex128)
    ap = ap.cpu().numpy().astype(np.complex128)
    assert np.abs(aq.conj().T @ aq - np.eye(30)).max() < 2e-5
    assert np.abs(aq @ ap - a / np.linalg.norm(a)).max() < 1e-5
    sig = np.linalg.norm(ap, axis=1)
    assert np.allclose(sig, sv / np.linalg.norm(sv), rtol=2e-2, atol=2e-6)


@pytest.mark.parametrize("m,n,target", SHAPES)
@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_tsvd_backward_matches_the_oracle(m, n, target, prec, ws32, ws64):
    ws = ws32 if prec == "c64" else ws64
    rng = np.random.default_rng(7 + m * 31 + n)
    a = _rand(rng, m, n)
    c = min(m, n)
    m1, w1, w2 = _rand(rng, m, n), rng.random((m, c)), rng.random((c, n))
    r = o_tsvd(a, target, 0, 1e-6)
    gq, gp = _cot(r["Aq"], r["Ap"], m1, w1, w2)
    want = o_backward(r["U"], r["S"], r["V"], r["k"], gq, gp)
    ta = torch.from_numpy(a).to(ws.dtype).cuda().requires_grad_(True)
    aq, ap, info = AD.tsvd(ws, ta, target)
    assert info["k"] == r["k"]
    tq, tp = _cot(aq.detach().cpu().numpy().astype(np.complex128), ap.detach().cpu().numpy().astype(np.complex128),
                  m1, w1, w2)
    torch.autograd.backward([aq, ap], [torch.from_numpy(tq).to(ws.dtype).cuda(), torch.from_numpy(tp).to(ws.dtype).cuda()])
    got = ta.grad.cpu().numpy().astype(np.complex128)
    rel = np.linalg.norm(got - want) / np.linalg.norm(want)
    # a rounding error e in the factors reaches the adjoint through 1/(s_j^2 - s_i^2): the bound is
    # a small multiple of e * s_0^2 / (the smallest gap coupled to a kept value)
    unit = 1.2e-7 if prec == "c64" else 2.2e-16
    assert rel < max(1e-5 if prec == "c64" else 1e-12, 20 * unit * _adjoint_condition(r["S"], r["k"])), rel


def test_tsvd_gradcheck_on_phase_invariant_outputs(ws64):
    """torch's own finite differences (FP64 handle) on outputs that do not depend on the phases of
    the singular vectors: A_q A_p, |A_q|^2, |A_p|^2 and the projector A_q A_q^H."""
    rng = np.random.default_rng(11)
    a = torch.from_numpy(_rand(rng, 7, 5)).cuda().requires_grad_(True)

    def f(x):
        aq, ap, _ = AD.tsvd(ws64, x, 1.0, 3)
        return aq @ ap, aq.abs() ** 2, ap.abs() ** 2, aq @ aq.mH

    assert torch.autograd.gradcheck(f, (a,), eps=1e-6, atol=1e-6, rtol=1e-5)


def test_gemm_gradcheck(ws64):
    rng = np.random.default_rng(12)
    a = torch.from_numpy(_rand(rng, 5, 7)).cuda().requires_grad_(True)
    b = torch.from_numpy(_rand(rng, 7, 3)).cuda().requires_grad_(True)
    assert torch.autograd.gradcheck(lambda x, y: AD.gemm(ws64, x, y), (a, b), eps=1e-6, atol=1e-7, rtol=1e-6)


def test_untruncated_gradient_is_the_exact_parameter_shift_gradient():
    n, layers = 10, 2
    p = W.ansatz_params(n, layers, 21)
    e, g, info = AD.energy_and_grad_ad(n, layers, p, chi_max=64)

    def e_exact(pp):
        c = W.ansatz_circuit(n, layers, pp)
        return zz_energy_dense(SV.run_circuit(n, c.gates()), n)

    assert abs(e - e_exact(p)) < 1e-5
    ps = np.zeros_like(p)
    for j in range(p.size):
        sh = np.zeros_like(p)
        sh[j] = math.pi / 2
        ps[j] = 0.5 * (e_exact(p + sh) - e_exact(p - sh))
    assert np.abs(g - ps).max() < 1e-4, np.abs(g - ps).max()
    assert abs(info["fidelity"] - 1.0) < 1e-12


@pytest.mark.parametrize("prec,tol", [(E.TF32X3, 2e-3), (E.FP64, 1e-7)])
def test_truncated_gradient_matches_oracle_finite_differences(prec, tol):
    """With a cut, the simulated energy is a smooth function of the angles between changes of k;
    its derivative with every k frozen (FP64 oracle, central differences) is what reverse mode
    computes."""
    n, layers, f_min = 10, 3, 0.9
    p = W.ansatz_params(n, layers, 22)
    e, g, info = AD.energy_and_grad_ad(n, layers, p, f_min=f_min, chi_max=64, precision=prec)

    rank_tol = 1e-6 if prec == E.TF32X3 else 1e-12

    def chain(pp, k_fixed=None):
        c = W.ansatz_circuit(n, layers, pp)
        ch = DiffChain(n, f_min=f_min, n_2q=c.n_2q, rank_tol=rank_tol, k_fixed=k_fixed)
        for q, u in c.gates():
            ch.apply_2q(q, u)
        return ch.energy_zz(), ch

    e0, ch0 = chain(p)
    assert ch0.k_log == info["k_log"]
    assert ch0.product < 0.999   # the run truncated
    assert abs(e - e0) < (1e-4 if prec == E.TF32X3 else 1e-10)
    h = 1e-5
    fd = np.zeros_like(p)
    for j in range(p.size):
        d = np.zeros_like(p)
        d[j] = h
        fd[j] = (chain(p + d, ch0.k_log)[0] - chain(p - d, ch0.k_log)[0]) / (2 * h)
    assert np.abs(g - fd).max() < tol * max(1.0, np.abs(fd).max()), np.abs(g - fd).max()


def test_autodiff_gradient_agrees_with_the_batched_parameter_shift():
    """The two gradient routes of the library on the same untruncated circuit."""
    from paper_2307_16870_gb300 import grad as G
    n, layers = 12, 2
    p = W.ansatz_params(n, layers, 23)
    e_ad, g_ad, _ = AD.energy_and_grad_ad(n, layers, p, chi_max=64)
    fn = lambda ang: W.ansatz_circuit(n, layers, ang)   # noqa: E731
    e_ps, g_ps, _ = G.energy_and_grad(fn, n, p, concurrency=8)
    assert abs(e_ad - e_ps) < 1e-5
    assert np.abs(g_ad - g_ps).max() < 1e-4


def test_per_layer_checkpointing_recomputes_and_gives_the_same_gradient():
    n, layers, f_min = 10, 3, 0.9
    p = W.ansatz_params(n, layers, 24)
    e0, g0, i0 = AD.energy_and_grad_ad(n, layers, p, f_min=f_min, chi_max=64)
    e1, g1, i1 = AD.energy_and_grad_ad(n, layers, p, f_min=f_min, chi_max=64, checkpoint=True)
    assert i1["k_log"] == i0["k_log"]
    assert i1["bond_dims"] == i0["bond_dims"]           # the live state survives the recomputation
    assert i0["tsvd_calls"] == len(i0["k_log"])
    assert i1["tsvd_calls"] > len(i1["k_log"])          # the layers ran again in the backward
    assert abs(e1 - e0) < 1e-12
    assert np.abs(g1 - g0).max() < 1e-6 * max(1.0, np.abs(g0).max())


def test_stateless_calls_refuse_bad_arguments(ws32):
    h = ws32.h
    a = torch.zeros((8, 8), dtype=torch.complex64, device="cuda")
    u = torch.zeros((8, 8), dtype=torch.complex64, device="cuda")
    s = torch.zeros(8, dtype=torch.float64, device="cuda")
    big = torch.zeros((4096, 4), dtype=torch.complex64, device="cuda")
    p = a.data_ptr()
    with pytest.raises(E.MpsError):      # rows beyond the handle's scratch
        E.mps_tsvd_device(h, 4096, 4, big.data_ptr(), 4, 1.0, 0, 0.0, p, s.data_ptr(), p, p, p)
    with pytest.raises(E.MpsError):      # negative target
        E.mps_tsvd_device(h, 8, 8, p, 8, -0.5, 0, 0.0, u.data_ptr(), s.data_ptr(), p, p, p)
    with pytest.raises(E.MpsError):      # lda < n
        E.mps_tsvd_device(h, 8, 8, p, 4, 1.0, 0, 0.0, u.data_ptr(), s.data_ptr(), p, p, p)
    with pytest.raises(E.MpsError):      # k above min(m, n)
        E.mps_tsvd_backward_device(h, 8, 4, 5, p, s.data_ptr(), p, 0, 0, 0.0, p)
    with pytest.raises(E.MpsError):      # K = 0
        E.mps_gemm_device(h, 4, 4, 0, p, 1, 1, 0, p, 1, 1, 0, p, 4, 1)
    # the handle still works after the refusals
    rng = np.random.default_rng(5)
    x = torch.from_numpy(_rand(rng, 8, 6)).to(torch.complex64).cuda()
    aq, ap, info = AD.tsvd(ws32, x, 1.0)
    assert info["k"] == 6


def test_tsvd_of_the_zero_matrix_is_refused():
    ws = AD.Workspace(8, 16, E.TF32X3)
    try:
        a = torch.zeros((8, 8), dtype=torch.complex64, device="cuda")
        u = torch.zeros((8, 8), dtype=torch.complex64, device="cuda")
        s = torch.zeros(8, dtype=torch.float64, device="cuda")
        with pytest.raises(E.MpsError):      # W_k = 0: no direction to keep
            E.mps_tsvd_device(ws.h, 8, 8, a.data_ptr(), 8, 1.0, 0, 0.0, u.data_ptr(), s.data_ptr(), u.data_ptr(),
                              u.data_ptr(), u.data_ptr())
    finally:
        ws.close()
