"""The complex64 contraction kernels (tcgen05 3xTF32 and CUDA-core FP32) against complex128 products."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
E = pytest.importorskip("paper_2307_16870_gb300")

SHAPES = [(1, 1, 1), (5, 3, 7), (64, 64, 64), (128, 128, 128), (130, 70, 33), (257, 129, 200),
          (512, 1024, 256), (1000, 300, 17), (64, 640, 512), (7, 1030, 129)]


def _rand(shape, seed):
    g = torch.Generator().manual_seed(seed)
    re = torch.randn(shape, generator=g, dtype=torch.float64)
    im = torch.randn(shape, generator=g, dtype=torch.float64)
    return torch.complex(re, im)


def _run(prec, M, N, K, layout_a, layout_b, conj_a, conj_b, seed):
    dev = torch.device("cuda")
    # storage of A: row-major (M x K) or column-major (K x M stored); same for B
    a64 = _rand((M, K), seed)
    b64 = _rand((K, N), seed + 1)
    if layout_a == "row":
        a_store = a64.clone()
        a_rs, a_cs = K, 1
    else:
        a_store = a64.t().contiguous()
        a_rs, a_cs = 1, M
    if layout_b == "row":
        b_store = b64.clone()
        b_rs, b_cs = N, 1
    else:
        b_store = b64.t().contiguous()
        b_rs, b_cs = 1, K
    # op(A) = conj(stored) when conj_a: the operand the kernel sees is conj(a64)
    a_dev = (a_store.conj() if conj_a else a_store).resolve_conj().to(torch.complex64).to(dev)
    b_dev = (b_store.conj() if conj_b else b_store).resolve_conj().to(torch.complex64).to(dev)
    c_dev = torch.full((M, N), complex(7.0, 7.0), dtype=torch.complex64, device=dev)
    alpha = 0.75
    E.mps_cgemm_c64(prec, M, N, K, alpha, a_dev.data_ptr(), a_rs, a_cs, conj_a, b_dev.data_ptr(), b_rs, b_cs,
                    conj_b, c_dev.data_ptr(), N, 1)
    # reference from the complex64-rounded inputs, in complex128
    a_in = a_dev.cpu().to(torch.complex128)
    b_in = b_dev.cpu().to(torch.complex128)
    a_op = (a_in.conj() if conj_a else a_in)
    b_op = (b_in.conj() if conj_b else b_in)
    a_mat = a_op if layout_a == "row" else a_op.t()
    b_mat = b_op if layout_b == "row" else b_op.t()
    ref = alpha * (a_mat @ b_mat)
    got = c_dev.cpu().to(torch.complex128)
    scale = (a_mat.abs() ** 2).sum(1, keepdim=True).sqrt() @ (b_mat.abs() ** 2).sum(0, keepdim=True).sqrt()
    err = ((got - ref).abs() / (alpha * scale + 1e-30)).max().item()
    return err


@pytest.mark.parametrize("M,N,K", SHAPES)
@pytest.mark.parametrize("prec_name", ["tf32x3", "fp32"])
def test_cgemm_shapes(M, N, K, prec_name):
    prec = E.TF32X3 if prec_name == "tf32x3" else E.FP32
    err = _run(prec, M, N, K, "row", "row", False, False, M * 7 + N)
    # FP32-level accuracy: relative to |row of A| |column of B|
    assert err < 2e-6, err


@pytest.mark.parametrize("la,lb,ca,cb", [("col", "row", True, False), ("row", "col", False, True),
                                          ("col", "col", True, True), ("row", "row", True, False)])
def test_cgemm_layouts_and_conjugation(la, lb, ca, cb):
    for prec in (E.TF32X3, E.FP32):
        err = _run(prec, 200, 96, 160, la, lb, ca, cb, 11)
        assert err < 2e-6, (la, lb, ca, cb, prec, err)


def test_tf32x3_is_more_accurate_than_one_tf32_product():
    """3xTF32 must beat a single TF32 product (~1e-3 relative) by orders of magnitude."""
    err = _run(E.TF32X3, 256, 256, 512, "row", "row", False, False, 3)
    assert err < 2e-6
