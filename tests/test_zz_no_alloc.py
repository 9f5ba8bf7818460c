"""The allocation-free tensor-core GEMM entry point, called through the C ABI.

Callers that manage every device allocation themselves (or must not trigger
the device synchronisation of cudaFree) use mps_cgemm_c64_noalloc, whose
workspace is a fixed array inside the library.  Its results must equal those
of the allocating entry point mps_cgemm_c64 on the same inputs, on two calls
in a row (the array keeps the previous call's contents)."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
E = pytest.importorskip("paper_2307_16870_gb300")


def _operands(M, N, K, seed):
    g = torch.Generator().manual_seed(seed)
    a = torch.complex(torch.randn(M, K, generator=g), torch.randn(M, K, generator=g)).to(torch.complex64)
    b = torch.complex(torch.randn(K, N, generator=g), torch.randn(K, N, generator=g)).to(torch.complex64)
    return a.cuda(), b.cuda()


def _pair(M, N, K, seed, conj_b=False):
    a, b = _operands(M, N, K, seed)
    c_ref = torch.zeros(M, N, dtype=torch.complex64, device="cuda")
    c_new = torch.full((M, N), complex(3.0, -3.0), dtype=torch.complex64, device="cuda")
    E.mps_cgemm_c64(E.TF32X3, M, N, K, 0.5, a.data_ptr(), K, 1, False, b.data_ptr(), N, 1, conj_b,
                    c_ref.data_ptr(), N, 1)
    E.mps_cgemm_c64_noalloc(M, N, K, 0.5, a.data_ptr(), K, 1, False, b.data_ptr(), N, 1, conj_b,
                            c_new.data_ptr(), N, 1)
    torch.cuda.synchronize()
    # same tolerance as the GEMM tests: relative to |row of A| |column of B|
    scale = 0.5 * (a.abs().pow(2).sum(1, keepdim=True).sqrt() @ b.abs().pow(2).sum(0, keepdim=True).sqrt())
    return ((c_new - c_ref).abs() / scale).max().item()


def test_noalloc_matches_allocating_entry_point_twice():
    # two calls in a row with different shapes: the second must not see the first one's contents
    assert _pair(300, 160, 200, 1) < 2e-6
    assert _pair(129, 257, 64, 2, conj_b=True) < 2e-6


def test_noalloc_rejects_oversized_shapes():
    a, b = _operands(8, 8, 8, 3)
    c = torch.zeros(8, 8, dtype=torch.complex64, device="cuda")
    with pytest.raises(E.MpsError) as ei:
        # 2K padded = 4096 floats per row: M * 4096 > 524288 for M = 200
        E.mps_cgemm_c64_noalloc(200, 8, 2048, 1.0, a.data_ptr(), 0, 0, False, b.data_ptr(), 0, 0, False,
                                c.data_ptr(), 8, 1)
    assert ei.value.code == 1
