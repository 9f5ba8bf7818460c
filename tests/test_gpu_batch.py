"""Batched runs of independent circuits (mps_batch_run): every circuit's results are
those of running it alone, whatever the concurrency, and agree with the oracle."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
E = pytest.importorskip("paper_2307_16870_gb300")

import workloads as W  # noqa: E402
from oracle import textbook_mps as T  # noqa: E402


def _upload(circ):
    ops = circ.ops_array()
    return torch.from_numpy(ops.view(np.float64).reshape(len(circ.qs), -1).copy()).cuda()


def _specs():
    # small circuits (single-CTA Jacobi) and mid-size ones (cluster and point-to-point kernels)
    return [(8, 6, 0.99, 0), (10, 8, 0.99, 0), (12, 8, 0.95, 0), (9, 5, 0.999, 0),
            (20, 16, 0.99, 128), (22, 14, 0.9, 96), (18, 18, 0.99, 128), (24, 12, 0.95, 64)]


def _single(circ, ops_dev, f_min, cap):
    m = E.MPS(circ.n_qubits, f_min=f_min, n_2q=circ.n_2q, chi_max=cap, log_truncations=False)
    E.mps_apply_circuit_device(m.h, circ.qs, ops_dev.data_ptr(), 4)
    return m


def _sites(m):
    return [m.site(i) for i in range(m.n)]


@pytest.fixture(scope="module")
def batch_inputs():
    circs, devs = [], []
    for i, (n, d, f, cap) in enumerate(_specs()):
        c = W.brickwork_circuit(n, d, 4000 + i)
        circs.append(c)
        devs.append(_upload(c))
    return circs, devs


def _items(circs, devs):
    out = []
    for c, dv, (n, d, f, cap) in zip(circs, devs, _specs()):
        out.append({"n_qubits": n, "qs": c.qs, "ops_dev": dv.data_ptr(), "op_dim": 4, "f_min": f,
                    "n_2q": c.n_2q, "chi_max": cap, "precision": E.TF32X3})
    return out


@pytest.mark.parametrize("concurrency", [1, 4])
def test_batch_equals_single_runs(batch_inputs, concurrency):
    circs, devs = batch_inputs
    code, res = E.mps_batch_run(_items(circs, devs), concurrency=concurrency, keep=True)
    assert code in (E.OK, E.WARN_CHI_CAP)
    for c, dv, r, (n, d, f, cap) in zip(circs, devs, res, _specs()):
        assert r["status"] in (E.OK, E.WARN_CHI_CAP)
        m = _single(c, dv, f, cap)
        b = r["mps"]
        assert r["fidelity"] == m.fidelity()
        assert b.bond_dims() == m.bond_dims()
        assert r["max_bond"] == max(m.bond_dims())
        assert b.centre() == m.centre()
        for x, y in zip(_sites(b), _sites(m)):
            assert np.array_equal(x, y)
        b.close()
        m.close()


def test_batch_against_oracle(batch_inputs):
    circs, devs = batch_inputs
    code, res = E.mps_batch_run(_items(circs, devs)[:4], concurrency=4, keep=True)
    assert code == E.OK
    for c, r, (n, d, f, cap) in zip(circs[:4], res, _specs()[:4]):
        o = T.TextbookMPS(n, f_min=f, n_2q=c.n_2q)
        for q, u in c.gates():
            o.apply_2q(q, u)
        assert abs(r["fidelity"] - o.product) < 1e-4
        assert r["mps"].bond_dims() == o.bond_dims()
        r["mps"].close()


def test_batch_reports_a_bad_item_and_runs_the_rest(batch_inputs):
    circs, devs = batch_inputs
    items = _items(circs, devs)[:3]
    items[1] = dict(items[1], n_qubits=1)      # invalid chain length
    code, res = E.mps_batch_run(items, concurrency=2)
    assert code == 1
    assert res[1]["status"] == 1
    assert res[0]["status"] == E.OK and res[2]["status"] == E.OK
    assert res[0]["fidelity"] > 0.99 and res[2]["fidelity"] > 0.95
