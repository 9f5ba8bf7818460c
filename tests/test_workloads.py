"""Seeded input generators: determinism, unitarity, distribution sanity."""
import json
import os

import numpy as np

import workloads as W

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))


def _splitmix_scalar(seed, i):
    # SplitMix64 as a sequential generator: state advances by gamma, then the finaliser.
    mask = (1 << 64) - 1
    state = (seed + (i + 1) * 0x9E3779B97F4A7C15) & mask
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
    return z ^ (z >> 31)


def test_splitmix_vectorised_matches_sequential():
    seed = 0x1234ABCD
    v = W.splitmix64(seed, np.arange(50, dtype=np.uint64))
    for i in range(50):
        assert int(v[i]) == _splitmix_scalar(seed, i)


def test_normals_moments():
    x = W.normals(7, 0, 200000)
    assert abs(x.mean()) < 0.01
    assert abs(x.var() - 1.0) < 0.01
    assert np.all(np.isfinite(x))


def test_haar_unitary_is_special_unitary():
    for i in range(20):
        u = W.haar_unitary(4, 11, i)
        assert np.abs(u.conj().T @ u - np.eye(4)).max() < 1e-13
        assert abs(np.linalg.det(u) - 1.0) < 1e-12


def test_haar_second_moment():
    g = GOLDEN["haar_second_moment"]
    us = np.stack([W.haar_unitary(g["d"], 3, i) for i in range(3000)])
    m = (np.abs(us) ** 2).mean(axis=0)
    assert np.abs(m - g["mean_abs2"]).max() < 0.02


def test_haar_deterministic_and_order_free():
    a = W.brickwork_circuit(8, 4, 99)
    b = W.brickwork_circuit(8, 4, 99)
    assert all(np.array_equal(x, y) for x, y in zip(a.ops, b.ops))
    assert np.array_equal(a.ops[5], W.haar_unitary(4, 99, 5))


def test_brickwork_counts_and_layout():
    for case in GOLDEN["brickwork_gate_counts"]["cases"]:
        pairs = W.brickwork_pairs(case["N"], case["D"])
        assert len(pairs) == case["n"] == W.count_brickwork_gates(case["N"], case["D"])
        f0 = case["f_min"] ** (1.0 / case["n"])
        assert abs((1 - f0) - case["one_minus_f0"]) < 1e-8
    pairs = W.brickwork_pairs(6, 3)
    assert pairs == [(0, 0), (0, 2), (0, 4), (1, 3), (1, 1), (2, 0), (2, 2), (2, 4)]


def test_noise_kraus_complete():
    for ks, dim in ((W.depolarizing_2q_kraus(0.01), 4), (W.amplitude_damping_kraus(0.3), 2)):
        acc = sum(k.conj().T @ k for k in ks)
        assert np.abs(acc - np.eye(dim)).max() < 1e-14


def test_batch_specs_ranges():
    specs = W.random_batch_specs(64, 5)
    assert len(specs) == 64
    assert all(20 <= s["n_qubits"] <= 80 and 10 <= s["depth"] <= 30 for s in specs)
    assert {s["f_min"] for s in specs} <= {0.9, 0.99}
