"""Seeded input generators: determinism, the host/device implementations of the counter-based
state generator agree, and the workload recipes have the stated shapes."""
import numpy as np
import torch

import synth


def test_counter_state_numpy_vs_torch_cpu():
    n = 12
    a = synth.gaussian_state_np(7, n)
    b = synth.gaussian_state_torch(7, n, torch.complex128, "cpu", chunk=1000).numpy()
    assert np.array_equal(a, b) or np.max(np.abs(a - b)) < 1e-15
    idx = np.array([0, 5, 4095, 1234])
    assert np.max(np.abs(synth.gaussian_amplitudes_at(7, n, idx) - a[idx])) == 0.0
    assert abs(np.vdot(a, a).real - 1.0) < 0.1


def test_generators_are_deterministic():
    p1, p2 = synth.hhl7_problem(1), synth.hhl7_problem(1)
    assert np.array_equal(p1["A"], p2["A"]) and np.array_equal(p1["b"], p2["b"])
    g1 = synth.gate_microbench_list(3, 20, ks=(1, 3), per_k=4)
    g2 = synth.gate_microbench_list(3, 20, ks=(1, 3), per_k=4)
    assert all(t1 == t2 and np.array_equal(u1, u2) for (t1, u1), (t2, u2) in zip(g1, g2))


def test_workload_shapes():
    p = synth.hhl7_problem()
    assert p["A"].shape == (4, 4) and p["m"] == 4
    w = np.linalg.eigvalsh(p["A"])
    assert np.max(np.abs(w - np.round(w))) < 1e-12 and w[-1] == 15.0 or abs(w[-1] - 15) < 1e-12
    q = synth.hhl27_problem()
    assert q["A"].shape == (64, 64) and q["m"] == 20
    assert np.all(np.linalg.eigvalsh(q["A"]) > 0)
    bp = synth.batched_problems(count=16)
    for x in bp:
        assert 2 <= x["nb"] <= 5 and 4 <= x["m"] <= 10
        assert x["A"].shape == (2 ** x["nb"], 2 ** x["nb"])
        assert np.all(np.linalg.eigvalsh(x["A"]) > 0)
    s = synth.serving_stream(count=50)
    for r in s:
        pr = r["problem"]
        assert r["n"] == pr["nb"] + pr["m"] + 1 and 8 <= r["n"] <= 30 and 2 <= pr["nb"] <= 7
    assert all(s[i]["arrival"] < s[i + 1]["arrival"] for i in range(len(s) - 1))


def test_grid_edges():
    rng = np.random.default_rng(0)
    edges = synth.random_connected_graph(rng, 65, n_edges=98)
    assert len(edges) == 98 and len(set(edges)) == 98
    A, b, _ = synth.grid_system(np.random.default_rng(1), 65)
    assert np.allclose(A, A.T)
