"""The paper's gate fusion (Sec. II-C, Fig. 4): four strategies on gates of at most two qubits,
in their priority order (one-qubit + one-qubit; one-qubit into the following, then into the
preceding two-qubit gate; two-qubit + two-qubit on the same pair).

Host-side only: the fused list is read back and applied with the FP64 oracle, against the
unfused list applied the same way."""
import numpy as np
import pytest

import synth
from oracle import core as ocore


@pytest.fixture(scope="module")
def qs():
    from paper_2402_08136_gb300 import build
    build.build()
    import paper_2402_08136_gb300 as q
    return q


def apply_list(psi, gates):
    for g in gates:
        assert g["kind"] == 0
        ocore.apply_gate(psi, g["targets"], g["U"], g["controls"])
    return psi


def random_circuit(qs, rng, n, count):
    c = qs.Circuit(n)
    for _ in range(count):
        r = rng.random()
        q = [int(x) for x in rng.permutation(n)]
        if r < 0.45:
            c.add_gate([q[0]], synth.haar_unitary(rng, 2))
        elif r < 0.75:
            c.add_gate(q[:2], synth.haar_unitary(rng, 4))
        elif r < 0.9:
            c.add_gate([q[0]], synth.haar_unitary(rng, 2), [q[1]])  # controlled one-qubit gate
        else:
            c.add_gate(q[:3], synth.haar_unitary(rng, 8))  # not mergeable: stays in place
    return c


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_paper_fusion_preserves_the_circuit(qs, seed):
    rng = np.random.default_rng(seed)
    n = 6
    c = random_circuit(qs, rng, n, 80)
    f = qs.qsim_fuse_paper(c)
    g0, g1 = qs.qsim_circuit_gates(c), qs.qsim_circuit_gates(f)
    assert len(g1) < len(g0)
    assert all(len(g["targets"]) + len(g["controls"]) <= 3 for g in g1)
    psi = synth.gaussian_state_np(seed, n)
    a = apply_list(psi.copy(), g0)
    b = apply_list(psi.copy(), g1)
    assert np.max(np.abs(a - b)) <= 1e-12


def test_paper_fusion_is_a_fixed_point(qs):
    """After the four passes no strategy applies any more: fusing the result (rebuilt as an
    unfused list) changes nothing."""
    rng = np.random.default_rng(9)
    n = 5
    f = qs.qsim_fuse_paper(random_circuit(qs, rng, n, 60))
    g1 = qs.qsim_circuit_gates(f)
    c2 = qs.Circuit(n)
    for g in g1:
        c2.add_gate(g["targets"], g["U"], g["controls"])
    g2 = qs.qsim_circuit_gates(qs.qsim_fuse_paper(c2))
    assert len(g2) == len(g1)


def test_one_qubit_gates_merge_before_joining_two_qubit_gates(qs):
    """Strategy 1 comes first: two one-qubit gates on qubit 0 around nothing else become one
    gate, which then joins the following two-qubit gate (strategy 2): a single gate equal to
    B (u2 u1 (x) I)."""
    rng = np.random.default_rng(4)
    u1, u2, B = synth.haar_unitary(rng, 2), synth.haar_unitary(rng, 2), synth.haar_unitary(rng, 4)
    c = qs.Circuit(2)
    c.add_gate([0], u1)
    c.add_gate([0], u2)
    c.add_gate([0, 1], B)
    g = qs.qsim_circuit_gates(qs.qsim_fuse_paper(c))
    assert len(g) == 1 and g[0]["targets"] == [0, 1]
    expect = B @ np.kron(np.eye(2), u2 @ u1)  # bit 0 of the index <-> qubit 0
    assert np.max(np.abs(g[0]["U"] - expect)) <= 1e-13


def test_following_two_qubit_gate_takes_priority_over_preceding_one(qs):
    """a (qubit 1), B (0, 1), c (qubit 1), D (1, 2): strategy 2 puts a into B and c into D before
    strategy 3 could put c into B; the greedy circuit-order fusion puts c into B instead."""
    rng = np.random.default_rng(5)
    a, cc = synth.haar_unitary(rng, 2), synth.haar_unitary(rng, 2)
    B, D = synth.haar_unitary(rng, 4), synth.haar_unitary(rng, 4)
    c = qs.Circuit(3)
    c.add_gate([1], a)
    c.add_gate([0, 1], B)
    c.add_gate([1], cc)
    c.add_gate([1, 2], D)
    g = qs.qsim_circuit_gates(qs.qsim_fuse_paper(c))
    assert [x["targets"] for x in g] == [[0, 1], [1, 2]]
    assert np.max(np.abs(g[0]["U"] - B @ np.kron(a, np.eye(2)))) <= 1e-13       # qubit 1 = bit 1
    assert np.max(np.abs(g[1]["U"] - D @ np.kron(np.eye(2), cc))) <= 1e-13      # qubit 1 = bit 0
    greedy = qs.qsim_circuit_gates(qs.qsim_fuse(c, 2))
    assert len(greedy) == 2
    assert np.max(np.abs(greedy[1]["U"] - D)) <= 1e-13


def test_controlled_gate_joins_as_a_two_qubit_gate(qs):
    """A one-qubit gate next to a controlled one-qubit gate on the same qubit merges into its
    dense 4 x 4 form; two-qubit gates on the same pair in either qubit order merge (strategy 4)."""
    rng = np.random.default_rng(6)
    u, v = synth.haar_unitary(rng, 2), synth.haar_unitary(rng, 2)
    W = synth.haar_unitary(rng, 4)
    c = qs.Circuit(2)
    c.add_gate([0], u, [1])  # controlled-u, control qubit 1
    c.add_gate([0], v)
    c.add_gate([1, 0], W)
    g = qs.qsim_circuit_gates(qs.qsim_fuse_paper(c))
    assert len(g) == 1 and not g[0]["controls"]
    psi = synth.gaussian_state_np(7, 2)
    a = apply_list(psi.copy(), qs.qsim_circuit_gates(c))
    b = apply_list(psi.copy(), g)
    assert np.max(np.abs(a - b)) <= 1e-13


def test_gate_level_hhl_keeps_its_structured_steps(qs):
    """The paper's gate-level HHL circuit (4 x 4 system, 4 clock qubits) under the paper's
    fusion: fewer gates; the operations it does not merge (the eigenvalue inversion and the
    multi-qubit controlled evolutions) are all still there, in order."""
    p = synth.hhl7_problem()
    h = qs.hhl_build(p["A"], p["b"], p["m"])
    c = h.as_circuit()
    g0 = qs.qsim_circuit_gates(c)
    g1 = qs.qsim_circuit_gates(qs.qsim_fuse_paper(c))
    assert len(g1) < len(g0)
    big = lambda gs: [(g["kind"], g["targets"], g["controls"]) for g in gs
                      if g["kind"] != 0 or len(g["targets"]) + len(g["controls"]) > 2]
    assert big(g1) == big(g0)
