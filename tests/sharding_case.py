"""A seeded random circuit for the sharding tests, built twice from the same draws: through the
library's public API (for the planner and the GPU path) and as the FP64 oracle's gate list
(applied gate by gate on the host).  Gates: dense 1- to 3-qubit Haar gates (some with
controls), uniformly controlled rotations, Fourier passes with twiddle sources, Walsh-Hadamard
passes."""
import numpy as np

import synth
from oracle import core as ocore
from oracle import hhl as ohhl


def random_case(qs, n, count, seed):
    rng = np.random.default_rng(seed)
    c = qs.Circuit(n)
    gates = []  # ("u", targets, U, controls) | ("ucry", target, controls, theta) | ("dft", field, sign, src, pre) | ("walsh", field)
    for i in range(count):
        kind = i % 6
        if kind in (0, 1, 2):
            k = 1 + (i % 3)
            q = [int(x) for x in rng.permutation(n)[: k + (1 if kind == 2 else 0)]]
            t, ctl = q[:k], q[k:]
            U = synth.haar_unitary(rng, 1 << k)
            c.add_gate(t, U, ctl)
            gates.append(("u", t, U, ctl))
        elif kind == 3:
            q = [int(x) for x in rng.permutation(n)[:3]]
            th = rng.uniform(-3, 3, size=4)
            c.add_ucry(q[0], q[1:], th)
            gates.append(("ucry", q[0], q[1:], th))
        elif kind == 4:
            f0 = int(rng.integers(0, n - 3))
            field = list(range(f0, f0 + 3))
            src = [int(x) for x in rng.permutation([q for q in range(n) if q not in field])[:2]]
            sign = int(rng.choice([-1, 1]))
            pre = bool(rng.integers(0, 2))
            c.add_dft(field, sign, src, twiddle_first=pre)
            gates.append(("dft", field, sign, src, pre))
        else:
            field = [int(x) for x in rng.permutation(n)[:2]]
            c.add_walsh(field)
            gates.append(("walsh", field))
    return c, gates


H = np.array([[1, 1], [1, -1]], dtype=np.complex128) / np.sqrt(2.0)


def apply_oracle_gate(psi, g, perm=None):
    """Apply one oracle gate to psi, its qubits renumbered by perm (logical -> physical)."""
    m = (lambda q: q) if perm is None else (lambda q: perm[q])
    if g[0] == "u":
        ocore.apply_gate(psi, [m(q) for q in g[1]], g[2], [m(q) for q in g[3]], [1] * len(g[3]))
    elif g[0] == "ucry":
        ocore.apply_ucry(psi, m(g[1]), [m(q) for q in g[2]], g[3])
    elif g[0] == "dft":
        ohhl.dft_pass(psi, [m(q) for q in g[1]], g[2], [m(q) for q in g[3]], g[4])
    else:
        for q in g[1]:
            ocore.apply_gate(psi, [m(q)], H)


def permute_qubits(psi, n, perm_from):
    """The vector whose qubit q is qubit perm_from[q] of psi (undo a logical -> physical map)."""
    t = psi.reshape([2] * n)
    # numpy axis a holds bit n-1-a
    axes = [n - 1 - perm_from[n - 1 - a] for a in range(n)]
    return np.ascontiguousarray(np.transpose(t, axes)).reshape(-1)
