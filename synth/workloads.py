"""The HHL workloads as seeded problem descriptions (matrices, right-hand sides, register sizes).

Each function returns plain data: ``dict(A=..., b=..., m=..., t=..., C=...)`` where ``t`` and
``C`` equal 0.0 when the solver's automatic choice is wanted.  Nothing here runs the method.

  * 7-qubit plain HHL: a random connected 5-bus grid (tree plus each other pair with
    probability 1/2), 4x4 reduced Laplacian with its spectrum snapped onto the 4-qubit clock grid
    (eigenvalues integers in 1..15, evolution time 2*pi/16), 4 clock qubits, 1 ancilla.
  * 27-qubit precision form: random 65-bus grid, average degree 3 (98 lines), 64x64 reduced
    Laplacian, 20 clock qubits, 1 ancilla; t and C automatic (off-grid).
  * batched: 512 N-1 contingencies, data qubits nb ~ U{2..5} on a (2^nb + 1)-bus grid of average
    degree 3 with one line removed (kept connected), clock qubits m ~ U{4..10}.
  * serving: Poisson arrivals; total qubits n = floor(exp(U[ln 8, ln 31))), nb uniform over
    {max(2, n-23) .. min(7, n-5)}, m = n - 1 - nb, contingency systems as above.
"""
from __future__ import annotations

import math

import numpy as np

from .grids import contingency_system, grid_system, spectral_snap


def hhl7_problem(seed: int = 1):
    rng = np.random.default_rng(seed)
    m = 4
    A, b, _ = grid_system(rng, 5, avg_degree=None, extra_prob=0.5)
    A = spectral_snap(A, m).astype(np.complex128)
    return dict(A=A, b=b, m=m, t=2 * math.pi / 2 ** m, C=0.0, nb=2)


def hhl27_problem(seed: int = 3):
    rng = np.random.default_rng(seed)
    A, b, _ = grid_system(rng, 65, avg_degree=3.0)
    return dict(A=A, b=b, m=20, t=0.0, C=0.0, nb=6)


def batched_problems(seed: int = 4, count: int = 512, nb_range=(2, 5), m_range=(4, 10)):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        nb = int(rng.integers(nb_range[0], nb_range[1] + 1))
        m = int(rng.integers(m_range[0], m_range[1] + 1))
        A, b = contingency_system(rng, 2 ** nb + 1, avg_degree=3.0)
        out.append(dict(A=A, b=b, m=m, t=0.0, C=0.0, nb=nb))
    return out


def serving_stream(seed: int = 5, count: int = 20000, rate: float = 2000.0,
                   n_range=(8, 30), max_n: int | None = None):
    """Poisson request stream.  Each item: dict(arrival=seconds, n=..., problem=dict(...)).

    ``max_n`` caps the drawn qubit count (for a load the box sustains); requests keep their
    draw order, so a capped stream is a prefix-compatible variant of the full one.
    """
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=count)
    arrivals = np.cumsum(gaps)
    lo, hi = math.log(n_range[0]), math.log(n_range[1] + 1)
    out = []
    for i in range(count):
        n = int(math.floor(math.exp(rng.uniform(lo, hi))))
        n = min(max(n, n_range[0]), n_range[1])
        if max_n is not None:
            n = min(n, max_n)
        nb_lo, nb_hi = max(2, n - 23), min(7, n - 5)
        nb = int(rng.integers(nb_lo, nb_hi + 1))
        m = n - 1 - nb
        A, b = contingency_system(rng, 2 ** nb + 1, avg_degree=3.0)
        out.append(dict(arrival=float(arrivals[i]), n=n,
                        problem=dict(A=A, b=b, m=m, t=0.0, C=0.0, nb=nb)))
    return out
