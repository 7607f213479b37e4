"""Haar-random gate matrices on random distinct target qubits (gate-apply microbenchmark inputs)."""
from __future__ import annotations

import numpy as np


def haar_unitary(rng: np.random.Generator, d: int) -> np.ndarray:
    """d x d Haar-distributed unitary (complex128, row-major).

    Mezzadri, "How to generate random matrices from the classical compact groups" (2007):
    QR of a complex Ginibre matrix, then multiply column j of Q by the phase of R[j, j] so that
    the distribution is exactly Haar.
    """
    Z = (rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))) / np.sqrt(2.0)
    Q, R = np.linalg.qr(Z)
    diag = np.diagonal(R)
    phase = diag / np.abs(diag)
    return np.ascontiguousarray(Q * phase[None, :])


def random_targets(rng: np.random.Generator, n: int, k: int) -> list[int]:
    """k distinct qubits drawn uniformly from 0..n-1, in draw order (order matters: target b of
    the list is bit b of the gate matrix's row/column index)."""
    return [int(q) for q in rng.choice(n, size=k, replace=False)]


def gate_microbench_list(seed: int, n: int, ks=(1, 2, 3, 4, 5, 6), per_k: int = 200):
    """Gate list of the dense-gate microbenchmark: ``per_k`` Haar 2^k x 2^k unitaries for each
    k in ``ks`` (grouped by k, in increasing k), each on k uniformly random distinct targets.

    Returns a list of ``(targets, U)`` with U complex128 of shape (2^k, 2^k).
    """
    rng = np.random.default_rng(seed)
    out = []
    for k in ks:
        for _ in range(per_k):
            t = random_targets(rng, n, k)
            out.append((t, haar_unitary(rng, 2 ** k)))
    return out
