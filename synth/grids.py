"""Synthetic reduced DC power-flow matrices (stand-ins for the paper's MATPOWER cases).

Recipe (stated once, used for every HHL workload):
  * a uniformly random labelled spanning tree on B buses, drawn from a random Pruefer sequence;
  * extra distinct random edges until the requested edge count (or, for the 5-bus case, each
    remaining pair with probability 1/2);
  * line susceptance per edge ~ U[5, 20] p.u.;
  * DC B-matrix = weighted graph Laplacian; deleting the slack bus 0 leaves an SPD matrix of
    size (B-1) x (B-1).
"""
from __future__ import annotations

import heapq

import numpy as np


def _pruefer_tree(rng: np.random.Generator, B: int) -> list[tuple[int, int]]:
    """Uniform random labelled tree on B >= 2 vertices via a random Pruefer sequence."""
    if B == 2:
        return [(0, 1)]
    seq = rng.integers(0, B, size=B - 2).tolist()
    degree = [1] * B
    for v in seq:
        degree[v] += 1
    leaves = [u for u in range(B) if degree[u] == 1]
    heapq.heapify(leaves)
    edges = []
    for v in seq:
        leaf = heapq.heappop(leaves)          # smallest current leaf
        edges.append((min(leaf, v), max(leaf, v)))
        degree[leaf] -= 1
        degree[v] -= 1
        if degree[v] == 1:
            heapq.heappush(leaves, v)
    u, w = sorted(leaves)
    edges.append((u, w))
    return edges


def _connected(B: int, edges) -> bool:
    parent = list(range(B))

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    for a, b in edges:
        parent[find(a)] = find(b)
    return len({find(x) for x in range(B)}) == 1


def random_connected_graph(rng: np.random.Generator, B: int, n_edges: int | None = None,
                           extra_prob: float | None = None) -> list[tuple[int, int]]:
    """Random connected simple graph: spanning tree plus extra distinct edges.

    Exactly one of ``n_edges`` (total edge count, clipped to [B-1, B(B-1)/2]) or
    ``extra_prob`` (each non-tree pair independently) selects the extra edges.
    """
    tree = _pruefer_tree(rng, B)
    have = set(tree)
    rest = [(a, b) for a in range(B) for b in range(a + 1, B) if (a, b) not in have]
    if extra_prob is not None:
        extra = [e for e in rest if rng.random() < extra_prob]
    else:
        target = B - 1 if n_edges is None else int(min(max(n_edges, B - 1), B * (B - 1) // 2))
        k = target - (B - 1)
        idx = rng.choice(len(rest), size=k, replace=False) if k > 0 else []
        extra = [rest[i] for i in sorted(idx)]
    return sorted(tree + extra)


def reduced_laplacian(B: int, edges, susceptance) -> np.ndarray:
    """Weighted Laplacian of the line graph with bus 0 (slack) removed: (B-1)x(B-1) SPD."""
    L = np.zeros((B, B))
    for (a, b), s in zip(edges, susceptance):
        L[a, a] += s
        L[b, b] += s
        L[a, b] -= s
        L[b, a] -= s
    return L[1:, 1:].copy()


def random_rhs(rng: np.random.Generator, N: int) -> np.ndarray:
    """Random injections b ~ N(0, 1)^N (complex dtype, zero imaginary part), not normalized."""
    return rng.standard_normal(N).astype(np.complex128)


def grid_system(rng: np.random.Generator, B: int, avg_degree: float | None = 3.0,
                extra_prob: float | None = None):
    """(A, b, edges) for a random connected B-bus grid; A is (B-1)x(B-1) complex128."""
    if extra_prob is not None:
        edges = random_connected_graph(rng, B, extra_prob=extra_prob)
    else:
        edges = random_connected_graph(rng, B, n_edges=int(np.ceil(B * avg_degree / 2)))
    s = rng.uniform(5.0, 20.0, size=len(edges))
    A = reduced_laplacian(B, edges, s).astype(np.complex128)
    b = random_rhs(rng, B - 1)
    return A, b, edges


def contingency_system(rng: np.random.Generator, B: int, avg_degree: float = 3.0):
    """N-1 contingency: a random B-bus grid with one random line removed, kept connected.

    The removed line is resampled until the remaining graph is connected (a grid whose every
    line is a bridge, i.e. a tree, loses no line).
    """
    edges = random_connected_graph(rng, B, n_edges=int(np.ceil(B * avg_degree / 2)))
    s = rng.uniform(5.0, 20.0, size=len(edges))
    order = rng.permutation(len(edges))
    keep = list(range(len(edges)))
    for j in order:
        trial = [e for i, e in enumerate(edges) if i != j]
        if _connected(B, trial):
            keep = [i for i in range(len(edges)) if i != j]
            break
    A = reduced_laplacian(B, [edges[i] for i in keep], s[keep]).astype(np.complex128)
    b = random_rhs(rng, B - 1)
    return A, b


def spectral_snap(A: np.ndarray, m: int) -> np.ndarray:
    """Move the spectrum of a Hermitian positive-definite A onto the integer grid {1..2^m-1}.

    Scale so that the largest eigenvalue becomes 2^m - 1, round every eigenvalue to the nearest
    integer in [1, 2^m - 1] (ties away from zero) and rebuild A = V diag(k) V^H with the same
    eigenvectors.  Repeated eigenvalues are allowed.  This is input construction: it makes a
    matrix whose phases are exactly representable by an m-qubit clock register when the
    evolution time is t = 2*pi / 2^m.
    """
    w, V = np.linalg.eigh(A)
    if w[0] <= 0:
        raise ValueError("spectral_snap needs a positive-definite matrix")
    top = 2 ** m - 1
    k = np.floor(w * (top / w[-1]) + 0.5)
    k = np.clip(k, 1, top)
    out = (V * k) @ V.conj().T
    return 0.5 * (out + out.conj().T)
