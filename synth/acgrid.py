"""Synthetic AC power-flow cases (stand-ins for the paper's MATPOWER IEEE cases, Sec. IV).

Recipe: a random connected grid (spanning tree plus extra lines, average degree 3); per line a
series reactance x ~ U[0.05, 0.25] p.u., resistance r = x / U[3, 10], line charging
b_sh ~ U[0, 0.05] p.u.; bus 0 is the slack (|V| = 1.02, angle 0); about a fifth of the other
buses are PV generators (P ~ U[0.2, 0.6] p.u., |V| ~ U[0.98, 1.04]); the rest are PQ loads
(P ~ -U[0.05, 0.3] p.u., Q ~ -U[0.0, 0.15] p.u., net injections, negative = consumption).
Only data is produced here; the power-flow equations live with the solver.
"""
from __future__ import annotations

import numpy as np

from .grids import random_connected_graph


def ac_case(seed: int, B: int, avg_degree: float = 3.0):
    rng = np.random.default_rng(seed)
    edges = random_connected_graph(rng, B, n_edges=int(np.ceil(B * avg_degree / 2)))
    L = len(edges)
    x = rng.uniform(0.05, 0.25, size=L)
    r = x / rng.uniform(3.0, 10.0, size=L)
    bsh = rng.uniform(0.0, 0.05, size=L)
    kind = np.full(B, "PQ", dtype=object)
    kind[0] = "slack"
    others = np.arange(1, B)
    npv = max(1, (B - 1) // 5)
    kind[rng.choice(others, size=npv, replace=False)] = "PV"
    P = np.zeros(B)
    Q = np.zeros(B)
    Vset = np.ones(B)
    Vset[0] = 1.02
    for i in range(1, B):
        if kind[i] == "PV":
            P[i] = rng.uniform(0.2, 0.6)
            Vset[i] = rng.uniform(0.98, 1.04)
        else:
            P[i] = -rng.uniform(0.05, 0.3)
            Q[i] = -rng.uniform(0.0, 0.15)
    return dict(B=B, edges=edges, r=r, x=x, bsh=bsh, kind=list(kind), P=P, Q=Q, Vset=Vset)
