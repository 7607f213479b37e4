"""Newton-Raphson AC power flow whose linear solves are HHL circuits run by this library.

The paper's application (Sec. III, "Newton-Raphson based AC power flow"): each Newton step
solves J dx = -F, where F are the active/reactive power mismatches of the non-slack buses and J
the power-flow Jacobian in polar coordinates.  J is not symmetric, so every step runs the HHL
solve of its Hermitian dilation (Sec. III-A step 1(c)), optionally Gauss-Seidel preconditioned
(step 1(a)); the right-hand side and solution scaling follow step 4 of the procedure.  The
power-flow equations themselves (admittance matrix, injections, Jacobian) are host-side numpy:
they are the application around the simulated solver, not the data-parallel path.
"""
from __future__ import annotations

import numpy as np

from . import _binding as qs


def admittance(case):
    """Bus admittance matrix Y = G + iB of the pi-model lines."""
    B = case["B"]
    Y = np.zeros((B, B), dtype=np.complex128)
    for (a, b), r, x, bsh in zip(case["edges"], case["r"], case["x"], case["bsh"]):
        y = 1.0 / complex(r, x)
        Y[a, a] += y + 0.5j * bsh
        Y[b, b] += y + 0.5j * bsh
        Y[a, b] -= y
        Y[b, a] -= y
    return Y


def _index(case):
    kind = case["kind"]
    pv_pq = [i for i in range(case["B"]) if kind[i] != "slack"]
    pq = [i for i in range(case["B"]) if kind[i] == "PQ"]
    return pv_pq, pq


def mismatch(case, Y, Vm, Va):
    """F = [P_calc - P_spec over PV and PQ buses; Q_calc - Q_spec over PQ buses]."""
    V = Vm * np.exp(1j * Va)
    S = V * np.conj(Y @ V)
    pv_pq, pq = _index(case)
    return np.concatenate([S.real[pv_pq] - case["P"][pv_pq], S.imag[pq] - case["Q"][pq]])


def jacobian(case, Y, Vm, Va):
    """d(P, Q) / d(angle of PV/PQ buses, |V| of PQ buses), polar form."""
    V = Vm * np.exp(1j * Va)
    I = Y @ V
    dS_dVa = 1j * np.diag(V) @ np.conj(np.diag(I) - Y @ np.diag(V))
    dS_dVm = np.diag(V) @ np.conj(Y @ np.diag(np.exp(1j * Va))) + np.diag(np.exp(1j * Va)) @ np.conj(np.diag(I))
    pv_pq, pq = _index(case)
    J11 = dS_dVa.real[np.ix_(pv_pq, pv_pq)]
    J12 = dS_dVm.real[np.ix_(pv_pq, pq)]
    J21 = dS_dVa.imag[np.ix_(pq, pv_pq)]
    J22 = dS_dVm.imag[np.ix_(pq, pq)]
    return np.block([[J11, J12], [J21, J22]])


def newton_raphson(case, solver="hhl", n_clock=10, dtype="c128", tol=1e-6, max_iter=20,
                   gauss_seidel=False, structured=True):
    """Solve the AC power flow.  solver "hhl": every Newton step is an HHL solve on the GPU
    (dilated Jacobian system); "direct": numpy's dense solve (for comparison).

    Returns dict(Vm, Va, iterations, mismatch_history, hhl_p_success)."""
    import torch

    Y = admittance(case)
    B = case["B"]
    Vm = np.array(case["Vset"], dtype=float)
    Va = np.zeros(B)
    for i, k in enumerate(case["kind"]):
        if k == "PQ":
            Vm[i] = 1.0
    pv_pq, pq = _index(case)
    hist, psucc = [], []
    tdt = torch.complex128 if dtype == "c128" else torch.complex64
    it = 0
    for it in range(max_iter):
        F = mismatch(case, Y, Vm, Va)
        hist.append(float(np.max(np.abs(F))))
        if hist[-1] < tol:
            break
        J = jacobian(case, Y, Vm, Va)
        if solver == "direct":
            dx = np.linalg.solve(J, -F)
        else:
            h = qs.hhl_build(J, -F.astype(np.complex128), n_clock, structured=structured,
                             gauss_seidel=gauss_seidel, dilate=True)
            info = h.info()
            circ = qs.qsim_fuse(h.as_circuit(), 4)
            st = torch.empty(1 << info["n"], dtype=tdt, device="cuda")
            qs.hhl_prepare_state(st, h)
            qs.qsim_apply(st, circ, n_qubits=info["n"])
            r = qs.hhl_readout(st, h)
            dx = r["x"].real
            psucc.append(r["p_success"])
        na = len(pv_pq)
        Va[pv_pq] += dx[:na]
        Vm[pq] += dx[na:]
    return dict(Vm=Vm, Va=Va, iterations=it, mismatch_history=hist, hhl_p_success=psucc)
