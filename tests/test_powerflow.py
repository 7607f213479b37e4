"""Newton-Raphson AC power flow (the paper's application, Sec. III) with HHL linear solves.

CPU: the host-side power-flow equations (Jacobian vs central finite differences of the
mismatch; the direct-solve Newton iteration converges quadratically to a consistent solution).
GPU: the same iteration with every Newton step solved by an HHL circuit (dilated, optionally
Gauss-Seidel preconditioned) reaches the direct-solve voltages."""
import numpy as np
import pytest

import synth
from paper_2402_08136_gb300 import powerflow as pf


def test_jacobian_matches_finite_differences():
    case = synth.ac_case(3, 12)
    Y = pf.admittance(case)
    rng = np.random.default_rng(0)
    Vm = 1.0 + 0.02 * rng.standard_normal(12)
    Va = 0.05 * rng.standard_normal(12)
    Va[0] = 0.0
    J = pf.jacobian(case, Y, Vm, Va)
    pv_pq, pq = pf._index(case)
    h = 1e-6
    cols = []
    for i in pv_pq:
        d = np.zeros(12); d[i] = h
        cols.append((pf.mismatch(case, Y, Vm, Va + d) - pf.mismatch(case, Y, Vm, Va - d)) / (2 * h))
    for i in pq:
        d = np.zeros(12); d[i] = h
        cols.append((pf.mismatch(case, Y, Vm + d, Va) - pf.mismatch(case, Y, Vm - d, Va)) / (2 * h))
    assert np.max(np.abs(J - np.array(cols).T)) < 1e-6


def test_direct_newton_converges():
    case = synth.ac_case(4, 14)
    r = pf.newton_raphson(case, solver="direct", tol=1e-11)
    h = r["mismatch_history"]
    assert h[-1] < 1e-11 and r["iterations"] <= 8
    assert h[2] < h[1] ** 1.5 or h[2] < 1e-9          # quadratic convergence


@pytest.mark.gpu
@pytest.mark.parametrize("dtype,gs", [("c128", False), ("c128", True), ("c64", False)])
def test_hhl_newton_reaches_direct_solution(cuda_device, dtype, gs):
    from paper_2402_08136_gb300 import build
    build.build()
    case = synth.ac_case(5, 9)
    ref = pf.newton_raphson(case, solver="direct", tol=1e-12)
    r = pf.newton_raphson(case, solver="hhl", n_clock=11, dtype=dtype, tol=1e-5, max_iter=25,
                          gauss_seidel=gs)
    assert r["mismatch_history"][-1] < 1e-5
    assert np.max(np.abs(r["Vm"] - ref["Vm"])) < 1e-4
    assert np.max(np.abs(r["Va"] - ref["Va"])) < 1e-4
