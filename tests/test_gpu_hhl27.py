"""The 27-qubit HHL workload at full size vs the FP64 oracle: the 64 x 64 reduced Laplacian of
a 65-bus grid (98 lines), nb = 6 data qubits, m = 20 clock qubits, one ancilla (Sec. III-A
procedure, Fig. 5 circuit).

One oracle run (plain gate-level HHL, FP64, every gate unfused: 20 controlled evolutions, the
textbook inverse QFT, the rotation and the uncomputation on a 2^27 state) serves both checks:
  * complex64, the product path (structured phase estimation, QFTs as Fourier passes, fused
    dense gates on the tensor cores, hhl_run + hhl_readout, the library's own eigensolver):
    every amplitude within 1e-5, fidelity >= 1 - 1e-6, readout within the implied bounds;
  * complex128 from the same spectral decomposition (hhl_build_spectral with the oracle's
    (lambda, V), t and C): every amplitude within 1e-12.
The library's default t and C must equal the oracle's (same readings, independent code).
"""
import math

import numpy as np
import pytest
import torch

import synth
from hhl_bounds import prob_bound, readout_bounds
from oracle import hhl as ohhl

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def qs(cuda_device):
    from paper_2402_08136_gb300 import build
    build.build()
    import paper_2402_08136_gb300 as q
    return q


def oracle_from_spectrum(lam, V, b, m):
    """The oracle's HHL with its controlled evolutions U_j = V diag(exp(i lam t 2^j)) V^H taken
    from the given eigendata (its default t and C, from the same eigenvalues)."""
    A = (V * lam) @ V.conj().T
    h = ohhl.build(0.5 * (A + A.conj().T), b, m)
    t = h["t"]
    forward = True
    gates = []
    for g in h["gates"]:
        if g[0] == "ucry":
            forward = False
        elif g[3]:
            j = g[3][0] - h["nb"]
            Uj = (V * np.exp(1j * lam * t * 2 ** j)) @ V.conj().T
            g = ("u", g[1], Uj if forward else Uj.conj().T, g[3], g[4])
        gates.append(g)
    h["gates"] = gates
    psi = ohhl.run(h)
    r = ohhl.readout(h, psi)
    r["psi"] = psi
    r["circuit"] = h
    return r


@pytest.fixture(scope="module")
def case():
    p = synth.hhl27_problem()
    assert p["A"].shape == (64, 64) and p["m"] == 20
    lam, V = np.linalg.eigh(p["A"])
    ref = oracle_from_spectrum(lam, V, p["b"], p["m"])
    assert ref["circuit"]["n"] == 27
    return p, lam, V, ref


def check_readout(r, ref, tol):
    """Readout within the bounds the state bound implies; returns the bound on each x entry."""
    h = ref["circuit"]
    bd = readout_bounds(ref, h["nb"], h["m"], tol, h["C"], h["bnorm"], 1 << h["nb"])
    assert abs(r["p_success"] - ref["P"]) <= bd["P"]
    assert abs(r["p_clock0"] - ref["P0"]) <= bd["P0"]
    assert abs(r["norm2"] - ref["norm2"]) <= prob_bound(ref["psi"], tol)
    assert np.all(np.abs(r["x_state"] - ref["x_state"]) <= bd["x_state"])
    dx = bd["x"][: len(ref["x"])]
    assert np.all(np.abs(r["x"] - ref["x"]) <= dx)
    return dx


def test_hhl27_complex64_product_path_matches_oracle(qs, case):
    p, _, _, ref = case
    h = qs.hhl_build(p["A"], p["b"], p["m"], structured=True, fft_qft=True)
    info = h.info()
    assert info["n"] == 27
    # the default evolution time and inversion constant: same readings as the oracle's
    assert abs(info["t"] - ref["circuit"]["t"]) <= 1e-13 * ref["circuit"]["t"]
    assert abs(info["C"] - ref["circuit"]["C"]) <= 1e-13 * ref["circuit"]["C"]
    st = torch.empty(1 << 27, dtype=torch.complex64, device="cuda")
    qs.hhl_run(st, h, qs.qsim_fuse(h.as_circuit(), 6))
    r = qs.hhl_readout(st, h)
    assert qs.qsim_device_status() == 0
    out = st.cpu().numpy().astype(np.complex128)
    del st
    err = float(np.max(np.abs(out - ref["psi"])))
    fid = abs(np.vdot(ref["psi"], out)) ** 2 / (np.vdot(out, out).real * np.vdot(ref["psi"], ref["psi"]).real)
    assert err <= 1e-5, "max|d amp| %.3e" % err
    assert fid >= 1 - 1e-6, "fidelity %.9f" % fid
    dx = check_readout(r, ref, 1e-5)
    # the HHL solution error against the classical A^-1 b is the method's (QPE discretisation):
    # the device's and the oracle's differ by at most ||x_dev - x_oracle|| / ||A^-1 b||
    xt = np.linalg.solve(p["A"], p["b"])
    e_dev = np.linalg.norm(r["x"] - xt) / np.linalg.norm(xt)
    e_ora = np.linalg.norm(ref["x"] - xt) / np.linalg.norm(xt)
    assert abs(e_dev - e_ora) <= np.linalg.norm(dx) / np.linalg.norm(xt)


def test_hhl27_complex128_shared_spectrum_matches_oracle_to_1e12(qs, case):
    p, lam, V, ref = case
    hc = ref["circuit"]
    h = qs.hhl_build_spectral(lam, V, p["b"], p["m"], hc["t"], hc["C"], structured=True, fft_qft=True)
    st = torch.empty(1 << 27, dtype=torch.complex128, device="cuda")
    qs.hhl_run(st, h, qs.qsim_fuse(h.as_circuit(), 2))
    r = qs.hhl_readout(st, h)
    out = st.cpu().numpy()
    del st
    err = float(np.max(np.abs(out - ref["psi"])))
    assert err <= 1e-12, "max|d amp| %.3e" % err
    check_readout(r, ref, 1e-12)
