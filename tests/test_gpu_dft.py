"""Fourier-transform passes (qsim_circuit_add_dft) and HHL circuits whose QFTs run as passes
(QSIM_HHL_FFT_QFT), against the FP64 oracle through the C ABI.

A single pass is compared with the oracle's `dft_pass` (the textbook dense-gate rule applied to
the DFT matrix and its twiddle, pinned against the gate-level QFT).  HHL circuits with passes are
compared with the oracle's gate-level HHL (H, controlled phases and swaps): the final states must
agree although the intermediate ones differ by a relabelling of the clock register.  Tolerances
as in test_gpu_parity: complex128 1e-12 (or the clock-conditioning bound when both sides
eigendecompose A), complex64 1e-5 with fidelity >= 1 - 1e-6.
"""
import functools
import math

import numpy as np
import pytest
import torch

import synth
from oracle import core as ocore
from oracle import hhl as ohhl
from test_gpu_parity import (DTYPES, TOL, _indefinite, _oracle_spectral, check, compare_hhl, cond_tol,
                             dev_state, host_input, run_product_hhl)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qs(cuda_device):
    from paper_2402_08136_gb300 import build
    build.build()
    import paper_2402_08136_gb300 as q
    return q


# (n, field, twiddle-source register, sign, twiddle first)
PASSES = [
    (16, list(range(10, 16)), list(range(4, 10)), -1, False),   # top clock field, as in an inverse QFT
    (16, list(range(10, 16)), list(range(4, 10)), +1, True),    # and its inverse
    (18, list(range(8, 18)), list(range(0, 8)), -1, False),     # 10-qubit field, 16-32 tiles
    (18, list(range(3, 12)), [0, 1, 2], +1, True),              # odd field (9), lanes above it
    (14, list(range(0, 5)), [], -1, False),                     # field holds qubit 0
    (14, [1, 3, 6, 7, 11], [0, 2, 13], +1, False),              # scattered field and source
    (12, [5], [0, 1, 2, 3, 4], -1, False),                      # one-qubit field
    (12, [2, 9], [], +1, False),
    (13, [4, 5, 6], [10, 11, 12], -1, True),                    # source above the field
    (15, list(range(8, 15)), list(range(8)), -1, False),        # field of 7, all bits below as source
    (16, list(range(0, 8)), list(range(8, 16)), +1, False),     # field of 8 at the bottom
    (6, list(range(6)), [], -1, False),                         # the field is the whole state
    (7, list(range(1, 7)), [0], +1, True),                      # one lane qubit
]


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("case", list(range(len(PASSES))))
def test_dft_pass_parity(qs, dtype, case):
    n, field, src, sign, pre = PASSES[case]
    psi = synth.gaussian_state_np(500 + case, n)
    x0 = host_input(psi, dtype)
    ref = x0.copy()
    ohhl.dft_pass(ref, field, sign, src, pre)
    c = qs.Circuit(n)
    c.add_dft(field, sign, src, twiddle_first=pre)
    st = dev_state(x0, dtype)
    qs.qsim_apply(st, c)
    torch.cuda.synchronize()
    check(st, ref, dtype)


@pytest.mark.parametrize("dtype", DTYPES)
def test_dft_passes_compose_to_qft_and_back(qs, dtype):
    """Inverse QFT as three passes and the QFT back: the identity, within rounding."""
    n, reg = 17, list(range(2, 17))
    fields = [reg[10:], reg[5:10], reg[:5]]
    psi = synth.gaussian_state_np(77, n)
    x0 = host_input(psi, dtype)
    c = qs.Circuit(n)
    for f in fields:
        c.add_dft(f, -1, [q for q in reg if q < min(f)])
    for f in reversed(fields):
        c.add_dft(f, +1, [q for q in reg if q < min(f)], twiddle_first=True)
    st = dev_state(x0, dtype)
    qs.qsim_apply(st, c)
    torch.cuda.synchronize()
    check(st, x0, dtype)


# ------------------------------------------------------------------ HHL with Fourier passes
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("structured", [False, True])
@pytest.mark.parametrize("max_k", [0, 4])
def test_hhl7_fft_qft_exact_grid(qs, dtype, structured, max_k):
    p = synth.hhl7_problem()
    h = qs.hhl_build(p["A"], p["b"], p["m"], p["t"], p["C"], structured=structured, fft_qft=True)
    assert h.as_circuit().info()["n_dft"] == 4
    ref = ohhl.solve(p["A"], p["b"], p["m"], p["t"], p["C"])
    st, r = run_product_hhl(qs, h, dtype, max_k)
    compare_hhl(st, r, ref, dtype, TOL[dtype])
    xt = np.linalg.solve(p["A"], p["b"])
    assert np.max(np.abs(r["x"] - xt)) / np.linalg.norm(xt) < (1e-11 if dtype == torch.complex128 else 1e-4)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("seed", [0, 1])
def test_hhl_fft_qft_offgrid_contingency(qs, dtype, seed):
    rng = np.random.default_rng(seed)
    nb = int(rng.integers(2, 5))
    m = int(rng.integers(5, 9))
    A, b = synth.contingency_system(rng, 2 ** nb + 1)
    h = qs.hhl_build(A, b, m, structured=True, fft_qft=True)
    ref = ohhl.solve(A, b, m)
    st, r = run_product_hhl(qs, h, dtype, 4)
    compare_hhl(st, r, ref, dtype, cond_tol(m) if dtype == torch.complex128 else TOL[dtype])


@functools.lru_cache(maxsize=None)
def _spectral_case(N, m, seed):
    rng = np.random.default_rng(seed)
    V = synth.haar_unitary(rng, N)
    lam = np.sort(rng.uniform(0.5, 9.0, size=N))
    b = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    t = 2 * math.pi * (2 ** m - 1) / (2 ** m * 9.0)
    return lam, V, b, t, 0.4, _oracle_spectral(lam, V, b, m, t, 0.4)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("N,m", [(6, 12), (2, 21)])
@pytest.mark.parametrize("structured", [False, True])
def test_hhl_fft_qft_two_and_three_fields(qs, dtype, N, m, structured):
    """12 clock qubits run as two passes each way, 21 as three (7 + 7 + 7): the rotation reads
    the clock value in field order and the QFT back restores the natural order."""
    lam, V, b, t, C, ref = _spectral_case(N, m, 21)
    h = qs.hhl_build_spectral(lam, V, b, m, t, C, structured=structured, fft_qft=True)
    assert h.as_circuit().info()["n_dft"] == 4 * ((m + 9) // 10)
    st, r = run_product_hhl(qs, h, dtype, 4)
    compare_hhl(st, r, ref, dtype, 1e-12 if dtype == torch.complex128 else TOL[dtype])


@pytest.mark.parametrize("dtype", DTYPES)
def test_hhl_fft_qft_indefinite_two_fields(qs, dtype):
    """Two's-complement clock (sign qubit) read through the field order."""
    m, N = 12, 5
    A, b = _indefinite(3, N, m, grid=True)
    t = 2 * math.pi / 2 ** m
    h = qs.hhl_build(A, b, m, t, structured=True, fft_qft=True)
    ref = ohhl.solve(A, b, m, t)
    st, r = run_product_hhl(qs, h, dtype, 3)
    compare_hhl(st, r, ref, dtype, cond_tol(m) if dtype == torch.complex128 else TOL[dtype])


@pytest.mark.parametrize("dtype", DTYPES)
def test_hhl_fft_qft_dilated(qs, dtype):
    rng = np.random.default_rng(31)
    N, m = 3, 11
    U, W = synth.haar_unitary(rng, N), synth.haar_unitary(rng, N)
    A = (U * np.array([2.0, 5.0, 31.0])) @ W.conj().T
    b = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    h = qs.hhl_build(A, b, m, dilate=True, structured=True, fft_qft=True)
    ref = ohhl.solve_general(A, b, m)
    st, r = run_product_hhl(qs, h, dtype, 3)
    compare_hhl(st, r, ref, dtype, cond_tol(m) if dtype == torch.complex128 else TOL[dtype])


# (n, field): H on every field qubit as one Walsh-Hadamard pass
WALSH = [(14, list(range(3, 13))), (12, [0, 1, 2]), (13, [2, 7, 5, 11]), (6, list(range(6))),
         (16, list(range(6, 15))), (9, [8])]


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("case", list(range(len(WALSH))))
def test_walsh_pass_parity(qs, dtype, case):
    n, field = WALSH[case]
    psi = synth.gaussian_state_np(700 + case, n)
    x0 = host_input(psi, dtype)
    ref = x0.copy()
    for q in field:
        ocore.apply_gate(ref, [q], ohhl.H)
    c = qs.Circuit(n)
    c.add_walsh(field)
    st = dev_state(x0, dtype)
    qs.qsim_apply(st, c)
    torch.cuda.synchronize()
    check(st, ref, dtype)
