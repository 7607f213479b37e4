"""The complex64 Fourier / Walsh-Hadamard pass with bulk-copy (TMA) tiles (bulk stores, or
thread stores with the next tile's load issued early) against the FP64 oracle, and against the
thread-load kernel, each selected through the kernel-choice table.

Shapes the bulk-copy kernel takes: a contiguous field of 9 or 10 qubits starting at qubit 3 or
above (the lanes are qubits 0..2), with the twiddle before or after the transform or none,
either sign, and the Walsh-Hadamard pass; inside HHL solves it also carries the structured
phase on its inputs or outputs and the eigenvalue inversion into the unwritten upper half.
Tolerance: 1e-5 per amplitude with fidelity >= 1 - 1e-6 (complex64).
"""
import numpy as np
import pytest
import torch

import synth
from hhl_bounds import cond_tol
from oracle import hhl as ohhl
from test_gpu_parity import TOL, check, compare_hhl, dev_state, host_input

pytestmark = pytest.mark.gpu

C64 = torch.complex64


@pytest.fixture(scope="module")
def qs(cuda_device):
    from paper_2402_08136_gb300 import build
    build.build()
    import paper_2402_08136_gb300 as q
    yield q
    q.qsim_tune_reset()


# (n, field, twiddle source, sign, twiddle first, walsh)
CASES = [
    (16, list(range(6, 16)), [], -1, False, False),             # the field right above 6 qubits
    (18, list(range(8, 18)), list(range(0, 8)), -1, False, False),  # top field, twiddle after
    (18, list(range(8, 18)), list(range(0, 8)), +1, True, False),   # and its inverse
    (17, list(range(3, 13)), list(range(13, 17)), +1, False, False),  # field at qubit 3, source above
    (15, list(range(5, 14)), [0, 1, 2, 3, 4], -1, False, False),    # field of 9, one qubit above
    (13, list(range(3, 13)), [], +1, False, False),             # the field fills the state above the lanes
    (16, list(range(6, 16)), [], +1, False, True),              # Walsh-Hadamard
    (19, list(range(4, 13)), [], +1, False, True),              # Walsh-Hadamard, 9 qubits, gap and qubits above
]


@pytest.mark.parametrize("tma", [4, 3, 2, 1, 0])
@pytest.mark.parametrize("case", list(range(len(CASES))))
def test_pass_matches_oracle_with_either_kernel(qs, tma, case):
    n, field, src, sign, pre, walsh = CASES[case]
    qs.qsim_tune_set(qs.QSIM_C64, qs.QSIM_TUNE_DFT_TMA, tma)
    try:
        psi = synth.gaussian_state_np(900 + case, n)
        x0 = host_input(psi, C64)
        ref = x0.copy()
        c = qs.Circuit(n)
        if walsh:
            c.add_walsh(field)
            H = np.array([[1, 1], [1, -1]]) / np.sqrt(2)
            from oracle import core as ocore
            for q in field:
                ocore.apply_gate(ref, [q], H)
        else:
            c.add_dft(field, sign, src, twiddle_first=pre)
            ohhl.dft_pass(ref, field, sign, src, pre)
        st = dev_state(x0, C64)
        qs.qsim_apply(st, c)
        torch.cuda.synchronize()
        check(st, ref, C64)
        assert qs.qsim_device_status() == 0
    finally:
        qs.qsim_tune_reset()


def test_both_kernels_agree_on_a_large_pass(qs):
    """A 24-qubit state (2048 tiles, several per CTA): the two kernels agree to rounding."""
    n = 24
    st0 = synth.gaussian_state_torch(5, n, C64, "cuda", normalize=True)
    c = qs.Circuit(n).add_dft(list(range(14, 24)), -1, list(range(4, 14)))
    outs = []
    for tma in (4, 3, 2, 1, 0):
        qs.qsim_tune_set(qs.QSIM_C64, qs.QSIM_TUNE_DFT_TMA, tma)
        st = st0.clone()
        qs.qsim_apply(st, c)
        torch.cuda.synchronize()
        outs.append(st)
    qs.qsim_tune_reset()
    for o in outs[1:]:
        assert float((outs[0] - o).abs().max()) <= 1e-6


@pytest.mark.parametrize("tma", [4, 3, 2, 1, 0])
def test_hhl_with_ten_qubit_clock_fields_matches_oracle(qs, tma):
    """A solve whose clock register splits into two 9-qubit fields (m = 18, qubits 3..11 and
    12..20): the passes with the structured phase on their inputs / outputs and the inversion
    fused into the inverse QFT's last pass, through hhl_run on a NaN-filled state (live width:
    the inversion writes the upper half, nothing reads an unwritten amplitude)."""
    rng = np.random.default_rng(77)
    A, b = synth.contingency_system(rng, 2 ** 3 + 1)      # nb = 3: the bottom clock field starts at qubit 3
    m = 18
    qs.qsim_tune_set(qs.QSIM_C64, qs.QSIM_TUNE_DFT_TMA, tma)
    try:
        h = qs.hhl_build(A, b, m, structured=True, fft_qft=True)
        info = h.info()
        assert info["n"] == 22
        ref = ohhl.solve(A, b, m)
        st = torch.empty(1 << info["n"], dtype=C64, device="cuda")
        st.fill_(float("nan"))
        qs.hhl_run(st, h, qs.qsim_fuse(h.as_circuit(), 4))
        r = qs.hhl_readout(st, h)
        compare_hhl(st, r, ref, C64, TOL[C64])
        assert qs.qsim_device_status() == 0
    finally:
        qs.qsim_tune_reset()


@pytest.mark.parametrize("m", [18, 20])
@pytest.mark.parametrize("tma", [4, 0])
def test_hhl_merged_passes_match_oracle(qs, m, tma):
    """nb = 4: both clock fields start at qubit 4 or above, so with 128-byte tile rows the executor
    runs the top field's H layer, the structured phase and the inverse QFT's first pass as one
    kernel with generated inputs, merges the inverse QFT's last pass, the inversion and the QFT's
    first pass into one kernel per half, and the QFT's last pass, the structured phase and the
    Walsh-Hadamard pass of the top field into another (tma = 4); tma = 0 runs the same circuit
    pass by pass.  Both against the oracle's gate-level HHL, on a NaN-filled state."""
    rng = np.random.default_rng(300 + m)
    A, b = synth.contingency_system(rng, 2 ** 4 + 1)      # nb = 4
    qs.qsim_tune_set(qs.QSIM_C64, qs.QSIM_TUNE_DFT_TMA, tma)
    qs.qsim_tune_set(qs.QSIM_C64, qs.QSIM_TUNE_DFT_MERGE, 7)   # every merge, whatever the default
    try:
        h = qs.hhl_build(A, b, m, structured=True, fft_qft=True)
        info = h.info()
        assert info["n"] == 4 + m + 1
        ref = ohhl.solve(A, b, m)
        st = torch.empty(1 << info["n"], dtype=C64, device="cuda")
        st.fill_(float("nan"))
        before = qs.qsim_launch_counts()
        qs.hhl_run(st, h, qs.qsim_fuse(h.as_circuit(), 4))
        r = qs.hhl_readout(st, h)
        after = qs.qsim_launch_counts()
        compare_hhl(st, r, ref, C64, TOL[C64])
        assert qs.qsim_device_status() == 0
        passes = after["fourier_tma"] - before["fourier_tma"] + after["fourier"] - before["fourier"]
        expands = after["expand"] - before["expand"]
        if tma == 4:
            # H layer + phase + inverse QFT on the top field with generated inputs, 2 merged launches
            # (inverse QFT's last pass, inversion, QFT's first pass), QFT top + phase + Walsh
            # merged, Walsh bottom field: 5 pass launches, and only the bottom field's H layer is a
            # write-only expansion (2 launches)
            assert after["fourier"] == before["fourier"]
            assert passes == 5 and expands == 2
        else:
            assert passes == 6 and expands == 4
    finally:
        qs.qsim_tune_reset()


def test_autotune_writes_its_size_class_and_results_stay_correct(qs):
    """qsim_autotune on a 22-qubit complex64 buffer: it writes the table entries of that size
    class only (marked tuned), reports positive timings, and a Fourier pass and a dense 5-qubit
    gate run with the tuned entries still match the oracle."""
    n = 22
    buf = torch.empty(1 << n, dtype=C64, device="cuda")
    try:
        rep = qs.qsim_autotune(buf)
        assert rep["n_qubits"] == n and rep["table"]["tuned"] == 1
        assert rep["dft_ms"] > 0 and all(v > 0 for v in rep["fuse_ms"].values())
        assert qs.qsim_tune_get(qs.QSIM_C64, qs.QSIM_TUNE_TUNED, n) == 1
        assert qs.qsim_tune_get(qs.QSIM_C64, qs.QSIM_TUNE_TUNED, 27) == 0      # another size class
        for k in ("dft_tma", "dft_lanes", "dft_prefetch", "dense_tc", "fuse_width"):
            key = getattr(qs, "QSIM_TUNE_" + k.upper())
            assert qs.qsim_tune_get(qs.QSIM_C64, key, n) == rep["table"][k]
        psi = host_input(synth.gaussian_state_np(71, n), C64)
        ref = psi.copy()
        field, src = list(range(12, 22)), list(range(2, 12))
        ohhl.dft_pass(ref, field, -1, src, False)
        rng = np.random.default_rng(72)
        U = synth.haar_unitary(rng, 32)
        t = synth.random_targets(rng, n, 5)
        from oracle import core as ocore
        ocore.apply_gate(ref, t, U)
        c = qs.Circuit(n).add_dft(field, -1, src).add_gate(t, U)
        st = dev_state(psi, C64)
        qs.qsim_apply(st, c)
        torch.cuda.synchronize()
        check(st, ref, C64)
    finally:
        qs.qsim_tune_reset()
