"""The C-ABI library loads and exports every symbol include/*.h declares; host-only calls and
their error paths (no device compute, runs without a GPU)."""
import ctypes
import glob
import math
import os
import re

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def qs():
    from paper_2402_08136_gb300 import build
    build.build()
    import paper_2402_08136_gb300 as q
    return q


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b((?:qsim|hhl)_\w+)\s*\(", text, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


def test_every_declared_symbol_is_exported(qs):
    names = declared_functions()
    assert len(names) >= 14
    lib = ctypes.CDLL(qs.library_path())
    for n in names:
        assert hasattr(lib, n), n


def test_version_and_error_text(qs):
    assert "sm_103a" in qs.qsim_version()
    with pytest.raises(qs.QsimError) as e:
        qs.Circuit(0)
    assert e.value.code == -1 and "n_qubits" in str(e.value)


def test_gate_argument_checks(qs):
    c = qs.Circuit(5)
    U = synth.haar_unitary(np.random.default_rng(0), 4)
    c.add_gate([0, 3], U, controls=[4])
    for bad in ([0, 0], [0, 5], [-1, 2]):
        with pytest.raises(qs.QsimError):
            c.add_gate(bad, U)
    with pytest.raises(qs.QsimError):
        c.add_gate([0, 1], U, controls=[1])
    Unan = U.copy()
    Unan[0, 0] = np.nan
    with pytest.raises(qs.QsimError):
        c.add_gate([0, 1], Unan)
    with pytest.raises(qs.QsimError):
        c.add_ucry(0, [0, 1], np.zeros(4))
    info = c.info()
    assert info["n_gates"] == 1 and info["n_dense"] == 1


def test_classification_of_specialised_gates(qs):
    c = qs.Circuit(4)
    c.add_gate([0, 1], np.diag([1, 1, 1, np.exp(0.3j)]))          # controlled phase
    c.add_gate([2], np.diag([np.exp(0.1j), np.exp(-0.1j)]))      # RZ: diagonal
    swap = np.eye(4)[[0, 2, 1, 3]]
    c.add_gate([1, 3], swap)                                      # swap
    c.add_gate([0], np.array([[0, 1], [1, 0]]))                   # X: dense
    c.add_ucry(3, [0, 1, 2], np.linspace(0, 1, 8))
    i = c.info()
    assert (i["n_diag"], i["n_perm"], i["n_dense"], i["n_ucry"]) == (2, 1, 1, 1)


def test_fusion_counts(qs):
    # QFT-like circuit on 6 qubits: fusion to width 2 and 6 reduces the executed gate count
    n = 6
    c = qs.Circuit(n)
    H = np.array([[1, 1], [1, -1]]) / math.sqrt(2)
    gates = 0
    for j in range(n - 1, -1, -1):
        c.add_gate([j], H)
        gates += 1
        for l in range(j - 1, -1, -1):
            c.add_gate([l, j], np.diag([1, 1, 1, np.exp(2j * math.pi / 2 ** (j - l + 1))]))
            gates += 1
    f2 = qs.qsim_fuse(c, 2).info()
    f6 = qs.qsim_fuse(c, 6).info()
    assert c.info()["n_gates"] == gates
    assert f2["fused"] == 1 and f2["max_k"] <= 2 and f2["n_gates"] < gates
    assert f6["n_gates"] == 1 and f6["max_k"] == 6


def test_fusion_keeps_controlled_and_ucry(qs):
    c = qs.Circuit(5)
    U = synth.haar_unitary(np.random.default_rng(1), 4)
    c.add_gate([0], np.eye(2))
    c.add_gate([0, 1], U, controls=[2])
    c.add_ucry(4, [2, 3], np.zeros(4))
    c.add_gate([1], np.eye(2))
    f = qs.qsim_fuse(c, 4).info()
    assert f["n_ucry"] == 1 and f["n_gates"] == 4


def test_hhl_build_host_side(qs):
    p = synth.hhl7_problem()
    h = qs.hhl_build(p["A"], p["b"], p["m"], p["t"], p["C"])
    i = h.info()
    assert (i["N"], i["nb"], i["m"], i["n"]) == (4, 2, 4, 7)
    w = np.linalg.eigvalsh(p["A"])
    assert abs(i["lambda_min"] - w[0]) < 1e-12 and abs(i["lambda_max"] - w[-1]) < 1e-12
    assert abs(i["C"] - w[0]) < 1e-9          # exact grid: C = lambda_min
    assert abs(i["norm_b"] - np.linalg.norm(p["b"])) < 1e-14
    # gate count: m H + m controlled-U + IQFT (m H + m(m-1)/2 CP + m/2 swaps) + UCRY, mirrored
    m = 4
    qpe = m + m + m + m * (m - 1) // 2 + m // 2
    assert i["n_gates"] == 2 * qpe + 1
    circ = h.as_circuit().info()
    assert circ["n_ucry"] == 1


def test_hhl_default_clock_count_follows_formula(qs):
    rng = np.random.default_rng(3)
    A, b, _ = synth.grid_system(rng, 17, avg_degree=3.0)
    h = qs.hhl_build(A, b)
    i = h.info()
    w = np.linalg.eigvalsh(A)
    kappa = w[-1] / w[0]
    assert i["m"] == max(4 + 1, math.ceil(math.log2(kappa + 1)))
    assert i["n_total_formula"] == i["nb"] + i["m"] + 1


def test_hhl_build_errors(qs):
    A = np.array([[2.0, 1.0], [0.0, 3.0]])
    with pytest.raises(qs.QsimError):
        qs.hhl_build(A, [1.0, 0.0], 3)                 # not Hermitian
    with pytest.raises(qs.QsimError):
        qs.hhl_build(np.diag([1.0, 0.0]), [1.0, 0.0], 3)   # singular
    qs.hhl_build(-np.eye(2), [1.0, 0.0], 3)            # negative definite: sign qubit, accepted
    with pytest.raises(qs.QsimError):
        qs.hhl_build(np.eye(2), [0.0, 0.0], 3)         # b = 0
    with pytest.raises(qs.QsimError):
        qs.hhl_build(np.diag([1.0, 2.0]), [1.0, 1.0], 3, C=1.5)   # C above lambda_min
    with pytest.raises(qs.QsimError):
        qs.hhl_build(np.diag([1.0, np.nan]), [1.0, 1.0], 3)


def test_hhl_build_matches_spectral_path(qs):
    rng = np.random.default_rng(8)
    V = synth.haar_unitary(rng, 5)
    lam = np.array([1.0, 2.5, 3.0, 7.0, 9.0])
    A = (V * lam) @ V.conj().T
    A = 0.5 * (A + A.conj().T)
    b = rng.standard_normal(5)
    h1 = qs.hhl_build(A, b, 5).info()
    h2 = qs.hhl_build_spectral(lam, V, b, 5).info()
    for key in ("N", "nb", "m", "n", "n_gates"):
        assert h1[key] == h2[key]
    for key in ("t", "C", "lambda_min", "lambda_max"):
        assert abs(h1[key] - h2[key]) < 1e-12 * max(1.0, abs(h2[key]))


def test_structured_qpe_gate_counts(qs):
    p = synth.hhl7_problem()
    m = p["m"]
    h = qs.hhl_build(p["A"], p["b"], m, p["t"], p["C"], structured=True)
    iqft = m + m * (m - 1) // 2 + m // 2
    assert h.info()["n_gates"] == 2 * m + 2 + 2 + 2 * iqft + 1
    ci = h.as_circuit().info()
    assert ci["n_ucry"] == 1 and ci["n_dense"] >= 2


def test_real_and_complex_eigensolvers_agree(qs):
    # the same spectrum as a real symmetric and as a complex Hermitian matrix (unitary similarity)
    rng = np.random.default_rng(21)
    Q, _ = np.linalg.qr(rng.standard_normal((24, 24)))
    lam = np.sort(rng.uniform(1.0, 50.0, 24))
    A = (Q * lam) @ Q.T
    A = 0.5 * (A + A.T)
    D = np.diag(np.exp(1j * rng.uniform(0, 6, 24)))
    Ac = D @ A @ D.conj().T
    b = rng.standard_normal(24)
    i1 = qs.hhl_build(A, b, 6).info()
    i2 = qs.hhl_build(0.5 * (Ac + Ac.conj().T), b, 6).info()
    for key in ("lambda_min", "lambda_max", "t", "C"):
        assert abs(i1[key] - lam[0 if key == "lambda_min" else -1]) < 1e-12 * lam[-1] \
            if key.startswith("lambda") else abs(i1[key] - i2[key]) < 1e-12 * max(1, abs(i2[key]))
    assert abs(i2["lambda_min"] - lam[0]) < 1e-12 * lam[-1]
    assert abs(i2["lambda_max"] - lam[-1]) < 1e-12 * lam[-1]


def test_indefinite_system_uses_sign_qubit(qs):
    rng = np.random.default_rng(5)
    V = np.linalg.qr(rng.standard_normal((6, 6)))[0]
    lam = np.array([-20.0, -3.0, 1.0, 2.0, 8.0, 16.0])
    A = (V * lam) @ V.T
    i = qs.hhl_build(0.5 * (A + A.T), rng.standard_normal(6)).info()
    assert i["m"] == max(3 + 1, math.ceil(math.log2(20.0 / 1.0 + 1))) + 1
    assert i["n_total_formula"] == i["nb"] + i["m"] + 1
    assert abs(i["t"] - 2 * math.pi * (2 ** (i["m"] - 1) - 1) / (2 ** i["m"] * 20.0)) < 1e-14
    assert abs(i["lambda_min"] + 20.0) < 1e-12 and abs(i["lambda_max"] - 16.0) < 1e-12


def test_gauss_seidel_and_dilation_host_side(qs):
    """Table I, 30-bus*: a Gauss-Seidel preconditioned 29 x 29 system is dilated to 58 rows
    (n_data = 6) and has negative eigenvalues (sign qubit)."""
    rng = np.random.default_rng(33)
    A, b, _ = synth.grid_system(rng, 30)
    h = qs.hhl_build(A, b, 0, gauss_seidel=True).info()
    assert (h["N"], h["N_eff"], h["nb"]) == (29, 58, 6)
    assert h["lambda_min"] < 0 < h["lambda_max"] and abs(h["lambda_min"] + h["lambda_max"]) < 1e-9 * h["lambda_max"]
    with pytest.raises(qs.QsimError):
        qs.hhl_build(np.array([[2.0, 1.0], [0.0, 3.0]]), [1.0, 0.0], 3)        # needs dilate
    d = qs.hhl_build(np.array([[2.0, 1.0], [0.0, 3.0]]), [1.0, 0.0], 3, dilate=True).info()
    assert d["N_eff"] == 4 and d["N"] == 2


def test_dft_argument_checks(qs):
    c = qs.Circuit(8)
    c.add_dft([4, 5, 6], -1, src=[0, 1, 2, 3])
    c.add_dft([0, 1], +1, twiddle_first=True)
    c.add_walsh([7, 2, 5])
    assert c.info()["n_dft"] == 3 and c.info()["n_gates"] == 3
    for bad in ([], [1, 1], [12], list(range(11))):
        with pytest.raises(qs.QsimError):
            qs.Circuit(12).add_walsh(bad)
    for bad in (dict(targets=[], sign=1), dict(targets=[1, 1], sign=1), dict(targets=[12], sign=1),
                dict(targets=[1, 2], sign=0), dict(targets=[1, 2], sign=1, src=[2]),
                dict(targets=list(range(11)), sign=1)):
        with pytest.raises(qs.QsimError):
            qs.Circuit(12).add_dft(**bad)


@pytest.mark.parametrize("m,fields", [(4, 1), (10, 1), (11, 2), (20, 2), (21, 3), (26, 3)])
def test_fft_qft_pass_counts(qs, m, fields):
    """QFTs as Fourier passes: one pass per field of at most 10 clock qubits, each way."""
    rng = np.random.default_rng(m)
    lam = np.array([1.0, 3.0])
    V = np.eye(2)
    b = rng.standard_normal(2)
    for structured in (False, True):
        h = qs.hhl_build_spectral(lam, V, b, m, structured=structured, fft_qft=True)
        ci = h.as_circuit().info()
        assert ci["n_dft"] == 4 * fields          # inverse QFT, QFT and the two Hadamard layers
        assert ci["n_perm"] == 0
        g = qs.hhl_build_spectral(lam, V, b, m, structured=structured)
        iqft = m + m * (m - 1) // 2 + m // 2
        assert g.info()["n_gates"] - h.info()["n_gates"] == 2 * (iqft + m) - 4 * fields
    fz = qs.qsim_fuse(h.as_circuit(), 4).info()
    assert fz["n_dft"] == 4 * fields


def test_run_and_solve_argument_checks(qs):
    """hhl_run, hhl_batch_solve, hhl_batch_results reject bad arguments before touching the
    device; qsim_launch_count needs no GPU."""
    import ctypes
    from paper_2402_08136_gb300 import _binding as B
    L = B.library()
    p = synth.hhl7_problem()
    h = qs.hhl_build(p["A"], p["b"], p["m"], p["t"], p["C"])
    fake = ctypes.c_void_p(256)  # never dereferenced: every call below fails its checks first
    assert L.hhl_run(None, B.QSIM_C64, h.ptr, None, None) != 0
    assert L.hhl_run(fake, 7, h.ptr, None, None) != 0                      # dtype
    assert L.hhl_run(fake, B.QSIM_C64, None, None, None) != 0              # no problem
    other = qs.Circuit(h.info()["n"] + 1)
    assert L.hhl_run(fake, B.QSIM_C64, h.ptr, other.ptr, None) != 0        # qubit count
    assert "qubit count" in L.qsim_last_error().decode()
    assert L.hhl_batch_solve(None, None, None, None) != 0
    assert L.hhl_batch_results(None, None, None, None) != 0
    n0 = qs.qsim_launch_count()
    assert isinstance(n0, int) and n0 >= 0


def test_host_eigensolver_matches_numpy(qs):
    """The eigensolver behind hhl_build: eigenvalues equal numpy's eigh, V is unitary and
    A V = V diag(lambda), for a real symmetric (power-flow) and a complex Hermitian matrix."""
    rng = np.random.default_rng(3)
    A_real, _ = synth.contingency_system(rng, 33)
    G = rng.standard_normal((24, 24)) + 1j * rng.standard_normal((24, 24))
    A_cplx = G + G.conj().T
    for A in (A_real, A_cplx):
        lam, V = qs.qsim_hermitian_eig(A)
        ref = np.linalg.eigvalsh(A)
        scale = np.max(np.abs(ref))
        assert np.max(np.abs(lam - ref)) <= 1e-13 * scale
        assert np.max(np.abs(V.conj().T @ V - np.eye(len(lam)))) <= 1e-13
        assert np.max(np.abs(A @ V - V * lam)) <= 1e-12 * scale


def test_eigensolver_reports_non_convergence(qs):
    """A capped iteration that stops before the matrix is diagonal is an error (EINVAL), not
    an unconverged V handed on to the circuit."""
    rng = np.random.default_rng(5)
    A_real, _ = synth.contingency_system(rng, 33)   # 32 x 32 real symmetric
    G = rng.standard_normal((32, 32)) + 1j * rng.standard_normal((32, 32))
    for A in (A_real, G + G.conj().T):
        with pytest.raises(qs.QsimError) as e:
            qs.qsim_hermitian_eig(A, max_iter=1)
        assert e.value.code == -1 and "did not converge" in str(e.value)
        lam, _ = qs.qsim_hermitian_eig(A)          # the default cap converges
        assert np.all(np.isfinite(lam))


def test_noalloc_readout_rejects_a_slice_beyond_its_scratch(qs):
    """nb = 11 (2^11 amplitudes in the solution slice) is beyond the allocation-free readout's
    fixed scratch: QSIM_EINVAL before any device access (the state pointer is never used)."""
    from paper_2402_08136_gb300._binding import _DP, _VP, _ReadoutStats, library
    f = library().hhl_readout_noalloc
    f.argtypes = [_VP, ctypes.c_int, _VP, _VP, _DP, _DP, ctypes.POINTER(_ReadoutStats)]
    f.restype = ctypes.c_int
    N = 1025
    h = qs.hhl_build_spectral(np.linspace(1.0, 2.0, N), np.eye(N), np.ones(N), 1, structured=True)
    assert h.info()["nb"] == 11
    x = np.zeros(N, dtype=np.complex128)
    rc = f(ctypes.c_void_p(256), qs.QSIM_C128, h.ptr, None, x.view(np.float64).ctypes.data_as(_DP),
           None, None)
    assert rc == -1
    assert "2^10" in library().qsim_last_error().decode()


def test_kernel_choice_table(qs):
    """The table that replaces environment knobs: defaults, per-size-class entries, range checks,
    reset."""
    t = qs.qsim_tune_table()
    for cls in ("le24", "25to28", "ge29"):
        assert t["c64"][cls]["dft_tma"] == 4 and t["c128"][cls]["dft_tma"] == 0
        assert t["c64"][cls]["fuse_width"] == 4 and t["c64"][cls]["tuned"] == 0
        assert t["c64"][cls]["dense_tc"] == (1 << 4) | (1 << 5) | (1 << 6) | (1 << 7)
    qs.qsim_tune_set(qs.QSIM_C64, qs.QSIM_TUNE_FUSE_WIDTH, 3)
    qs.qsim_tune_set(qs.QSIM_C64, qs.QSIM_TUNE_DFT_TMA, 1, n_qubits=31)   # one size class only
    try:
        assert qs.qsim_tune_get(qs.QSIM_C64, qs.QSIM_TUNE_FUSE_WIDTH) == 3
        assert qs.qsim_tune_get(qs.QSIM_C64, qs.QSIM_TUNE_DFT_TMA, 30) == 1
        assert qs.qsim_tune_get(qs.QSIM_C64, qs.QSIM_TUNE_DFT_TMA, 27) == 4
        assert qs.qsim_tune_get(qs.QSIM_C64, qs.QSIM_TUNE_DFT_TMA, 20) == 4
        # qsim_fuse(max_k = 0) takes the table's width
        n = 6
        c = qs.Circuit(n)
        H = np.array([[1, 1], [1, -1]]) / math.sqrt(2)
        for q in range(n):
            c.add_gate([q], H)
        assert qs.qsim_fuse(c, 0).info()["max_k"] == 3
        for key, bad in ((qs.QSIM_TUNE_FUSE_WIDTH, 7), (qs.QSIM_TUNE_DFT_TMA, 5), (99, 1)):
            with pytest.raises(qs.QsimError):
                qs.qsim_tune_set(qs.QSIM_C64, key, bad)
        with pytest.raises(qs.QsimError):
            qs.qsim_tune_get(3, 0)
        with pytest.raises(qs.QsimError):
            qs.qsim_tune_get(qs.QSIM_C64, 0, 35)
    finally:
        qs.qsim_tune_reset()
    assert qs.qsim_tune_get(qs.QSIM_C64, qs.QSIM_TUNE_FUSE_WIDTH) == 4
    assert qs.qsim_tune_get(qs.QSIM_C64, qs.QSIM_TUNE_DFT_TMA, 31) == 4
