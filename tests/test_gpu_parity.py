"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (absolute, per amplitude): complex128 1e-12, complex64 1e-5 with fidelity
>= 1 - 1e-6 (complex64 inputs are the complex128 inputs rounded to complex64 on both sides).
HHL circuits whose clock register amplifies eigenvalue rounding (phases lambda t 2^j) get the
conditioning bound max(1e-12, 2^m * 2 pi * 8 eps) when both sides eigendecompose A themselves;
with a shared spectral decomposition the 1e-12 bound applies at every m.
"""
import math

import numpy as np
import pytest
import torch

import synth
from hhl_bounds import cond_tol, prob_bound, readout_bounds
from oracle import core as ocore
from oracle import hhl as ohhl

pytestmark = pytest.mark.gpu

TOL = {torch.complex128: 1e-12, torch.complex64: 1e-5}
EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def qs(cuda_device):
    from paper_2402_08136_gb300 import build
    build.build()
    import paper_2402_08136_gb300 as q
    return q


def dev_state(psi, dtype):
    return torch.from_numpy(np.ascontiguousarray(psi)).to(dtype).cuda()


def host_input(psi, dtype):
    """The input both sides start from: rounded to complex64 for the complex64 path."""
    if dtype == torch.complex64:
        return psi.astype(np.complex64).astype(np.complex128)
    return psi.copy()


def check(out_dev, ref, dtype, fidelity=True):
    out = out_dev.cpu().numpy().astype(np.complex128)
    err = np.max(np.abs(out - ref)) if ref.size else 0.0
    assert err <= TOL[dtype], "max|d amp| = %.3e" % err
    if fidelity and dtype == torch.complex64 and ref.size:
        f = abs(np.vdot(ref, out)) ** 2 / (np.vdot(ref, ref).real * np.vdot(out, out).real)
        assert f >= 1 - 1e-6
    return err


DTYPES = [torch.complex128, torch.complex64]


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6, 7])
def test_dense_gate_parity(qs, dtype, k):
    rng = np.random.default_rng(100 + k)
    n = 14
    psi = synth.gaussian_state_np(k, n)
    x0 = host_input(psi, dtype)
    c = qs.Circuit(n)
    ref = x0.copy()
    cases = [list(range(k)),                                    # all-low targets
             [n - 1 - i for i in range(k)],                     # all-high targets
             synth.random_targets(rng, n, k),
             synth.random_targets(rng, n, k)]
    for i, t in enumerate(cases):
        U = synth.haar_unitary(rng, 1 << k)
        ctl = []
        if i == 3 and k + 2 <= n:
            ctl = [q for q in rng.permutation(n) if q not in t][:2]
            ctl = [int(q) for q in ctl]
        c.add_gate(t, U, ctl)
        ocore.apply_gate(ref, t, U, ctl)
    st = dev_state(x0, dtype)
    qs.qsim_apply(st, c)
    torch.cuda.synchronize()
    check(st, ref, dtype)


@pytest.fixture
def tc_on(qs):
    """Select the tensor-core kernel for dense gates of k targets (every size class); the
    kernel-choice table is put back afterwards."""
    def on(*ks):
        mask = qs.qsim_tune_get(qs.QSIM_C64, qs.QSIM_TUNE_DENSE_TC, 17)
        for k in ks:
            mask |= 1 << k
        qs.qsim_tune_set(qs.QSIM_C64, qs.QSIM_TUNE_DENSE_TC, mask)
    yield on
    qs.qsim_tune_reset()


@pytest.mark.parametrize("k", [3, 4, 5, 6])
def test_tensor_core_dense_parity_complex64(qs, k, tc_on):
    """complex64 gates with 3..6 targets and at least 128 groups run on the tcgen05 3xTF32
    kernel: low, high and random targets, with and without controls, vs the FP64 oracle.  4 and
    5 targets on qubits 0 and 1 run widened to the 6-target transposed form."""
    tc_on(k, 6)
    before = qs.qsim_launch_counts()["dense_tc"]
    rng = np.random.default_rng(500 + k)
    n = 17
    psi = host_input(synth.gaussian_state_np(500 + k, n), torch.complex64)
    c = qs.Circuit(n)
    ref = psi.copy()
    cases = [(list(range(k)), []), ([n - 1 - i for i in range(k)], []),
             (synth.random_targets(rng, n, k), []), (list(range(k))[::-1], [k + 3]),
             (synth.random_targets(rng, n, k), None)]
    for t, ctl in cases:
        if ctl is None:
            ctl = [int(q) for q in rng.permutation(n) if q not in t][:3]
        U = synth.haar_unitary(rng, 1 << k)
        c.add_gate(t, U, ctl)
        ocore.apply_gate(ref, t, U, ctl)
    st = dev_state(psi, torch.complex64)
    qs.qsim_apply(st, c)
    torch.cuda.synchronize()
    assert qs.qsim_device_status() == 0
    assert qs.qsim_launch_counts()["dense_tc"] - before == len(cases)
    check(st, ref, torch.complex64)


def test_real_six_target_gates_on_low_qubits(qs):
    """complex64 real 6-target gates whose targets include qubits 0 and 1 (the eigenvector
    rotation of a 64 x 64 system on the data register) run in the transposed tensor-core form:
    targets contiguous, with gaps, with controls above and between them; applied alone and in one
    circuit."""
    dtype = torch.complex64
    rng = np.random.default_rng(66)
    n = 14
    psi = host_input(synth.gaussian_state_np(44, n), dtype)
    cases = [([0, 1, 2, 3, 4, 5], []), ([0, 1, 3, 4, 5, 7], []), ([0, 1, 2, 4, 6, 8], [13]),
             ([0, 1, 3, 4, 5, 6], [2])]
    c_all = qs.Circuit(n)
    ref_all = psi.copy()
    for t, ctl in cases:
        Q, _ = np.linalg.qr(rng.standard_normal((64, 64)))
        U = Q.astype(np.complex128)
        c_all.add_gate(t, U, ctl)
        ocore.apply_gate(ref_all, t, U, ctl)
        ref = psi.copy()
        ocore.apply_gate(ref, t, U, ctl)
        st = dev_state(psi, dtype)
        qs.qsim_apply(st, qs.Circuit(n).add_gate(t, U, ctl))
        torch.cuda.synchronize()
        check(st, ref, dtype)
    st = dev_state(psi, dtype)
    qs.qsim_apply(st, c_all)
    torch.cuda.synchronize()
    check(st, ref_all, dtype)


@pytest.mark.parametrize("real", [False, True])
def test_widened_low_qubit_gates(qs, real, tc_on):
    """complex64 gates of 4..5 targets on qubit 0 or 1, widened with identity qubits to the
    6-target transposed form where the group-major form's loads are poor, and 6-target gates on
    the low qubits in the transposed form itself.  The added qubits are qubits 0 and 1 when
    free, qubit 2 when that leaves exactly one of qubits 2 and 3 free, then free qubits from 4
    up: above the targets, between them, moved up by controls.  6-target gates with qubit 0 and
    at most one free qubit among 0..3 run in the transposed form unwidened (qubit 1 a group
    bit); with qubit 1 and qubit 0 the only free one, in its sibling-group variant (each 16-byte
    load one amplitude of two groups).  Gates with qubit 0 or 1 a control, or with free low
    qubits, stay in the group-major form.  Each gate alone (one tensor-core launch) and all in
    one circuit."""
    tc_on(6, 7)
    dtype = torch.complex64
    rng = np.random.default_rng(77 + real)
    n = 16
    psi = host_input(synth.gaussian_state_np(78, n), dtype)
    cases = [([0, 1, 2, 3], []), ([0, 1, 3, 6], []), ([0, 1, 2, 3], [4, 5]), ([1, 0, 5, 2, 9], [3]),
             ([0, 1, 2, 3, 4], []), ([0, 1, 4, 7, 8], [2, 15]),
             ([1, 2, 3, 4], []), ([0, 2, 3, 9], [12]), ([0, 1, 2, 9], []), ([0, 1, 3, 7, 9], [4]),
             ([0, 5, 9, 13], [2]), ([1, 3, 6, 8, 10], []),
             ([0, 2, 3, 4, 5, 6], []), ([0, 2, 3, 7, 9, 11], [13]),  # complex: transposed, qubit 1 free
             ([1, 2, 3, 4, 5, 6], []), ([1, 2, 5, 7, 9, 11], [3]),  # complex: sibling-group loads
             ([1, 3, 6, 8], [0]), ([0, 3, 4, 6, 7], [1])]  # the last two: qubit 0 or 1 a control
    if real:
        cases += [([0, 1, 2, 3, 4, 5], [6]), ([0, 1, 3, 5, 7, 9], [2, 4]), ([1, 2, 3, 4, 5, 6], []),
                  ([0, 1, 2, 3, 9, 13], []), ([0, 1, 2, 9, 13, 15], []),
                  ([0, 2, 4, 6, 8, 10], [1]), ([6, 5, 4, 3, 2, 0], [13, 14])]
    c_all = qs.Circuit(n)
    ref_all = psi.copy()
    for t, ctl in cases:
        D = 1 << len(t)
        if real:
            Q, _ = np.linalg.qr(rng.standard_normal((D, D)))
            U = Q.astype(np.complex128)
        else:
            U = synth.haar_unitary(rng, D)
        c_all.add_gate(t, U, ctl)
        ocore.apply_gate(ref_all, t, U, ctl)
        ref = psi.copy()
        ocore.apply_gate(ref, t, U, ctl)
        st = dev_state(psi, dtype)
        before = qs.qsim_launch_counts()["dense_tc"]
        qs.qsim_apply(st, qs.Circuit(n).add_gate(t, U, ctl))
        torch.cuda.synchronize()
        assert qs.qsim_device_status() == 0
        assert qs.qsim_launch_counts()["dense_tc"] - before == 1, (t, ctl)
        check(st, ref, dtype)
    st = dev_state(psi, dtype)
    qs.qsim_apply(st, c_all)
    torch.cuda.synchronize()
    check(st, ref_all, dtype)


def test_widened_small_gates_on_low_qubits(qs, tc_on):
    """complex64 gates of 1..3 targets on qubit 0 or 1 run widened to the 6-target transposed
    tensor-core form on states of at least 2^24 amplitudes (one tensor-core launch each), and stay
    in the SIMT kernels with qubit 0 or 1 a control or on smaller states."""
    tc_on(6)
    dtype = torch.complex64
    rng = np.random.default_rng(79)
    cases = [(24, [0], [], 1), (24, [1], [7], 1), (24, [1, 0], [], 1), (24, [0, 2], [3], 1),
             (24, [1, 5], [], 1), (24, [0, 1, 2], [], 1), (24, [3, 1, 2], [23], 1),
             (24, [0, 3, 7], [1], 0), (24, [4, 9], [], 0), (20, [0, 1], [], 0)]
    for n, t, ctl, expect_tc in cases:
        psi = host_input(synth.gaussian_state_np(80 + n, n), dtype)
        U = synth.haar_unitary(rng, 1 << len(t))
        ref = psi.copy()
        ocore.apply_gate(ref, t, U, ctl)
        st = dev_state(psi, dtype)
        before = qs.qsim_launch_counts()["dense_tc"]
        qs.qsim_apply(st, qs.Circuit(n).add_gate(t, U, ctl))
        torch.cuda.synchronize()
        assert qs.qsim_device_status() == 0
        assert qs.qsim_launch_counts()["dense_tc"] - before == expect_tc, (n, t, ctl)
        check(st, ref, dtype)


@pytest.mark.parametrize("dtype", DTYPES)
def test_real_matrix_gates(qs, dtype):
    """Real orthogonal gates (the eigenvector matrices of real symmetric systems) run the SIMT
    kernels' real-matrix variant (two multiply-adds per entry), k = 1..7, with low, high and
    random targets and a control; k = 7 on complex64 uses the wider tile, or the real tensor-core
    form when qubits 0 and 1 are targets."""
    rng = np.random.default_rng(61)
    n = 15
    psi = host_input(synth.gaussian_state_np(61, n), dtype)
    c = qs.Circuit(n)
    ref = psi.copy()
    for k in range(1, 8):
        cases = [(list(range(k)), []), (synth.random_targets(rng, n, k), []),
                 ([n - 1 - i for i in range(k)], [0] if k < 7 else [])]
        if k == 7:  # the complex64 tensor-core form for real 7-target gates on the lowest qubits
            cases += [([1, 0, 6, 5, 4, 3, 2], [n - 1]), (list(range(7)), [9, 12])]
        for t, ctl in cases:
            Q, _ = np.linalg.qr(rng.standard_normal((1 << k, 1 << k)))
            c.add_gate(t, Q, ctl)
            ocore.apply_gate(ref, t, Q.astype(np.complex128), ctl)
    st = dev_state(psi, dtype)
    qs.qsim_apply(st, c)
    torch.cuda.synchronize()
    check(st, ref, dtype)


@pytest.mark.parametrize("k", [3, 4, 5, 6])
def test_tensor_core_low_target_layouts(qs, k, tc_on):
    """Gates whose targets include qubits 0 and 1 (vector loads across a group's amplitudes,
    shuffle-transposed stores), in any given order, with scattered upper targets and controls;
    and gates with qubit 0 but not qubit 1 (the group-major layout)."""
    tc_on(k)
    rng = np.random.default_rng(900 + k)
    n = 19
    psi = host_input(synth.gaussian_state_np(900 + k, n), torch.complex64)
    c = qs.Circuit(n)
    ref = psi.copy()
    up = [int(q) for q in rng.permutation(range(2, n))]
    cases = [([1, 0] + up[:k - 2], []),
             (up[:k - 2][::-1] + [0, 1], [up[k]]),
             (list(range(k)), [n - 1, n - 2]),
             ([0] + up[:k - 1], []),
             ([1] + up[:k - 1], [0])]
    for t, ctl in cases:
        U = synth.haar_unitary(rng, 1 << k)
        c.add_gate(t, U, ctl)
        ocore.apply_gate(ref, t, U, ctl)
    st = dev_state(psi, torch.complex64)
    qs.qsim_apply(st, c)
    torch.cuda.synchronize()
    assert qs.qsim_device_status() == 0
    check(st, ref, torch.complex64)


@pytest.mark.parametrize("dtype", DTYPES)
def test_control_on_low_qubits_and_small_states(qs, dtype):
    rng = np.random.default_rng(7)
    for n in (3, 5, 9):
        psi = host_input(synth.gaussian_state_np(n, n), dtype)
        c = qs.Circuit(n)
        ref = psi.copy()
        for _ in range(6):
            k = int(rng.integers(1, min(3, n - 1) + 1))
            q = [int(v) for v in rng.permutation(n)]
            t, ctl = q[:k], [0] if 0 not in q[:k] else []
            U = synth.haar_unitary(rng, 1 << k)
            c.add_gate(t, U, ctl)
            ocore.apply_gate(ref, t, U, ctl)
        U = synth.haar_unitary(rng, 1 << n) if n <= 7 else None
        if U is not None:                                 # gate on every qubit: one tile
            c.add_gate(list(range(n))[::-1], U)
            ocore.apply_gate(ref, list(range(n))[::-1], U)
        st = dev_state(psi, dtype)
        qs.qsim_apply(st, c)
        torch.cuda.synchronize()
        check(st, ref, dtype)


@pytest.mark.parametrize("dtype", DTYPES)
def test_empty_circuit_is_identity(qs, dtype):
    psi = host_input(synth.gaussian_state_np(1, 10), dtype)
    st = dev_state(psi, dtype)
    qs.qsim_apply(st, qs.Circuit(10))
    torch.cuda.synchronize()
    check(st, psi, dtype)


@pytest.mark.parametrize("dtype", DTYPES)
def test_specialised_ops_parity(qs, dtype):
    rng = np.random.default_rng(3)
    n = 13
    psi = host_input(synth.gaussian_state_np(3, n), dtype)
    c = qs.Circuit(n)
    ref = psi.copy()

    def add(t, U, ctl=()):
        c.add_gate(t, U, list(ctl))
        ocore.apply_gate(ref, t, U, list(ctl))

    add([0, 7], np.diag([1, 1, 1, np.exp(0.7j)]))                    # phase, low + high
    add([12, 3], np.diag([1, 1, 1, np.exp(-1.3j)]))
    add([5], np.diag([1, np.exp(0.2j)]), [9, 1])                      # controlled phase
    add([4], np.diag([np.exp(0.4j), np.exp(-0.9j)]))                  # diagonal
    add([2, 11], np.diag(np.exp(1j * rng.uniform(0, 6, 4))), [6])     # controlled diagonal
    sw = np.eye(4)[[0, 2, 1, 3]]
    add([0, 12], sw)
    add([3, 8], sw, [10])
    theta = rng.uniform(-3, 3, size=16)
    c.add_ucry(12, [4, 5, 6, 7], theta)                               # contiguous register
    ocore.apply_ucry(ref, 12, [4, 5, 6, 7], theta)
    theta2 = rng.uniform(-3, 3, size=8)
    c.add_ucry(1, [9, 0, 6], theta2)                                  # scattered register
    ocore.apply_ucry(ref, 1, [9, 0, 6], theta2)
    info = c.info()
    assert info["n_diag"] == 5 and info["n_perm"] == 2 and info["n_ucry"] == 2
    st = dev_state(psi, dtype)
    qs.qsim_apply(st, c)
    torch.cuda.synchronize()
    check(st, ref, dtype)


def random_small_gate_circuit(rng, n, count):
    H = np.array([[1, 1], [1, -1]]) / math.sqrt(2)
    out = []
    for _ in range(count):
        r = rng.random()
        if r < 0.3:
            out.append(([int(rng.integers(n))], H))
        elif r < 0.55:
            out.append((synth.random_targets(rng, n, 2),
                        np.diag([1, 1, 1, np.exp(1j * rng.uniform(-3, 3))])))
        elif r < 0.65:
            out.append((synth.random_targets(rng, n, 2), np.eye(4)[[0, 2, 1, 3]]))
        elif r < 0.85:
            out.append(([int(rng.integers(n))], synth.haar_unitary(rng, 2)))
        else:
            out.append((synth.random_targets(rng, n, 2), synth.haar_unitary(rng, 4)))
    return out


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("max_k", [1, 2, 3, 4, 5, 6])
def test_fusion_parity(qs, dtype, max_k):
    rng = np.random.default_rng(40 + max_k)
    n = 12
    gates = random_small_gate_circuit(rng, n, 150)
    psi = host_input(synth.gaussian_state_np(9, n), dtype)
    ref = psi.copy()
    c = qs.Circuit(n)
    for t, U in gates:
        c.add_gate(t, U)
        ocore.apply_gate(ref, t, U)
    f = qs.qsim_fuse(c, max_k)
    fi = f.info()
    # gates wider than max_k pass through unfused
    assert fi["max_k"] <= max(max_k, 2) and fi["n_gates"] <= 150
    st = dev_state(psi, dtype)
    qs.qsim_apply(st, f)
    torch.cuda.synchronize()
    check(st, ref, dtype)


# ------------------------------------------------------------------------------- HHL
def run_product_hhl(qs, h, dtype, max_k):
    info = h.info()
    circ = h.as_circuit()
    if max_k:
        circ = qs.qsim_fuse(circ, max_k)
    st = torch.empty(1 << info["n"], dtype=dtype, device="cuda")
    qs.hhl_prepare_state(st, h)
    qs.qsim_apply(st, circ, n_qubits=info["n"])
    r = qs.hhl_readout(st, h)
    return st, r


def compare_hhl(st, r, ref, dtype, tol_state):
    """State element by element within tol_state (and fidelity for complex64); the readout
    within the bounds that the state bound implies (tests/hhl_bounds.py)."""
    out = st.cpu().numpy().astype(np.complex128)
    err = np.max(np.abs(out - ref["psi"]))
    assert err <= tol_state, "state max|d| %.3e > %.1e" % (err, tol_state)
    if dtype == torch.complex64:
        f = abs(np.vdot(ref["psi"], out)) ** 2 / np.vdot(out, out).real
        assert f >= 1 - 1e-6
    h = ref["circuit"]
    xs_b = readout_bounds(ref, h["nb"], h["m"], tol_state, h["C"], h["bnorm"], 1 << h["nb"])
    assert abs(r["p_success"] - ref["P"]) <= xs_b["P"]
    assert abs(r["p_clock0"] - ref["P0"]) <= xs_b["P0"]
    assert abs(r["norm2"] - ref["norm2"]) <= prob_bound(ref["psi"], tol_state)
    assert np.all(np.abs(r["x_state"] - ref["x_state"]) <= xs_b["x_state"])
    N = len(ref["x"])
    off = len(ref["x_eff"]) - N if "x_eff" in ref else 0
    x_b = readout_bounds(ref, h["nb"], h["m"], tol_state, h["C"], h["bnorm"], N, off)
    assert np.all(np.abs(r["x"] - ref["x"]) <= x_b["x"])


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("max_k", [0, 2, 4, 6])
def test_hhl7_parity_and_exact_grid(qs, dtype, max_k):
    p = synth.hhl7_problem()
    h = qs.hhl_build(p["A"], p["b"], p["m"], p["t"], p["C"])
    ref = ohhl.solve(p["A"], p["b"], p["m"], p["t"], p["C"])
    st, r = run_product_hhl(qs, h, dtype, max_k)
    compare_hhl(st, r, ref, dtype, TOL[dtype])
    xt = np.linalg.solve(p["A"], p["b"])
    rel = np.max(np.abs(r["x"] - xt)) / np.linalg.norm(xt)
    assert rel < (1e-11 if dtype == torch.complex128 else 1e-4)
    if dtype == torch.complex128:
        assert abs(r["leakage"]) < 1e-13


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("max_k", [0, 3, 6])
def test_hhl7_structured_qpe_parity(qs, dtype, max_k):
    """Diagonalised phase estimation vs the oracle's controlled-evolution circuit."""
    p = synth.hhl7_problem()
    h = qs.hhl_build(p["A"], p["b"], p["m"], p["t"], p["C"], structured=True)
    ref = ohhl.solve(p["A"], p["b"], p["m"], p["t"], p["C"])
    st, r = run_product_hhl(qs, h, dtype, max_k)
    compare_hhl(st, r, ref, dtype, TOL[dtype])


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_hhl_structured_offgrid_parity(qs, dtype, seed):
    rng = np.random.default_rng(seed)
    nb = int(rng.integers(2, 5))
    m = int(rng.integers(5, 9))
    A, b = synth.contingency_system(rng, 2 ** nb + 1)
    h = qs.hhl_build(A, b, m, structured=True)
    ref = ohhl.solve(A, b, m)
    st, r = run_product_hhl(qs, h, dtype, 4)
    tol = cond_tol(m) if dtype == torch.complex128 else TOL[dtype]
    compare_hhl(st, r, ref, dtype, tol)


@pytest.mark.parametrize("dtype", DTYPES)
def test_hhl_structured_spectral_large_clock(qs, dtype):
    rng = np.random.default_rng(21)
    N, m = 6, 12
    V = synth.haar_unitary(rng, N)
    lam = np.sort(rng.uniform(0.5, 9.0, size=N))
    b = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    t = 2 * math.pi * (2 ** m - 1) / (2 ** m * 9.0)
    h = qs.hhl_build_spectral(lam, V, b, m, t, 0.4, structured=True)
    ref = _oracle_spectral(lam, V, b, m, t, 0.4)
    st, r = run_product_hhl(qs, h, dtype, 4)
    compare_hhl(st, r, ref, dtype, 1e-12 if dtype == torch.complex128 else TOL[dtype])


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_hhl_offgrid_contingency_parity(qs, dtype, seed):
    rng = np.random.default_rng(seed)
    nb = int(rng.integers(2, 5))
    m = int(rng.integers(5, 9))
    A, b = synth.contingency_system(rng, 2 ** nb + 1)
    h = qs.hhl_build(A, b, m)
    ref = ohhl.solve(A, b, m)
    st, r = run_product_hhl(qs, h, dtype, 4)
    tol = cond_tol(m) if dtype == torch.complex128 else TOL[dtype]
    compare_hhl(st, r, ref, dtype, tol)


@pytest.mark.parametrize("dtype", DTYPES)
def test_hhl_spectral_path_large_clock(qs, dtype):
    """Shared spectral decomposition: 1e-12 holds even with 12 clock qubits, off-grid."""
    rng = np.random.default_rng(21)
    N, m = 6, 12
    V = synth.haar_unitary(rng, N)
    lam = np.sort(rng.uniform(0.5, 9.0, size=N))
    b = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    t = 2 * math.pi * (2 ** m - 1) / (2 ** m * 9.0)
    C = 0.4
    h = qs.hhl_build_spectral(lam, V, b, m, t, C)
    ref = _oracle_spectral(lam, V, b, m, t, C)
    st, r = run_product_hhl(qs, h, dtype, 4)
    compare_hhl(st, r, ref, dtype, TOL[dtype])


def _oracle_spectral(lam, V, b, m, t, C):
    """Oracle HHL with a given spectrum: feed the oracle's builder A's eigendata through a
    matrix whose eigh reproduces it, then replace the controlled evolutions by ones computed
    from (lam, V) directly (the oracle's own formula U_j = V diag(e^{i lam t 2^j}) V^H)."""
    N = len(lam)
    A = (V * lam) @ V.conj().T
    A = 0.5 * (A + A.conj().T)
    h = ohhl.build(A, b, m, t, C)
    D = 1 << h["nb"]
    lam_p = np.concatenate([lam, np.full(D - N, lam.max())])
    Vp = np.eye(D, dtype=np.complex128)
    Vp[:N, :N] = V
    gates = []
    forward = True
    for g in h["gates"]:
        if g[0] == "ucry":
            forward = False
            gates.append(g)
            continue
        if g[3]:  # controlled evolution
            jj = g[3][0] - h["nb"]
            Uj = (Vp * np.exp(1j * lam_p * t * 2 ** jj)) @ Vp.conj().T
            gates.append(("u", g[1], Uj if forward else Uj.conj().T, g[3], g[4]))
        else:
            gates.append(g)
    h["gates"] = gates
    psi = ohhl.run(h)
    out = ohhl.readout(h, psi)
    out["psi"] = psi
    out["circuit"] = h
    return out


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n", [7, 16, 23])
def test_readout_sums_match_compensated_fp64(qs, dtype, n):
    """||psi||^2, P(ancilla = 1) and P(ancilla = 1, clock = 0) of an arbitrary state against the
    oracle's compensated FP64 sums of the same (rounded) amplitudes: relative 1e-13 for both
    dtypes (complex64 squares are formed exactly and summed in double-single groups)."""
    m = n - 2
    h = qs.hhl_build_spectral([1.0, 3.0], np.eye(2), [1.0, 0.5], m)
    psi = synth.gaussian_state_np(40 + n, n)
    psi[::7] *= 1e-6                                  # a wide dynamic range
    psi = host_input(psi, dtype)
    st = dev_state(psi, dtype)
    r = qs.hhl_readout(st, h)
    anc = 1 << (n - 1)
    clock = ((1 << m) - 1) << 1
    want = {"norm2": ocore.masked_norm2(psi, 0, 0), "p_success": ocore.masked_norm2(psi, anc, anc),
            "p_clock0": ocore.masked_norm2(psi, anc | clock, anc)}
    for key, v in want.items():
        assert abs(r[key] - v) <= 1e-13 * v, (key, r[key], v)


# --------------------------------------------------------------- full-size sampled checks
@pytest.mark.parametrize("dtype,n", [(torch.complex128, 30), (torch.complex64, 31)])
def test_full_size_gate_apply_sampled(qs, dtype, n):
    """At the benchmark's sizes: one Haar gate per k applied to the seeded Gaussian state; 48
    sampled groups per gate recomputed by the oracle from the generator's amplitudes."""
    free = torch.cuda.mem_get_info()[0]
    if free < (1 << n) * (16 if dtype == torch.complex128 else 8) * 1.3:
        pytest.skip("not enough device memory")
    seed = 77
    gates = synth.gate_microbench_list(seed, n, per_k=1)
    rng = np.random.default_rng(5)
    for t, U in gates:
        st = synth.gaussian_state_torch(seed, n, dtype, "cuda")
        c = qs.Circuit(n).add_gate(t, U)
        qs.qsim_apply(st, c)
        torch.cuda.synchronize()
        k = len(t)
        others = [q for q in range(n) if q not in t]
        offs = np.array([sum(((r >> b) & 1) << t[b] for b in range(k)) for r in range(1 << k)],
                        dtype=np.int64)
        for _ in range(48):
            base = 0
            for q in others:
                if rng.random() < 0.5:
                    base |= 1 << q
            idx = base + offs
            x = synth.gaussian_amplitudes_at(seed, n, idx.astype(np.uint64))
            x = host_input(x, dtype)
            ocore.apply_gate(x, list(range(k)), U)     # the group as a k-qubit system
            got = st[torch.from_numpy(idx).cuda()].cpu().numpy().astype(np.complex128)
            assert np.max(np.abs(got - x)) <= TOL[dtype]
        del st
        torch.cuda.empty_cache()


def _sample_groups(rng, n, group_qubits, count):
    """`count` random assignments of the qubits outside `group_qubits`, as base indices."""
    others = [q for q in range(n) if q not in group_qubits]
    bases = []
    for _ in range(count):
        base = 0
        for q in others:
            if rng.random() < 0.5:
                base |= 1 << q
        bases.append(base)
    return bases


@pytest.mark.parametrize("dtype,n", [(torch.complex64, 34), (torch.complex128, 33)])
def test_maximum_size_sampled(qs, dtype, n):
    """The largest states the library accepts (2^34 complex64 = 2^33 complex128 = 128 GiB,
    amplitude indices beyond 2^32): a dense gate on the top qubit, a dense gate with random
    targets (tensor cores for complex64), a Fourier pass on the top 10 qubits with a twiddle and
    a Walsh-Hadamard pass on scattered qubits, each on the seeded state, checked on sampled
    groups recomputed by the oracle from the generator's amplitudes."""
    free = torch.cuda.mem_get_info()[0]
    if free < (1 << n) * (16 if dtype == torch.complex128 else 8) * 1.15:
        pytest.skip("not enough device memory")
    seed, rng = 91, np.random.default_rng(8)
    k2 = 6 if dtype == torch.complex64 else 3
    U1 = synth.haar_unitary(rng, 2)
    t2 = [n - 1] + [int(q) for q in rng.permutation(n - 1)[:k2 - 1]]
    U2 = synth.haar_unitary(rng, 1 << k2)
    field, src = list(range(n - 10, n)), list(range(n - 13, n - 10))
    walsh = [0, 5, 17, n - 1]

    def apply_and_get(build):
        st = synth.gaussian_state_torch(seed, n, dtype, "cuda")
        c = qs.Circuit(n)
        build(c)
        qs.qsim_apply(st, c)
        torch.cuda.synchronize()
        return st

    def check_groups(st, qubits, bases, expect):
        offs = np.array([sum(((r >> b) & 1) << qubits[b] for b in range(len(qubits)))
                         for r in range(1 << len(qubits))], dtype=np.int64)
        for base in bases:
            idx = base + offs
            x = host_input(synth.gaussian_amplitudes_at(seed, n, idx.astype(np.uint64)), dtype)
            want = expect(x, base)
            got = st[torch.from_numpy(idx).cuda()].cpu().numpy().astype(np.complex128)
            assert np.max(np.abs(got - want)) <= TOL[dtype]

    def dense(U, k):
        def f(x, base):
            ocore.apply_gate(x, list(range(k)), U)
            return x
        return f

    def fourier(x, base):  # the group as a (10 + 3)-qubit system with the source bits of base
        w = sum(((base >> q) & 1) << j for j, q in enumerate(src))
        mini = np.zeros(1 << 13, dtype=np.complex128)
        mini[w << 10: (w << 10) + 1024] = x
        ohhl.dft_pass(mini, list(range(10)), -1, [10, 11, 12], False)
        return mini[w << 10: (w << 10) + 1024]

    def hadamards(x, base):
        for q in range(4):
            ocore.apply_gate(x, [q], ohhl.H)
        return x

    for qubits, build, expect, count in (
            ([n - 1], lambda c: c.add_gate([n - 1], U1), dense(U1, 1), 64),
            (t2, lambda c: c.add_gate(t2, U2), dense(U2, k2), 32),
            (field, lambda c: c.add_dft(field, -1, src), fourier, 8),
            (walsh, lambda c: c.add_walsh(walsh), hadamards, 32)):
        st = apply_and_get(build)
        check_groups(st, qubits, _sample_groups(rng, n, qubits, count), expect)
        del st
        torch.cuda.empty_cache()


@pytest.mark.parametrize("dtype,n", [(torch.complex128, 30), (torch.complex64, 31)])
def test_full_size_forward_inverse_roundtrip(qs, dtype, n):
    """Property at full size: the benchmark's gate kinds (4 per k) followed by their inverses
    return the state to itself, and the norm is preserved."""
    seed = 78
    st = synth.gaussian_state_torch(seed, n, dtype, "cuda")
    x0 = st.clone()
    gates = synth.gate_microbench_list(seed, n, per_k=4)
    c = qs.Circuit(n)
    for t, U in gates:
        c.add_gate(t, U)
    for t, U in reversed(gates):
        c.add_gate(t, U.conj().T)
    n0 = torch.linalg.vector_norm(torch.view_as_real(x0), dtype=torch.float64).item()
    qs.qsim_apply(st, c)
    torch.cuda.synchronize()
    err = (st - x0).abs().max().item()
    n1 = torch.linalg.vector_norm(torch.view_as_real(st), dtype=torch.float64).item()
    assert err <= TOL[dtype]
    if dtype == torch.complex128:
        assert abs(n1 - n0) <= 1e-12
    else:
        # a complex64 dense gate on 2^k amplitudes changes the norm by at most ~2^k * 2^-22
        # relative (FP32 dot products of length 2^(k+1); 3xTF32 keeps ~22 bits per product)
        bound = 2 * sum(2.0 ** len(t) for t, _ in gates) * 2.0 ** -22
        assert abs(n1 - n0) / n0 <= bound
        ov = 0j
        for s0 in range(0, x0.numel(), 1 << 28):   # torch.vdot takes < 2^31 elements
            ov += torch.vdot(x0[s0:s0 + (1 << 28)].to(torch.complex128),
                             st[s0:s0 + (1 << 28)].to(torch.complex128)).item()
        fid = abs(ov) ** 2 / (n0 ** 2 * n1 ** 2)
        assert fid >= 1 - 1e-6


# ------------------------------------------------------------------ degenerate HHL systems
def _degenerate_cases():
    rng = np.random.default_rng(77)
    yield "1x1", np.array([[3.0]]), np.array([2.0]), 4, 2 * math.pi / 16, 0.0
    yield "scaled identity", 5.0 * np.eye(4), rng.standard_normal(4), 5, 0.0, 0.0
    A, _, _ = synth.grid_system(rng, 9)
    w, V = np.linalg.eigh(A)
    yield "b is an eigenvector", A, V[:, 3].astype(np.complex128), 6, 0.0, 0.0
    # eigenvalues far below the first grid step: clock value 0 carries weight, theta_0 = 0
    A2 = np.diag([1e-3, 0.5, 40.0, 100.0])
    yield "eigenvalues under the grid", A2, np.ones(4), 4, 0.0, 0.0


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("case", list(range(4)))
def test_hhl_degenerate_systems(qs, dtype, case):
    name, A, b, m, t, C = list(_degenerate_cases())[case]
    for structured in (False, True):
        h = qs.hhl_build(A, b, m, t, C, structured=structured)
        ref = ohhl.solve(A, b, m, t, C)
        st, r = run_product_hhl(qs, h, dtype, 3)
        tol = cond_tol(m) if dtype == torch.complex128 else TOL[dtype]
        compare_hhl(st, r, ref, dtype, tol)



# ------------------------------------------------------------ indefinite systems (sign qubit)
def _indefinite(seed, N, m, grid):
    rng = np.random.default_rng(seed)
    V = synth.haar_unitary(rng, N)
    if grid:
        top = 2 ** (m - 1) - 1
        lam = rng.integers(1, top + 1, size=N).astype(float) * rng.choice([-1.0, 1.0], size=N)
        lam[0], lam[-1] = -top, top
    else:
        lam = rng.uniform(0.5, 10.0, size=N) * rng.choice([-1.0, 1.0], size=N)
        lam[0] = -abs(lam[0])
    A = (V * lam) @ V.conj().T
    return 0.5 * (A + A.conj().T), rng.standard_normal(N) + 1j * rng.standard_normal(N)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("structured", [False, True])
def test_hhl_indefinite_exact_grid(qs, dtype, structured):
    m, N = 6, 5
    A, b = _indefinite(3, N, m, grid=True)
    t = 2 * math.pi / 2 ** m
    h = qs.hhl_build(A, b, m, t, structured=structured)
    ref = ohhl.solve(A, b, m, t)
    st, r = run_product_hhl(qs, h, dtype, 3)
    compare_hhl(st, r, ref, dtype, TOL[dtype])
    xt = np.linalg.solve(A, b)
    assert np.linalg.norm(r["x"] - xt) / np.linalg.norm(xt) < (1e-10 if dtype == torch.complex128 else 1e-4)


@pytest.mark.parametrize("dtype", DTYPES)
def test_hhl_indefinite_offgrid(qs, dtype):
    m = 8
    A, b = _indefinite(4, 6, m, grid=False)
    h = qs.hhl_build(A, b, m, structured=True)
    ref = ohhl.solve(A, b, m)
    st, r = run_product_hhl(qs, h, dtype, 3)
    compare_hhl(st, r, ref, dtype, cond_tol(m) if dtype == torch.complex128 else TOL[dtype])


# ------------------------------------------- Gauss-Seidel preconditioning, Hermitian dilation
@pytest.mark.parametrize("dtype", DTYPES)
def test_dilation_exact_grid(qs, dtype):
    rng = np.random.default_rng(31)
    N, m = 3, 6
    U, W = synth.haar_unitary(rng, N), synth.haar_unitary(rng, N)
    A = (U * np.array([2.0, 5.0, 31.0])) @ W.conj().T
    b = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    t = 2 * math.pi / 2 ** m
    for structured in (False, True):
        h = qs.hhl_build(A, b, m, t, dilate=True, structured=structured)
        ref = ohhl.solve_general(A, b, m, t)
        st, r = run_product_hhl(qs, h, dtype, 3)
        compare_hhl(st, r, ref, dtype, TOL[dtype])
        xt = np.linalg.solve(A, b)
        assert np.linalg.norm(r["x"] - xt) / np.linalg.norm(xt) < (1e-10 if dtype == torch.complex128 else 1e-4)


@pytest.mark.parametrize("dtype", DTYPES)
def test_gauss_seidel_dilated_offgrid(qs, dtype):
    rng = np.random.default_rng(8)
    A, b, _ = synth.grid_system(rng, 9)
    m = 9
    h = qs.hhl_build(A, b, m, gauss_seidel=True, structured=True)
    ref = ohhl.solve_general(A, b, m, gauss_seidel=True)
    st, r = run_product_hhl(qs, h, dtype, 3)
    # Both sides form A' = M^-1 A with their own triangular solve: the results differ by up to
    # cond(M) eps relative (forward error of a triangular solve), which the dilation's
    # eigenvalues inherit; the phase estimation amplifies that like any eigenvalue rounding.
    condM = np.linalg.cond(np.tril(A))
    compare_hhl(st, r, ref, dtype, cond_tol(m) * max(1.0, condM) if dtype == torch.complex128 else TOL[dtype])


def test_dilated_batch_readout_offset(qs):
    """The batched executor returns x from the lower half of the dilated slice."""
    rng = np.random.default_rng(12)
    probs = []
    for _ in range(3):
        N = 3
        U, W = synth.haar_unitary(rng, N), synth.haar_unitary(rng, N)
        probs.append(((U * np.array([1.0, 3.0, 7.0])) @ W.conj().T, rng.standard_normal(N)))
    m, t = 4, 2 * math.pi / 16
    hs = [qs.hhl_build(A, b, m, t, dilate=True, structured=True) for A, b in probs]
    fused = [qs.qsim_fuse(h.as_circuit(), 3) for h in hs]
    states = [torch.empty(1 << h.info()["n"], dtype=torch.complex128, device="cuda") for h in hs]
    bt = qs.hhl_batch_create(hs, states, fused)
    bt.run()
    for (A, b), r in zip(probs, bt.results()):
        xt = np.linalg.solve(A, b)
        assert np.linalg.norm(r["x"] - xt) / np.linalg.norm(xt) < 1e-10
