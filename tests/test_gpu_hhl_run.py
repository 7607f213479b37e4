"""hhl_run (state preparation plus the circuit, every operation before the first one on the
ancilla run on the lower half of the state, which is exactly zero above) against
hhl_prepare_state + qsim_apply of the same circuit and against the FP64 oracle.  The state is
filled with NaN first: an amplitude that hhl_run reads before writing would poison the
result."""
import math

import numpy as np
import pytest
import torch

import synth
from oracle import core as ocore
from oracle import hhl as ohhl

DTYPES = [torch.complex128, torch.complex64]
TOL = {torch.complex128: 1e-12, torch.complex64: 1e-5}


@pytest.fixture(scope="module")
def qs():
    from paper_2402_08136_gb300 import build
    build.build()
    import paper_2402_08136_gb300 as q
    return q


def nan_state(n, dtype):
    return torch.full((1 << n,), complex(float("nan"), float("nan")), dtype=dtype, device="cuda")


def both_ways(qs, h, circ, dtype):
    n = h.info()["n"]
    a = nan_state(n, dtype)
    qs.hhl_run(a, h, circ)
    b = torch.empty(1 << n, dtype=dtype, device="cuda")
    qs.hhl_prepare_state(b, h)
    qs.qsim_apply(b, circ if circ is not None else h.as_circuit(), n_qubits=n)
    torch.cuda.synchronize()
    a_np = a.cpu().numpy().astype(np.complex128)
    b_np = b.cpu().numpy().astype(np.complex128)
    assert np.all(np.isfinite(a_np)), "hhl_run left or read unwritten amplitudes"
    return a, a_np, b_np


FORMS = [("gates", 0), ("gates", 4), ("structured", 3), ("structured_fft", 4), ("structured_fft", 0)]


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("form,max_k", FORMS)
@pytest.mark.parametrize("problem", ["hhl7", "contingency"])
def test_hhl_run_matches_two_step_path_and_oracle(qs, cuda_device, dtype, form, max_k, problem):
    if problem == "hhl7":
        p = synth.hhl7_problem()
        A, b, m, t, C = p["A"], p["b"], p["m"], p["t"], p["C"]
    else:
        A, b = synth.contingency_system(np.random.default_rng(5), 9)
        m, t, C = 7, 0.0, 0.0
    h = qs.hhl_build(A, b, m, t, C, structured=form != "gates", fft_qft=form == "structured_fft")
    circ = qs.qsim_fuse(h.as_circuit(), max_k) if max_k else None
    st, a_np, b_np = both_ways(qs, h, circ, dtype)
    # same operations on the same values: equal up to rounding of the reordered launches
    assert np.max(np.abs(a_np - b_np)) <= TOL[dtype] / 10
    ref = ohhl.solve(A, b, m, t, C)
    tol = max(TOL[dtype], 2.0 ** m * 2 * math.pi * 8 * np.finfo(float).eps) if dtype == torch.complex128 \
        else TOL[dtype]
    assert np.max(np.abs(a_np - ref["psi"])) <= tol
    r = qs.hhl_readout(st, h)
    assert abs(r["p_success"] - ref["P"]) <= 10 * tol
    assert abs(r["norm2"] - 1.0) <= (1e-12 if dtype == torch.complex128 else 1e-5)


def reference_state(p):
    """|0>|0>|b> from the oracle (complex128)."""
    return ohhl.initial_state(ohhl.build(p["A"], p["b"], p["m"], p["t"], p["C"]))


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", DTYPES)
def test_hhl_run_first_top_operation_not_an_inversion(qs, cuda_device, dtype):
    """A dense gate reaches the ancilla first: the upper half is zeroed before it."""
    p = synth.hhl7_problem()
    h = qs.hhl_build(p["A"], p["b"], p["m"], p["t"], p["C"])
    n = h.info()["n"]
    rng = np.random.default_rng(3)
    gates = [([1, 2], synth.haar_unitary(rng, 4)), ([n - 1, 0], synth.haar_unitary(rng, 4)),
             ([3, 4, 5], synth.haar_unitary(rng, 8)), ([n - 1], synth.haar_unitary(rng, 2))]
    c = qs.Circuit(n)
    for t, U in gates:
        c.add_gate(t, U)
    _, a_np, b_np = both_ways(qs, h, c, dtype)
    ref = reference_state(p)
    for t, U in gates:
        ocore.apply_gate(ref, t, U)
    assert np.max(np.abs(a_np - b_np)) <= TOL[dtype] / 10
    assert np.max(np.abs(a_np - ref)) <= TOL[dtype]


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", DTYPES)
def test_hhl_run_rotation_on_the_ancilla_first(qs, cuda_device, dtype):
    """A uniformly controlled RY on the ancilla is the first operation on it: it writes the upper
    half without reading it."""
    p = synth.hhl7_problem()
    h = qs.hhl_build(p["A"], p["b"], p["m"], p["t"], p["C"])
    n = h.info()["n"]
    rng = np.random.default_rng(4)
    U = synth.haar_unitary(rng, 8)
    reg = [2, 3, 4]
    th = rng.uniform(-3, 3, size=8)
    U2 = synth.haar_unitary(rng, 4)
    c = qs.Circuit(n).add_gate([0, 1, 5], U).add_ucry(n - 1, reg, th).add_gate([n - 1, 2], U2)
    _, a_np, b_np = both_ways(qs, h, c, dtype)
    assert np.max(np.abs(a_np - b_np)) <= TOL[dtype] / 10
    ref = reference_state(p)
    ocore.apply_gate(ref, [0, 1, 5], U)
    ocore.apply_ucry(ref, n - 1, reg, th)
    ocore.apply_gate(ref, [n - 1, 2], U2)
    assert np.max(np.abs(a_np - ref)) <= 10 * TOL[dtype]


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", DTYPES)
def test_hhl_run_circuit_that_never_touches_the_ancilla(qs, cuda_device, dtype):
    """No operation on the ancilla: the upper half is zeroed at the end."""
    p = synth.hhl7_problem()
    h = qs.hhl_build(p["A"], p["b"], p["m"], p["t"], p["C"])
    n = h.info()["n"]
    rng = np.random.default_rng(6)
    c = qs.Circuit(n).add_gate([0, 4], synth.haar_unitary(rng, 4)).add_gate([5], synth.haar_unitary(rng, 2))
    _, a_np, b_np = both_ways(qs, h, c, dtype)
    assert np.max(np.abs(a_np - b_np)) <= TOL[dtype] / 10
    assert np.all(a_np[1 << (n - 1):] == 0)


@pytest.mark.gpu
@pytest.mark.parametrize("fft", [False, True])
def test_one_circuit_in_both_dtypes(qs, cuda_device, fft):
    """The same circuit object applied in complex128, then complex64 (its device tables are
    packed per dtype, the structured phase's second and per-chunk tables included)."""
    A, b = synth.contingency_system(np.random.default_rng(8), 9)
    m = 7
    h = qs.hhl_build(A, b, m, structured=True, fft_qft=fft)
    circ = qs.qsim_fuse(h.as_circuit(), 3)
    ref = ohhl.solve(A, b, m)
    n = h.info()["n"]
    for dtype in (torch.complex128, torch.complex64):
        st = torch.empty(1 << n, dtype=dtype, device="cuda")
        qs.hhl_prepare_state(st, h)
        qs.qsim_apply(st, circ, n_qubits=n)
        torch.cuda.synchronize()
        out = st.cpu().numpy().astype(np.complex128)
        tol = max(TOL[dtype], 2.0 ** m * 2 * math.pi * 8 * np.finfo(float).eps) \
            if dtype == torch.complex128 else TOL[dtype]
        assert np.max(np.abs(out - ref["psi"])) <= tol


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("m", [12, 17])
def test_hhl_run_multi_field_clock(qs, cuda_device, dtype, m):
    """Clock registers of two Fourier fields: the inverse QFT's last pass carries the inversion
    rotation into the unwritten upper half, the opening layer expands field by field."""
    A, b = synth.contingency_system(np.random.default_rng(12), 5)
    h = qs.hhl_build(A, b, m, structured=True, fft_qft=True)
    circ = qs.qsim_fuse(h.as_circuit(), 4)
    st, a_np, b_np = both_ways(qs, h, circ, dtype)
    assert np.max(np.abs(a_np - b_np)) <= TOL[dtype] / 10
    ref = ohhl.solve(A, b, m)
    tol = max(TOL[dtype], 2.0 ** m * 2 * math.pi * 8 * np.finfo(float).eps) if dtype == torch.complex128 \
        else TOL[dtype]
    assert np.max(np.abs(a_np - ref["psi"])) <= tol
    r = qs.hhl_readout(st, h)
    assert abs(r["p_success"] - ref["P"]) <= 10 * tol


@pytest.mark.gpu
def test_launch_counter_counts_kernels(qs, cuda_device):
    """qsim_launch_count: one launch per applied gate here, two for the readout reductions."""
    rng = np.random.default_rng(9)
    st = torch.from_numpy(synth.gaussian_state_np(1, 12)).cuda()
    c = qs.Circuit(12).add_gate([0], synth.haar_unitary(rng, 2)).add_gate([3, 4], synth.haar_unitary(rng, 4))
    l0 = qs.qsim_launch_count()
    qs.qsim_apply(st, c)
    torch.cuda.synchronize()
    assert qs.qsim_launch_count() - l0 == 2
    p = synth.hhl7_problem()
    h = qs.hhl_build(p["A"], p["b"], p["m"], p["t"], p["C"])
    s2 = torch.empty(1 << h.info()["n"], dtype=torch.complex128, device="cuda")
    qs.hhl_run(s2, h)
    l1 = qs.qsim_launch_count()
    qs.hhl_readout(s2, h)
    assert qs.qsim_launch_count() - l1 == 2


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", [torch.complex64, torch.complex128])
def test_hhl_run_replays_from_a_cuda_graph(qs, dtype, cuda_device):
    """hhl_run only enqueues stream work after its first call (which uploads the circuit's
    tables), so it can be captured into a CUDA graph: a replay gives the same bits as the eager
    call, solve after solve (the graph rewrites every amplitude it reads)."""
    import synth as _s
    rng = np.random.default_rng(61)
    A, b = _s.contingency_system(rng, 2 ** 4 + 1)
    h = qs.hhl_build(A, b, 18, structured=True, fft_qft=True)
    c = qs.qsim_fuse(h.as_circuit(), 6 if dtype == torch.complex64 else 2)
    n = h.info()["n"]
    st = torch.empty(1 << n, dtype=dtype, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        qs.hhl_run(st, h, c, s)
    s.synchronize()
    eager = st.clone()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        qs.hhl_run(st, h, c, s)
    for _ in range(2):
        st.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(st, eager)


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", [torch.complex64, torch.complex128])
def test_readout_sums_inside_the_run(qs, dtype, cuda_device):
    """hhl_run_sums + hhl_readout_sums against hhl_run + hhl_readout on a 64 x 64 system with
    12 clock qubits (19 qubits): complex64 ends with V on the 6 data qubits in the transposed
    tensor-core form, whose epilogue writes the readout partial sums (no reduction pass of its
    own: one readout launch instead of two); complex128 takes the reduction pass and gives the
    same sums bit for bit.  The kernel adds a tile's 128 squares per thread in FP32 (at most 24
    roundings: within 1.5e-6 of their sum) and the tiles in FP64, so the complex64 sums agree to 2e-6 relative with the
    reduction pass (far inside what the state's own 1e-5 per amplitude allows), the solutions
    likewise; both match the FP64 oracle's P and P0."""
    p = synth.hhl27_problem()
    m = 12
    h = qs.hhl_build(p["A"], p["b"], m, structured=True, fft_qft=True)
    circ = qs.qsim_fuse(h.as_circuit(), 4)
    n = h.info()["n"]
    a = torch.empty(1 << n, dtype=dtype, device="cuda")
    b = torch.empty(1 << n, dtype=dtype, device="cuda")
    sums = torch.full((qs.QSIM_READOUT_SUMS_DOUBLES,), float("nan"), dtype=torch.float64, device="cuda")
    qs.hhl_run(a, h, circ)
    r0 = qs.hhl_readout(a, h)
    c0 = qs.qsim_launch_counts()
    qs.hhl_run_sums(b, h, sums, circ)
    c1 = qs.qsim_launch_counts()
    r1 = qs.hhl_readout_sums(b, h, sums)
    c2 = qs.qsim_launch_counts()
    torch.cuda.synchronize()
    assert torch.equal(a, b)  # the same state either way
    fused = dtype == torch.complex64
    assert c1["readout"] - c0["readout"] == (0 if fused else 1)
    assert c2["readout"] - c1["readout"] == 1
    for key in ("p_success", "p_clock0", "norm2"):
        if fused:
            assert abs(r1[key] - r0[key]) <= 2e-6 * abs(r0[key])
        else:
            assert r1[key] == r0[key]
    assert np.max(np.abs(r1["x"] - r0["x"])) <= 2e-6 * np.max(np.abs(r0["x"]))
    ref = ohhl.solve(p["A"], p["b"], m)
    tol = 1e-5 if fused else max(1e-12, 2.0 ** m * 2 * math.pi * 8 * np.finfo(float).eps)
    bound = 2 * tol * np.sum(np.abs(ref["psi"])) + (1 << n) * tol * tol
    assert abs(r1["p_success"] - ref["P"]) <= bound
    assert abs(r1["p_clock0"] - ref["P0"]) <= bound


@pytest.mark.gpu
def test_readout_sums_replay_from_a_cuda_graph(qs, cuda_device):
    """hhl_run_sums is device-only after its first call: captured once, replayed, read out."""
    p = synth.hhl27_problem()
    h = qs.hhl_build(p["A"], p["b"], 12, structured=True, fft_qft=True)
    circ = qs.qsim_fuse(h.as_circuit(), 4)
    n = h.info()["n"]
    st = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    sums = torch.zeros(qs.QSIM_READOUT_SUMS_DOUBLES, dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        qs.hhl_run_sums(st, h, sums, circ, stream=s)
    s.synchronize()
    r0 = qs.hhl_readout_sums(st, h, sums, stream=s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        qs.hhl_run_sums(st, h, sums, circ, stream=s)
    sums.zero_()
    g.replay()
    r1 = qs.hhl_readout_sums(st, h, sums, stream=s)
    assert r1["p_success"] == r0["p_success"] and r1["p_clock0"] == r0["p_clock0"]
    assert np.array_equal(r1["x"], r0["x"])
