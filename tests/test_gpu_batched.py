"""Batched executor (one persistent launch for many circuits) vs the FP64 oracle; a circuit's
result is bit-identical alone and in a mixed batch; HHL batches reproduce the oracle's readout;
the run can be captured in a CUDA graph."""
import ctypes
import math

import numpy as np
import pytest
import torch

import synth
from hhl_bounds import cond_tol, prob_bound, readout_bounds
from oracle import core as ocore
from oracle import hhl as ohhl

TOL = {torch.complex128: 1e-12, torch.complex64: 1e-5}
DTYPES = [torch.complex128, torch.complex64]


@pytest.fixture(scope="module")
def qs():
    from paper_2402_08136_gb300 import build
    build.build()
    import paper_2402_08136_gb300 as q
    return q


def random_circuit(qs, rng, n, count):
    """Gates the batched executor supports: dense up to 5 targets (with controls), phases,
    diagonals, swaps, a contiguous-register UCRY."""
    c = qs.Circuit(n)
    ref_gates = []
    for _ in range(count):
        r = rng.random()
        if r < 0.5:
            k = int(rng.integers(1, min(5, n - 1) + 1))
            q = [int(v) for v in rng.permutation(n)]
            t = q[:k]
            ctl = q[k:k + int(rng.integers(0, 2))] if n - k >= 1 else []
            U = synth.haar_unitary(rng, 1 << k)
            c.add_gate(t, U, ctl)
            ref_gates.append(("u", t, U, ctl))
        elif r < 0.7:
            t = synth.random_targets(rng, n, 2)
            U = np.diag([1, 1, 1, np.exp(1j * rng.uniform(-3, 3))])
            c.add_gate(t, U)
            ref_gates.append(("u", t, U, []))
        elif r < 0.8:
            t = [int(rng.integers(n))]
            U = np.diag(np.exp(1j * rng.uniform(-3, 3, 2)))
            c.add_gate(t, U)
            ref_gates.append(("u", t, U, []))
        elif r < 0.9:
            t = synth.random_targets(rng, n, 2)
            U = np.eye(4)[[0, 2, 1, 3]]
            c.add_gate(t, U)
            ref_gates.append(("u", t, U, []))
        else:
            nr = min(3, n - 1)
            c0 = int(rng.integers(0, n - nr))
            reg = list(range(c0, c0 + nr))
            tgt = [q for q in range(n) if q not in reg][int(rng.integers(0, n - nr))]
            th = rng.uniform(-3, 3, size=1 << nr)
            c.add_ucry(tgt, reg, th)
            ref_gates.append(("ucry", tgt, reg, th))
    return c, ref_gates


def oracle_apply(psi, gates):
    for g in gates:
        if g[0] == "u":
            ocore.apply_gate(psi, g[1], g[2], g[3])
        else:
            ocore.apply_ucry(psi, g[1], g[2], g[3])
    return psi


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", DTYPES)
def test_batched_matches_oracle_and_is_batch_independent(qs, dtype, cuda_device):
    rng = np.random.default_rng(31)
    sizes = [5, 9, 12, 13, 14, 15, 16, 7, 11, 3]
    circs, refs, inputs = [], [], []
    for i, n in enumerate(sizes):
        c, g = random_circuit(qs, rng, n, 40)
        psi = synth.gaussian_state_np(100 + i, n)
        if dtype == torch.complex64:
            psi = psi.astype(np.complex64).astype(np.complex128)
        circs.append(c)
        refs.append(oracle_apply(psi.copy(), g))
        inputs.append(psi)
    states = [torch.from_numpy(x).to(dtype).cuda() for x in inputs]
    qs.qsim_apply_batched(states, circs)
    torch.cuda.synchronize()
    for st, ref in zip(states, refs):
        out = st.cpu().numpy().astype(np.complex128)
        assert np.max(np.abs(out - ref)) <= TOL[dtype]
    # each circuit alone in a batch of one: bit-identical to its result in the mix
    for i in (0, 3, 6, 9):
        alone = torch.from_numpy(inputs[i]).to(dtype).cuda()
        qs.qsim_apply_batched([alone], [circs[i]])
        torch.cuda.synchronize()
        assert torch.equal(alone, states[i])


def ref_solve(p):
    return ohhl.solve(p["A"], p["b"], p["m"])


def check_hhl_result(st, r, ref, m, dtype):
    """Batched HHL result vs the oracle: the state element by element (cond_tol for complex128,
    where both sides eigendecompose A; 1e-5 and fidelity >= 1 - 1e-6 for complex64), and P, P0,
    the normalized solution and x within the bounds that the state bound implies."""
    tol = cond_tol(m) if dtype == torch.complex128 else TOL[dtype]
    out = st.cpu().numpy().astype(np.complex128)
    assert np.max(np.abs(out - ref["psi"])) <= tol
    if dtype == torch.complex64:
        f = abs(np.vdot(ref["psi"], out)) ** 2 / (np.vdot(out, out).real * np.vdot(ref["psi"], ref["psi"]).real)
        assert f >= 1 - 1e-6
    h = ref["circuit"]
    N = len(ref["x"])
    bd = readout_bounds(ref, h["nb"], h["m"], tol, h["C"], h["bnorm"], N)
    assert abs(r["p_success"] - ref["P"]) <= bd["P"]
    assert abs(r["p_clock0"] - ref["P0"]) <= bd["P0"]
    assert abs(r["norm2"] - ref["norm2"]) <= prob_bound(ref["psi"], tol)
    xs = r["x"] / (r["norm_x"] * r["norm_b"])   # the normalized slice the kernel read out
    assert np.all(np.abs(xs - ref["x_state"][:N]) <= bd["x_state"])
    assert np.all(np.abs(r["x"] - ref["x"]) <= bd["x"])


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", DTYPES)
def test_hhl_batch_matches_oracle(qs, dtype, cuda_device):
    probs = synth.batched_problems(seed=9, count=12)
    hs, fused, states, refs = [], [], [], []
    for p in probs:
        h = qs.hhl_build(p["A"], p["b"], p["m"])
        hs.append(h)
        fused.append(qs.qsim_fuse(h.as_circuit(), 4))
        states.append(torch.empty(1 << h.info()["n"], dtype=dtype, device="cuda"))
        refs.append(ohhl.solve(p["A"], p["b"], p["m"]))
    b = qs.hhl_batch_create(hs, states, fused)
    b.run()
    res = b.results()
    for p, h, st, r, ref in zip(probs, hs, states, res, refs):
        check_hhl_result(st, r, ref, p["m"], dtype)


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", DTYPES)
def test_hhl_batch_structured_matches_oracle(qs, dtype, cuda_device):
    probs = synth.batched_problems(seed=19, count=10)
    hs = [qs.hhl_build(p["A"], p["b"], p["m"], structured=True) for p in probs]
    fused = [qs.qsim_fuse(h.as_circuit(), 3) for h in hs]
    states = [torch.empty(1 << h.info()["n"], dtype=dtype, device="cuda") for h in hs]
    b = qs.hhl_batch_create(hs, states, fused)
    b.run()
    res = b.results()
    for p, st, r in zip(probs, states, res):
        check_hhl_result(st, r, ref_solve(p), p["m"], dtype)


@pytest.mark.gpu
def test_batch_run_captures_in_cuda_graph(qs, cuda_device):
    probs = synth.batched_problems(seed=10, count=6)
    hs = [qs.hhl_build(p["A"], p["b"], p["m"]) for p in probs]
    fused = [qs.qsim_fuse(h.as_circuit(), 3) for h in hs]
    states = [torch.empty(1 << h.info()["n"], dtype=torch.complex64, device="cuda") for h in hs]
    b = qs.hhl_batch_create(hs, states, fused)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b.run(s)
    s.synchronize()
    eager = b.results(s)
    snap = [st.clone() for st in states]
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        b.run(s)
    for st in states:
        st.zero_()
    g.replay()
    torch.cuda.synchronize()
    replay = b.results(s)
    for a, c in zip(snap, states):
        assert torch.equal(a, c)
    for a, c in zip(eager, replay):
        assert a["p_success"] == c["p_success"] and np.array_equal(a["x"], c["x"])


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", DTYPES)
def test_repeated_runs_reset_the_work_counter(qs, dtype, cuda_device):
    """More circuits than CTAs (each CTA takes several), run three times eagerly and twice from
    a CUDA graph: every run must apply every circuit once more (the kernel leaves its work
    counter at zero for the next launch), so each state ends at U^5 psi."""
    rng = np.random.default_rng(41)
    count = 400
    circs, refs, inputs = [], [], []
    for i in range(count):
        n = int(rng.integers(3, 9))
        c, g = random_circuit(qs, rng, n, 8)
        psi = synth.gaussian_state_np(500 + i, n)
        if dtype == torch.complex64:
            psi = psi.astype(np.complex64).astype(np.complex128)
        ref = psi.copy()
        for _ in range(5):
            oracle_apply(ref, g)
        circs.append(c)
        refs.append(ref)
        inputs.append(psi)
    states = [torch.from_numpy(x).to(dtype).cuda() for x in inputs]
    b = qs.qsim_batch_create(circs, states)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for _ in range(3):
            b.run(s)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    snap = [st.clone() for st in states]
    with torch.cuda.graph(g, stream=s):
        b.run(s)
    for st, x in zip(states, snap):  # capturing records the launch without running it
        assert torch.equal(st, x)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    for st, ref in zip(states, refs):
        out = st.cpu().numpy().astype(np.complex128)
        assert np.max(np.abs(out - ref)) <= 5 * TOL[dtype]


@pytest.mark.gpu
def test_hhl_batch_solve_single_call(qs, cuda_device):
    """hhl_batch_solve (launch, copy, synchronize, host scaling in one call) gives the same
    bits as a run followed by hhl_batch_results, every time, and the oracle's solution."""
    p = synth.hhl7_problem()
    h = qs.hhl_build(p["A"], p["b"], p["m"], p["t"], p["C"])
    st = torch.empty(1 << h.info()["n"], dtype=torch.complex128, device="cuda")
    b = qs.hhl_batch_create([h], [st], [qs.qsim_fuse(h.as_circuit(), 2)])
    b.run()
    x0, s0 = (a.copy() for a in b.results_arrays())
    ref = ohhl.solve(p["A"], p["b"], p["m"], p["t"], p["C"])
    assert np.max(np.abs(x0 - ref["x"])) <= 1e-11 * np.linalg.norm(ref["x"])
    for _ in range(50):
        x, stats = b.solve()
        assert np.array_equal(x, x0) and np.array_equal(stats, s0)
    assert qs.qsim_device_status() == 0


def test_batch_rejects_wide_dense_gate(qs):
    c = qs.Circuit(8).add_gate(list(range(6)), synth.haar_unitary(np.random.default_rng(0), 64))
    fake = ctypes.c_void_p(256)  # never dereferenced: the op check fails before any CUDA call
    with pytest.raises(qs.QsimError) as e:
        qs._binding.library()
        p = ctypes.c_void_p()
        arr_c = (ctypes.c_void_p * 1)(c.ptr)
        arr_s = (ctypes.c_void_p * 1)(fake)
        qs._binding._check(qs._binding.library().qsim_batch_create(arr_c, arr_s, 1, qs.QSIM_C64,
                                                                   ctypes.byref(p)))
    assert "max_k <= 5" in str(e.value)


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", DTYPES)
def test_batched_fourier_and_walsh_passes_match_oracle(qs, dtype, cuda_device):
    """Fourier passes (contiguous fields, twiddle before / after / none) and Walsh-Hadamard
    passes inside the batched executor, states in shared memory (n = 11) and in place (n = 16),
    vs the oracle; a circuit's result is the same alone and in the batch."""
    rng = np.random.default_rng(44)
    circs, states, refs = [], [], []
    for n, f0, K, src, sign, pre in [(11, 5, 6, [1, 2, 3, 4], -1, False), (11, 0, 5, [5, 6], +1, True),
                                     (16, 8, 8, list(range(2, 8)), -1, False), (16, 3, 10, [], +1, False)]:
        field = list(range(f0, f0 + K))
        psi = synth.gaussian_state_np(int(rng.integers(1 << 30)), n)
        x0 = psi.astype(np.complex64).astype(np.complex128) if dtype == torch.complex64 else psi
        c = qs.Circuit(n)
        c.add_walsh(field[::-1])
        c.add_dft(field, sign, src, twiddle_first=pre)
        ref = x0.copy()
        for q in field:
            ocore.apply_gate(ref, [q], ohhl.H)
        ohhl.dft_pass(ref, field, sign, src, pre)
        circs.append(c)
        states.append(torch.from_numpy(x0).to(dtype).cuda())
        refs.append(ref)
    batch_states = [s.clone() for s in states]
    qs.qsim_apply_batched(batch_states, circs)
    torch.cuda.synchronize()
    for i, (st, ref) in enumerate(zip(batch_states, refs)):
        out = st.cpu().numpy().astype(np.complex128)
        assert np.max(np.abs(out - ref)) <= TOL[dtype]
        alone = states[i].clone()
        qs.qsim_apply_batched([alone], [circs[i]])
        torch.cuda.synchronize()
        assert torch.equal(alone, st)


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", DTYPES)
def test_hhl_batch_with_qft_passes_matches_oracle(qs, dtype, cuda_device):
    """HHL circuits whose QFTs and Hadamard layers are passes, in one batched launch: one field
    (m <= 10) and two fields (m = 12, 13: the rotation reads the clock register rotated)."""
    probs = synth.batched_problems(seed=29, count=8)
    rng = np.random.default_rng(3)
    for m in (12, 13):
        A, b = synth.contingency_system(rng, 5)
        probs.append({"A": A, "b": b, "m": m})
    hs = [qs.hhl_build(p["A"], p["b"], p["m"], structured=True, fft_qft=True) for p in probs]
    fused = [qs.qsim_fuse(h.as_circuit(), 3) for h in hs]
    states = [torch.empty(1 << h.info()["n"], dtype=dtype, device="cuda") for h in hs]
    b = qs.hhl_batch_create(hs, states, fused)
    b.run()
    res = b.results()
    for p, st, r in zip(probs, states, res):
        ref = ohhl.solve(p["A"], p["b"], p["m"])
        m = p["m"]
        tol = max(1e-12, 2.0 ** m * 2 * math.pi * 8 * np.finfo(float).eps) \
            if dtype == torch.complex128 else TOL[dtype]
        out = st.cpu().numpy().astype(np.complex128)
        assert np.max(np.abs(out - ref["psi"])) <= tol
        assert abs(r["p_success"] - ref["P"]) <= 10 * tol
        assert abs(r["p_clock0"] - ref["P0"]) <= 10 * tol


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", DTYPES)
def test_batch_autotune_returns_its_fastest_candidate_and_every_width_is_correct(qs, dtype, cuda_device):
    """hhl_batch_autotune: the width it returns is the one with the smallest measured time, and the
    batch fused at every candidate width reproduces the oracle (the state within the dtype's
    bound, the readout within the bounds that implies)."""
    probs = synth.batched_problems(seed=23, count=16)
    hs = [qs.hhl_build(p["A"], p["b"], p["m"], structured=True, fft_qft=True) for p in probs]
    states = [torch.empty(1 << h.info()["n"], dtype=dtype, device="cuda") for h in hs]
    cands = (1, 2, 3, 4, 5)
    k, tmap = qs.hhl_batch_autotune(hs, states, cands)
    assert set(tmap) == set(cands) and all(v > 0 for v in tmap.values())
    assert k == min(tmap, key=tmap.get)
    refs = [ref_solve(p) for p in probs]
    for kk in cands:
        fused = [qs.qsim_fuse(h.as_circuit(), kk) for h in hs]
        b = qs.hhl_batch_create(hs, states, fused)
        b.run()
        for p, st, r, ref in zip(probs, states, b.results(), refs):
            check_hhl_result(st, r, ref, p["m"], dtype)
