"""Pins of the FP64 oracle against things other than itself (no GPU needed).

  * gate rule          -> brute-force full 2^n x 2^n operator built from Kronecker products
  * UCRY               -> brute-force block-diagonal operator
  * QFT / inverse QFT  -> numpy's FFT (the DFT up to normalisation)
  * DFT passes         -> the textbook QFT gate circuit (H, controlled phases, swaps): the
                          Cooley-Tukey field passes plus a relabelling of the register equal it
  * QPE                -> an eigenvector whose phase lies on the clock grid lands on exactly |k>
  * HHL (exact grid)   -> the postselected slice equals A^-1 b / ||A^-1 b||, P = C^2 ||A^-1 b||^2,
                          no leakage, and x = A^-1 b (Sec. III-A)
  * resource formula   -> the qubit counts printed in Table I (tests/golden)
  * compensated sums   -> math.fsum (exactly rounded)
Mutation tests plant a plausible mistake in the oracle and check that a pin catches it.
"""
import math
import os

import numpy as np
import pytest

import synth
from oracle import core, hhl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def full_operator(n, targets, U, controls=(), vals=()):
    """2^n x 2^n operator of U on `targets` controlled on `controls` == `vals`, built as
    I (x) G in a basis where the gate's qubits are the lowest bits, then permuted back."""
    k, c = len(targets), len(controls)
    dk = 1 << k
    if c:
        pv = sum(int(v) << j for j, v in enumerate(vals))
        P = np.zeros((1 << c, 1 << c))
        P[pv, pv] = 1.0
        G = np.kron(P, U) + np.kron(np.eye(1 << c) - P, np.eye(dk))
    else:
        G = U
    Fp = np.kron(np.eye(1 << (n - k - c)), G)
    order = list(targets) + list(controls) + [q for q in range(n) if q not in targets and q not in controls]
    idx = np.arange(1 << n)
    pi = np.zeros(1 << n, dtype=np.int64)
    for j, q in enumerate(order):
        pi |= ((idx >> q) & 1) << j
    return Fp[np.ix_(pi, pi)]


def rand_state(rng, n):
    v = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    return v / np.linalg.norm(v)


def test_threaded_oracle_is_deterministic():
    """The C oracle's parallel loops (gate groups, UCRY pairs, Neumaier partial sums) give the
    same bits with 1 thread and with several: its groups are disjoint and its sums are combined
    in a fixed order, so a race or an order that depends on the thread count would show."""
    rng = np.random.default_rng(5)
    n = 16
    psi0 = rand_state(rng, n)
    gates = []
    for _ in range(12):
        k = int(rng.integers(1, 5))
        qs = [int(q) for q in rng.choice(n, size=k + 1, replace=False)]
        gates.append((qs[:k], synth.haar_unitary(rng, 1 << k), qs[k:], [1]))
    th = rng.uniform(-3, 3, size=8)
    saved = core.num_threads()
    outs = []
    try:
        for t in (1, max(2, saved)):
            core.set_num_threads(t)
            psi = psi0.copy()
            for tg, U, ctl, vals in gates:
                core.apply_gate(psi, tg, U, ctl, vals)
            core.apply_ucry(psi, n - 1, [3, 4, 5], th)
            outs.append((psi, core.masked_norm2(psi, 1 << (n - 1), 1 << (n - 1))))
    finally:
        core.set_num_threads(saved)
    assert np.array_equal(outs[0][0], outs[1][0])
    assert outs[0][1] == outs[1][1]


@pytest.mark.parametrize("seed", range(6))
def test_gate_rule_matches_bruteforce(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(3, 9))
    for _ in range(8):
        k = int(rng.integers(1, min(4, n) + 1))
        c = int(rng.integers(0, min(2, n - k) + 1))
        qs = [int(q) for q in rng.choice(n, size=k + c, replace=False)]
        t, ctl = qs[:k], qs[k:]
        vals = [int(v) for v in rng.integers(0, 2, size=c)]
        U = synth.haar_unitary(rng, 1 << k)
        psi = rand_state(rng, n)
        ref = full_operator(n, t, U, ctl, vals) @ psi
        out = psi.copy()
        core.apply_gate(out, t, U, ctl, vals)
        assert np.max(np.abs(out - ref)) < 1e-13


def test_ucry_matches_bruteforce():
    rng = np.random.default_rng(11)
    n, target, ctl = 6, 5, [1, 2, 4]
    theta = rng.uniform(-np.pi, np.pi, size=8)
    F = np.eye(1 << n, dtype=np.complex128)
    for v in range(8):  # the eight controlled rotations act on disjoint subspaces
        vals = [(v >> j) & 1 for j in range(3)]
        F = full_operator(n, [target], hhl.RY(theta[v]), ctl, vals) @ F
    psi = rand_state(rng, n)
    out = psi.copy()
    core.apply_ucry(out, target, ctl, theta)
    assert np.max(np.abs(out - F @ psi)) < 1e-13


def test_norm_preserved_by_random_circuit():
    rng = np.random.default_rng(5)
    n = 11
    psi = rand_state(rng, n)
    gates = 60
    for _ in range(gates):
        k = int(rng.integers(1, 5))
        t = synth.random_targets(rng, n, k)
        core.apply_gate(psi, t, synth.haar_unitary(rng, 1 << k))
    assert abs(np.vdot(psi, psi).real - 1.0) < 1e-13 * gates


def test_haar_unitary():
    rng = np.random.default_rng(2)
    for k in range(1, 7):
        U = synth.haar_unitary(rng, 1 << k)
        assert np.max(np.abs(U.conj().T @ U - np.eye(1 << k))) < 1e-13


@pytest.mark.parametrize("m", [1, 2, 3, 4, 5, 7])
def test_qft_matches_fft(m):
    rng = np.random.default_rng(m)
    psi = rand_state(rng, m)
    fwd = psi.copy()
    for g in hhl.qft_gates(list(range(m)), inverse=False):
        core.apply_gate(fwd, g[1], g[2])
    N = 1 << m
    assert np.max(np.abs(fwd - np.fft.ifft(psi) * math.sqrt(N))) < 1e-13
    inv = psi.copy()
    for g in hhl.qft_gates(list(range(m)), inverse=True):
        core.apply_gate(inv, g[1], g[2])
    assert np.max(np.abs(inv - np.fft.fft(psi) / math.sqrt(N))) < 1e-13


def test_qft_on_embedded_register():
    # register on qubits 2,4,5 of a 6-qubit state, others spectators
    rng = np.random.default_rng(9)
    reg = [2, 4, 5]
    psi = rand_state(rng, 6)
    out = psi.copy()
    for g in hhl.qft_gates(reg, inverse=True):
        core.apply_gate(out, g[1], g[2])
    # reference: reshape so the register value is an axis, FFT along it
    idx = np.arange(64)
    val = sum(((idx >> q) & 1) << j for j, q in enumerate(reg))
    rest = idx & ~sum(1 << q for q in reg)
    ref = np.zeros_like(psi)
    for r in np.unique(rest):
        sel = np.where(rest == r)[0]
        order = sel[np.argsort(val[sel])]
        ref[order] = np.fft.fft(psi[order]) / math.sqrt(8)
    assert np.max(np.abs(out - ref)) < 1e-13


def _grid_problem(seed, N, m, complex_vectors=False):
    rng = np.random.default_rng(seed)
    top = 2 ** m - 1
    k = np.sort(rng.integers(1, top + 1, size=N)).astype(float)
    k[-1] = top
    if complex_vectors:
        V = synth.haar_unitary(rng, N)
    else:
        V, _ = np.linalg.qr(rng.standard_normal((N, N)))
    A = (V * k) @ V.conj().T
    A = 0.5 * (A + A.conj().T)
    b = rng.standard_normal(N) + (1j * rng.standard_normal(N) if complex_vectors else 0)
    return A, b, k, V


def test_qpe_exact_on_grid_eigenvector():
    m, N = 5, 4
    A, _, k, V = _grid_problem(3, N, m)
    for i in range(N):
        h = hhl.build(A, V[:, i], m, t=2 * math.pi / 2 ** m)
        qpe = []
        for g in h["gates"]:
            if g[0] == "ucry":
                break
            qpe.append(g)
        psi = hhl.initial_state(h)
        for g in qpe:
            core.apply_gate(psi, g[1], g[2], g[3], g[4])
        nb = h["nb"]
        clock_val = int(round(k[i]))
        sl = psi[clock_val << nb: (clock_val << nb) + (1 << nb)]
        assert abs(np.linalg.norm(sl) - 1.0) < 1e-12


@pytest.mark.parametrize("m,N,cplx,seed", [(3, 2, False, 0), (4, 4, False, 1), (5, 3, False, 2),
                                           (6, 5, True, 3), (7, 8, True, 4), (8, 4, False, 5)])
def test_hhl_exact_grid(m, N, cplx, seed):
    A, b, k, V = _grid_problem(seed, N, m, cplx)
    r = hhl.solve(A, b, m, t=2 * math.pi / 2 ** m)
    xt = np.linalg.solve(A, b)
    bh = b / np.linalg.norm(b)
    y = np.linalg.solve(A, bh)
    C = r["circuit"]["C"]
    assert abs(C - k[0]) < 1e-9
    assert np.max(np.abs(r["x_state"][:N] - y / np.linalg.norm(y))) < 1e-12
    assert abs(r["P"] - C ** 2 * np.vdot(y, y).real) < 1e-12
    assert abs(r["leakage"]) < 1e-14
    assert abs(r["norm_x"] - np.linalg.norm(y)) < 1e-12 * np.linalg.norm(y)
    assert np.max(np.abs(r["x"] - xt)) < 1e-11 * np.linalg.norm(xt)
    assert abs(r["norm2"] - 1.0) < 1e-12


@pytest.mark.parametrize("m,N,cplx,seed", [(4, 3, False, 10), (5, 4, True, 11), (6, 6, False, 12),
                                           (7, 8, True, 13)])
def test_hhl_exact_grid_indefinite(m, N, cplx, seed):
    """Signed eigenvalues: integers in +-[1, 2^(m-1) - 1] with t = 2 pi / 2^m land exactly on the
    two's-complement clock grid; the slice is then exactly A^-1 b / ||A^-1 b||."""
    rng = np.random.default_rng(seed)
    top = 2 ** (m - 1) - 1
    k = rng.integers(1, top + 1, size=N).astype(float) * rng.choice([-1.0, 1.0], size=N)
    k[0], k[-1] = -top, top
    V = synth.haar_unitary(rng, N) if cplx else np.linalg.qr(rng.standard_normal((N, N)))[0]
    A = (V * k) @ V.conj().T
    A = 0.5 * (A + A.conj().T)
    b = rng.standard_normal(N) + (1j * rng.standard_normal(N) if cplx else 0)
    r = ohhl_solve_signed(A, b, m)
    bh = b / np.linalg.norm(b)
    y = np.linalg.solve(A, bh)
    assert r["circuit"]["signed"]
    assert np.max(np.abs(r["x_state"][:N] - y / np.linalg.norm(y))) < 1e-12
    assert abs(r["leakage"]) < 1e-14
    assert abs(r["norm_x"] - np.linalg.norm(y)) < 1e-12 * np.linalg.norm(y)
    assert np.max(np.abs(r["x"] - np.linalg.solve(A, b))) < 1e-11 * np.linalg.norm(np.linalg.solve(A, b))


def ohhl_solve_signed(A, b, m):
    return hhl.solve(A, b, m, t=2 * math.pi / 2 ** m)


def test_resource_formula_counts_sign_qubit_by_default():
    rng = np.random.default_rng(3)
    V = np.linalg.qr(rng.standard_normal((5, 5)))[0]
    lam = np.array([-9.0, -2.0, 1.5, 4.0, 12.0])
    A = (V * lam) @ V.T
    h = hhl.build(0.5 * (A + A.T), rng.standard_normal(5), 0)
    assert h["signed"]
    assert h["m"] == max(3 + 1, math.ceil(math.log2(12.0 / 1.5 + 1))) + 1


def test_dilation_exact_grid():
    """Non-Hermitian A' = U diag(sigma) W^H with integer singular values: the dilation has
    eigenvalues +-sigma, exactly on the signed clock grid, and HHL returns A'^-1 b exactly."""
    rng = np.random.default_rng(31)
    N, m = 3, 6
    U, W = synth.haar_unitary(rng, N), synth.haar_unitary(rng, N)
    sig = np.array([2.0, 5.0, 31.0])
    A = (U * sig) @ W.conj().T
    b = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    r = hhl.solve_general(A, b, m, t=2 * math.pi / 2 ** m)
    xt = np.linalg.solve(A, b)
    assert r["circuit"]["signed"] and r["circuit"]["N"] == 2 * N
    assert np.max(np.abs(r["x"] - xt)) < 1e-11 * np.linalg.norm(xt)
    assert np.max(np.abs(r["x_eff"][:N])) < 1e-12 * np.linalg.norm(xt)   # y = 0
    assert abs(r["leakage"]) < 1e-14


def test_gauss_seidel_on_lower_triangular_is_identity():
    """For a lower-triangular A the Gauss-Seidel splitting is A itself: A' = I, b' = A^-1 b,
    and the (dilated, signed) HHL solve is exact with eigenvalues +-1."""
    rng = np.random.default_rng(32)
    N = 4
    A = np.tril(rng.standard_normal((N, N))) + 4 * np.eye(N)
    b = rng.standard_normal(N)
    Ae, be, off, _ = hhl.preprocess(A, b, gauss_seidel=True)
    assert off == 0 and np.max(np.abs(Ae - np.eye(N))) < 1e-14          # Hermitian: no dilation
    r = hhl.solve_general(A, b, 3, t=2 * math.pi / 8, gauss_seidel=True, dilate=True)
    assert np.max(np.abs(r["x"] - np.linalg.solve(A, b))) < 1e-12 * np.linalg.norm(np.linalg.solve(A, b))


def test_dilated_resources_match_table1_30bus_star():
    """Table I, 30-bus*: a preconditioned (non-Hermitian) 29 x 29 system is dilated to 58 rows,
    n_data = 6."""
    rng = np.random.default_rng(33)
    A, b, _ = synth.grid_system(rng, 30)
    Ae, be, off, N = hhl.preprocess(A, b, gauss_seidel=True)
    assert Ae.shape == (58, 58) and off == 29 and N == 29
    assert hhl.resource_counts(Ae.shape[0], 109.3, True)[1] == 6


def test_hhl_padding_gives_zero_tail():
    A, b, _, _ = _grid_problem(7, 3, 5)
    r = hhl.solve(A, b, 5, t=2 * math.pi / 32)
    assert r["circuit"]["nb"] == 2
    assert abs(r["x_state"][3]) < 1e-13
    assert np.max(np.abs(r["x"] - np.linalg.solve(A, b))) < 1e-11


def test_hhl7_problem_exact():
    p = synth.hhl7_problem()
    r = hhl.solve(p["A"], p["b"], p["m"], p["t"], p["C"])
    xt = np.linalg.solve(p["A"], p["b"])
    assert np.max(np.abs(r["x"] - xt)) < 1e-12 * np.linalg.norm(xt)
    assert r["circuit"]["n"] == 7


def test_resource_formula_matches_table1():
    rows = []
    with open(os.path.join(GOLDEN, "table1_resources.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append(line.split())
    assert len(rows) == 3
    for name, nrows, kappa, neg, n_total, n_data, n_qpe in rows:
        got = hhl.resource_counts(int(nrows), float(kappa), bool(int(neg)))
        assert got == (int(n_total), int(n_data), int(n_qpe)), name


def test_compensated_sum_vs_fsum():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(10000) * 1e8, rng.standard_normal(10000),
                        -rng.standard_normal(10000) * 1e8])
    rng.shuffle(x)
    assert abs(core.compensated_sum(x) - math.fsum(x)) <= 1e-16 * np.sum(np.abs(x))
    psi = rand_state(rng, 10)
    sq = np.concatenate([psi.real ** 2, psi.imag ** 2])
    assert abs(core.masked_norm2(psi, 0, 0) - math.fsum(sq)) < 1e-15


# ---------------------------------------------------------------- planted mistakes
def test_planted_missing_swaps_is_caught(monkeypatch):
    orig = hhl.qft_gates

    def no_swaps(qubits, inverse):
        return [g for g in orig(qubits, inverse) if not (len(g[1]) == 2 and np.allclose(g[2], hhl.SWAP))]

    monkeypatch.setattr(hhl, "qft_gates", no_swaps)
    psi = rand_state(np.random.default_rng(1), 4)
    out = psi.copy()
    for g in hhl.qft_gates(list(range(4)), inverse=False):
        core.apply_gate(out, g[1], g[2])
    assert np.max(np.abs(out - np.fft.ifft(psi) * 4.0)) > 1e-3


def test_planted_wrong_evolution_sign_is_caught(monkeypatch):
    A, b, _, _ = _grid_problem(1, 4, 4)
    orig_build = hhl.build

    def conj_build(*args, **kw):
        h = orig_build(*args, **kw)
        # plant: controlled evolutions become exp(-iAt) (complex conjugate for real A)
        h["gates"] = [("u", g[1], g[2].conj(), g[3], g[4]) if g[0] == "u" and g[3] else g
                      for g in h["gates"]]
        return h

    monkeypatch.setattr(hhl, "build", conj_build)
    r = hhl.solve(A, b, 4, t=2 * math.pi / 16)
    y = np.linalg.solve(A, b / np.linalg.norm(b))
    err = np.max(np.abs(r["x_state"][:4] - y / np.linalg.norm(y))) if r["P0"] > 1e-30 else 1.0
    assert err > 1e-3 or abs(r["leakage"]) > 1e-3


# ------------------------------------------------------------------ QFT as Cooley-Tukey passes
def _split_fields(reg, sizes):
    """Fields of `reg` (bit j <-> reg[j]) from the top down: sizes[0] top bits first."""
    out, hi = [], len(reg)
    for s in sizes:
        out.append(list(reg[hi - s: hi]))
        hi -= s
    assert hi == 0
    return out


def _relabel(psi, reg, order, to_natural=True):
    """Move register value v between the layouts 'bit j of v at order[j]' and 'at reg[j]'."""
    idx = np.arange(psi.size)
    src, dst = (order, reg) if to_natural else (reg, order)
    v = sum(((idx >> q) & 1) << j for j, q in enumerate(src))
    rest = idx & ~sum(1 << q for q in reg)
    dest = rest | sum(((v >> j) & 1) << q for j, q in enumerate(dst))
    out = np.empty_like(psi)
    out[dest] = psi
    return out


def _check_dft_factorisation(m, sizes, dft):
    rng = np.random.default_rng(100 + m)
    n = m + 2
    reg = list(range(1, m + 1))  # spectator qubits 0 and m+1
    fields = _split_fields(reg, sizes)
    order = [q for f in fields for q in f]
    psi = rand_state(rng, n)
    # inverse QFT: passes top field first, each with the twiddle of the bits below it
    p = psi.copy()
    for f in fields:
        dft(p, f, -1, [q for q in reg if q < min(f)], False)
    ref = psi.copy()
    for g in hhl.qft_gates(reg, inverse=True):
        core.apply_gate(ref, g[1], g[2])
    assert np.max(np.abs(_relabel(p, reg, order) - ref)) < 1e-13
    # QFT from the field-ordered layout: the passes reversed, conjugated, twiddle first
    for f in reversed(fields):
        dft(p, f, +1, [q for q in reg if q < min(f)], True)
    assert np.max(np.abs(p - psi)) < 1e-13
    # forward QFT of a natural-order state
    q2 = _relabel(psi, reg, order, to_natural=False)
    for f in reversed(fields):
        dft(q2, f, +1, [q for q in reg if q < min(f)], True)
    ref2 = psi.copy()
    for g in hhl.qft_gates(reg, inverse=False):
        core.apply_gate(ref2, g[1], g[2])
    assert np.max(np.abs(q2 - ref2)) < 1e-13


@pytest.mark.parametrize("m,sizes", [(5, [5]), (6, [3, 3]), (7, [4, 3]), (8, [3, 5]), (9, [3, 3, 3])])
def test_dft_passes_factor_the_textbook_qft(m, sizes):
    _check_dft_factorisation(m, sizes, hhl.dft_pass)


def test_planted_twiddle_mistakes_are_caught():
    def wrong_denominator(psi, targets, sign, src, pre):
        hhl.dft_pass(psi, targets, sign, list(src)[1:], pre)   # drops the lowest twiddle bit

    def wrong_side(psi, targets, sign, src, pre):
        hhl.dft_pass(psi, targets, sign, src, not pre)         # twiddle on the wrong side

    def wrong_sign(psi, targets, sign, src, pre):
        hhl.dft_pass(psi, targets, sign, (), pre)              # twiddle left out
    for bad in (wrong_denominator, wrong_side, wrong_sign):
        with pytest.raises(AssertionError):
            _check_dft_factorisation(6, [3, 3], bad)


# ------------------------------------------------------------ default evolution time and C
def _clock_distribution(h, b_vec):
    """Run the phase-estimation part of the oracle's gate list (everything before the
    rotation) from |0>|b_vec> and return the probability of each clock value."""
    h = dict(h)
    bp = np.zeros(1 << h["nb"], dtype=np.complex128)
    bp[: len(b_vec)] = b_vec / np.linalg.norm(b_vec)
    h["b_pad"] = bp
    psi = hhl.initial_state(h)
    for g in h["gates"]:
        if g[0] == "ucry":
            break
        core.apply_gate(psi, g[1], g[2], g[3], g[4])
    nb, m = h["nb"], h["m"]
    return (np.abs(psi.reshape(-1, 1 << nb)) ** 2).sum(axis=1)[: 1 << m]


def _default_t_problems():
    """An off-grid power-flow matrix (positive definite) and an indefinite one."""
    A, b = synth.contingency_system(np.random.default_rng(21), 9)     # 8 x 8 SPD, generic spectrum
    rng = np.random.default_rng(22)
    V = np.linalg.qr(rng.standard_normal((6, 6)))[0]
    lam = np.array([-7.3, -2.2, 0.9, 1.7, 4.4, 9.1])
    Ai = (V * lam) @ V.T
    return [(A, b, False), (0.5 * (Ai + Ai.T), rng.standard_normal(6), True)]


@pytest.mark.parametrize("m", [5, 7])
def test_default_t_puts_the_largest_eigenvalue_on_the_top_clock_value(m):
    """With the default evolution time, phase estimation of the eigenvector of the largest
    |lambda| lands exactly on the top clock value: 2^m - 1 for a positive definite A, and
    +-(2^(m-1) - 1) in two's complement for an indefinite A (the sign qubit of Sec. III-B).
    The spectrum is off the grid, so only the extreme eigenvector is exact."""
    for A, b, signed in _default_t_problems():
        h = hhl.build(A, b, m)
        assert h["signed"] == signed
        w, V = np.linalg.eigh(A)
        i = int(np.argmax(np.abs(w)))
        M = 1 << m
        if signed:
            want = (M // 2 - 1) if w[i] > 0 else M - (M // 2 - 1)
        else:
            want = M - 1
        prob = _clock_distribution(h, V[:, i])
        assert abs(prob[want] - 1.0) < 1e-12
        # an off-grid eigenvalue spreads over several clock values
        j = int(np.argmin(np.abs(w)))
        assert _clock_distribution(h, V[:, j]).max() < 1.0 - 1e-6


def test_default_c_is_the_largest_grid_value_below_lambda_min_and_hhl_is_exact_on_it():
    """Default C: a clock grid value (C / step an integer, with the grid step fixed by where the
    largest eigenvalue lands) not above min|lambda|, and the next grid value is above it.  With
    b the (on-grid) top eigenvector, HHL is exact even though A is off the grid: P = (C /
    lambda_max)^2, no leakage, x = A^-1 b."""
    m = 6
    for A, _, signed in _default_t_problems():
        h = hhl.build(A, np.ones(A.shape[0]), m)
        w, V = np.linalg.eigh(A)
        amin, amax = np.abs(w).min(), np.abs(w).max()
        top = (2 ** (m - 1) - 1) if signed else (2 ** m - 1)
        step = amax / top                                 # where the largest eigenvalue lands
        C = h["C"]
        q = C / step
        assert abs(q - round(q)) < 1e-9 and round(q) >= 1
        assert C <= amin * (1 + 1e-12) and C + step > amin
        i = int(np.argmax(np.abs(w)))
        bi = V[:, i]
        r = hhl.solve(A, bi, m)
        assert abs(r["P"] - (C / w[i]) ** 2) < 1e-12
        assert abs(r["leakage"]) < 1e-13
        assert np.max(np.abs(r["x"] - bi / w[i])) < 1e-11 / amin


def test_planted_off_by_one_evolution_time_is_caught():
    """t = 2 pi 2^m / (2^m lambda_max) (top = 2^m instead of 2^m - 1) wraps the largest
    eigenvalue around the clock: the pin above sees it."""
    m = 5
    A, b, _ = _default_t_problems()[0]
    w, V = np.linalg.eigh(A)
    M = 1 << m
    h = hhl.build(A, b, m, t=2 * math.pi * M / (M * w[-1]))
    assert _clock_distribution(h, V[:, -1])[M - 1] < 0.5
