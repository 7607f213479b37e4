"""HHL as the paper's procedure, step by step, in FP64 -- test infrastructure only.

Follows the "Practical HHL procedures" box of Sec. III-A (steps 1-4), the HHL decomposition
|x> = sum_i lambda_i^-1 b_i |v_i> of Sec. III-A, the circuit structure of Fig. 5 (state
preparation, quantum phase estimation, eigenvalue-inversion rotation on an ancilla, inverse
phase estimation) and the resource formula of Sec. III-B.

Readings of points the paper leaves open (the same list is kept with the design notes):
  * qubit order little-endian; data qubits 0..nb-1, clock qubit j is nb+j (bit j of the clock
    value), the ancilla is qubit nb+m;
  * evolution U = exp(+iAt); clock qubit j controls U^(2^j); an eigenvalue lambda lands on clock
    value k = lambda t 2^m / (2 pi); the inverse QFT includes the final qubit-reversal swaps;
  * default t = 2 pi (2^m - 1) / (2^m lambda_max) (lambda_max on the top grid value); for an
    indefinite A the clock register is two's complement (its top bit is the sign qubit of
    Sec. III-B) and t = 2 pi (2^(m-1) - 1) / (2^m max|lambda|);
    grid value of clock k: lt_k = 2 pi k / (t 2^m); default C = the largest grid value not above
    lambda_min (at least one grid step); theta_k = 2 asin(C / lt_k), clamped to pi where
    C / lt_k > 1, and theta_0 = 0;
  * padding to 2^nb: block-diag(A, lambda_max I), b padded with zeros;
  * readout: P = P(ancilla = 1); P0 = P(ancilla = 1 and clock = 0); |x> is the
    (ancilla = 1, clock = 0) slice divided by sqrt(P0); ||x|| = sqrt(P) / C (the printed
    ||x|| = |lambda_0| sqrt(P) holds when C = |lambda_0|); x = ||x|| ||b|| |x>;
  * n_total counts the ancilla, and Table I's n_QPE column includes the sign qubit n_negval.
"""
from __future__ import annotations

import math

import numpy as np

from . import core

# ---------------------------------------------------------------- textbook gate matrices
SQRT1_2 = 1.0 / math.sqrt(2.0)
H = np.array([[SQRT1_2, SQRT1_2], [SQRT1_2, -SQRT1_2]], dtype=np.complex128)
SWAP = np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], dtype=np.complex128)


def RY(theta: float) -> np.ndarray:
    c, s = math.cos(theta / 2), math.sin(theta / 2)
    return np.array([[c, -s], [s, c]], dtype=np.complex128)


def CP(phi: float) -> np.ndarray:
    """Controlled phase on two qubits: diag(1, 1, 1, e^{i phi})."""
    return np.diag([1, 1, 1, np.exp(1j * phi)]).astype(np.complex128)


# A gate of the unfused list: ("u", targets, U, controls, ctrl_vals) or
# ("ucry", target, controls, thetas).


def qft_gates(qubits, inverse: bool):
    """QFT |x> = 2^{-m/2} sum_k exp(2 pi i x k / 2^m) |k> on `qubits` (qubits[j] = bit j).

    Textbook circuit (Nielsen & Chuang Sec. 5.1) for the most significant qubit first: H on a
    qubit, then controlled phases 2 pi / 2^(d+1) from each lower qubit at distance d, and the
    bit-reversal swaps at the end.  The inverse is the reversed sequence with conjugate phases.
    """
    m = len(qubits)
    seq = []
    for j in range(m - 1, -1, -1):
        seq.append(("u", [qubits[j]], H, [], []))
        for l in range(j - 1, -1, -1):
            seq.append(("u", [qubits[l], qubits[j]], CP(2 * math.pi / 2 ** (j - l + 1)), [], []))
    for j in range(m // 2):
        seq.append(("u", [qubits[j], qubits[m - 1 - j]], SWAP, [], []))
    if not inverse:
        return seq
    out = []
    for g in reversed(seq):
        out.append(("u", g[1], g[2].conj().T, [], []))
    return out


def dft_pass(psi: np.ndarray, targets, sign: int, src=(), pre: bool = False) -> None:
    """In place: one Cooley-Tukey stage of a (inverse) QFT on the register `targets`.

    With y the value of `targets` (bit j <-> targets[j], k bits) and w the value of `src`
    (bit j <-> src[j], s bits), for every w apply the 2^k x 2^k unitary
        F[y', y] = 2^{-k/2} exp(sign 2 pi i y y' / 2^k)
    followed (pre=False) or preceded (pre=True) by the diagonal twiddle
        T_w[y] = exp(sign 2 pi i w y / 2^(k+s)).
    A QFT on m qubits splits into such passes by the Cooley-Tukey factorisation of the DFT of
    size 2^m (Cooley & Tukey 1965): the top field's pass carries the twiddle of the bits below
    it, and the result is the QFT with its output digits in field order.  Written with the
    textbook dense-gate rule: one gate per value w, conditioned on src == w.
    """
    k, s = len(targets), len(src)
    K = 1 << k
    y = np.arange(K, dtype=np.int64)
    F = np.exp(sign * 2j * np.pi * ((np.outer(y, y) % K) / K)) / math.sqrt(K)
    for w in range(1 << s):
        T = np.exp(sign * 2j * np.pi * (((w * y) % (1 << (k + s))) / (1 << (k + s))))
        G = F * T[None, :] if pre else T[:, None] * F
        vals = [(w >> j) & 1 for j in range(s)]
        core.apply_gate(psi, list(targets), G, list(src), vals)


def resource_counts(n_rows: int, kappa: float, has_negative: bool):
    """Sec. III-B qubit count, with Table I's conventions (ancilla counted, sign qubit in n_QPE).

    Returns (n_total, n_data, n_qpe_table)."""
    n_data = int(math.ceil(math.log2(n_rows))) if n_rows > 1 else 1
    n_qpe = max(n_data + 1, int(math.ceil(math.log2(kappa + 1))))
    n_neg = 1 if has_negative else 0
    return n_data + n_qpe + n_neg + 1, n_data, n_qpe + n_neg


def check_problem(A: np.ndarray, b: np.ndarray):
    """Shape, finiteness and Hermiticity checks (step 1 takes A Hermitian)."""
    A = np.asarray(A, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128).ravel()
    N = A.shape[0]
    if A.shape != (N, N) or b.size != N or N < 1:
        raise ValueError("shape")
    if not (np.all(np.isfinite(A)) and np.all(np.isfinite(b))):
        raise ValueError("non-finite input")
    scale = max(1.0, float(np.max(np.abs(A))))
    if np.max(np.abs(A - A.conj().T)) > 1e-12 * scale:
        raise ValueError("A is not Hermitian")
    if np.linalg.norm(b) == 0:
        raise ValueError("b = 0")
    return A, b


def build(A, b, m: int, t: float = 0.0, C: float = 0.0):
    """Step 1 and 2 of the procedure: normalize b, pad, and emit the unfused HHL gate list.

    A positive definite A uses the clock value k as is.  An indefinite A (Sec. III-B's sign
    qubit, n_negval = 1) reads the clock register as a two's-complement number: clock value c
    stands for c - 2^m when c >= 2^(m-1), t maps the largest |lambda| to 2^(m-1) - 1, and the
    rotation angle takes the sign of the grid value."""
    A, b = check_problem(A, b)
    N = A.shape[0]
    bnorm = float(np.linalg.norm(b))
    bhat = b / bnorm
    nb = max(1, int(math.ceil(math.log2(N))))
    lam_A = np.linalg.eigvalsh(A)
    absl = np.abs(lam_A)
    if absl.min() == 0 or absl.min() <= 1e-14 * absl.max():
        raise ValueError("A is singular")
    signed = bool(lam_A[0] < 0)
    lam_amax, lam_amin = float(absl.max()), float(absl.min())
    D = 1 << nb
    Ap = np.zeros((D, D), dtype=np.complex128)
    Ap[:N, :N] = A
    for i in range(N, D):
        Ap[i, i] = lam_amax
    bp = np.zeros(D, dtype=np.complex128)
    bp[:N] = bhat
    lam, V = np.linalg.eigh(Ap)
    if m <= 0:
        m = resource_counts(N, lam_amax / lam_amin, signed)[2]
    M = 1 << m
    if t <= 0:
        top = (M // 2 - 1) if signed else (M - 1)
        t = 2 * math.pi * top / (M * lam_amax)
    step = 2 * math.pi / (t * M)              # grid value of clock k is k * step
    if C <= 0:
        C = max(1.0, math.floor(lam_amin / step * (1 + 1e-9))) * step
    elif C > lam_amin * (1 + 1e-9):
        raise ValueError("C above the smallest |eigenvalue|")
    k = np.arange(M, dtype=np.float64)
    if signed:
        k = np.where(k >= M // 2, k - M, k)   # two's complement clock value
    theta = np.zeros(M)
    nz = k != 0
    r = np.zeros(M)
    r[nz] = C / (k[nz] * step)
    theta[nz] = 2.0 * np.arcsin(np.clip(r[nz], -1.0, 1.0))

    data = list(range(nb))
    clock = [nb + j for j in range(m)]
    anc = nb + m
    gates = []
    qpe = []
    for q in clock:
        qpe.append(("u", [q], H, [], []))
    for j in range(m):
        Uj = (V * np.exp(1j * lam * t * 2 ** j)) @ V.conj().T
        qpe.append(("u", data, Uj, [clock[j]], [1]))
    qpe += qft_gates(clock, inverse=True)
    gates += qpe
    gates.append(("ucry", anc, clock, theta))
    for g in reversed(qpe):
        gates.append(("u", g[1], g[2].conj().T, g[3], g[4]))
    return dict(N=N, nb=nb, m=m, n=nb + m + 1, t=t, C=C, bnorm=bnorm, b_pad=bp, gates=gates,
                theta=theta, lam=lam, signed=signed)


def preprocess(A, b, gauss_seidel: bool = False, dilate: bool = False):
    """Sec. III-A step 1(a) and 1(c).

    (a) Gauss-Seidel preconditioning: with M the lower triangle of A including the diagonal
        (the Gauss-Seidel splitting), solve M A' = A and M b' = b; A' is generally not Hermitian.
    (c) Hermitian dilation: a non-Hermitian A' (or `dilate`) becomes [[0, A'], [A'^H, 0]] with
        right-hand side [b'; 0]; its solution is [0; x], so x is the lower half.
    Returns (A_eff, b_eff, x_offset, N)."""
    A = np.asarray(A, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128).ravel()
    N = A.shape[0]
    if gauss_seidel:
        M = np.tril(A)
        A = np.linalg.solve(M, A)
        b = np.linalg.solve(M, b)
    herm = np.max(np.abs(A - A.conj().T)) <= 1e-12 * max(1.0, float(np.max(np.abs(A))))
    if dilate or not herm:
        Z = np.zeros((N, N), dtype=np.complex128)
        A = np.block([[Z, A], [A.conj().T, Z]])
        b = np.concatenate([b, np.zeros(N, dtype=np.complex128)])
        return A, b, N, N
    return A, b, 0, N


def solve_general(A, b, m: int, t: float = 0.0, C: float = 0.0, gauss_seidel: bool = False,
                  dilate: bool = False):
    """HHL with the optional preprocessing of Sec. III-A step 1; x is mapped back to A x = b."""
    Ae, be, off, N = preprocess(A, b, gauss_seidel, dilate)
    r = solve(Ae, be, m, t, C)
    r["x_eff"] = r["x"]
    r["x"] = r["x"][off: off + N]
    return r


def initial_state(h) -> np.ndarray:
    """|0>_anc |0>_clock |b>: the normalized, padded b in the lowest 2^nb amplitudes."""
    psi = np.zeros(1 << h["n"], dtype=np.complex128)
    psi[: 1 << h["nb"]] = h["b_pad"]
    return psi


def run(h, psi: np.ndarray | None = None) -> np.ndarray:
    """Apply every gate of the unfused list in order (step 2), from the initial state."""
    if psi is None:
        psi = initial_state(h)
    for g in h["gates"]:
        if g[0] == "u":
            core.apply_gate(psi, g[1], g[2], g[3], g[4])
        else:
            core.apply_ucry(psi, g[1], g[2], g[3])
    return psi


def readout(h, psi: np.ndarray):
    """Steps 3-4: read |x>, P(ancilla = 1) and the solution x from the final state."""
    nb, m = h["nb"], h["m"]
    anc_bit = 1 << (nb + m)
    clock_mask = ((1 << m) - 1) << nb
    norm2 = core.masked_norm2(psi, 0, 0)
    P = core.masked_norm2(psi, anc_bit, anc_bit)
    P0 = core.masked_norm2(psi, anc_bit | clock_mask, anc_bit)
    sl = psi[anc_bit: anc_bit + (1 << nb)].copy()
    x_state = sl / math.sqrt(P0)
    norm_x = math.sqrt(P) / h["C"]
    x = norm_x * h["bnorm"] * x_state[: h["N"]]
    return dict(x=x, x_state=x_state, P=P, P0=P0, leakage=P - P0, norm2=norm2, norm_x=norm_x)


def solve(A, b, m: int, t: float = 0.0, C: float = 0.0):
    h = build(A, b, m, t, C)
    psi = run(h)
    r = readout(h, psi)
    r["psi"] = psi
    r["circuit"] = h
    return r


def classical_solution(A, b) -> np.ndarray:
    return np.linalg.solve(np.asarray(A, dtype=np.complex128), np.asarray(b, dtype=np.complex128))
