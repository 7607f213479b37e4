"""Readout tolerances derived from a per-amplitude state bound.

If every amplitude of the device state is within `tol` of the oracle's, the readout quantities
of Sec. III-A steps 3-4 (P = P(ancilla = 1), P0 = P(ancilla = 1, clock = 0), the normalized
slice |x> = slice / sqrt(P0), and x = (sqrt(P) / C) ||b|| |x>) are within the bounds below,
computed from the oracle's state (triangle inequality on | |a|^2 - |b|^2 | <= (|a| + |b|) |a - b|
and first-order bounds on the square root and the division, taken with the worst case of the
perturbed denominator).  The readout's own FP64 summation error is far below these.
"""
import math

import numpy as np


def prob_bound(ref_amps: np.ndarray, tol: float) -> float:
    """|sum |a_i|^2 - sum |b_i|^2| over a set of amplitudes, |a_i - b_i| <= tol."""
    return float(tol * np.sum(2.0 * np.abs(ref_amps) + tol))


def readout_bounds(ref: dict, nb: int, m: int, tol: float, C: float, norm_b: float, N: int, x_off: int = 0):
    """Bounds on |dP|, |dP0|, |d x_state_i| (first N entries from x_off) and |d x_i| given the
    oracle result `ref` (psi, P, P0, x_state) and the per-amplitude state bound `tol`."""
    psi = ref["psi"]
    n = nb + m + 1
    half = 1 << (n - 1)
    dP = prob_bound(psi[half:], tol)
    sl = psi[half: half + (1 << nb)]
    dP0 = prob_bound(sl, tol)
    P, P0 = ref["P"], ref["P0"]
    if not (dP0 < P0 and dP < P):
        return dict(P=dP, P0=dP0, x_state=np.inf, x=np.inf)
    s = np.abs(sl[x_off: x_off + N])
    lo0 = P0 - dP0
    dxs = tol / math.sqrt(lo0) + s * dP0 / (2.0 * lo0 ** 1.5)
    xs = np.abs(ref["x_state"][x_off: x_off + N])
    dsqrtP = dP / math.sqrt(P - dP)
    dx = (norm_b / C) * (math.sqrt(P + dP) * dxs + xs * dsqrtP)
    return dict(P=dP, P0=dP0, x_state=dxs, x=dx)


def cond_tol(m: int) -> float:
    """Per-amplitude state bound when the library and the oracle each eigendecompose A: two
    correct eigensolvers give eigenvalues that differ by a few ulps of ||A||, and the phase
    estimation multiplies the difference by t 2^j <= 2 pi 2^m / lambda_max, so the phases
    differ by up to 2^m 2 pi 8 eps."""
    return max(1e-12, 2.0 ** m * 2 * math.pi * 8 * np.finfo(np.float64).eps)
