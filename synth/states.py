"""Random complex-Gaussian initial state vectors from a counter-based generator.

Amplitude i of a state with seed s is a pure function of (s, i), so a sampled parity check can
regenerate any input amplitude on the host without holding the whole 2^n vector.  One
definition, two implementations (numpy on the host, torch integer ops on a device) that a CPU
test checks against each other:

  * counter c -> 64-bit word: the c-th output of a SplitMix64 sequence whose state starts at
    key(s) (Steele, Lea & Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014:
    state += 0x9E3779B97F4A7C15, then the xor-shift/multiply finaliser with constants
    0xBF58476D1CE4E5B9 and 0x94D049BB133111EB);
  * word -> uniform in [0, 1): top 53 bits times 2^-53;
  * amplitude i: Box-Muller on the uniforms of counters 2i and 2i+1,
    r = sqrt(-2 ln(1 - u1)), amp = r (cos 2 pi u2 + i sin 2 pi u2), times 2^(-(n+1)/2) so that
    the expected squared norm is exactly 1.
"""
from __future__ import annotations

import numpy as np

STATE_SCALE_NOTE = "complex Gaussian amplitudes scaled by 2^-(n+1)/2 (E||psi||^2 = 1)"

_GOLDEN = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB
_MASK64 = (1 << 64) - 1


def _key(seed: int) -> int:
    return (int(seed) * 0xD1B54A32D192ED03 + 0x632BE59BD9B4E019) & _MASK64


def _mix_np(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * np.uint64(_M1)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(_M2)
    return z ^ (z >> np.uint64(31))


def counter_uniform_np(seed: int, counters: np.ndarray) -> np.ndarray:
    """Uniform doubles in [0, 1) for the given uint64 counters."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(_key(seed)) + (c + np.uint64(1)) * np.uint64(_GOLDEN)
        z = _mix_np(z)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def gaussian_amplitudes_at(seed: int, n: int, idx) -> np.ndarray:
    """Amplitudes psi[idx] of the n-qubit seeded Gaussian state (complex128)."""
    idx = np.asarray(idx, dtype=np.uint64)
    u1 = counter_uniform_np(seed, idx * np.uint64(2))
    u2 = counter_uniform_np(seed, idx * np.uint64(2) + np.uint64(1))
    r = np.sqrt(-2.0 * np.log1p(-u1))
    scale = 2.0 ** (-(n + 1) / 2.0)
    return (r * scale) * np.exp(2j * np.pi * u2)


def gaussian_state_np(seed: int, n: int, chunk: int = 1 << 22) -> np.ndarray:
    """Whole n-qubit seeded Gaussian state as a complex128 numpy array (host)."""
    N = 1 << n
    out = np.empty(N, dtype=np.complex128)
    for s in range(0, N, chunk):
        e = min(N, s + chunk)
        out[s:e] = gaussian_amplitudes_at(seed, n, np.arange(s, e, dtype=np.uint64))
    return out


def _signed(x: int) -> int:
    return x - (1 << 64) if x >= (1 << 63) else x


def _srl_t(x, s: int):
    # logical right shift of int64 tensors (torch's >> is arithmetic)
    return (x >> s) & ((1 << (64 - s)) - 1)


def _counter_uniform_t(seed: int, c):
    """torch int64 version of counter_uniform_np (two's-complement wrapping arithmetic)."""
    z = (c + 1) * _signed(_GOLDEN) + _signed(_key(seed))
    z = (z ^ _srl_t(z, 30)) * _signed(_M1)
    z = (z ^ _srl_t(z, 27)) * _signed(_M2)
    z = z ^ _srl_t(z, 31)
    return _srl_t(z, 11).to(dtype=__import__("torch").float64) * (1.0 / 9007199254740992.0)


def gaussian_state_torch(seed: int, n: int, dtype, device, chunk: int = 1 << 24, normalize=False):
    """Whole n-qubit seeded Gaussian state as a torch tensor (complex64/complex128) on `device`.

    Element i equals ``gaussian_amplitudes_at(seed, n, i)`` (rounded to complex64 for that
    dtype).  With ``normalize`` the vector is divided by its exact norm afterwards (used for
    benchmarks, which do not compare against sampled host values).
    """
    import torch

    N = 1 << n
    out = torch.empty(N, dtype=dtype, device=device)
    scale = 2.0 ** (-(n + 1) / 2.0)
    for s in range(0, N, chunk):
        e = min(N, s + chunk)
        i = torch.arange(s, e, dtype=torch.int64, device=device)
        u1 = _counter_uniform_t(seed, 2 * i)
        u2 = _counter_uniform_t(seed, 2 * i + 1)
        r = torch.sqrt(-2.0 * torch.log1p(-u1)) * scale
        ang = 2.0 * np.pi * u2
        out[s:e] = torch.complex(r * torch.cos(ang), r * torch.sin(ang)).to(dtype)
        del i, u1, u2, r, ang
    if normalize:
        real = torch.view_as_real(out)
        nrm = torch.linalg.vector_norm(real, dtype=torch.float64)
        out /= nrm.to(out.real.dtype)
    return out
