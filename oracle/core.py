"""ctypes binding of the C oracle (sv_oracle.c) -- test infrastructure only.

``build()`` compiles sv_oracle.c with gcc (OpenMP) into oracle/_build/libsv_oracle.so.
The library is loaded lazily on first use.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sv_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "libsv_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc -O2 -fopenmp, no machine-specific flags)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        L.ora_apply.argtypes = [dp, ctypes.c_int, ctypes.c_int, ip, ctypes.c_int, ip, ip, dp]
        L.ora_apply.restype = ctypes.c_int
        L.ora_apply_ucry.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ip, dp]
        L.ora_apply_ucry.restype = ctypes.c_int
        L.ora_masked_norm2.argtypes = [dp, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64]
        L.ora_masked_norm2.restype = ctypes.c_double
        L.ora_sum.argtypes = [dp, ctypes.c_int64]
        L.ora_sum.restype = ctypes.c_double
        L.ora_num_threads.restype = ctypes.c_int
        L.ora_set_num_threads.argtypes = [ctypes.c_int]
        _lib = L
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _iarr(v):
    a = np.ascontiguousarray(np.asarray(v, dtype=np.int32))
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def apply_gate(psi: np.ndarray, targets, U: np.ndarray, controls=(), ctrl_vals=None) -> None:
    """In place: psi <- (U on targets, conditioned on controls == ctrl_vals) psi.

    psi: complex128 C-contiguous of length 2^n.  U: complex128 (2^k, 2^k); bit b of its
    row/column index is qubit targets[b].  ctrl_vals defaults to all ones.
    """
    assert psi.dtype == np.complex128 and psi.flags.c_contiguous
    n = int(psi.size).bit_length() - 1
    assert psi.size == 1 << n
    k = len(targets)
    U = np.ascontiguousarray(U, dtype=np.complex128)
    assert U.shape == (1 << k, 1 << k)
    if ctrl_vals is None:
        ctrl_vals = [1] * len(controls)
    ta, tp = _iarr(targets)
    ca, cp = _iarr(list(controls) if len(controls) else [0])
    va, vp = _iarr(list(ctrl_vals) if len(controls) else [0])
    rc = lib().ora_apply(_dptr(psi.view(np.float64)), n, k, tp, len(controls), cp, vp,
                         _dptr(U.view(np.float64)))
    if rc != 0:
        raise ValueError("oracle: bad gate (targets %r controls %r)" % (targets, controls))


def apply_ucry(psi: np.ndarray, target: int, controls, theta: np.ndarray) -> None:
    """In place: for each value v of the control register, RY(theta[v]) on target if the
    controls hold v (controls[j] is bit j of v)."""
    n = int(psi.size).bit_length() - 1
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    assert theta.size == 1 << len(controls)
    ca, cp = _iarr(list(controls) if len(controls) else [0])
    rc = lib().ora_apply_ucry(_dptr(psi.view(np.float64)), n, int(target), len(controls), cp,
                              _dptr(theta))
    if rc != 0:
        raise ValueError("oracle: bad uniformly controlled rotation")


def masked_norm2(psi: np.ndarray, mask: int, want: int) -> float:
    """Compensated sum of |psi_i|^2 over indices with (i & mask) == want."""
    n = int(psi.size).bit_length() - 1
    return float(lib().ora_masked_norm2(_dptr(psi.view(np.float64)), n, mask, want))


def compensated_sum(x: np.ndarray) -> float:
    x = np.ascontiguousarray(x, dtype=np.float64)
    return float(lib().ora_sum(_dptr(x), x.size))


def num_threads() -> int:
    return int(lib().ora_num_threads())


def set_num_threads(t: int) -> None:
    lib().ora_set_num_threads(int(t))
