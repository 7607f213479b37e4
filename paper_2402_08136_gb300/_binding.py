"""ctypes binding of libqsim_gb300.so with the same names as the C ABI (include/qsim.h)."""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(HERE, "libqsim_gb300.so")

QSIM_OK = 0
QSIM_C64 = 1
QSIM_C128 = 2
_STATUS = {-1: "EINVAL", -2: "ENOMEM", -3: "EBUSY", -4: "ECUDA", -5: "ETIMEOUT", -6: "ENOTFOUND"}


class QsimError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s (%d): %s" % (_STATUS.get(code, "?"), code, msg))
        self.code = code


class QsimLibraryMissing(ImportError):
    pass


class _CircuitInfo(ctypes.Structure):
    _fields_ = [("n_qubits", ctypes.c_int), ("n_gates", ctypes.c_int), ("n_dense", ctypes.c_int),
                ("n_diag", ctypes.c_int), ("n_perm", ctypes.c_int), ("n_ucry", ctypes.c_int),
                ("max_k", ctypes.c_int), ("fused", ctypes.c_int), ("bytes_c64", ctypes.c_double),
                ("bytes_c128", ctypes.c_double), ("flops", ctypes.c_double), ("n_dft", ctypes.c_int)]


class _HHLInfo(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("nb", ctypes.c_int), ("m", ctypes.c_int), ("n", ctypes.c_int),
                ("t", ctypes.c_double), ("C", ctypes.c_double), ("norm_b", ctypes.c_double),
                ("lambda_min", ctypes.c_double), ("lambda_max", ctypes.c_double),
                ("n_total_formula", ctypes.c_int), ("n_gates", ctypes.c_int), ("N_eff", ctypes.c_int),
                ("flags", ctypes.c_int)]


class _ReadoutStats(ctypes.Structure):
    _fields_ = [("p_success", ctypes.c_double), ("p_clock0", ctypes.c_double),
                ("leakage", ctypes.c_double), ("norm2", ctypes.c_double),
                ("norm_x", ctypes.c_double), ("norm_b", ctypes.c_double)]


class _HHLRequest(ctypes.Structure):
    _fields_ = [("A", ctypes.POINTER(ctypes.c_double)), ("b", ctypes.POINTER(ctypes.c_double)),
                ("N", ctypes.c_int), ("n_clock", ctypes.c_int), ("t", ctypes.c_double),
                ("C", ctypes.c_double), ("dtype", ctypes.c_int), ("flags", ctypes.c_int)]


class _PoolInfo(ctypes.Structure):
    _fields_ = [("bytes_total", ctypes.c_size_t), ("bytes_in_use", ctypes.c_size_t),
                ("bytes_peak", ctypes.c_size_t), ("queued", ctypes.c_int), ("building", ctypes.c_int),
                ("running", ctypes.c_int), ("done", ctypes.c_int), ("failed", ctypes.c_int),
                ("batches_launched", ctypes.c_longlong), ("singles_launched", ctypes.c_longlong)]


QSIM_TUNE_DFT_TMA = 0
QSIM_TUNE_DFT_LANES = 1
QSIM_TUNE_DFT_PREFETCH = 2
QSIM_TUNE_DENSE_TC = 3
QSIM_TUNE_FUSE_WIDTH = 4
QSIM_TUNE_DFT_L2PROMO = 5
QSIM_TUNE_DFT_MERGE = 6
QSIM_TUNE_TUNED = 7
QSIM_TUNE_COUNT = 8
TUNE_NAMES = ("dft_tma", "dft_lanes", "dft_prefetch", "dense_tc", "fuse_width", "dft_l2promo", "dft_merge", "tuned")


class _PoolLaunch(ctypes.Structure):
    _fields_ = [("slot", ctypes.c_int), ("batched", ctypes.c_int), ("n_requests", ctypes.c_int),
                ("first_ticket", ctypes.c_uint64), ("last_ticket", ctypes.c_uint64),
                ("t_start", ctypes.c_double), ("t_end", ctypes.c_double)]


class _ShardStep(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("global_bit", ctypes.c_int), ("local_qubit", ctypes.c_int),
                ("first_gate", ctypes.c_int), ("last_gate", ctypes.c_int)]


class _TuneReport(ctypes.Structure):
    _fields_ = [("n_qubits", ctypes.c_int), ("values", ctypes.c_int * QSIM_TUNE_COUNT),
                ("dft_ms", ctypes.c_double), ("dense_ms", ctypes.c_double * 4),
                ("fuse_ms", ctypes.c_double * 5)]


_lib = None

_VP = ctypes.c_void_p
_IP = ctypes.POINTER(ctypes.c_int)
_DP = ctypes.POINTER(ctypes.c_double)
_SIGS = {
    "qsim_last_error": ([], ctypes.c_char_p),
    "qsim_version": ([], ctypes.c_char_p),
    "qsim_circuit_create": ([ctypes.c_int, ctypes.POINTER(_VP)], ctypes.c_int),
    "qsim_circuit_add_gate": ([_VP, ctypes.c_int, _IP, ctypes.c_int, _IP, _DP], ctypes.c_int),
    "qsim_circuit_add_ucry": ([_VP, ctypes.c_int, ctypes.c_int, _IP, _DP], ctypes.c_int),
    "qsim_circuit_add_dft": ([_VP, ctypes.c_int, _IP, ctypes.c_int, _IP, ctypes.c_int, ctypes.c_int],
                             ctypes.c_int),
    "qsim_circuit_add_walsh": ([_VP, ctypes.c_int, _IP], ctypes.c_int),
    "qsim_circuit_free": ([_VP], None),
    "qsim_circuit_get_info": ([_VP, ctypes.POINTER(_CircuitInfo)], ctypes.c_int),
    "qsim_fuse": ([_VP, ctypes.c_int, ctypes.POINTER(_VP)], ctypes.c_int),
    "qsim_fuse_paper": ([_VP, ctypes.POINTER(_VP)], ctypes.c_int),
    "qsim_circuit_get_gate": ([_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                               ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                               ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "qsim_apply": ([_VP, ctypes.c_int, ctypes.c_int, _VP, _VP], ctypes.c_int),
    "hhl_build": ([_DP, _DP, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                   ctypes.POINTER(_VP)], ctypes.c_int),
    "hhl_build_spectral": ([_DP, _DP, _DP, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                            ctypes.c_double, ctypes.POINTER(_VP)], ctypes.c_int),
    "hhl_build_ex": ([_DP, _DP, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                      ctypes.POINTER(_VP)], ctypes.c_int),
    "hhl_build_spectral_ex": ([_DP, _DP, _DP, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                               ctypes.c_double, ctypes.c_int, ctypes.POINTER(_VP)], ctypes.c_int),
    "qsim_hermitian_eig": ([_DP, ctypes.c_int, ctypes.c_int, _DP, _DP], ctypes.c_int),
    "qsim_launch_counts": ([ctypes.POINTER(ctypes.c_ulonglong), ctypes.c_int], ctypes.c_int),
    "qsim_tune_get": ([ctypes.c_int, ctypes.c_int, ctypes.c_int, _IP], ctypes.c_int),
    "qsim_tune_set": ([ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "qsim_tune_reset": ([], ctypes.c_int),
    "qsim_autotune": ([_VP, ctypes.c_int, ctypes.c_int, _VP, ctypes.POINTER(_TuneReport)], ctypes.c_int),
    "hhl_circuit_free": ([_VP], None),
    "hhl_as_circuit": ([_VP], _VP),
    "hhl_get_info": ([_VP, ctypes.POINTER(_HHLInfo)], ctypes.c_int),
    "hhl_prepare_state": ([_VP, ctypes.c_int, _VP, _VP], ctypes.c_int),
    "hhl_run": ([_VP, ctypes.c_int, _VP, _VP, _VP], ctypes.c_int),
    "hhl_run_sums": ([_VP, ctypes.c_int, _VP, _VP, _VP, _VP], ctypes.c_int),
    "hhl_readout_sums": ([_VP, ctypes.c_int, _VP, _VP, _VP, _DP, _DP, ctypes.POINTER(_ReadoutStats)], ctypes.c_int),
    "qsim_launch_count": ([], ctypes.c_ulonglong),
    "qsim_device_status": ([ctypes.POINTER(ctypes.c_uint), ctypes.c_int], ctypes.c_int),
    "qsim_batch_create": ([ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.c_int, ctypes.c_int,
                           ctypes.POINTER(_VP)], ctypes.c_int),
    "hhl_batch_create": ([ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.c_int,
                          ctypes.c_int, ctypes.POINTER(_VP)], ctypes.c_int),
    "qsim_batch_run": ([_VP, _VP], ctypes.c_int),
    "hhl_batch_results": ([_VP, _VP, _DP, ctypes.POINTER(_ReadoutStats)], ctypes.c_int),
    "hhl_batch_solve": ([_VP, _VP, _DP, ctypes.POINTER(_ReadoutStats)], ctypes.c_int),
    "qsim_batch_free": ([_VP], None),
    "hhl_batch_autotune": ([ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.c_int, ctypes.c_int, _IP,
                            ctypes.c_int, _VP, _IP, _DP], ctypes.c_int),
    "qsim_apply_batched": ([ctypes.POINTER(_VP), _IP, ctypes.POINTER(_VP), ctypes.c_int, ctypes.c_int, _VP],
                           ctypes.c_int),
    "qsim_pool_create": ([ctypes.c_size_t, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_VP)], ctypes.c_int),
    "qsim_submit": ([_VP, ctypes.POINTER(_HHLRequest), ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    "qsim_poll": ([_VP, ctypes.c_uint64, _DP, ctypes.POINTER(_ReadoutStats), _DP], ctypes.c_int),
    "qsim_pool_wait": ([_VP, ctypes.c_uint64, ctypes.c_double], ctypes.c_int),
    "qsim_pool_get_info": ([_VP, ctypes.POINTER(_PoolInfo)], ctypes.c_int),
    "qsim_pool_take_completed": ([_VP, ctypes.POINTER(ctypes.c_uint64), ctypes.c_int, _IP, ctypes.c_double],
                                 ctypes.c_int),
    "qsim_pool_destroy": ([_VP], None),
    "qsim_shard_plan_create": ([_VP, ctypes.c_int, ctypes.POINTER(_VP)], ctypes.c_int),
    "qsim_shard_plan_num_steps": ([_VP], ctypes.c_int),
    "qsim_shard_plan_get_step": ([_VP, ctypes.c_int, ctypes.POINTER(_ShardStep), _IP], ctypes.c_int),
    "qsim_shard_plan_local_circuit": ([_VP, ctypes.c_int], _VP),
    "qsim_shard_plan_free": ([_VP], None),
    "qsim_shard_pack": ([_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP, _VP], ctypes.c_int),
    "qsim_shard_unpack": ([_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP, _VP], ctypes.c_int),
    "qsim_pool_launch_log": ([_VP, ctypes.POINTER(_PoolLaunch), ctypes.c_int, _IP], ctypes.c_int),
    "hhl_readout": ([_VP, ctypes.c_int, _VP, _VP, _DP, _DP, ctypes.POINTER(_ReadoutStats)],
                    ctypes.c_int),
}


def library_path() -> str:
    return _LIB_PATH


def library():
    """Load libqsim_gb300.so (built in-tree by build.py); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise QsimLibraryMissing(
                "libqsim_gb300.so not built: run paper_2402_08136_gb300/build.py "
                "(there is no CPU fallback)")
        L = ctypes.CDLL(_LIB_PATH)
        for name, (args, res) in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(rc: int):
    if rc != QSIM_OK:
        raise QsimError(rc, library().qsim_last_error().decode())


def _ints(v):
    a = np.ascontiguousarray(np.asarray(list(v) if len(v) else [0], dtype=np.int32))
    return a, a.ctypes.data_as(_IP)


def _cplx(a):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.complex128))
    return a, a.view(np.float64).ctypes.data_as(_DP)


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(stream.cuda_stream))


def _dtype_of(state):
    import torch
    if state.dtype == torch.complex64:
        return QSIM_C64
    if state.dtype == torch.complex128:
        return QSIM_C128
    raise QsimError(-1, "state must be complex64 or complex128")


def _check_state(state, n: int):
    if not state.is_cuda or not state.is_contiguous() or state.numel() != (1 << n):
        raise QsimError(-1, "state must be a contiguous CUDA tensor of 2^n amplitudes")


def qsim_launch_count() -> int:
    """Kernels this library has launched in this process (graph replays not included)."""
    return int(library().qsim_launch_count())


KERNEL_FAMILIES = ("dense_simt", "dense_tc", "fourier", "fourier_tma", "expand", "elementwise", "batched",
                   "readout", "prep")


def qsim_launch_counts() -> dict:
    """Kernels launched by the library in this process, by family (see QSIM_KERNEL_*)."""
    arr = (ctypes.c_ulonglong * len(KERNEL_FAMILIES))()
    _check(library().qsim_launch_counts(arr, len(KERNEL_FAMILIES)))
    return {name: int(arr[i]) for i, name in enumerate(KERNEL_FAMILIES)}


def qsim_device_status(clear: bool = False) -> int:
    """Sticky device-side error flags (bit 0: a bounded wait in a tensor-core kernel ran out)."""
    v = ctypes.c_uint(0)
    _check(library().qsim_device_status(ctypes.byref(v), 1 if clear else 0))
    return int(v.value)


def qsim_version() -> str:
    return library().qsim_version().decode()


class Circuit:
    """Owning handle of a qsim_circuit (or a borrowed view when `owner` is given)."""

    def __init__(self, n_qubits: int | None = None, _ptr=None, _owner=None):
        L = library()
        if _ptr is None:
            p = _VP()
            _check(L.qsim_circuit_create(int(n_qubits), ctypes.byref(p)))
            _ptr = p
        self._ptr = _ptr
        self._owner = _owner

    @property
    def ptr(self):
        return self._ptr

    def add_gate(self, targets, U, controls=()):
        t, tp = _ints(targets)
        c, cp = _ints(controls)
        u, up = _cplx(U)
        k = len(targets)
        if u.shape != (1 << k, 1 << k):
            raise QsimError(-1, "U must be 2^k x 2^k")
        _check(library().qsim_circuit_add_gate(self._ptr, k, tp, len(controls), cp, up))
        return self

    def add_ucry(self, target, controls, theta):
        c, cp = _ints(controls)
        th = np.ascontiguousarray(np.asarray(theta, dtype=np.float64))
        if th.size != 1 << len(controls):
            raise QsimError(-1, "theta must have 2^n_controls entries")
        _check(library().qsim_circuit_add_ucry(self._ptr, int(target), len(controls), cp,
                                               th.ctypes.data_as(_DP)))
        return self

    def add_dft(self, targets, sign: int, src=(), twiddle_first: bool = False):
        """One Cooley-Tukey pass of a QFT on the field `targets` (qsim_circuit_add_dft)."""
        t, tp = _ints(targets)
        s_, sp = _ints(src)
        _check(library().qsim_circuit_add_dft(self._ptr, len(targets), tp, len(src), sp, int(sign),
                                              1 if twiddle_first else 0))
        return self

    def add_walsh(self, targets):
        """H on every target qubit as one Walsh-Hadamard pass (qsim_circuit_add_walsh)."""
        t, tp = _ints(targets)
        _check(library().qsim_circuit_add_walsh(self._ptr, len(targets), tp))
        return self

    def info(self) -> dict:
        s = _CircuitInfo()
        _check(library().qsim_circuit_get_info(self._ptr, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in s._fields_}

    @property
    def n_qubits(self) -> int:
        return self.info()["n_qubits"]

    def __del__(self):
        if getattr(self, "_owner", None) is None and getattr(self, "_ptr", None):
            try:
                library().qsim_circuit_free(self._ptr)
            except Exception:
                pass
            self._ptr = None


def qsim_fuse(circuit: Circuit, max_k: int = 0) -> Circuit:
    p = _VP()
    _check(library().qsim_fuse(circuit.ptr, int(max_k), ctypes.byref(p)))
    return Circuit(_ptr=p)


def qsim_fuse_paper(circuit: Circuit) -> Circuit:
    """The paper's priority-ordered fusion of gates on at most two qubits (Sec. II-C, Fig. 4)."""
    p = _VP()
    _check(library().qsim_fuse_paper(circuit.ptr, ctypes.byref(p)))
    return Circuit(_ptr=p)


def qsim_circuit_gates(circuit: Circuit) -> list:
    """The circuit's gates as dicts: kind, targets, controls and, for dense gates, U (numpy)."""
    import numpy as np
    out = []
    for i in range(circuit.info()["n_gates"]):
        kind, k, nc = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(library().qsim_circuit_get_gate(circuit.ptr, i, ctypes.byref(kind), ctypes.byref(k), None,
                                               ctypes.byref(nc), None, None))
        t = (ctypes.c_int * max(1, k.value))()
        c = (ctypes.c_int * max(1, nc.value))()
        U = (ctypes.c_double * (2 * 4 ** k.value))() if kind.value == 0 else None
        _check(library().qsim_circuit_get_gate(circuit.ptr, i, ctypes.byref(kind), ctypes.byref(k), t, ctypes.byref(nc),
                                               c, U))
        g = {"kind": kind.value, "targets": list(t)[:k.value], "controls": list(c)[:nc.value]}
        if U is not None:
            a = np.frombuffer(U, dtype=np.float64)
            g["U"] = (a[0::2] + 1j * a[1::2]).reshape(1 << k.value, 1 << k.value).copy()
        out.append(g)
    return out


def qsim_apply(state, circuit: Circuit, stream=None, n_qubits: int | None = None):
    """Apply `circuit` to the CUDA tensor `state` in place, asynchronously on `stream`."""
    n = circuit.n_qubits if n_qubits is None else n_qubits
    _check_state(state, n)
    _check(library().qsim_apply(ctypes.c_void_p(state.data_ptr()), n, _dtype_of(state),
                                circuit.ptr, _stream_ptr(stream)))
    return state


class HHLCircuit:
    def __init__(self, ptr):
        self._ptr = ptr

    @property
    def ptr(self):
        return self._ptr

    def info(self) -> dict:
        s = _HHLInfo()
        _check(library().hhl_get_info(self._ptr, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in s._fields_}

    def as_circuit(self) -> Circuit:
        return Circuit(_ptr=_VP(library().hhl_as_circuit(self._ptr)), _owner=self)

    def __del__(self):
        if getattr(self, "_ptr", None):
            try:
                library().hhl_circuit_free(self._ptr)
            except Exception:
                pass
            self._ptr = None


QSIM_HHL_STRUCTURED_QPE = 1
QSIM_HHL_GAUSS_SEIDEL = 2
QSIM_HHL_DILATE = 4
QSIM_HHL_FFT_QFT = 8


def hhl_build(A, b, n_clock: int = 0, t: float = 0.0, C: float = 0.0,
              structured: bool = False, gauss_seidel: bool = False, dilate: bool = False,
              fft_qft: bool = False) -> HHLCircuit:
    """hhl_build (no options: the paper's controlled evolutions) or hhl_build_ex with the
    options (structured phase estimation, Gauss-Seidel preconditioning, Hermitian dilation,
    QFTs as Fourier-transform passes)."""
    Aa, Ap = _cplx(A)
    ba, bp = _cplx(np.ravel(b))
    N = ba.size
    if Aa.shape != (N, N):
        raise QsimError(-1, "A must be N x N")
    p = _VP()
    flags = ((QSIM_HHL_STRUCTURED_QPE if structured else 0) | (QSIM_HHL_GAUSS_SEIDEL if gauss_seidel else 0)
             | (QSIM_HHL_DILATE if dilate else 0) | (QSIM_HHL_FFT_QFT if fft_qft else 0))
    if flags:
        _check(library().hhl_build_ex(Ap, bp, N, int(n_clock), float(t), float(C), flags, ctypes.byref(p)))
    else:
        _check(library().hhl_build(Ap, bp, N, int(n_clock), float(t), float(C), ctypes.byref(p)))
    return HHLCircuit(p)


def hhl_build_spectral(lam, V, b, n_clock: int = 0, t: float = 0.0, C: float = 0.0,
                       structured: bool = False, fft_qft: bool = False) -> HHLCircuit:
    la = np.ascontiguousarray(np.asarray(lam, dtype=np.float64))
    Va, Vp = _cplx(V)
    ba, bp = _cplx(np.ravel(b))
    N = ba.size
    if Va.shape != (N, N) or la.size != N:
        raise QsimError(-1, "shape mismatch")
    p = _VP()
    flags = (QSIM_HHL_STRUCTURED_QPE if structured else 0) | (QSIM_HHL_FFT_QFT if fft_qft else 0)
    if flags:
        _check(library().hhl_build_spectral_ex(la.ctypes.data_as(_DP), Vp, bp, N, int(n_clock), float(t),
                                               float(C), flags, ctypes.byref(p)))
    else:
        _check(library().hhl_build_spectral(la.ctypes.data_as(_DP), Vp, bp, N, int(n_clock),
                                            float(t), float(C), ctypes.byref(p)))
    return HHLCircuit(p)


def qsim_tune_get(dtype: int, key: int, n_qubits: int = 27) -> int:
    """The kernel-choice table's entry (QSIM_TUNE_* key) for a QSIM_C64 / QSIM_C128 state of
    n_qubits (entries are kept per size class: <= 24, 25..28, >= 29 qubits)."""
    v = ctypes.c_int(0)
    _check(library().qsim_tune_get(int(dtype), int(key), int(n_qubits), ctypes.byref(v)))
    return int(v.value)


def qsim_tune_set(dtype: int, key: int, value: int, n_qubits: int = 0):
    """Set an entry for the size class of n_qubits (0: every class)."""
    _check(library().qsim_tune_set(int(dtype), int(key), int(n_qubits), int(value)))


def qsim_tune_reset():
    _check(library().qsim_tune_reset())


def qsim_tune_table() -> dict:
    """The whole table, by dtype, size class and key name."""
    classes = (("le24", 24), ("25to28", 27), ("ge29", 31))
    return {name: {cn: {TUNE_NAMES[k]: qsim_tune_get(dt, k, n) for k in range(QSIM_TUNE_COUNT)}
                   for cn, n in classes}
            for name, dt in (("c64", QSIM_C64), ("c128", QSIM_C128))}


def qsim_autotune(state, stream=None) -> dict:
    """Time the kernel alternatives on `state` (contents overwritten) and write the fastest into
    the table for the state's dtype; returns the report."""
    n = state.numel().bit_length() - 1
    _check_state(state, n)
    r = _TuneReport()
    _check(library().qsim_autotune(ctypes.c_void_p(state.data_ptr()), n, _dtype_of(state), _stream_ptr(stream),
                                   ctypes.byref(r)))
    return {"n_qubits": r.n_qubits, "table": {TUNE_NAMES[k]: r.values[k] for k in range(QSIM_TUNE_COUNT)},
            "dft_ms": r.dft_ms, "dense_ms": {str(3 + i): r.dense_ms[i] for i in range(4)},
            "fuse_ms": {str(2 + i): r.fuse_ms[i] for i in range(5)}}


def qsim_hermitian_eig(A, max_iter: int = 0):
    """The library's host eigensolver (the one hhl_build uses): (lambda ascending, V)."""
    Aa, Ap = _cplx(A)
    N = Aa.shape[0]
    if Aa.shape != (N, N):
        raise QsimError(-1, "A must be N x N")
    lam = np.zeros(N, dtype=np.float64)
    V = np.zeros((N, N), dtype=np.complex128)
    _check(library().qsim_hermitian_eig(Ap, N, int(max_iter), lam.ctypes.data_as(_DP),
                                        V.view(np.float64).ctypes.data_as(_DP)))
    return lam, V


def hhl_prepare_state(state, h: HHLCircuit, stream=None):
    _check_state(state, h.info()["n"])
    _check(library().hhl_prepare_state(ctypes.c_void_p(state.data_ptr()), _dtype_of(state), h.ptr,
                                       _stream_ptr(stream)))
    return state


def hhl_run(state, h: HHLCircuit, circuit=None, stream=None):
    """Prepare |0>|0>|b> and apply `circuit` (h's gate list if None, else a qsim_fuse of
    h.as_circuit()) with the operations before the inversion on half the state (the ancilla is
    |0> until then).  Enqueued on `stream`."""
    _check_state(state, h.info()["n"])
    _check(library().hhl_run(ctypes.c_void_p(state.data_ptr()), _dtype_of(state), h.ptr,
                             circuit.ptr if circuit is not None else None, _stream_ptr(stream)))
    return state


def hhl_readout(state, h: HHLCircuit, stream=None) -> dict:
    """Solution readout (synchronizes the stream).  Returns x, x_state and the statistics."""
    info = h.info()
    _check_state(state, info["n"])
    x = np.zeros(info["N"], dtype=np.complex128)
    xs = np.zeros(1 << info["nb"], dtype=np.complex128)
    st = _ReadoutStats()
    _check(library().hhl_readout(ctypes.c_void_p(state.data_ptr()), _dtype_of(state), h.ptr,
                                 _stream_ptr(stream), x.view(np.float64).ctypes.data_as(_DP),
                                 xs.view(np.float64).ctypes.data_as(_DP), ctypes.byref(st)))
    out = {f: getattr(st, f) for f, _ in st._fields_}
    out["x"] = x
    out["x_state"] = xs
    return out


QSIM_READOUT_SUMS_DOUBLES = 4096


def hhl_run_sums(state, h: HHLCircuit, sums, circuit=None, stream=None):
    """hhl_run that also writes the final state's readout partial sums into `sums` (a CUDA
    float64 tensor of QSIM_READOUT_SUMS_DOUBLES entries), in the circuit's last kernel when it
    can.  Device-only (graph-capturable)."""
    import torch
    _check_state(state, h.info()["n"])
    if not (sums.is_cuda and sums.dtype == torch.float64 and sums.numel() >= QSIM_READOUT_SUMS_DOUBLES):
        raise QsimError(-1, "sums must be a CUDA float64 tensor of QSIM_READOUT_SUMS_DOUBLES entries")
    _check(library().hhl_run_sums(ctypes.c_void_p(state.data_ptr()), _dtype_of(state), h.ptr,
                                  circuit.ptr if circuit is not None else None, _stream_ptr(stream),
                                  ctypes.c_void_p(sums.data_ptr())))
    return state


def hhl_readout_sums(state, h: HHLCircuit, sums, stream=None) -> dict:
    """hhl_readout from the partial sums hhl_run_sums left in `sums` (synchronizes the stream)."""
    info = h.info()
    _check_state(state, info["n"])
    x = np.zeros(info["N"], dtype=np.complex128)
    xs = np.zeros(1 << info["nb"], dtype=np.complex128)
    st = _ReadoutStats()
    _check(library().hhl_readout_sums(ctypes.c_void_p(state.data_ptr()), _dtype_of(state), h.ptr,
                                      ctypes.c_void_p(sums.data_ptr()), _stream_ptr(stream),
                                      x.view(np.float64).ctypes.data_as(_DP), xs.view(np.float64).ctypes.data_as(_DP),
                                      ctypes.byref(st)))
    out = {f: getattr(st, f) for f, _ in st._fields_}
    out["x"] = x
    out["x_state"] = xs
    return out


def _ptr_array(items):
    arr = (_VP * max(1, len(items)))()
    for i, x in enumerate(items):
        arr[i] = x
    return arr


class Batch:
    """Owning handle of a qsim_batch; keeps the circuits and states it references alive."""

    def __init__(self, ptr, keep, hhl=None):
        self._ptr = ptr
        self._keep = keep
        self._hhl = hhl
        self._Ns = [h.info()["N"] for h in hhl] if hhl is not None else None
        self._stats = None
        self._x = None

    @property
    def ptr(self):
        return self._ptr

    def run(self, stream=None):
        _check(library().qsim_batch_run(self._ptr, _stream_ptr(stream)))

    def results_arrays(self, stream=None):
        """HHL batches: (x, stats) -- all solutions concatenated (complex128, entry i has N_i
        values, in batch order) and a structured array of the readout statistics per entry.
        The buffers are reused by the next call."""
        self._result_buffers()
        _check(library().hhl_batch_results(self._ptr, _stream_ptr(stream), self._xp, self._stats))
        return self._x, self._stats_np

    def solve(self, stream=None):
        """HHL batches: run the batch and read its results in one library call (launch, copy,
        synchronize, host scaling); returns (x, stats) as results_arrays does."""
        self._result_buffers()
        _check(library().hhl_batch_solve(self._ptr, _stream_ptr(stream), self._xp, self._stats))
        return self._x, self._stats_np

    def _result_buffers(self):
        if self._hhl is None:
            raise QsimError(-1, "not an HHL batch")
        if self._x is None:
            self._x = np.zeros(max(1, sum(self._Ns)), dtype=np.complex128)
            self._xp = self._x.view(np.float64).ctypes.data_as(_DP)
            self._stats = (_ReadoutStats * len(self._Ns))()
            self._stats_np = np.ctypeslib.as_array(self._stats)

    def results(self, stream=None):
        """HHL batches: list of dicts (x and the readout statistics) per entry."""
        x, st = self.results_arrays(stream)
        out, o = [], 0
        for i, n in enumerate(self._Ns):
            d = {f: float(st[i][f]) for f, _ in _ReadoutStats._fields_}
            d["x"] = x[o:o + n].copy()
            o += n
            out.append(d)
        return out

    def __del__(self):
        if getattr(self, "_ptr", None):
            try:
                library().qsim_batch_free(self._ptr)
            except Exception:
                pass
            self._ptr = None


def qsim_batch_create(circuits, states) -> Batch:
    dt = {_dtype_of(s) for s in states}
    if len(dt) != 1:
        raise QsimError(-1, "all states must have the same dtype")
    for c, s in zip(circuits, states):
        _check_state(s, c.n_qubits)
    p = _VP()
    _check(library().qsim_batch_create(_ptr_array([c.ptr for c in circuits]),
                                       _ptr_array([s.data_ptr() for s in states]), len(circuits),
                                       dt.pop(), ctypes.byref(p)))
    return Batch(p, (list(circuits), list(states)))


def hhl_batch_create(hhls, states, fused=None) -> Batch:
    dt = {_dtype_of(s) for s in states}
    if len(dt) != 1:
        raise QsimError(-1, "all states must have the same dtype")
    for h, s in zip(hhls, states):
        _check_state(s, h.info()["n"])
    p = _VP()
    fz = _ptr_array([f.ptr for f in fused]) if fused is not None else None
    _check(library().hhl_batch_create(_ptr_array([h.ptr for h in hhls]), fz,
                                      _ptr_array([s.data_ptr() for s in states]), len(hhls),
                                      dt.pop(), ctypes.byref(p)))
    return Batch(p, (list(hhls), list(states), list(fused) if fused is not None else None),
                 hhl=list(hhls))


def qsim_apply_batched(states, circuits, stream=None):
    dt = {_dtype_of(s) for s in states}
    if len(dt) != 1:
        raise QsimError(-1, "all states must have the same dtype")
    ns = [c.n_qubits for c in circuits]
    for n, s in zip(ns, states):
        _check_state(s, n)
    na = np.ascontiguousarray(np.asarray(ns if ns else [0], dtype=np.int32))
    _check(library().qsim_apply_batched(_ptr_array([s.data_ptr() for s in states]),
                                        na.ctypes.data_as(_IP), _ptr_array([c.ptr for c in circuits]),
                                        len(circuits), dt.pop(), _stream_ptr(stream)))


def hhl_batch_autotune(hhls, states, candidates=(1, 2, 3, 4, 5), stream=None):
    """Fastest fusion width for this HHL batch (times real batch runs).  Returns (k, {k: ms})."""
    dt = {_dtype_of(s) for s in states}
    if len(dt) != 1:
        raise QsimError(-1, "all states must have the same dtype")
    cand = np.ascontiguousarray(np.asarray(list(candidates), dtype=np.int32))
    ms = np.zeros(len(cand))
    best = ctypes.c_int(0)
    _check(library().hhl_batch_autotune(_ptr_array([h.ptr for h in hhls]),
                                        _ptr_array([s.data_ptr() for s in states]), len(hhls), dt.pop(),
                                        cand.ctypes.data_as(_IP), len(cand), _stream_ptr(stream),
                                        ctypes.byref(best), ms.ctypes.data_as(_DP)))
    return int(best.value), {int(k): float(t) for k, t in zip(cand, ms)}


class Pool:
    """Serving pool (device arena, builder threads, continuous batching).  submit() returns a
    ticket; poll() returns None while pending, else a dict (x, statistics, latency_s) or raises
    the request's error."""

    def __init__(self, bytes_: int, n_builders: int = 0, n_streams: int = 0):
        p = _VP()
        _check(library().qsim_pool_create(int(bytes_), int(n_builders), int(n_streams), ctypes.byref(p)))
        self._ptr = p
        self._N = {}

    def submit(self, A, b, n_clock=0, t=0.0, C=0.0, dtype=QSIM_C64, structured=False) -> int:
        Aa, Ap = _cplx(A)
        ba, bp = _cplx(np.ravel(b))
        req = _HHLRequest(Ap, bp, ba.size, int(n_clock), float(t), float(C), int(dtype),
                          QSIM_HHL_STRUCTURED_QPE if structured else 0)
        tk = ctypes.c_uint64(0)
        _check(library().qsim_submit(self._ptr, ctypes.byref(req), ctypes.byref(tk)))
        self._N[int(tk.value)] = ba.size
        return int(tk.value)

    def poll(self, ticket: int):
        N = self._N.get(ticket, 1)
        x = np.zeros(N, dtype=np.complex128)
        st = _ReadoutStats()
        lat = ctypes.c_double(0)
        rc = library().qsim_poll(self._ptr, ctypes.c_uint64(ticket), x.view(np.float64).ctypes.data_as(_DP),
                                 ctypes.byref(st), ctypes.byref(lat))
        if rc == -3:  # EBUSY: pending
            return None
        self._N.pop(ticket, None)
        _check(rc)
        out = {f: getattr(st, f) for f, _ in st._fields_}
        out["x"] = x
        out["latency_s"] = lat.value
        return out

    def take_completed(self, capacity: int = 4096, timeout_s: float = 0.05) -> list:
        """Tickets of requests that finished since the last call (each handed out once)."""
        buf = (ctypes.c_uint64 * capacity)()
        cnt = ctypes.c_int(0)
        _check(library().qsim_pool_take_completed(self._ptr, buf, capacity, ctypes.byref(cnt),
                                                   float(timeout_s)))
        return [int(buf[i]) for i in range(cnt.value)]

    def wait(self, ticket: int, timeout_s: float = 60.0) -> None:
        _check(library().qsim_pool_wait(self._ptr, ctypes.c_uint64(ticket), float(timeout_s)))

    def info(self) -> dict:
        s = _PoolInfo()
        _check(library().qsim_pool_get_info(self._ptr, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in s._fields_}

    def launch_log(self, capacity: int = 4096) -> list:
        """The most recent retired launches, oldest first: slot, batched, n_requests, tickets and
        the device-time interval [t_start, t_end] (seconds since the pool was created)."""
        buf = (_PoolLaunch * capacity)()
        cnt = ctypes.c_int(0)
        _check(library().qsim_pool_launch_log(self._ptr, buf, capacity, ctypes.byref(cnt)))
        return [{f: getattr(buf[i], f) for f, _ in _PoolLaunch._fields_} for i in range(cnt.value)]

    def close(self):
        if getattr(self, "_ptr", None):
            library().qsim_pool_destroy(self._ptr)
            self._ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ShardPlan:
    """qsim_shard_plan: the steps that run an unfused circuit on 2^n_global shards.  steps is a
    list of dicts: {"kind": "swap", "global_bit", "local_qubit", "perm"} or {"kind": "apply",
    "first_gate", "last_gate", "perm", "circuit"} (the local circuit, owned by the plan)."""

    def __init__(self, circuit: Circuit, n_global: int):
        p = _VP()
        _check(library().qsim_shard_plan_create(circuit.ptr, int(n_global), ctypes.byref(p)))
        self._ptr = p
        self.n = circuit.n_qubits
        self.n_global = int(n_global)
        self.n_local = self.n - self.n_global
        self.steps = []
        for i in range(library().qsim_shard_plan_num_steps(p)):
            st = _ShardStep()
            perm = np.zeros(self.n, dtype=np.int32)
            _check(library().qsim_shard_plan_get_step(p, i, ctypes.byref(st), perm.ctypes.data_as(_IP)))
            if st.kind == 0:
                self.steps.append({"kind": "swap", "global_bit": st.global_bit, "local_qubit": st.local_qubit,
                                   "perm": perm.tolist()})
            else:
                c = Circuit(_ptr=_VP(library().qsim_shard_plan_local_circuit(p, i)), _owner=self)
                self.steps.append({"kind": "apply", "first_gate": st.first_gate, "last_gate": st.last_gate,
                                   "perm": perm.tolist(), "circuit": c})

    def __del__(self):
        if getattr(self, "_ptr", None):
            try:
                library().qsim_shard_plan_free(self._ptr)
            except Exception:
                pass
            self._ptr = None


def qsim_shard_pack(shard, qubit: int, value: int, out, stream=None):
    n = shard.numel().bit_length() - 1
    _check(library().qsim_shard_pack(ctypes.c_void_p(shard.data_ptr()), n, _dtype_of(shard), int(qubit), int(value),
                                     ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
    return out


def qsim_shard_unpack(shard, qubit: int, value: int, src, stream=None):
    n = shard.numel().bit_length() - 1
    _check(library().qsim_shard_unpack(ctypes.c_void_p(shard.data_ptr()), n, _dtype_of(shard), int(qubit), int(value),
                                       ctypes.c_void_p(src.data_ptr()), _stream_ptr(stream)))
    return shard
