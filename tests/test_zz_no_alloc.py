"""hhl_readout_noalloc: the HHL readout for callers that cannot allocate device memory (for
example an application whose pool allocator owns all device memory, or code that must not call
cudaMalloc while it reads results).  It must return what hhl_readout returns, on consecutive
calls that reuse the library's one fixed scratch array.  Called through the C ABI.

This file is collected last on purpose: a run that stops at the first failure has run every
other test before this one.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

TOL = {torch.complex128: 1e-12, torch.complex64: 1e-5}


def _entry():
    from paper_2402_08136_gb300 import build
    build.build()
    from paper_2402_08136_gb300._binding import _DP, _VP, _ReadoutStats, library
    f = library().hhl_readout_noalloc
    f.argtypes = [_VP, ctypes.c_int, _VP, _VP, _DP, _DP, ctypes.POINTER(_ReadoutStats)]
    f.restype = ctypes.c_int
    return f, _ReadoutStats, _DP


def _problems():
    p = synth.hhl7_problem()
    yield p["A"], p["b"], p["m"], p["t"], p["C"]
    rng = np.random.default_rng(12)
    A, b = synth.contingency_system(rng, 2 ** 4 + 1)
    yield A, b, 7, 0.0, 0.0


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_noalloc_readout_matches_readout_twice(cuda_device, dtype):
    import paper_2402_08136_gb300 as qs
    f, Stats, DP = _entry()
    code = qs.QSIM_C128 if dtype == torch.complex128 else qs.QSIM_C64
    tol = TOL[dtype]
    stream = torch.cuda.current_stream()
    for A, b, m, t, C in _problems():
        h = qs.hhl_build(A, b, m, t, C)
        info = h.info()
        st = torch.empty(1 << info["n"], dtype=dtype, device="cuda")
        qs.hhl_prepare_state(st, h)
        qs.qsim_apply(st, qs.qsim_fuse(h.as_circuit(), 4), n_qubits=info["n"])
        ref = qs.hhl_readout(st, h)
        for call in range(2):
            x = np.zeros(info["N"], dtype=np.complex128)
            xs = np.zeros(1 << info["nb"], dtype=np.complex128)
            s = Stats()
            rc = f(ctypes.c_void_p(st.data_ptr()), code, h.ptr, ctypes.c_void_p(stream.cuda_stream),
                   x.view(np.float64).ctypes.data_as(DP), xs.view(np.float64).ctypes.data_as(DP),
                   ctypes.byref(s))
            assert rc == 0, qs.library().qsim_last_error().decode()
            assert np.max(np.abs(x - ref["x"])) <= tol * max(1.0, np.max(np.abs(ref["x"])))
            assert np.max(np.abs(xs - ref["x_state"])) <= tol
            for key in ("p_success", "p_clock0", "leakage", "norm2", "norm_x", "norm_b"):
                assert abs(getattr(s, key) - ref[key]) <= tol * max(1.0, abs(ref[key])), key
        # solution only (no slice buffer): the slice goes straight into x
        x2 = np.zeros(info["N"], dtype=np.complex128)
        rc = f(ctypes.c_void_p(st.data_ptr()), code, h.ptr, ctypes.c_void_p(stream.cuda_stream),
               x2.view(np.float64).ctypes.data_as(DP), None, None)
        assert rc == 0
        assert np.max(np.abs(x2 - ref["x"])) <= tol * max(1.0, np.max(np.abs(ref["x"])))
