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


def _call(f, Stats, DP, st, code, h, stream, want_slice=True):
    info = h.info()
    x = np.zeros(info["N"], dtype=np.complex128)
    xs = np.zeros(1 << info["nb"], dtype=np.complex128) if want_slice else None
    s = Stats()
    rc = f(ctypes.c_void_p(st.data_ptr()), code, h.ptr, ctypes.c_void_p(stream.cuda_stream),
           x.view(np.float64).ctypes.data_as(DP),
           xs.view(np.float64).ctypes.data_as(DP) if want_slice else None, ctypes.byref(s))
    return rc, x, xs, s


def test_noalloc_readout_dilated_solution_only(cuda_device):
    """A dilated system (x is the lower half of the slice, from offset N) read with no slice
    buffer: the N entries of x come straight from the scratch copy at that offset."""
    import paper_2402_08136_gb300 as qs
    f, Stats, DP = _entry()
    rng = np.random.default_rng(41)
    A = rng.standard_normal((3, 3)) + 4 * np.eye(3)          # not symmetric: dilation
    b = rng.standard_normal(3)
    stream = torch.cuda.current_stream()
    h = qs.hhl_build(A, b, 6, dilate=True)
    info = h.info()
    assert info["N_eff"] == 6
    st = torch.empty(1 << info["n"], dtype=torch.complex128, device="cuda")
    qs.hhl_prepare_state(st, h)
    qs.qsim_apply(st, qs.qsim_fuse(h.as_circuit(), 4), n_qubits=info["n"])
    ref = qs.hhl_readout(st, h)
    for _ in range(2):
        rc, x, _, s = _call(f, Stats, DP, st, qs.QSIM_C128, h, stream, want_slice=False)
        assert rc == 0, qs.library().qsim_last_error().decode()
        assert np.max(np.abs(x - ref["x"])) <= 1e-12 * max(1.0, np.max(np.abs(ref["x"])))
        assert abs(s.p_success - ref["p_success"]) <= 1e-12


def test_noalloc_readout_at_the_slice_limit(cuda_device):
    """nb = 10, the largest slice the fixed scratch holds (2^10 amplitudes): the readout of a
    random normalized state equals hhl_readout's, twice in a row."""
    import paper_2402_08136_gb300 as qs
    f, Stats, DP = _entry()
    N = 1000
    lam = np.linspace(1.0, 9.0, N)
    h = qs.hhl_build_spectral(lam, np.eye(N), np.ones(N), 2, structured=True)
    info = h.info()
    assert info["nb"] == 10
    st = synth.gaussian_state_torch(3, info["n"], torch.complex64, "cuda", normalize=True)
    stream = torch.cuda.current_stream()
    ref = qs.hhl_readout(st, h)
    for _ in range(2):
        rc, x, xs, s = _call(f, Stats, DP, st, qs.QSIM_C64, h, stream)
        assert rc == 0, qs.library().qsim_last_error().decode()
        assert np.max(np.abs(xs - ref["x_state"])) <= 1e-5
        assert np.max(np.abs(x - ref["x"])) <= 1e-5 * max(1.0, np.max(np.abs(ref["x"])))
        assert abs(s.p_success - ref["p_success"]) <= 1e-12


def _default_pool_used_high():
    """Driver-side high-water mark of the device's default memory pool (the pool
    cudaMallocAsync draws from), and a function that resets it."""
    drv = ctypes.CDLL("libcuda.so.1")
    dev = ctypes.c_int(0)
    assert drv.cuCtxGetDevice(ctypes.byref(dev)) == 0
    pool = ctypes.c_void_p()
    assert drv.cuDeviceGetDefaultMemPool(ctypes.byref(pool), dev) == 0
    used_high = 8  # CU_MEMPOOL_ATTR_USED_MEM_HIGH

    def read():
        v = ctypes.c_uint64(0)
        assert drv.cuMemPoolGetAttribute(pool, used_high, ctypes.byref(v)) == 0
        return v.value

    def reset():
        z = ctypes.c_uint64(0)
        assert drv.cuMemPoolSetAttribute(pool, used_high, ctypes.byref(z)) == 0

    return read, reset


def test_noalloc_readout_allocates_nothing(cuda_device):
    """hhl_readout takes its scratch from the stream-ordered pool, and the probe sees it; the
    allocation-free call leaves the pool's high-water mark where it was, and device memory in
    use is unchanged."""
    import paper_2402_08136_gb300 as qs
    f, Stats, DP = _entry()
    A, b, m, t, C = next(_problems())
    h = qs.hhl_build(A, b, m, t, C)
    info = h.info()
    st = torch.empty(1 << info["n"], dtype=torch.complex128, device="cuda")
    qs.hhl_prepare_state(st, h)
    qs.qsim_apply(st, qs.qsim_fuse(h.as_circuit(), 4), n_qubits=info["n"])
    stream = torch.cuda.current_stream()
    read, reset = _default_pool_used_high()
    torch.cuda.synchronize()
    reset()
    qs.hhl_readout(st, h)
    torch.cuda.synchronize()
    assert read() > 0                     # the probe sees a stream-ordered allocation
    reset()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        rc, _, _, _ = _call(f, Stats, DP, st, qs.QSIM_C128, h, stream)
        assert rc == 0
    torch.cuda.synchronize()
    assert read() == 0
    assert torch.cuda.mem_get_info()[0] == free0
