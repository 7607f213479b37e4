"""Serving pool: results alone vs in a mixed, overlapping stream; parity with the oracle;
memory-budget admission; failures injected on the host (poisoned systems, a request larger
than the pool, a wait that times out, an unknown ticket).  No test faults or hangs a GPU."""
import math
import time

import numpy as np
import pytest
import torch

import synth
from hhl_bounds import cond_tol, readout_bounds
from oracle import hhl as ohhl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qs(cuda_device):
    from paper_2402_08136_gb300 import build
    build.build()
    import paper_2402_08136_gb300 as q
    return q


def stream_items(count, max_n, seed=11):
    return [r["problem"] for r in synth.serving_stream(seed=seed, count=count, max_n=max_n)]


def run_all(pool, items, dtype):
    tks = [pool.submit(p["A"], p["b"], p["m"], dtype=dtype) for p in items]
    out = []
    for t in tks:
        pool.wait(t, 120.0)
        out.append(pool.poll(t))
    return out


@pytest.mark.parametrize("dtype_name", ["c64", "c128"])
def test_pool_mix_equals_alone_and_oracle(qs, dtype_name):
    dtype = qs.QSIM_C64 if dtype_name == "c64" else qs.QSIM_C128
    items = stream_items(40, max_n=17)
    ns = [p["nb"] + p["m"] + 1 for p in items]
    assert min(ns) <= 14 < max(ns)            # both batched and full-GPU launches
    pool = qs.Pool(1 << 30, n_builders=4, n_streams=4)
    mix = run_all(pool, items, dtype)
    info = pool.info()
    assert info["batches_launched"] >= 1 and info["singles_launched"] >= 1
    alone = []
    for p in items[:12]:
        alone += run_all(pool, [p], dtype)
    pool.close()
    for a, b in zip(alone, mix[:12]):
        assert np.max(np.abs(a["x"] - b["x"])) <= 1e-12 * max(1.0, np.max(np.abs(b["x"])))
        assert abs(a["p_success"] - b["p_success"]) <= 1e-12
    # FP64 oracle on every request of at most 16 qubits: the served normalized solution and x
    # element by element, P and P0, within the bounds implied by the per-amplitude state bound
    # (tests/hhl_bounds.py); complex64 also by fidelity of the normalized solution
    checked = 0
    for p, r in zip(items, mix):
        if p["nb"] + p["m"] + 1 > 16:
            continue
        ref = ohhl.solve(p["A"], p["b"], p["m"])
        tol = 1e-5 if dtype_name == "c64" else cond_tol(p["m"])
        h = ref["circuit"]
        N = len(ref["x"])
        bd = readout_bounds(ref, h["nb"], h["m"], tol, h["C"], h["bnorm"], N)
        assert abs(r["p_success"] - ref["P"]) <= bd["P"]
        assert abs(r["p_clock0"] - ref["P0"]) <= bd["P0"]
        xs = r["x"] / (r["norm_x"] * r["norm_b"])
        assert np.all(np.abs(xs - ref["x_state"][:N]) <= bd["x_state"])
        assert np.all(np.abs(r["x"] - ref["x"]) <= bd["x"])
        if dtype_name == "c64":
            a, b = xs, ref["x_state"][:N]
            assert abs(np.vdot(b, a)) ** 2 / (np.vdot(a, a).real * np.vdot(b, b).real) >= 1 - 1e-6
        checked += 1
    assert checked >= 10


def test_pool_memory_budget_admission(qs):
    # 20-qubit complex64 states are 8 MiB; a 20 MiB arena holds two at a time
    rng = np.random.default_rng(3)
    items = []
    for _ in range(6):
        A, b = synth.contingency_system(rng, 2 ** 3 + 1)
        items.append(dict(A=A, b=b, m=16))
    pool = qs.Pool(20 << 20, n_builders=2, n_streams=4)
    res = run_all(pool, items, qs.QSIM_C64)
    info = pool.info()
    pool.close()
    assert all(r is not None for r in res)
    assert info["bytes_peak"] <= 20 << 20 and info["done"] == 6


def test_pool_failures_injected_on_host(qs):
    pool = qs.Pool(16 << 20, n_builders=2, n_streams=2)
    good = stream_items(3, max_n=12, seed=4)
    bad_A = np.array([[2.0, 1.0], [0.0, 3.0]])               # not Hermitian
    nan_b = np.array([1.0, np.nan])
    tk_good = [pool.submit(p["A"], p["b"], p["m"]) for p in good]
    tk_bad = [pool.submit(bad_A, [1.0, 0.0], 3), pool.submit(np.eye(2), nan_b, 3)]
    rng = np.random.default_rng(0)
    A, b = synth.contingency_system(rng, 5)
    tk_big = pool.submit(A, b, 20)                            # 23 qubits: 64 MiB > 16 MiB arena
    with pytest.raises(qs.QsimError) as e:
        pool.wait(tk_big + 1000, 0.0)
    assert e.value.code == -6                                  # unknown ticket
    for t in tk_bad:
        pool.wait(t, 60.0)
        with pytest.raises(qs.QsimError) as e:
            pool.poll(t)
        assert e.value.code == -1
    pool.wait(tk_big, 60.0)
    with pytest.raises(qs.QsimError) as e:
        pool.poll(tk_big)
    assert e.value.code == -2
    for t in tk_good:
        pool.wait(t, 60.0)
        assert pool.poll(t) is not None
    with pytest.raises(qs.QsimError) as e:
        pool.poll(tk_good[0])                                  # released
    assert e.value.code == -6
    pool.close()


def test_pool_wait_times_out(qs):
    pool = qs.Pool(64 << 20, n_builders=1, n_streams=1)
    rng = np.random.default_rng(1)
    A, b = synth.contingency_system(rng, 2 ** 4 + 1)
    t = pool.submit(A, b, 14)
    with pytest.raises(qs.QsimError) as e:
        pool.wait(t, 0.0)
    assert e.value.code == -5
    pool.wait(t, 60.0)
    assert pool.poll(t) is not None
    pool.close()


def test_pool_completion_queue_hands_out_each_ticket_once(qs):
    pool = qs.Pool(256 << 20, n_builders=2, n_streams=2)
    items = stream_items(12, max_n=14, seed=21)
    tks = {pool.submit(p["A"], p["b"], p["m"]) for p in items}
    seen = []
    while len(seen) < len(tks):
        got = pool.take_completed(5, 30.0)
        assert got, "completion queue timed out"
        seen += got
    assert sorted(seen) == sorted(tks)
    assert pool.take_completed(5, 0.0) == []
    for t in seen:
        assert pool.poll(t) is not None
    pool.close()


def test_pool_launches_overlap_on_the_device(qs):
    """Continuous batching, not a queue: launches on different stream slots run at the same time
    (their device-time intervals, from CUDA events on each slot's stream, intersect), and both
    batched and full-GPU launches take part."""
    items = stream_items(60, max_n=20, seed=31)
    pool = qs.Pool(1 << 30, n_builders=4, n_streams=4)
    res = run_all(pool, items, qs.QSIM_C64)
    log = pool.launch_log()
    pool.close()
    assert all(r is not None for r in res)
    assert {e["batched"] for e in log} == {0, 1}
    assert sum(e["n_requests"] for e in log) == len(items)
    ok = [e for e in log if e["t_start"] >= 0]
    overlaps = 0
    for i, a in enumerate(ok):
        for b in ok[i + 1:]:
            if a["slot"] != b["slot"] and a["t_start"] < b["t_end"] and b["t_start"] < a["t_end"]:
                overlaps += 1
    assert overlaps >= 1, "no two launches on different streams overlapped"


def test_pool_admits_new_work_while_earlier_work_runs(qs):
    """Mid-run admission under a memory budget.  Two 26-qubit complex128 requests (1 GiB states,
    tens of ms each on the FP64 pipe) start; while they are on the GPU two 26-qubit complex64
    requests (512 MiB) arrive, with room in the arena for only one of them.  That one is
    admitted at once and runs alongside the first wave (device-time intervals intersect); the
    other must wait for memory, so its launch starts only after an earlier launch has ended.
    The arena's peak stays within its size, and every result equals the same request run alone."""
    rng = np.random.default_rng(13)
    probs = []
    for _ in range(4):
        A, b = synth.contingency_system(rng, 2 ** 5 + 1)
        probs.append(dict(A=A, b=b, m=20))                    # 5 + 20 + 1 = 26 qubits
    dts = [qs.QSIM_C128, qs.QSIM_C128, qs.QSIM_C64, qs.QSIM_C64]
    arena = 2 * (1 << 30) + (512 << 20) + (64 << 20)
    pool = qs.Pool(arena, n_builders=2, n_streams=4)
    wave1 = [pool.submit(p["A"], p["b"], p["m"], dtype=d, structured=True) for p, d in zip(probs[:2], dts[:2])]
    t0 = time.perf_counter()
    while pool.info()["running"] == 0 and time.perf_counter() - t0 < 30.0:
        pass
    assert pool.info()["running"] > 0
    wave2 = [pool.submit(p["A"], p["b"], p["m"], dtype=d, structured=True) for p, d in zip(probs[2:], dts[2:])]
    out = {}
    for t in wave1 + wave2:
        pool.wait(t, 120.0)
        out[t] = pool.poll(t)
    info = pool.info()
    log = {e["first_ticket"]: e for e in pool.launch_log()}
    alone = []
    for p, d in zip(probs, dts):
        t = pool.submit(p["A"], p["b"], p["m"], dtype=d, structured=True)
        pool.wait(t, 120.0)
        alone.append(pool.poll(t))
    pool.close()
    assert info["bytes_peak"] <= arena and info["done"] == 4
    first, late = log[wave2[0]], log[wave2[1]]
    assert any(first["t_start"] < log[t]["t_end"] and log[t]["t_start"] < first["t_end"] for t in wave1), \
        "the request that arrived mid-run did not run alongside the first wave"
    assert late["t_start"] >= min(log[t]["t_end"] for t in wave1 + wave2[:1]), \
        "a request started without memory for its state"
    for a, t in zip(alone, wave1 + wave2):
        b = out[t]
        assert np.max(np.abs(a["x"] - b["x"])) <= 1e-12 * max(1.0, np.max(np.abs(b["x"])))
