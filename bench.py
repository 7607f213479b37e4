"""Benchmark of the GB300 HHL state-vector simulator.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload W]

Default workload ("gates"): the gate-apply microbenchmark on a 31-qubit complex64 state
(16 GiB): 200 Haar-random 2^k x 2^k unitaries for each k in 1..6 on uniformly random distinct
targets (1200 gates), initial state a seeded complex Gaussian, normalized.  One step applies
the 1200 gates in order through the C ABI (one qsim_apply per gate).  The metric is the
algorithmic HBM bandwidth of gate application, 2 x 8 bytes x 2^31 per gate, divided by the
step time (inputs far larger than L2, so no flush is needed).

Other workloads (one JSON line each): "gates-c128" (30-qubit complex128 state, same gates),
"hhl7" (7-qubit exact-grid HHL, complex128, solves/s and latency), "hhl27" (27-qubit
precision-form HHL: complex64 vs complex128, solves/s and error vs the oracle).

Multi-GPU (torchrun): every rank runs the same workload on its own GPU (independent replicas,
no collective on the data path); value = work of all ranks / max over ranks of the time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402


# ------------------------------------------------------------------------------ helpers
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d.get("bf16_tflops", 1946.5)), "measured"
    except Exception:
        return 6800.0, 1900.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def dist_setup(gpus: int, backend: str = "nccl"):
    """Rank, world size and local rank from the torchrun environment; one process per GPU.
    backend "gloo" (tests) keeps everything on the CPU."""
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        if backend == "nccl":
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group("gloo")
    elif backend == "nccl":
        torch.cuda.set_device(0)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, v: float) -> float:
    """Maximum of a per-rank value (the job's time is its slowest rank's)."""
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_seed(base: int, rank: int) -> int:
    """Each replica (rank) solves its own independent problems: weak scaling, no collective."""
    return base + 1000003 * rank


# DRAM bytes (read + write) per amplitude for one launch of each kernel family, from an ncu
# capture of the current kernel on a 27-qubit state (the full-size launch is linear in 2^n).
# An entry is removed whenever its kernel changes, until it is captured again.
TRAFFIC = {
    ("dense_tc_gm_kernel+dense_tc_tr_kernel", "c64"): {
        "bytes_per_amp": 2.0865e9 / 2 ** 27,
        "source": "profiles/dense_gate_kernels_c64_27q.md (group-major form, k=4..6 mean) and "
                  "profiles/dense_tc_tr_kernel_c64_27q.md (transposed form, 2.087e9), 27-qubit "
                  "captures scaled by 2^n"},
    ("dense_pipe_kernel", "c64"): {"bytes_per_amp": 2.0874e9 / 2 ** 27,
                                   "source": "profiles/dense_gate_kernels_c64_27q.md (k=1..3 mean, "
                                             "27-qubit capture scaled by 2^n)"},
}


FP64_PEAK_TFLOPS = 1.25


# the library counts launches per family; the tensor-core family is the group-major and the
# transposed form (gates on qubit 0 or 1)
FAMILY_KERNEL = {"dense_simt": "dense_pipe_kernel", "dense_tc": "dense_tc_gm_kernel+dense_tc_tr_kernel",
                 "fourier": "dft_kernel", "fourier_tma": "dft_tma_kernel"}


def launched_family(qs, fn):
    """Run fn() and return the kernel family the library reports for the launch it made."""
    before = qs.qsim_launch_counts()
    fn()
    after = qs.qsim_launch_counts()
    fams = [f for f in after if after[f] != before[f]]
    return FAMILY_KERNEL.get(fams[0], fams[0]) if len(fams) == 1 else "+".join(sorted(fams))


# ------------------------------------------------------------------------ oracle baseline
ORACLE_MIN_SECONDS = 10.0  # host work per oracle sample (the sample repeats until this is reached)


def oracle_gate_sample(seed: int, n_sample: int = 24, per_k: int = 4):
    """The oracle (FP64, OpenMP over the host cores) on a bounded sample of the gate
    workload: rounds of `per_k` Haar gates per k = 1..6 on an n_sample-qubit complex128 state,
    repeated until ORACLE_MIN_SECONDS of work."""
    from oracle import core as ocore
    gates = synth.gate_microbench_list(seed, n_sample, per_k=per_k)
    psi = synth.gaussian_state_np(seed, n_sample)
    done = 0
    t0 = time.perf_counter()
    while True:
        for t, U in gates:
            ocore.apply_gate(psi, t, U)
        done += len(gates)
        dt = time.perf_counter() - t0
        if dt >= ORACLE_MIN_SECONDS:
            break
    byts = done * 2 * 16 * (1 << n_sample)
    return {"value": byts / dt / 1e9, "unit": "GB/s", "cores": ocore.num_threads(),
            "kind": "oracle", "seconds": dt,
            "sample": "%d Haar gates (%d per k=1..6 per round) on a %d-qubit complex128 state (FP64 "
                      "oracle, algorithmic bytes 2x16x2^n per gate; GB/s is independent of n for this "
                      "streaming rule)" % (done, per_k, n_sample)}


def oracle_hhl_sample(problems, what: str, min_seconds: float = ORACLE_MIN_SECONDS):
    """The oracle solving a bounded list of HHL problems one after another, the list repeated
    until `min_seconds` of work: solves/s."""
    from oracle import core as ocore
    from oracle import hhl as ohhl
    done = 0
    t0 = time.perf_counter()
    while True:
        for p in problems:
            ohhl.solve(p["A"], p["b"], p["m"], p.get("t", 0.0), p.get("C", 0.0))
        done += len(problems)
        dt = time.perf_counter() - t0
        if dt >= min_seconds:
            break
    return {"value": done / dt, "unit": "solves/s", "cores": ocore.num_threads(),
            "kind": "oracle", "seconds": dt, "sample": "%d solves in rounds of %s" % (done, what)}


def oracle_hhl_both(problems, what: str, min_seconds: float = 3.0):
    """The oracle on all host cores (OpenMP) and on one thread: the all-core figure at the top,
    the single-thread one under "single_thread"."""
    from oracle import core as ocore
    allc = ocore.num_threads()
    rec = oracle_hhl_sample(problems, what, min_seconds)
    try:
        ocore.set_num_threads(1)
        one = oracle_hhl_sample(problems, what, min_seconds)
    finally:
        ocore.set_num_threads(allc)
    rec["single_thread"] = {k: one[k] for k in ("value", "unit", "cores", "seconds")}
    return rec


def oracle_baseline(workload: str, rank: int = 0):
    if workload in ("gates", "gates-c128"):
        return oracle_gate_sample(2402)
    if workload == "hhl7":
        return oracle_hhl_sample([synth.hhl7_problem()] * 20, "20 solves of the 7-qubit problem")
    if workload == "hhl27":
        p = dict(synth.hhl27_problem())
        p["m"] = 12
        return oracle_hhl_sample([p], "one solve of the same 64x64 system with 12 instead of 20 "
                                      "clock qubits (19 qubits; the 27-qubit solve has 2^8 x the "
                                      "amplitudes)")
    if workload == "batched":
        probs = synth.batched_problems(seed=rank_seed(4, rank), count=512)[:16]
        return oracle_hhl_sample(probs, "the first 16 circuits of the 512-circuit batch")
    if workload == "serving":
        items = synth.serving_stream(seed=rank_seed(5, rank), count=200, max_n=16)
        return oracle_hhl_sample([it["problem"] for it in items[:16]],
                                 "16 requests of the stream (qubits capped at 16)")
    raise ValueError(workload)


# ------------------------------------------------------------------------- gate workload
def run_gates(args, ws, rank, dtype_name):
    import torch
    import paper_2402_08136_gb300 as qs

    dtype = torch.complex64 if dtype_name == "c64" else torch.complex128
    n = args.n or (31 if dtype_name == "c64" else 30)
    S = 8 if dtype_name == "c64" else 16
    seed = 2402
    gates = synth.gate_microbench_list(seed, n, per_k=args.per_k)
    circs = [qs.Circuit(n).add_gate(t, U) for t, U in gates]
    ks = [len(t) for t, _ in gates]
    stream = torch.cuda.current_stream()
    # the library's autotuner picks its kernel variants on this state buffer first (it
    # overwrites the contents), then the benchmark's input is written
    st = torch.empty(1 << n, dtype=dtype, device="cuda")
    t0 = time.perf_counter()
    tune = {} if args.no_autotune else qs.qsim_autotune(st, stream)
    tune["seconds"] = round(time.perf_counter() - t0, 2)
    st.copy_(synth.gaussian_state_torch(seed, n, dtype, "cuda", normalize=True))
    bytes_per_gate = 2.0 * S * (1 << n)
    step_bytes = bytes_per_gate * len(gates)

    def step(evs=None):
        for i, c in enumerate(circs):
            if evs is not None:
                evs[i][0].record(stream)
            qs.qsim_apply(st, c, stream)
            if evs is not None:
                evs[i][1].record(stream)

    # which kernel the library launches for each gate (its per-family launch counters)
    fam_of = [launched_family(qs, lambda c=c: qs.qsim_apply(st, c, stream)) for c in circs]
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    evs = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            for _ in circs] for _ in range(args.steps)]
    barrier(ws)
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        l0 = qs.qsim_launch_count()
        t_start.record(stream)
        for s in range(args.steps):
            step(evs[s])
        t_end.record(stream)
        launches = qs.qsim_launch_count() - l0
        torch.cuda.synchronize()
    barrier(ws)
    ms_total = t_start.elapsed_time(t_end)
    ms_total = max_over_ranks(ws, ms_total)
    ms_step = ms_total / args.steps
    value = ws * step_bytes * args.steps / (ms_total / 1e3) / 1e9
    durs = np.array([[a.elapsed_time(b) for a, b in row] for row in evs])  # ms
    per_k = {}
    for k in sorted(set(ks)):
        sel = [i for i, kk in enumerate(ks) if kk == k]
        d = durs[:, sel].mean()
        per_k[str(k)] = {"ms_per_gate": round(float(d), 4),
                         "gbs": round(bytes_per_gate / (d / 1e3) / 1e9, 1),
                         "kernel": "/".join(sorted({fam_of[i] for i in sel}))}
    # per kernel family: launches, time, share of the timed gate time
    fams = {}
    for i, k in enumerate(ks):
        f = fam_of[i]
        e = fams.setdefault(f, {"launches": 0, "ms_total": 0.0})
        e["launches"] += args.steps
        e["ms_total"] += float(durs[:, i].sum())
    tot = sum(e["ms_total"] for e in fams.values())
    for f, e in fams.items():
        e["share"] = round(e["ms_total"] / tot, 4)
        e["achieved_gbs"] = round(bytes_per_gate * e["launches"] / (e["ms_total"] / 1e3) / 1e9, 1)
        e["ms_total"] = round(e["ms_total"], 2)
    dom = max(fams, key=lambda f: fams[f]["ms_total"])
    hbm, _, peak_kind = measured_peaks()
    achieved = fams[dom]["achieved_gbs"]
    tr = TRAFFIC.get((dom, dtype_name))
    traffic = None
    if tr is not None:
        traffic = round(tr["bytes_per_amp"] * (1 << n))
    if dtype_name == "c64":
        roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm,
                    "peak_kind": peak_kind + " copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                    "unit": "GB/s", "frac": round(achieved / hbm, 4), "traffic": traffic,
                    "traffic_source": tr["source"] if tr else None,
                    "bytes_per_launch": bytes_per_gate}
    else:
        # complex128: FP64 FMA bound (a dense k-qubit gate is 8 * 2^k real flops per amplitude)
        sel = [i for i, k in enumerate(ks) if fam_of[i] == dom]
        fl = sum(8.0 * (2 ** ks[i]) * (1 << n) for i in sel) * args.steps
        tf = fl / (fams[dom]["ms_total"] / 1e3) / 1e12
        roofline = {"bound": "alu", "kernel": dom, "achieved": round(tf, 4),
                    "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "peak_kind": "nominal GB300 FP64 rate (1.25 TFLOP/s; a probe measured 1.21)",
                    "frac": round(tf / FP64_PEAK_TFLOPS, 4), "traffic": traffic,
                    "traffic_source": tr["source"] if tr else None,
                    "hbm_achieved_gbs": achieved}

    # end to end through the public API from pinned host memory
    host_in = synth.gaussian_state_torch(seed, n, dtype, "cpu", chunk=1 << 22, normalize=True) \
        if args.e2e_from_host_gen else st.cpu()
    host_in = host_in.pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    e2e_steps = min(args.steps, 5)  # 2 x 16 GiB of host copies per step: a few steps suffice

    def e2e_step():
        st.copy_(host_in, non_blocking=True)
        step()
        host_out.copy_(st, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    barrier(ws)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(e2e_steps):
        e2e_step()
    b.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(ws, a.elapsed_time(b))
    e2e_val = ws * step_bytes * e2e_steps / (e2e_ms / 1e3) / 1e9
    nbytes = host_in.numel() * host_in.element_size()
    return {
        "metric": "gate-apply HBM GB/s (algorithmic, 2 x bytes/amp x 2^n per gate)",
        "value": round(value, 1), "unit": "GB/s", "ms_per_step": round(ms_step, 2),
        "higher_is_better": True, "dtype": dtype_name,
        "config": {"workload": "gate-apply microbenchmark: %d-qubit %s state, %d Haar gates per "
                               "k=1..6 on random distinct targets" % (n, "complex64" if S == 8
                                                                       else "complex128", args.per_k),
                   "n_qubits": n, "gates_per_step": len(gates), "state_bytes": S << n,
                   "l2": "inputs larger than L2 (state %d GiB vs 129 MB L2)" % ((S << n) >> 30),
                   "seed": seed},
        "per_k": per_k, "kernels": fams, "roofline": roofline, "autotune": tune,
        "e2e": {"value": round(e2e_val, 1), "unit": "GB/s", "h2d_bytes_per_step": nbytes,
                "d2h_bytes_per_step": nbytes},
        "gpu_launches": launches,  # counted by the library's launch sites
        "clocks": clk.summary(),
    }


# -------------------------------------------------------------------------- HHL workloads
def run_hhl(args, ws, rank, which):
    import torch
    import paper_2402_08136_gb300 as qs

    assert which == "hhl7"
    p = synth.hhl7_problem()
    dtypes = [("c128", torch.complex128)]
    tb = time.perf_counter()
    h = qs.hhl_build(p["A"], p["b"], p["m"], p["t"], p["C"], structured=args.structured,
                     fft_qft=args.fft_qft)
    build_ms = 1e3 * (time.perf_counter() - tb)  # host: eigendecomposition and gate list
    info = h.info()
    n = info["n"]
    xt = np.linalg.solve(p["A"], p["b"])
    stream = torch.cuda.current_stream()
    res = {}
    for name, dt in dtypes:
        # complex64: widest fusion (dense 4..6 run on the tensor cores); complex128: FP64-bound,
        # narrow fusion keeps the flops per amplitude low
        max_k = args.max_k or (6 if name == "c64" else 2)
        tf = time.perf_counter()
        circ = qs.qsim_fuse(h.as_circuit(), max_k)
        fuse_ms = 1e3 * (time.perf_counter() - tf)
        ci = circ.info()
        st = torch.empty(1 << n, dtype=dt, device="cuda")

        def solve():
            # preparation and circuit; the operations before the inversion on the lower half
            # (the ancilla is |0> until then)
            qs.hhl_run(st, h, circ, stream)
            return qs.hhl_readout(st, h, stream)

        for _ in range(args.warmup):
            solve()
        torch.cuda.synchronize()
        lat = []
        barrier(ws)
        t0 = time.perf_counter()
        reps = args.steps * 200
        l0 = qs.qsim_launch_count()
        for _ in range(reps):
            a = time.perf_counter()
            r = solve()
            lat.append(time.perf_counter() - a)
        torch.cuda.synchronize()
        dt_s = max_over_ranks(ws, time.perf_counter() - t0)
        n_launch = qs.qsim_launch_count() - l0
        rel = float(np.linalg.norm(r["x"] - xt) / np.linalg.norm(xt))
        res[name] = {"solves_per_s": ws * reps / dt_s, "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                     "p99_ms": 1e3 * float(np.percentile(lat, 99)), "rel_err_vs_classical": rel,
                     "p_success": r["p_success"], "leakage": r["leakage"], "max_k": max_k,
                     "gpu_launches": n_launch, "launches_per_solve": n_launch / reps,
                     "host_fuse_ms": round(fuse_ms, 3),
                     "fused_ops": ci["n_gates"], "algorithmic_gb": ci["bytes_c64" if name == "c64" else "bytes_c128"] / 1e9}
        del st
    if True:
        # single-launch form: the whole circuit, state preparation and readout in one persistent
        # kernel (batched executor with one circuit, fusion width autotuned on it); each solve
        # is one library call (launch, synchronization, host scaling of the readout sums the
        # kernel wrote into pinned host memory)
        st = torch.empty(1 << n, dtype=torch.complex128, device="cuda")
        k1, tmap1 = qs.hhl_batch_autotune([h], [st], (1, 2, 3, 4), stream)
        circ = qs.qsim_fuse(h.as_circuit(), k1)
        b = qs.hhl_batch_create([h], [st], [circ])
        for _ in range(max(args.warmup, 3) * 10):
            b.solve(stream)
        reps = max(10000, args.steps * 2000)
        lat = []
        barrier(ws)
        t0 = time.perf_counter()
        l0 = qs.qsim_launch_count()
        for _ in range(reps):
            a = time.perf_counter()
            x, stats = b.solve(stream)
            lat.append(time.perf_counter() - a)
        dt_s = max_over_ranks(ws, time.perf_counter() - t0)
        n_single = qs.qsim_launch_count() - l0
        rel = float(np.linalg.norm(x - xt) / np.linalg.norm(xt))
        res["c128_single_launch"] = {"solves_per_s": ws * reps / dt_s,
                                     "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                                     "p99_ms": 1e3 * float(np.percentile(lat, 99)),
                                     "rel_err_vs_classical": rel, "solves_timed": reps,
                                     "fusion_k": k1, "fused_ops": circ.info()["n_gates"],
                                     "autotune_ms": {str(kk): round(v, 4) for kk, v in tmap1.items()},
                                     "p_success": float(stats[0]["p_success"]),
                                     "leakage": float(stats[0]["leakage"])}
        res["c128_single_launch"]["gpu_launches"] = n_single
        flops = circ.info()["flops"]
        main_name = "c128_single_launch"
    main = res[main_name]
    tf = flops * main["solves_per_s"] / 1e12
    roof = {"bound": "alu", "kernel": "batched_kernel<double> (one circuit)", "achieved": round(tf, 6),
            "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": round(tf / FP64_PEAK_TFLOPS, 6),
            "traffic": None, "flops_per_solve": flops,
            "peak_kind": "nominal GB300 FP64 rate (1.25 TFLOP/s; a probe measured 1.21)",
            "note": "a 7-qubit solve (2 KiB state) is launch- and latency-bound: one CTA, a barrier per op"}
    return {
        "metric": "HHL solves/s", "value": round(main["solves_per_s"], 3), "unit": "solves/s",
        "ms_per_step": round(1e3 / main["solves_per_s"], 4), "higher_is_better": True,
        "dtype": "c128",
        "config": {"workload": which, "n_qubits": n, "nb": info["nb"], "m": info["m"],
                   "unfused_gates": info["n_gates"], "structured_qpe": bool(args.structured),
                   "qft": "fourier passes" if args.fft_qft else "gates",
                   "host_build_ms": round(build_ms, 3)},
        "latency_ms": {"p50": round(main["p50_ms"], 4), "p99": round(main["p99_ms"], 4)},
        "paths": res, "roofline": roof,
        "gpu_launches": main["gpu_launches"],  # counted by the library's launch sites
    }


# ------------------------------------------------------------- 27-qubit HHL (precision form)
# Fourier-pass shapes of the 27-qubit solve (nb = 6, m = 20: two clock fields of 10 qubits):
# the inverse QFT's top-field pass with its twiddle from the 10 clock bits below, the
# bottom-field pass, and a Walsh-Hadamard pass; each streams a 2^27 state once
PASS_SHAPES = (("dft_top_field_twiddle", lambda c: c.add_dft(list(range(16, 26)), -1, src=list(range(6, 16)))),
               ("dft_bottom_field", lambda c: c.add_dft(list(range(6, 16)), -1)),
               ("walsh_top_field", lambda c: c.add_walsh(list(range(16, 26)))))


def fourier_pass_roofline(qs, torch, launches: int = 10):
    """Average launch time of each Fourier-pass shape on a 27-qubit complex64 state (1 GiB,
    larger than L2), CUDA events on the launching stream; algorithmic bytes 2 x 8 x 2^27."""
    n = 27
    st = synth.gaussian_state_torch(27, n, torch.complex64, "cuda", normalize=True)
    stream = torch.cuda.current_stream()
    out = {}
    for name, add in PASS_SHAPES:
        c = qs.Circuit(n)
        add(c)
        for _ in range(3):
            qs.qsim_apply(st, c, stream)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(launches)]
        for a, b in evs:
            a.record(stream)
            qs.qsim_apply(st, c, stream)
            b.record(stream)
        torch.cuda.synchronize()
        ms = float(np.mean([a.elapsed_time(b) for a, b in evs]))
        out[name] = {"us_per_launch": round(1e3 * ms, 2), "gbs": round(2.0 * 8 * (1 << n) / (ms / 1e3) / 1e9, 1)}
    del st
    return out


def sub_hhl27(args, ws, rank):
    """The 27-qubit precision-form solve: complex64 (structured phase estimation, QFTs as
    passes, fused dense gates on the tensor cores) and complex128 (FP64 SIMT), both through
    hhl_run + hhl_readout; solves/s, latency, readout error against the classical A^-1 b; the
    Fourier-pass kernel's roofline; the final states kept on the host for the comparison with
    the full-size oracle (oracle_hhl27_compare, run after every GPU measurement)."""
    import torch
    import paper_2402_08136_gb300 as qs

    p = synth.hhl27_problem()
    tb = time.perf_counter()
    h = qs.hhl_build(p["A"], p["b"], p["m"], structured=True, fft_qft=True)
    build_ms = 1e3 * (time.perf_counter() - tb)
    info = h.info()
    n = info["n"]
    xt = np.linalg.solve(p["A"], p["b"])
    stream = torch.cuda.current_stream()
    paths, keep = {}, {}
    reps = {"c64": 20, "c128": 5}
    tune = {}
    for name, dt, max_k in (("c64", torch.complex64, 6), ("c128", torch.complex128, 2)):
        tf = time.perf_counter()
        circ = qs.qsim_fuse(h.as_circuit(), max_k)
        fuse_ms = 1e3 * (time.perf_counter() - tf)
        ci = circ.info()
        st = torch.empty(1 << n, dtype=dt, device="cuda")
        if not args.no_autotune and not qs.qsim_tune_get(qs.QSIM_C64 if name == "c64" else qs.QSIM_C128,
                                                         qs.QSIM_TUNE_TUNED):
            tune[name] = qs.qsim_autotune(st, stream)
        # the readout's partial sums come out of the circuit's last kernel (hhl_run_sums)
        sums = torch.zeros(qs.QSIM_READOUT_SUMS_DOUBLES, dtype=torch.float64, device="cuda")
        for _ in range(3):
            qs.hhl_run_sums(st, h, sums, circ, stream)
            qs.hhl_readout_sums(st, h, sums, stream)
        torch.cuda.synchronize()
        lat = []
        with ClockSampler(torch.cuda.current_device()) as clk:
            l0 = qs.qsim_launch_count()
            t0 = time.perf_counter()
            for _ in range(reps[name]):
                a = time.perf_counter()
                qs.hhl_run_sums(st, h, sums, circ, stream)
                r = qs.hhl_readout_sums(st, h, sums, stream)
                lat.append(time.perf_counter() - a)
            dt_s = time.perf_counter() - t0
            nl = qs.qsim_launch_count() - l0
        dt_s = max_over_ranks(ws, dt_s)
        rel = float(np.linalg.norm(r["x"] - xt) / np.linalg.norm(xt))
        paths[name] = {"solves_per_s": round(ws * reps[name] / dt_s, 2), "ms_per_solve": round(1e3 * dt_s / reps[name], 3),
                       "p50_ms": round(1e3 * float(np.percentile(lat, 50)), 3),
                       "p99_ms": round(1e3 * float(np.percentile(lat, 99)), 3),
                       "readout_rel_err_vs_classical": rel, "p_success": r["p_success"],
                       "leakage": r["leakage"], "max_k": max_k, "fused_ops": ci["n_gates"],
                       "launches_per_solve": nl / reps[name], "host_fuse_ms": round(fuse_ms, 3),
                       "solves_timed": reps[name], "clocks": clk.summary()}
        # the same solve with hhl_run replayed from a CUDA graph (captured once; every launch of
        # the solve's circuit in one replay), the readout eager: no per-operation host work
        g = torch.cuda.CUDAGraph()
        cs = torch.cuda.Stream()
        cs.wait_stream(stream)
        with torch.cuda.stream(cs):
            qs.hhl_run_sums(st, h, sums, circ, cs)
        cs.synchronize()
        with torch.cuda.graph(g, stream=cs):
            qs.hhl_run_sums(st, h, sums, circ, cs)
        for _ in range(3):
            g.replay()
            qs.hhl_readout_sums(st, h, sums, stream)
        torch.cuda.synchronize()
        glat = []
        l0 = qs.qsim_launch_count()
        t0 = time.perf_counter()
        for _ in range(reps[name]):
            a = time.perf_counter()
            g.replay()
            rg = qs.hhl_readout_sums(st, h, sums, stream)
            glat.append(time.perf_counter() - a)
        gdt = max_over_ranks(ws, time.perf_counter() - t0)
        paths[name]["graph"] = {"solves_per_s": round(ws * reps[name] / gdt, 2),
                                "ms_per_solve": round(1e3 * gdt / reps[name], 3),
                                "p50_ms": round(1e3 * float(np.percentile(glat, 50)), 3),
                                "p99_ms": round(1e3 * float(np.percentile(glat, 99)), 3),
                                "readout_rel_err_vs_classical": float(np.linalg.norm(rg["x"] - xt) / np.linalg.norm(xt)),
                                "library_launches_outside_graph": qs.qsim_launch_count() - l0}
        del g
        keep[name] = (st.cpu().numpy(), r)
        del st
        torch.cuda.empty_cache()
    passes = fourier_pass_roofline(qs, torch)
    hbm, _, peak_kind = measured_peaks()
    ach = float(np.mean([v["gbs"] for v in passes.values()]))
    roof = {"bound": "hbm", "kernel": "dft_kernel", "achieved": round(ach, 1), "peak": hbm,
            "peak_kind": peak_kind + " copy bandwidth (MEASURED_PEAKS.json hbm_gbs)", "unit": "GB/s",
            "frac": round(ach / hbm, 4), "traffic": None,
            "bytes_per_launch": 2.0 * 8 * (1 << n), "per_shape": passes,
            "note": "mean of the three pass shapes of the solve, each timed alone on a 27-qubit complex64 state"}
    oracle_p = dict(p)
    oracle_p["m"] = 12
    best = paths["c64"]["graph"] if paths["c64"]["graph"]["solves_per_s"] > paths["c64"]["solves_per_s"] else paths["c64"]
    rec = {
        "metric": "HHL solves/s (27 qubits, complex64 precision form)", "value": best["solves_per_s"],
        "unit": "solves/s", "ms_per_solve": best["ms_per_solve"], "dtype": "c64",
        "solve_path": "hhl_run_sums replayed from a CUDA graph + hhl_readout_sums (readout partial sums from the circuit's last kernel)" if best is not paths["c64"]
                      else "hhl_run_sums + hhl_readout_sums (eager)",
        "config": {"workload": "27-qubit HHL: 64x64 reduced Laplacian of a random 65-bus grid (98 lines), "
                               "nb=6, m=20, structured phase estimation, QFTs as Fourier passes",
                   "n_qubits": n, "nb": info["nb"], "m": info["m"], "host_build_ms": round(build_ms, 3),
                   "l2": "state 1 GiB (c64) / 2 GiB (c128), larger than L2"},
        "latency_ms": {"p50": best["p50_ms"], "p99": best["p99_ms"]},
        "paths": paths, "roofline": roof, "tuning": qs.qsim_tune_table(), "autotune": tune,
        "speedup_c64_vs_c128": round(paths["c64"]["solves_per_s"] / paths["c128"]["solves_per_s"], 2),
        "gpu_launches": int(paths["c64"]["launches_per_solve"] * reps["c64"]),
    }
    if rank == 0:
        rec["cpu_baseline"] = oracle_hhl_both(
            [oracle_p], "one solve of the same 64x64 system with 12 instead of 20 clock qubits (19 "
                        "qubits; the 27-qubit solve has 2^8 x the amplitudes)")
    return rec, keep, p


def oracle_hhl27_compare(rec, keep, p):
    """The full-size FP64 oracle (plain gate-level HHL on 2^27 amplitudes, all host cores) and
    the error of each kept device state against it: max |d amp|, fidelity, and the readout
    relative error of the oracle itself against A^-1 b."""
    from oracle import core as ocore
    from oracle import hhl as ohhl
    t0 = time.perf_counter()
    ref = ohhl.solve(p["A"], p["b"], p["m"])
    secs = time.perf_counter() - t0
    xt = np.linalg.solve(p["A"], p["b"])
    rec["oracle_full_size"] = {"seconds": round(secs, 1), "cores": ocore.num_threads(),
                               "readout_rel_err_vs_classical": float(np.linalg.norm(ref["x"] - xt) / np.linalg.norm(xt)),
                               "p_success": ref["P"]}
    ps = ref["psi"]
    nps = np.vdot(ps, ps).real
    for name, (psi, r) in keep.items():
        z = psi.astype(np.complex128)
        fid = abs(np.vdot(ps, z)) ** 2 / (np.vdot(z, z).real * nps)
        rec["paths"][name]["err_vs_oracle"] = {"max_abs_amp": float(np.max(np.abs(z - ps))), "fidelity": float(fid),
                                               "p_success": abs(r["p_success"] - ref["P"])}
    rec["error_note"] = ("both library paths eigendecompose A themselves, like the oracle: complex64 is held "
                         "to 1e-5 per amplitude; complex128 here differs from the oracle by the eigensolvers' "
                         "rounding times t 2^m (bound 2^m 2 pi 8 eps = 1.2e-8); with a shared spectral "
                         "decomposition the complex128 path is held to 1e-12 (tests/test_gpu_hhl27.py)")


def with_args(args, **kw):
    a = argparse.Namespace(**vars(args))
    for k, v in kw.items():
        setattr(a, k, v)
    return a


def sub_records(args, ws, rank):
    """Configs 1, 3, 4 and 5 as sub-records of the default line, each at a fixed, bounded size
    (not scaled by --steps): the 7-qubit plain FP64 solve, the 27-qubit precision form, the
    512-circuit batch and a serving stream at a rate the box sustains; the full-size 27-qubit
    oracle last, after every GPU measurement."""
    import torch
    out = {}
    t0 = time.perf_counter()
    r7 = run_hhl(with_args(args, steps=2, warmup=3, structured=False, fft_qft=False, max_k=0), ws, rank, "hhl7")
    if rank == 0:
        r7["cpu_baseline"] = oracle_hhl_both([synth.hhl7_problem()] * 20, "20 solves of the 7-qubit problem")
    out["hhl7"] = r7
    r27, keep, p27 = sub_hhl27(args, ws, rank)
    out["hhl27"] = r27
    rb = run_batched(with_args(args, steps=20, warmup=3, count=512, structured=True, fft_qft=True), ws, rank)
    if rank == 0:
        probs = synth.batched_problems(seed=rank_seed(4, rank), count=512)[:16]
        rb["cpu_baseline"] = oracle_hhl_both(probs, "the first 16 circuits of the 512-circuit batch")
    out["batched512"] = rb
    torch.cuda.empty_cache()
    rs = run_serving(with_args(args, count=4000, rate=2000.0, max_n=22, pool_gb=150.0), ws, rank)
    if rank == 0:
        items = synth.serving_stream(seed=rank_seed(5, rank), count=200, max_n=16)
        rs["cpu_baseline"] = oracle_hhl_both([it["problem"] for it in items[:16]],
                                             "16 requests of the stream (qubits capped at 16)")
    out["serving"] = rs
    # the full qubit range 8..30 (7.5 % of the requests need 28-30 qubits, 2-8 GiB states): a
    # shorter stream at the same offered rate, to show the service rate and latency the box
    # reaches when the offered load exceeds it
    rf = run_serving(with_args(args, count=1000, rate=2000.0, max_n=30, pool_gb=150.0), ws, rank)
    out["serving_full_range"] = rf
    if rank == 0 and not args.no_oracle27:
        oracle_hhl27_compare(r27, keep, p27)
    del keep
    out["seconds"] = round(time.perf_counter() - t0, 1)
    return out


# ----------------------------------------------------------------------- batched workload
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12  # SMs x FP32 lanes x 2 flops x max clock


def run_batched(args, ws, rank):
    """512 N-1 contingency HHL solves of uneven size (7..16 qubits) per step, one persistent
    launch (replayed from a CUDA graph) plus the result copy; complex64 and complex128 with the
    autotuned fusion width; against the plain form (one circuit at a time, complex128,
    per-operation kernels + readout)."""
    import torch
    import paper_2402_08136_gb300 as qs

    count = args.count or 512
    probs = synth.batched_problems(seed=rank_seed(4, rank), count=count)
    t0 = time.perf_counter()
    hs = [qs.hhl_build(p["A"], p["b"], p["m"], structured=args.structured, fft_qft=args.fft_qft)
          for p in probs]
    t_build = time.perf_counter() - t0
    infos = [h.info() for h in hs]
    xt = [np.linalg.solve(p["A"], p["b"]) for p in probs]
    stream = torch.cuda.current_stream()
    paths = {}
    main_line = None
    for name, dt in (("c64", torch.complex64), ("c128", torch.complex128)):
        states = [torch.empty(1 << i["n"], dtype=dt, device="cuda") for i in infos]
        k, tmap = qs.hhl_batch_autotune(hs, states, (2, 3, 4, 5))
        t0 = time.perf_counter()
        fused = [qs.qsim_fuse(h.as_circuit(), k) for h in hs]
        t_fuse = time.perf_counter() - t0
        b = qs.hhl_batch_create(hs, states, fused)
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(stream)
        with torch.cuda.stream(s):
            b.run(s)
        s.synchronize()
        with torch.cuda.graph(g, stream=s):
            b.run(s)
        for _ in range(args.warmup):
            g.replay()
            b.results(stream)
        torch.cuda.synchronize()
        barrier(ws)
        a = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        ka = torch.cuda.Event(enable_timing=True)
        ke = torch.cuda.Event(enable_timing=True)
        kern_ms = 0.0
        with ClockSampler(torch.cuda.current_device()) as clk:
            a.record(stream)
            for _ in range(args.steps):
                ka.record(stream)
                g.replay()
                ke.record(stream)
                b.results_arrays(stream)  # every solution and statistic of the batch, on the host
                kern_ms += ka.elapsed_time(ke)
            e.record(stream)
            torch.cuda.synchronize()
        ms = max_over_ranks(ws, a.elapsed_time(e))
        sps = ws * count * args.steps / (ms / 1e3)
        res = b.results(stream)  # the same results as dicts, after the timed region
        rel = [float(np.linalg.norm(r["x"] - x) / np.linalg.norm(x)) for r, x in zip(res, xt)]
        sub_e = list(range(0, count, max(1, count // 64)))  # the plain form's subset
        flops = sum(f.info()["flops"] for f in fused)
        tf = flops * args.steps / (kern_ms / 1e3) / 1e12
        # the same circuits alone (batch of one) give bit-identical states
        ident = True
        for i in range(0, count, max(1, count // 8)):
            alone = torch.empty_like(states[i])
            b1 = qs.hhl_batch_create([hs[i]], [alone], [fused[i]])
            b1.run(stream)
            torch.cuda.synchronize()
            ident &= bool(torch.equal(alone, states[i]))
        paths[name] = {"solves_per_s": round(sps, 1), "ms_per_batch": round(ms / args.steps, 3),
                       "kernel_ms_per_batch": round(kern_ms / args.steps, 3), "fusion_k": k,
                       "autotune_ms": {str(kk): round(v, 3) for kk, v in tmap.items()},
                       "rel_err_vs_classical_median": float(np.median(rel)),
                       "rel_err_vs_classical_max": float(np.max(rel)),
                       "rel_err_vs_classical_median_plain_subset": float(np.median([rel[i] for i in sub_e])),
                       "alone_equals_in_batch": ident, "alu_tflops": round(tf, 3),
                       "fuse_s": round(t_fuse, 2), "clocks": clk.summary()}
        if name == "c64":
            bound = {"bound": "alu", "kernel": "batched_kernel<float>", "achieved": round(tf, 3),
                     "peak": round(FP32_PEAK_TFLOPS, 1), "unit": "TFLOP/s",
                     "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz (states are "
                                  "shared-memory / L2 resident, HBM is not the bound)",
                     "frac": round(tf / FP32_PEAK_TFLOPS, 4), "traffic": None}
            main_line = (sps, ms / args.steps, bound, clk.summary())
        del b, g, states
    # plain form: the paper's circuit (controlled evolutions, gate-level QFT), one circuit at a
    # time, complex128, per-operation kernels and readout
    sub = list(range(0, count, max(1, count // 64)))
    hp = {i: qs.hhl_build(probs[i]["A"], probs[i]["b"], probs[i]["m"]) for i in sub}
    fused_plain = {i: qs.qsim_fuse(hp[i].as_circuit(), 4) for i in sub}
    for i in sub[:4]:
        st = torch.empty(1 << infos[i]["n"], dtype=torch.complex128, device="cuda")
        qs.hhl_prepare_state(st, hp[i], stream)
        qs.qsim_apply(st, fused_plain[i], stream, n_qubits=infos[i]["n"])
        qs.hhl_readout(st, hp[i], stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rel_plain = []
    for i in sub:
        st = torch.empty(1 << infos[i]["n"], dtype=torch.complex128, device="cuda")
        qs.hhl_prepare_state(st, hp[i], stream)
        qs.qsim_apply(st, fused_plain[i], stream, n_qubits=infos[i]["n"])
        r = qs.hhl_readout(st, hp[i], stream)
        rel_plain.append(float(np.linalg.norm(r["x"] - xt[i]) / np.linalg.norm(xt[i])))
    t_plain = time.perf_counter() - t0
    paths["plain_c128"] = {"solves_per_s": round(len(sub) / t_plain, 1), "circuits_timed": len(sub),
                           "rel_err_vs_classical_median": float(np.median(rel_plain)),
                           "rel_err_vs_classical_max": float(np.max(rel_plain))}
    sps, ms_step, roof, clocks = main_line
    return {
        "metric": "HHL solves/s (batched, 512 contingency circuits per launch)",
        "value": round(sps, 1), "unit": "solves/s", "ms_per_step": round(ms_step, 3),
        "higher_is_better": True, "dtype": "c64",
        "config": {"workload": "batched: 512 N-1 contingency HHL circuits (nb 2..5, m 4..10, "
                               "7..16 qubits), one persistent launch per step from a CUDA graph",
                   "count": count, "host_build_s": round(t_build, 2),
                   "structured_qpe": bool(args.structured),
                   "qft": "fourier passes" if args.fft_qft else "gates",
                   "l2": "states shared-memory / L2 resident (working set < 129 MB)"},
        "paths": paths, "roofline": roof, "clocks": clocks,
        "speedup_vs_plain_c128": round(sps / paths["plain_c128"]["solves_per_s"], 1),
        "gpu_launches": args.steps,
    }


# ----------------------------------------------------------------------- serving workload
def _oracle_solve_job(job):
    """(index, A, b, m) -> oracle x (runs in a spawned worker process)."""
    import sys as _sys
    if ROOT not in _sys.path:
        _sys.path.insert(0, ROOT)
    from oracle import hhl as ohhl
    i, A, b, m = job
    r = ohhl.solve(A, b, m)
    return i, r["x"], r["P"]


def run_serving(args, ws, rank):
    """Poisson stream of HHL contingency solves (serving form): arrivals replayed in real time
    into the pool; latency = completion - arrival."""
    import multiprocessing as mp
    import threading as th
    import torch
    import paper_2402_08136_gb300 as qs

    count = args.count or 20000
    rate = args.rate
    max_n = args.max_n or 30
    t0 = time.perf_counter()
    items = synth.serving_stream(seed=rank_seed(5, rank), count=count, rate=rate, max_n=max_n)
    t_gen = time.perf_counter() - t0
    dtype = qs.QSIM_C64
    arena = int(args.pool_gb * (1 << 30))
    nproc = os.cpu_count() or 8
    pool = qs.Pool(arena, n_builders=max(2, nproc - 4), n_streams=8)
    # warm-up: one request of each path
    for it in items[:8]:
        tk = pool.submit(it["problem"]["A"], it["problem"]["b"], it["problem"]["m"], dtype=dtype,
                         structured=True)
        pool.wait(tk, 300.0)
        pool.poll(tk)
    while pool.take_completed(8192, 0.0):   # drop the warm-up tickets from the completion queue
        pass
    t_arr = [0.0] * count
    start = time.perf_counter() + 0.2
    index = {}

    def submitter():
        for i, it in enumerate(items):
            due = start + it["arrival"]
            d = due - time.perf_counter()
            if d > 0:
                time.sleep(d)
            p = it["problem"]
            t_arr[i] = time.perf_counter()
            tk = pool.submit(p["A"], p["b"], p["m"], dtype=dtype, structured=True)
            index[tk] = i

    with ClockSampler(torch.cuda.current_device()) as clk:
        thr = th.Thread(target=submitter)
        thr.start()
        results = [None] * count
        left = count
        t_last = start
        while left:
            for tk in pool.take_completed(8192, 0.05):   # completion queue: finished tickets only
                while tk not in index:                     # submit() returned, mapping not yet set
                    time.sleep(0)
                results[index[tk]] = pool.poll(tk)
                left -= 1
                t_last = time.perf_counter()
        thr.join()
    info = pool.info()
    pool.close()
    lat = np.array([r["latency_s"] for r in results])
    span = t_last - start
    sps = count / span
    xt_err = []
    for it, r in zip(items, results):
        p = it["problem"]
        xt = np.linalg.solve(p["A"], p["b"])
        xt_err.append(float(np.linalg.norm(r["x"] - xt) / np.linalg.norm(xt)))
    # FP64 oracle on a seeded 1% sample (requests of at most 16 qubits; larger sampled requests
    # are compared with the classical solution only)
    rng = np.random.default_rng(7)
    sample = sorted(rng.choice(count, size=max(1, count // 100), replace=False).tolist())
    jobs = [(i, items[i]["problem"]["A"], items[i]["problem"]["b"], items[i]["problem"]["m"])
            for i in sample if items[i]["n"] <= 16]
    t0 = time.perf_counter()
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(len(jobs), nproc) or 1) as op:
        ora = op.map(_oracle_solve_job, jobs)
    t_ora = time.perf_counter() - t0
    err_or = [float(np.linalg.norm(results[i]["x"] - x) / max(np.linalg.norm(x), 1e-300))
              for i, x, _ in ora]
    dp = [abs(results[i]["p_success"] - P) for i, _, P in ora]
    ns = np.array([it["n"] for it in items])
    # algorithmic HBM bytes of the served stream: per request, its full-state circuit (structured
    # phase estimation, QFTs as passes) in complex64; the live-width executor moves fewer
    shape_bytes = {}
    for it in items:
        pp = it["problem"]
        key = (pp["nb"], pp["m"])
        if key not in shape_bytes:
            hh = qs.hhl_build(pp["A"], pp["b"], pp["m"], structured=True, fft_qft=True)
            shape_bytes[key] = qs.qsim_fuse(hh.as_circuit(), 4).info()["bytes_c64"]
    tot_bytes = sum(shape_bytes[(it["problem"]["nb"], it["problem"]["m"])] for it in items)
    hbm, _, peak_kind = measured_peaks()
    gbs = tot_bytes / span / 1e9
    roof = {"bound": "hbm", "kernel": "whole served stream (batched_kernel, dft_kernel, dense kernels)",
            "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s", "frac": round(gbs / hbm, 4),
            "traffic": None, "peak_kind": peak_kind + " copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
            "note": "full-state algorithmic bytes of every request over the span from the first arrival "
                    "to the last completion; arrival-limited when the offered rate is below capacity"}
    return {
        "metric": "HHL solves/s served (Poisson arrivals) with p50/p99 latency",
        "roofline": roof,
        "value": round(sps, 1), "unit": "solves/s", "ms_per_step": round(1e3 * span, 1),
        "higher_is_better": True, "dtype": "c64",
        "config": {"workload": "serving: Poisson stream of N-1 contingency HHL solves, qubits "
                               "log-uniform 8..30 (capped at %d), structured phase estimation, "
                               "complex64" % max_n,
                   "requests": count, "rate_per_s": rate, "max_n": max_n,
                   "arena_gib": args.pool_gb, "stream_gen_s": round(t_gen, 1),
                   "requests_n_ge_28": int((ns >= 28).sum())},
        "latency_ms": {"p50": round(1e3 * float(np.percentile(lat, 50)), 3),
                       "p99": round(1e3 * float(np.percentile(lat, 99)), 3),
                       "max": round(1e3 * float(lat.max()), 3)},
        "offered_rate": rate, "achieved_rate": round(sps, 1),
        "pool": info,
        "error": {"rel_vs_classical_median": float(np.median(xt_err)),
                  "rel_vs_oracle_max": float(max(err_or)) if err_or else None,
                  "p_success_vs_oracle_max": float(max(dp)) if dp else None,
                  "oracle_sample": len(jobs), "oracle_seconds": round(t_ora, 1)},
        "clocks": clk.summary(), "gpu_launches": int(info["batches_launched"] + info["singles_launched"]),
    }

# ---------------------------------------------------------------------------------- main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="gates",
                    choices=["gates", "gates-c128", "hhl7", "hhl27", "batched", "serving"])
    ap.add_argument("--rate", type=float, default=2000.0, help="arrivals per second (serving)")
    ap.add_argument("--max-n", type=int, default=0, help="cap on qubits per request (serving)")
    ap.add_argument("--pool-gb", type=float, default=150.0, help="device arena (serving)")
    ap.add_argument("--count", type=int, default=0, help="circuits per batch (batched workload)")
    ap.add_argument("--n", type=int, default=0, help="override qubit count (gates workloads)")
    ap.add_argument("--per-k", type=int, default=200)
    ap.add_argument("--max-k", type=int, default=0)
    ap.add_argument("--structured", action="store_true", help="diagonalised phase estimation")
    ap.add_argument("--fft-qft", action="store_true", help="QFTs as Fourier-transform passes")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-from-host-gen", action="store_true")
    ap.add_argument("--no-subrecords", action="store_true",
                    help="default workload only: skip the configs 1, 3, 4, 5 sub-records")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the kernel-choice table's defaults (for profiling runs with a fixed launch sequence)")
    ap.add_argument("--no-oracle27", action="store_true",
                    help="skip the full-size 27-qubit oracle comparison (about 2 minutes of host time)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3) if args.impl == "ours" else args.warmup

    if args.impl == "reference":
        # the reference is a paper without code: this arm times the FP64 oracle on the host cores
        ws = int(os.environ.get("WORLD_SIZE", "1"))
        rank = int(os.environ.get("RANK", "0"))
        if rank != 0:
            return
        for _ in range(args.warmup):
            oracle_baseline(args.workload)
        vals = [oracle_baseline(args.workload) for _ in range(args.steps)]
        v = sum(x["value"] for x in vals) / len(vals)
        cb = dict(vals[-1])
        cb["value"] = round(v, 4)
        metric = {"gates": "gate-apply HBM GB/s (algorithmic, 2 x bytes/amp x 2^n per gate)",
                  "gates-c128": "gate-apply HBM GB/s (algorithmic, 2 x bytes/amp x 2^n per gate)",
                  "batched": "HHL solves/s (batched, 512 contingency circuits per launch)",
                  "serving": "HHL solves/s served (Poisson arrivals) with p50/p99 latency"}.get(
                      args.workload, "HHL solves/s")
        line = {"impl": "reference", "metric": metric, "value": round(v, 4), "unit": cb["unit"],
                "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(1e3 * cb["seconds"], 1), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": args.workload + " (bounded oracle sample: " + cb["sample"] + ")"},
                "cpu_baseline": cb,
                "e2e": {"value": round(v, 4), "unit": cb["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    from paper_2402_08136_gb300 import build as qbuild
    qbuild.build()
    ws, rank, local = dist_setup(args.gpus)
    if args.workload in ("gates", "gates-c128"):
        out = run_gates(args, ws, rank, "c64" if args.workload == "gates" else "c128")
        if args.workload == "gates" and not args.no_subrecords:
            out["workloads"] = sub_records(args, ws, rank)
    elif args.workload == "batched":
        out = run_batched(args, ws, rank)
    elif args.workload == "serving":
        out = run_serving(args, ws, rank)
    elif args.workload == "hhl27":
        out, keep, p27 = sub_hhl27(args, ws, rank)
        if rank == 0 and not args.no_oracle27:
            oracle_hhl27_compare(out, keep, p27)
        out["ms_per_step"] = out.pop("ms_per_solve")
        out["higher_is_better"] = True
        out.pop("cpu_baseline", None)
    else:
        out = run_hhl(args, ws, rank, args.workload)
    line = {"metric": out.pop("metric"), "value": out.pop("value"), "unit": out.pop("unit"),
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": out.pop("ms_per_step"), "higher_is_better": out.pop("higher_is_better"),
            "scaling": "weak", "vs_baseline": None, "dtype": out.pop("dtype"), "data": "synthetic",
            "config": dict(out.pop("config"), parallelism="replicas x%d" % ws)}
    line.update(out)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_baseline(args.workload, rank)
    if rank == 0:
        print(json.dumps(line))
    barrier(ws)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
