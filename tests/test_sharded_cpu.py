"""State sharding with the qubit-swap exchange, on CPU ranks (gloo, world size 2 and 4): the
library's planner (host code) and the exchange protocol of paper_2402_08136_gb300.sharded (the
pairwise half-shard send/receive) drive the shards; the local gates are applied by the FP64
oracle on each shard with the plan's qubit map.  The gathered shards equal the oracle's full
state within 1e-12, so the plan (where it swaps, which halves move, the final reordering) and
the exchange are right.  No GPU: the library's pack/unpack kernels are replaced by numpy views
of the same halves."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as tmp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N = 10


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _half_view(shard, n_local, qubit, value):
    t = shard.reshape(-1, 2, 1 << qubit)
    return t[:, value, :]


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch
    import torch.distributed as dist
    import paper_2402_08136_gb300 as qs
    import synth
    from paper_2402_08136_gb300 import build, sharded
    from sharding_case import apply_oracle_gate, random_case
    build.build()
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    g = ws.bit_length() - 1
    nl = N - g
    c, gates = random_case(qs, N, 40, seed=17)
    plan = qs.ShardPlan(c, g)
    psi = synth.gaussian_state_np(5, N)
    shard = psi[rank << nl:(rank + 1) << nl].copy()
    current = {}

    def on_step(i, step):
        current["i"] = i

    def apply(sh, circuit):
        st = plan.steps[current["i"]]
        if st["first_gate"] == st["last_gate"]:
            # final local reordering: the SWAP gates of the local circuit, taken from the map before it
            prev = plan.steps[current["i"] - 1]["perm"] if current["i"] > 0 else list(range(N))
            from sharding_case import permute_qubits
            local_from = [prev[qq] for qq in range(nl)]
            sh[:] = permute_qubits(sh, nl, local_from)
            return
        for k in range(st["first_gate"], st["last_gate"]):
            apply_oracle_gate(sh, gates[k], st["perm"])

    def pack(sh, qubit, value):
        return torch.from_numpy(np.ascontiguousarray(_half_view(sh, nl, qubit, value)).reshape(-1))

    def unpack(sh, qubit, value, buf):
        _half_view(sh, nl, qubit, value)[:] = buf.numpy().reshape(-1, 1 << qubit)

    sharded.run_sharded(shard, plan, rank, apply=apply, pack=pack, unpack=unpack, on_step=on_step)
    parts = [torch.empty(1 << nl, dtype=torch.complex128) for _ in range(ws)]
    dist.all_gather(parts, torch.from_numpy(shard))
    if rank == 0:
        full = np.concatenate([p.numpy() for p in parts])
        ref = psi.copy()
        for gt in gates:
            apply_oracle_gate(ref, gt)
        swaps = sum(1 for s in plan.steps if s["kind"] == "swap")
        q.put((float(np.max(np.abs(full - ref))), swaps, len(plan.steps)))
    dist.destroy_process_group()


@pytest.mark.parametrize("ws", [2, 4])
def test_sharded_state_over_gloo_ranks_matches_oracle(ws):
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    err, swaps, steps = q.get(timeout=10)
    assert swaps >= 1
    assert err <= 1e-12, "gathered shards differ from the oracle by %.3e" % err
