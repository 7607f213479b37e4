"""State sharding with the qubit-swap exchange on one GPU: G = 2, 4, 8 shards of one state held
as separate device buffers in one process (each rank's shard), the library's planner, its
local circuits (fused, applied with qsim_apply), and its pack / unpack kernels for the pairwise
half-shard exchange, the partner's buffer handed over directly instead of sent.  The shards in
rank order must equal the oracle's full state: 1e-12 (complex128), 1e-5 with fidelity
>= 1 - 1e-6 (complex64).  (Several GPUs are not available here; the multi-process exchange over
torch.distributed is covered on CPU ranks in test_sharded_cpu.py.)"""
import numpy as np
import pytest
import torch

import synth
from oracle import hhl as ohhl
from sharding_case import apply_oracle_gate, random_case
from test_gpu_parity import TOL, check, host_input

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qs(cuda_device):
    from paper_2402_08136_gb300 import build
    build.build()
    import paper_2402_08136_gb300 as q
    return q


def run_all_shards(qs, plan, shards, max_k=4):
    from paper_2402_08136_gb300 import sharded
    apply, pack, unpack = sharded._library_ops(max_k)
    G = len(shards)
    for step in plan.steps:
        if step["kind"] == "apply":
            for sh in shards:
                apply(sh, step["circuit"])
            continue
        b, p = step["global_bit"], step["local_qubit"]
        bufs = [pack(shards[r], p, 1 - ((r >> b) & 1)) for r in range(G)]
        for r in range(G):
            unpack(shards[r], p, 1 - ((r >> b) & 1), bufs[r ^ (1 << b)])
    torch.cuda.synchronize()
    return torch.cat(shards)


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
@pytest.mark.parametrize("g", [1, 2, 3])
def test_sharded_random_circuit_matches_oracle(qs, dtype, g):
    n = 16
    c, gates = random_case(qs, n, 60, seed=100 + g)
    plan = qs.ShardPlan(c, g)
    assert any(s["kind"] == "swap" for s in plan.steps)
    psi = host_input(synth.gaussian_state_np(9 + g, n), dtype)
    ref = psi.copy()
    for gt in gates:
        apply_oracle_gate(ref, gt)
    nl = n - g
    shards = [torch.from_numpy(psi[r << nl:(r + 1) << nl].copy()).to(dtype).cuda() for r in range(1 << g)]
    out = run_all_shards(qs, plan, shards)
    check(out, ref, dtype)


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_sharded_hhl_matches_oracle(qs, dtype):
    """A gate-level HHL solve (controlled evolutions, QFTs as passes, the inversion) over 4 shards:
    the ancilla and the top clock qubit are global, so the rotation and the passes on the top
    field need swaps."""
    rng = np.random.default_rng(5)
    A, b = synth.contingency_system(rng, 2 ** 3 + 1)
    m = 9
    h = qs.hhl_build(A, b, m, fft_qft=True)
    info = h.info()
    n = info["n"]
    ref = ohhl.solve(A, b, m)
    g = 2
    nl = n - g
    plan = qs.ShardPlan(h.as_circuit(), g)
    st = torch.empty(1 << n, dtype=dtype, device="cuda")
    qs.hhl_prepare_state(st, h)
    torch.cuda.synchronize()
    shards = [st[r << nl:(r + 1) << nl].clone() for r in range(1 << g)]
    out = run_all_shards(qs, plan, shards)
    tol = TOL[dtype] if dtype == torch.complex64 else max(1e-12, 2.0 ** m * 2 * np.pi * 8 * np.finfo(float).eps)
    err = float(np.max(np.abs(out.cpu().numpy().astype(np.complex128) - ref["psi"])))
    assert err <= tol, err
