"""One state vector sharded over the ranks of a process group (the paper's simulator spreads
its state over several GPUs, Sec. II-C; Sec. III-B reaches 42 qubits that way).

Rank r of a group of 2^g ranks holds the 2^(n-g) amplitudes whose top g qubits equal r.  The
library's planner (`ShardPlan`, C ABI `qsim_shard_plan_create`) turns an unfused circuit into
local circuits and qubit swaps; this module executes a plan: a local circuit runs on the shard
with the library's kernels (qsim_fuse + qsim_apply), a swap of global bit b with local qubit p
is a pairwise exchange with rank r ^ 2^b of half of each shard (packed into a contiguous buffer
by the library's kernel, sent and received with torch.distributed -- NCCL between GPUs, or any
backend whose tensors live where the shard lives -- and unpacked into the same positions).
No collective other than these point-to-point pairs is used.

`run_sharded` takes the three operations as arguments so that the exchange protocol can be
driven with other implementations (the CPU tests use numpy views and the FP64 oracle); the
defaults are the library's.
"""
from __future__ import annotations

from . import _binding as B


def _library_ops(max_k: int):
    import torch

    def apply(shard, circuit, stream=None):
        B.qsim_apply(shard, B.qsim_fuse(circuit, max_k), stream, n_qubits=shard.numel().bit_length() - 1)

    def pack(shard, qubit, value, stream=None):
        out = torch.empty(shard.numel() // 2, dtype=shard.dtype, device=shard.device)
        return B.qsim_shard_pack(shard, qubit, value, out, stream)

    def unpack(shard, qubit, value, buf, stream=None):
        B.qsim_shard_unpack(shard, qubit, value, buf, stream)

    return apply, pack, unpack


def exchange_halves(send_buf, partner: int, rank: int, group=None):
    """Swap send_buf with the partner rank's buffer of the same shape (the lower rank sends
    first, so the blocking pair cannot deadlock); returns the received buffer."""
    import torch
    import torch.distributed as dist
    recv = torch.empty_like(send_buf)
    if rank < partner:
        dist.send(send_buf, partner, group=group)
        dist.recv(recv, partner, group=group)
    else:
        dist.recv(recv, partner, group=group)
        dist.send(send_buf, partner, group=group)
    return recv


def run_sharded(shard, plan: "B.ShardPlan", rank: int, group=None, apply=None, pack=None, unpack=None,
                exchange=None, max_k: int = 4, on_step=None):
    """Execute `plan` on this rank's shard in place.  apply(shard, circuit), pack(shard, qubit,
    value) -> buffer, unpack(shard, qubit, value, buffer) and exchange(buffer, partner, rank) ->
    buffer default to the library's kernels and torch.distributed point-to-point transfers.
    on_step(i, step), if given, is called before each step."""
    la, lp, lu = _library_ops(max_k)
    apply = apply or la
    pack = pack or lp
    unpack = unpack or lu
    exchange = exchange or (lambda buf, partner, r: exchange_halves(buf, partner, r, group))
    for i, step in enumerate(plan.steps):
        if on_step is not None:
            on_step(i, step)
        if step["kind"] == "apply":
            apply(shard, step["circuit"])
            continue
        b, p = step["global_bit"], step["local_qubit"]
        v = 1 - ((rank >> b) & 1)          # the half whose bit p differs from bit b of the rank
        partner = rank ^ (1 << b)
        got = exchange(pack(shard, p, v), partner, rank)
        unpack(shard, p, v, got)
    return shard
