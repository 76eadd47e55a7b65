"""Partition of the nested probe sequence across ranks (host logic only).

Probe quadratures are independent (Section 2.2: each q_m is one solve per
dilution index), so rank r of W solves the contiguous block
[r * n, (r + 1) * n) of every round of W * n probes and no collective is
needed while the solves run.  At the end one all-gather exchanges the FP64
quadratures of every rank's blocks; concatenated in probe order they give the
nested sequence q_0, q_1, ... from which every prefix estimate
T_s = (1/s) sum_{m<s} q_m follows (the library's hp_trace_prefix sums them in
the same order as a one-rank run, so the ranks' T_s agree with it bit for bit).
"""
from __future__ import annotations

import numpy as np


def probe_block(rank: int, world: int, per_rank: int, round_index: int = 0) -> tuple[int, int]:
    """(first, count) of the probes rank ``rank`` solves in round ``round_index``."""
    if world < 1 or not (0 <= rank < world) or per_rank < 0 or round_index < 0:
        raise ValueError("bad partition arguments")
    first = (round_index * world + rank) * per_rank
    return first, per_rank


def assemble(blocks: list[tuple[int, list]]) -> list:
    """Concatenate (first, q-values) blocks from all ranks into one sequence, checking that they
    tile [0, total) without gaps or overlaps."""
    blocks = sorted(blocks, key=lambda b: b[0])
    out: list = []
    for first, vals in blocks:
        if first != len(out):
            raise ValueError("probe blocks do not tile the sequence (gap or overlap at %d)" % first)
        out.extend(vals)
    return out


def gather_quadratures(q: np.ndarray, rank: int, world: int, per_rank: int, rounds: int,
                       device: str = "cpu") -> np.ndarray:
    """The full sequence q[0 .. rounds * world * per_rank) on every rank, from each rank's own
    blocks of rounds 0 .. rounds-1 (``q`` complex128 on the host; the other ranks' entries are
    ignored).  One all-gather of the FP64 (re, im) pairs (``device``: where the exchanged
    tensor lives, "cuda:i" for NCCL, "cpu" for gloo); the values are copied, never added, so
    every rank receives every q_m bit for bit."""
    total = rounds * world * per_rank
    if q.dtype != np.complex128 or q.shape[0] < total:
        raise ValueError("q must be complex128 with at least %d entries" % total)
    mine = np.empty((rounds, per_rank), dtype=np.complex128)
    for r in range(rounds):
        first, n = probe_block(rank, world, per_rank, r)
        mine[r] = q[first:first + n]
    if world == 1:
        parts = [mine]
    else:
        import torch
        import torch.distributed as dist

        t = torch.from_numpy(mine.view(np.float64).copy()).to(device)
        recv = [torch.empty_like(t) for _ in range(world)]
        dist.all_gather(recv, t)
        parts = [x.cpu().numpy().view(np.complex128) for x in recv]
    full = np.zeros(total, dtype=np.complex128)
    for src, vals in enumerate(parts):
        for r in range(rounds):
            first, n = probe_block(src, world, per_rank, r)
            full[first:first + n] = vals[r]
    return full
