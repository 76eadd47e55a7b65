"""Partition of the nested probe sequence across ranks (host logic only).

Probe quadratures are independent (Section 2.2: each q_m is one solve per
dilution index), so rank r of W solves the contiguous block
[r * n, (r + 1) * n) of every round of W * n probes and no collective is
needed on the data path.  Concatenating the ranks' blocks in rank order gives
the nested sequence q_0, q_1, ... from which any prefix estimate
T_s = (1/s) sum_{m<s} q_m follows.
"""
from __future__ import annotations


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
