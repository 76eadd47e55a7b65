"""The N > 1 path on CPU with world_size-2 gloo process groups: disjoint probe blocks per rank,
no data-path collective, max-over-ranks timing, and a rank that leaves before the barrier."""
import os
import socket
import time

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1302_4018_gb300.sharding import assemble, gather_quadratures, probe_block


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _init(rank, world, port, timeout_s=60):
    import datetime

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=timeout_s))


def _worker_quadratures(rank, world, port, out_q):
    from oracle import estimator as E

    _init(rank, world, port)
    dims = (4, 4, 2, 2)
    per_rank = 3
    blocks = []
    for rnd in range(2):
        first, count = probe_block(rank, world, per_rank, rnd)
        q = E.laplacian_quadratures(dims, 0.3, first, count, 7, method="dense")
        blocks.append((first, [complex(v) for v in q]))
    # timing as bench.py does it: each rank measures, the max is taken
    t = torch.tensor([float(rank + 1)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    gathered = [None] * world
    dist.all_gather_object(gathered, blocks)
    if rank == 0:
        out_q.put((t.item(), [b for g in gathered for b in g]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_tile_the_nested_sequence():
    from oracle import estimator as E

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker_quadratures, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    tmax, blocks = q.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert tmax == 2.0
    seq = assemble(blocks)
    assert len(seq) == 12
    ref = E.laplacian_quadratures((4, 4, 2, 2), 0.3, 0, 12, 7, method="dense")
    assert np.allclose(seq, ref, rtol=1e-13)
    T = E.trace_prefix(seq)
    assert np.allclose(T, E.trace_prefix(ref), rtol=1e-13)


def _worker_gather(rank, world, port, out_q):
    """Each rank fills only its own probe blocks (the others stay zero, as in bench.py at N > 1),
    then the all-gather helper gives every rank the whole nested sequence."""
    from oracle import estimator as E

    _init(rank, world, port)
    dims, per_rank, rounds = (4, 4, 2, 2), 2, 3
    q = np.zeros(rounds * world * per_rank + 5, dtype=np.complex128)
    for rnd in range(rounds):
        first, count = probe_block(rank, world, per_rank, rnd)
        q[first:first + count] = E.laplacian_quadratures(dims, 0.3, first, count, 7, method="dense")
    full = gather_quadratures(q, rank, world, per_rank, rounds)
    out_q.put((rank, full.tobytes()))
    dist.barrier()
    dist.destroy_process_group()


def test_gathered_quadratures_equal_the_one_rank_sequence_bitwise():
    from oracle import estimator as E

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker_gather, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=240) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # the one-rank run solves the same probes block by block in sequence order
    one = np.concatenate([E.laplacian_quadratures((4, 4, 2, 2), 0.3, f, 2, 7, method="dense")
                          for f in range(0, 12, 2)]).astype(np.complex128)
    for r in range(2):
        seq = np.frombuffer(got[r], dtype=np.complex128)
        assert seq.tobytes() == one.tobytes(), r
        assert E.trace_prefix(seq).tobytes() == E.trace_prefix(one).tobytes()


def test_gather_on_one_rank_is_the_identity():
    q = np.arange(8, dtype=np.float64).astype(np.complex128) * (1 + 0.5j)
    assert np.array_equal(gather_quadratures(q, 0, 1, 4, 2), q)
    with pytest.raises(ValueError):
        gather_quadratures(q[:5], 0, 1, 4, 2)


def _worker_leaves(rank, world, port, out_q):
    _init(rank, world, port, timeout_s=5)
    if rank == 1:
        os._exit(0)            # leaves between steps, before the barrier
    t0 = time.time()
    try:
        dist.barrier()
        out_q.put("no error")
    except Exception as e:      # the survivor learns of it through the process-group timeout
        out_q.put("error after %.1f s: %s" % (time.time() - t0, type(e).__name__))


def test_rank_that_leaves_is_detected_by_timeout():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker_leaves, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    msg = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
    assert msg.startswith("error"), msg


def test_partition_arguments():
    assert probe_block(1, 4, 5, 2) == ((2 * 4 + 1) * 5, 5)
    with pytest.raises(ValueError):
        probe_block(4, 4, 5)
    with pytest.raises(ValueError):
        assemble([(0, [1, 2]), (3, [4])])
