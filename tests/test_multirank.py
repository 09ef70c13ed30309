"""Replica parallelism across ranks (what `bench.py --gpus N` runs), tested with gloo on CPU.

Each rank runs its own GA replica, drawing its random numbers with stream id
= rank; there is no collective on the data path, only the final totals
(evaluations summed, time the maximum over ranks).  Here the replicas are the
CPU oracle's GA, so no GPU is needed.
"""

import multiprocessing as mp
import os
import socket
import time

import numpy as np

import oracle
from paper_1610_10061_gb300.inputs import graph_instance


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    d = graph_instance(60, 150, seed=4)
    pi, de = oracle.tables(d, 6)
    t0 = time.perf_counter()
    st, trace, _, _ = oracle.ga_run(pi, de, 60, 6, seed=0, P=64, D=32, gens=3, inst=rank)
    ms = 1000 * (time.perf_counter() - t0) + rank  # ranks report different times on purpose
    tot, mx = bench.combine_ranks(st.evals, ms)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, st.evals, ms, tot, mx, trace.tolist()))


def test_two_replicas_combine_without_data_collectives():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=240) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, e0, m0, t0, x0, tr0), (_, e1, m1, t1, x1, tr1) = out
    assert t0 == t1 == e0 + e1
    assert x0 == x1 == max(m0, m1)
    # the replicas are independent runs (different stream ids) and each equals the standalone run
    d = graph_instance(60, 150, seed=4)
    pi, de = oracle.tables(d, 6)
    for r, tr in ((0, tr0), (1, tr1)):
        _, want, _, _ = oracle.ga_run(pi, de, 60, 6, seed=0, P=64, D=32, gens=3, inst=r)
        assert tr == want.tolist()
    st0, _, pops0, _ = oracle.ga_run(pi, de, 60, 6, seed=0, P=64, D=32, gens=1, inst=0, record=True)
    st1, _, pops1, _ = oracle.ga_run(pi, de, 60, 6, seed=0, P=64, D=32, gens=1, inst=1, record=True)
    assert not np.array_equal(pops0, pops1)


# ---------------------------------------------------------------------------
# Client-sharded evaluation: partial costs over client blocks, one all-reduce.
# ---------------------------------------------------------------------------

def test_client_blocks_partition_the_clients():
    from paper_1610_10061_gb300.shard import client_block

    for n in (1, 7, 100, 901):
        for world in (1, 2, 3, 8):
            if world > n:
                continue
            blocks = [client_block(n, r, world) for r in range(world)]
            assert blocks[0][0] == 0 and blocks[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(blocks, blocks[1:]))
            sizes = [hi - lo for lo, hi in blocks]
            assert max(sizes) - min(sizes) <= 1


def _shard_worker(rank, world, port, q):
    import torch.distributed as dist

    from paper_1610_10061_gb300.inputs import random_masks
    from paper_1610_10061_gb300.shard import ShardedEvaluator

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1610_10061_gb300.shard import client_block

    d = graph_instance(90, 200, seed=7)
    p = 9
    # on CPU ranks the slice evaluator is the oracle's scan over this rank's truncated rows
    lo, hi = client_block(90, rank, world)
    pi, de = oracle.tables(d[lo:hi], p)
    ev = ShardedEvaluator(d, p, slice_evaluator=lambda masks: oracle.eval_scan(pi, de, masks))
    masks = random_masks(40, 90, p, seed=11)
    full = ev.eval(masks)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ev.lo, ev.hi, full.tolist()))


def test_two_ranks_client_sharded_costs_equal_the_full_cost():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=240) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, lo0, hi0, c0), (_, lo1, hi1, c1) = out
    assert (lo0, hi0, lo1, hi1) == (0, 45, 45, 90)
    from paper_1610_10061_gb300.inputs import random_masks

    d = graph_instance(90, 200, seed=7)
    expect = oracle.eval_direct(d, random_masks(40, 90, 9, seed=11))
    np.testing.assert_array_equal(c0, expect)
    np.testing.assert_array_equal(c1, expect)
