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
