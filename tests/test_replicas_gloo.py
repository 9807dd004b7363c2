"""The multi-GPU path of bench.py is replicas: every rank solves its own,
independently seeded batch and the only collective is the max over ranks of
the step time.  Checked here with two gloo ranks on the CPU."""
import multiprocessing as mp
import os
import socket

import numpy as np


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from inputs import lattice as L
    cfg = L.CONFIGS["wilson_4x4x4x4"]
    src = bench.rank_sources(cfg, rank, 2)
    t = bench.max_over_ranks(10.0 + 5.0 * rank)
    q.put((rank, float(np.abs(src).sum()), src[0, 0, 0, 0], t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, e0, t0), (r1, s1, e1, t1) = out
    assert t0 == t1 == 15.0          # max over ranks
    assert e0 != e1                   # independent sources per rank


def test_single_process_max_is_identity():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
