"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2): each rank
solves its own problem (independent replicas, no data-path collective) and
the whole-job numbers are the slowest rank's time and the summed work."""
import os
import socket
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        t, f = bench.reduce_over_ranks(1.5 + rank, 10.0 * (rank + 1), world, device="cpu")
        # the replicas' problems: cas16_m512 seeds 3 + rank, and batched
        # problem s of rank r from seed s + 64 r
        class A:
            batch_sweeps, tol, precision, refine = 1, 1e-6, "bf16", 0
        p = bench.batched_problems(A, rank)
        h0 = torch.tensor(float(np.abs(p[0][0]).sum()), dtype=torch.float64)
        hs = [torch.zeros((), dtype=torch.float64) for _ in range(world)]
        dist.all_gather(hs, h0)
        q.put((rank, t, f, [float(x) for x in hs], len(p)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_replicas_over_two_gloo_ranks():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, f, hs, n in out:
        assert t == 2.5 and f == 30.0        # max of 1.5, 2.5; 10 + 20
        assert n == 64
        assert hs[0] != hs[1]                # the ranks' problems differ
