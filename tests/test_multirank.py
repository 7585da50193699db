"""The N > 1 paths of bench.py on CPU ranks (gloo):
* replicas: the whole-job numbers are the slowest rank's time and the summed
  work;
* partitioned batches: the 64 active spaces of the batched workload are split
  by the library's LPT partition, every problem is solved by exactly one rank,
  the load is within the greedy bound, and the results gathered on rank 0
  equal a one-rank run bit for bit.  The per-problem solve here is the CPU
  oracle's FCI energy of small problems (no GPU), which exercises the same
  partition and gather code as the GPU runs."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class _Args:
    batch_sweeps, tol, precision, refine = 1, 1e-6, "bf16", 0


def _small_problems():
    # 13 half-filled active spaces of 2..4 orbitals (S_z = 1/2 when odd)
    from gbd_synth import make_integrals
    out = []
    for s in range(13):
        n = 2 + s % 3
        h, chol = make_integrals(n, 3, 500 + s)
        out.append((h, chol, n, n % 2, [16] * (1 + s % 2), [1e-8] * (1 + s % 2), {"seed": s}))
    return out


def _fci_energy(p):
    from oracle import fock
    h, chol, ne, sz = p[:4]
    w, _, _ = fock.ground_state(h, fock.eri_from_chol(chol), (ne + sz) // 2, (ne - sz) // 2)
    return float(w[0])


def _rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        t, f = bench.reduce_over_ranks(1.5 + rank, 10.0 * (rank + 1), world, device="cpu")
        # the batched workload's partition: the same on every rank
        owner64, load64 = bench.partition_problems(bench.batched_problems(_Args), world)
        mine64 = [i for i in range(64) if owner64[i] == rank]
        # partitioned solve of small problems, gathered on rank 0
        probs = _small_problems()
        owner, _ = bench.partition_problems(probs, world)
        mine = [(i, _fci_energy(probs[i])) for i in range(len(probs)) if owner[i] == rank]
        gathered = bench.gather_results(mine, len(probs), world)
        q.put((rank, t, f, mine64, [float(x) for x in load64], gathered))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _run(world):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted([q.get(timeout=300) for _ in procs])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return out


@pytest.mark.parametrize("world", [2, 3])
def test_partitioned_batches_over_gloo_ranks(world):
    sys.path.insert(0, ROOT)
    import bench
    from paper_2609_09990_gb300 import gbdmrg as G
    out = _run(world)
    # reduce: max of the times, sum of the work
    for rank, t, f, *_ in out:
        assert t == 1.5 + (world - 1) and f == 10.0 * world * (world + 1) / 2
    # every one of the 64 problems on exactly one rank
    owned = [i for o in out for i in o[3]]
    assert sorted(owned) == list(range(64))
    # greedy list-scheduling bound: makespan <= total / m + (1 - 1/m) max cost
    cost = G.host_batch_costs(bench.batched_problems(_Args))
    load = np.array(out[0][4])
    assert np.allclose([cost[o[3]].sum() for o in out], load)
    assert load.max() <= cost.sum() / world + (1 - 1 / world) * cost.max() + 1e-9 * cost.sum()
    # gathered results on rank 0 equal a one-rank run bit for bit
    one = [_fci_energy(p) for p in _small_problems()]
    assert out[0][5] == one
    assert all(o[5] is None for o in out[1:])
