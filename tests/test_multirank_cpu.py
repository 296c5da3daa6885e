"""The multi-GPU path of bench.py (one process per GPU, weak scaling over chains) run as
two gloo ranks on CPU: distinct chains and keys per rank, the slowest rank's time taken
by every rank, the whole-job rate over all ranks' chains."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    from paper_1908_09359_gb300 import inputs
    w = inputs.WORKLOADS["peps_24x24"] | {"seed": inputs.SEED_BASE + 3}
    seeds = bench.rank_seeds(w, rank)
    slowest = bench.max_over_ranks(10.0 + rank, dist, "cpu")
    rate = bench.whole_job_rate(world, 512, 2, slowest)
    gathered = [None] * world
    dist.all_gather_object(gathered, seeds)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, seeds, slowest, rate, gathered))


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, t0, v0, g0), (r1, s1, t1, v1, g1) = res
    assert (r0, r1) == (0, 1)
    assert s0["spins"] != s1["spins"] and s0["key"] != s1["key"]   # independent chains
    assert g0 == g1 == [s0, s1]
    assert t0 == t1 == pytest.approx(11.0)                        # the slowest rank's time
    assert v0 == v1 == pytest.approx(2 * 512 * 2 / 11.0)          # all ranks' samples
