"""The multi-GPU path (one process per GPU) run as two gloo ranks on CPU.

* bench.py's sharding: every rank runs its own slice of the job's chains with the job's
  one Philox key and a chain offset (so its draws are those of the same chains in a
  one-rank job), the slowest rank's time is taken by every rank, and the whole-job rate
  counts all ranks' chains.
* The one exchange of the path (Algorithm 1's gradient step, Sec. II B): the float64 sums
  E_tot, E_tot^2, n, P1 = sum G E_loc and P2 = sum G of each rank's samples are
  all-reduced (paper_1908_09359_gb300.dist) before the sign-SGD step.  Each rank's sums
  come from the FP64 oracle on its own configurations; after the exchange both ranks hold
  bit-identical gradients and updated tensors, equal to those of one rank holding every
  configuration.
"""
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


def _spawn(target, world):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=target, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return res


def _shard_rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    from paper_1908_09359_gb300 import inputs
    w = dict(inputs.WORKLOADS["peps_8x8"], seed=inputs.SEED_BASE + 1, n_chains=16)
    share = bench.rank_share(w, rank, world)
    slowest = bench.max_over_ranks(10.0 + rank, dist, "cpu")
    rate = bench.whole_job_rate(world, 16, 2, slowest)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, share["spins"], share["chain_offset"], share["key"], slowest, rate))


def test_two_gloo_ranks_share_the_chains():
    sys.path.insert(0, ROOT)
    import bench
    from paper_1908_09359_gb300 import inputs
    res = _spawn(_shard_rank, 2)
    (r0, s0, o0, k0, t0, v0), (r1, s1, o1, k1, t1, v1) = res
    whole = bench.rank_share(dict(inputs.WORKLOADS["peps_8x8"], seed=inputs.SEED_BASE + 1, n_chains=32), 0, 1)
    assert np.array_equal(np.concatenate([s0, s1]), whole["spins"])   # slices of the one-rank job
    assert (o0, o1) == (0, 16) and k0 == k1 == whole["key"]
    assert t0 == t1 == pytest.approx(11.0)                            # the slowest rank's time
    assert v0 == v1 == pytest.approx(2 * 16 * 2 / 11.0)               # all ranks' samples


def _oracle_case():
    from oracle import vmc
    from paper_1908_09359_gb300 import inputs
    t = inputs.peps_tensors(4, 4, 2, 8)
    sk = inputs.sketch(4, 4, 2, 8)
    g = vmc.unpack(t, 4, 4, 2)
    configs = inputs.start_spins(8, 4, 4, 21, "random")
    return t, sk, g, configs


def _sums(g, sk, configs):
    from oracle import vmc
    acc = vmc.Accumulator(g)
    for s in configs:
        r = vmc.measure(g, s, 4, sk, 1, 1.0, 0.0)
        acc.add(s, r["eloc"], r["G"])
    return np.array([acc.sE, acc.sE2, float(acc.n)]), vmc.pack(acc.P1), vmc.pack(acc.P2)


def _update(g, t, scalars, P1, P2):
    from oracle import vmc
    acc = vmc.Accumulator(g)
    acc.sE, acc.sE2, acc.n = scalars[0], scalars[1], scalars[2]
    acc.P1, acc.P2 = vmc.unpack(P1, 4, 4, 2), vmc.unpack(P2, 4, 4, 2)
    grad, _ = acc.gradient()
    return vmc.pack(grad), vmc.sign_sgd(t, vmc.pack(grad), 0.05, 11, 3)


def _exchange_rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    from paper_1908_09359_gb300 import dist as xdist
    t, sk, g, configs = _oracle_case()
    mine = configs[rank::world]
    sc, p1, p2 = _sums(g, sk, mine)
    sc, p1, p2 = xdist.allreduce_host(sc, p1, p2)
    grad, new = _update(g, t, sc, p1, p2)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, sc, grad, new))


def test_gradient_sums_all_reduced_over_two_gloo_ranks():
    sys.path.insert(0, ROOT)
    res = _spawn(_exchange_rank, 2)
    (_, sc0, g0, n0), (_, sc1, g1, n1) = res
    assert np.array_equal(sc0, sc1) and np.array_equal(g0, g1) and np.array_equal(n0, n1)
    t, sk, g, configs = _oracle_case()
    sc, p1, p2 = _sums(g, sk, configs)
    grad, new = _update(g, t, sc, p1, p2)
    assert sc0[2] == 8.0
    assert np.allclose(sc0, sc, rtol=1e-14, atol=0)
    assert np.allclose(g0, grad, rtol=1e-12, atol=1e-14 * np.abs(grad).max())
    # sign-SGD moves each entry by r delta sgn(grad): identical wherever the sign is clear
    clear = np.abs(grad) > 1e-12 * np.abs(grad).max()
    assert np.array_equal(n0[clear], new[clear])
