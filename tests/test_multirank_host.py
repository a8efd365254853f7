"""The N > 1 path of bench.py on CPU: two gloo ranks.  Each rank takes its own seeded
sums (weak scaling, no data exchange); the job time is the slowest rank's time (MAX
all-reduce) and the whole-job rate counts every rank's sums.  The oracle computes one
sum per rank and rank 0 gathers them: sharded results equal single-process results."""
import os
import socket

import pytest


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist

    import bench
    import oracle
    from paper_2504_11989_gb300 import workloads as W

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        items = bench.workload(rank, 3)
        rate, ms = bench.job_rate(10.0 * (rank + 1), len(items), 2, dist)
        # one small sum per rank through the oracle, gathered on every rank
        name, s = items[0]
        prob = W.nbody_problem(name, 3.0, 3, W.Quad(n_u=8, n_v=8, lam=s, r_real=6 * s, r_recip=6 / s), scale=s)
        val = torch.tensor([float(oracle.nbody(prob, threads=1)[0])], dtype=torch.float64)
        got = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(got, val)
        q.put((rank, items, rate, ms, [float(g.item()) for g in got]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_sums_and_time_by_slowest_rank(oracle_mod):
    import torch.multiprocessing as mp

    import bench
    from paper_2504_11989_gb300 import workloads as W

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, items0, rate0, ms0, g0), (r1, items1, rate1, ms1, g1) = out
    # disjoint seeded sums per rank, each rank's own list reproducible in one process
    assert items0 == bench.workload(0, 3) and items1 == bench.workload(1, 3)
    assert not set(items0) & set(items1)
    # the job is timed by its slowest rank, and counts both ranks' sums
    assert ms0 == ms1 == 20.0
    assert rate0 == rate1 == pytest.approx(2 * 6 * 2 / 0.020)
    # the gathered per-rank results equal the single-process oracle values
    assert g0 == g1
    for rank, items in ((0, items0), (1, items1)):
        name, s = items[0]
        prob = W.nbody_problem(name, 3.0, 3, W.Quad(n_u=8, n_v=8, lam=s, r_real=6 * s, r_recip=6 / s), scale=s)
        assert g0[rank] == float(oracle_mod.nbody(prob, threads=1)[0])


def test_single_process_rate_has_no_exchange():
    import bench

    rate, ms = bench.job_rate(50.0, 10, 5)
    assert ms == 50.0 and rate == pytest.approx(10 * 5 / 0.05)
