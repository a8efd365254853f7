"""The N > 1 paths of bench.py on CPU, as two gloo ranks.

Weak scaling: each rank takes its own seeded sums (no data exchange); the job time is the
slowest rank's time (MAX all-reduce) and the whole-job rate counts every rank's sums.  The
oracle computes one sum per rank and the ranks gather them: sharded results equal
single-process results.

Split sum: one sum's Duffy lines are divided into contiguous parts; each rank holds its
part's values and every rank adds the gathered parts in rank order, so all ranks get the
same, deterministic total, equal to the single-process sum of the parts."""
import os
import socket

import numpy as np
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
        probs = bench.config2_problems(rank, 3)
        scales = [float(p.quad.lam) for p in probs]
        rate, ms = bench.job_rate(10.0 * (rank + 1), len(probs), 2, dist)
        # one small sum per rank through the oracle, gathered on every rank
        s = scales[0]
        prob = W.nbody_problem("square", 3.0, 3, W.Quad(n_u=8, n_v=8, lam=s, r_real=6 * s, r_recip=6 / s), scale=s)
        val = torch.tensor([float(oracle.nbody(prob, threads=1)[0])], dtype=torch.float64)
        got = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(got, val)
        # split sum: this rank's part of a d = 3 ATM sum = the sum of its contiguous share of
        # the far lines (the near lines belong to part 0), from the oracle's per-line values
        pa = W.atm_problem("fcc", W.Quad(n_u=2, n_v=3, u_rule=2, lam=1.0, r_real=4.0, r_recip=4.0))
        _, far, near = oracle.nbody(pa, threads=1, lines=True)
        flat = far.reshape(-1, far.shape[-1])
        lo, hi = rank * len(flat) // world, (rank + 1) * len(flat) // world
        part = flat[lo:hi].sum(axis=0) + (near.sum(axis=0) if rank == 0 else 0.0)
        total = bench.add_parts_in_rank_order(part[None, :], dist)[0]
        q.put((rank, scales, rate, ms, [float(g.item()) for g in got], total.tolist(), part.tolist()))
    finally:
        dist.destroy_process_group()


@pytest.fixture(scope="module")
def two_ranks(oracle_mod):
    import torch.multiprocessing as mp

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
    return out


def test_two_gloo_ranks_shard_sums_and_time_by_slowest_rank(two_ranks, oracle_mod):
    import bench
    from paper_2504_11989_gb300 import workloads as W

    (r0, sc0, rate0, ms0, g0, *_), (r1, sc1, rate1, ms1, g1, *_) = two_ranks
    # disjoint seeded sums per rank, each rank's own list reproducible in one process
    assert sc0 == [p.quad.lam for p in bench.config2_problems(0, 3)]
    assert sc1 == [p.quad.lam for p in bench.config2_problems(1, 3)]
    assert not set(sc0) & set(sc1)
    # the job is timed by its slowest rank, and counts both ranks' sums
    assert ms0 == ms1 == 20.0
    assert rate0 == rate1 == pytest.approx(2 * 6 * 2 / 0.020)
    # the gathered per-rank results equal the single-process oracle values
    assert g0 == g1
    for rank, sc in ((0, sc0), (1, sc1)):
        s = sc[0]
        prob = W.nbody_problem("square", 3.0, 3, W.Quad(n_u=8, n_v=8, lam=s, r_real=6 * s, r_recip=6 / s), scale=s)
        assert g0[rank] == float(oracle_mod.nbody(prob, threads=1)[0])


def test_split_sum_parts_add_up_in_rank_order(two_ranks, oracle_mod):
    from paper_2504_11989_gb300 import workloads as W

    (_, _, _, _, _, tot0, part0), (_, _, _, _, _, tot1, part1) = two_ranks
    assert tot0 == tot1  # every rank holds the same total
    assert tot0 == (np.asarray(part0) + np.asarray(part1)).tolist()  # rank order, bit for bit
    pa = W.atm_problem("fcc", W.Quad(n_u=2, n_v=3, u_rule=2, lam=1.0, r_real=4.0, r_recip=4.0))
    whole = oracle_mod.nbody(pa, threads=1)
    assert np.allclose(tot0, whole[: len(tot0)], rtol=1e-14, atol=0)


def test_single_process_rate_has_no_exchange():
    import bench

    rate, ms = bench.job_rate(50.0, 10, 5)
    assert ms == 50.0 and rate == pytest.approx(10 * 5 / 0.05)
    assert bench.add_parts_in_rank_order(np.ones((2, 3))).tolist() == np.ones((2, 3)).tolist()
