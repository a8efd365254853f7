"""One lattice sum split over two processes, as bench.py --split-sum does on N GPUs.

Both processes run on the one GPU here (their kernels never wait on each other: each
computes its own part, then the hosts exchange a few doubles over gloo).  Rank r computes
part r of n_parts = 2 (a contiguous range of Duffy line groups; the near part in part 0)
of a config-3-shaped ATM sum; the parts are added in rank order on every rank.  The total
equals the whole sum computed in one process to 1e-14 relative, and each part's lines equal
the whole sum's lines bitwise on its range."""
import os
import socket

import numpy as np
import pytest

from paper_2504_11989_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    return W.atm_problem("bcc", W.Quad(n_u=4, n_v=24, u_rule=2, lam=0.0, r_real=0.0, r_recip=0.0))


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist

    import bench
    from paper_2504_11989_gb300 import ezeta as ez

    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = _problem()
        L = ez.Lattice(p.A)
        spec = ez.sum_spec(p.nu, p.expo)
        q_part = ez.quadrature(p.quad, part=rank, n_parts=world)
        vals, lines, offs = ez.ez_lattice_sums([L], [spec], [q_part], lines=True)
        npr = len(p.expo)
        total = bench.add_parts_in_rank_order(vals[:, :npr], dist)[0]
        q.put((rank, total.tolist(), lines[offs[0]: offs[1], :npr].tolist()))
    finally:
        dist.destroy_process_group()


def test_split_sum_over_two_processes_equals_the_whole():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import torch.multiprocessing as mp

    from paper_2504_11989_gb300 import build, ezeta as ez

    build.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    out = sorted(q.get(timeout=600) for _ in procs)
    for pr in procs:
        pr.join(timeout=120)
        assert pr.exitcode == 0
    (_, tot0, l0), (_, tot1, l1) = out
    assert tot0 == tot1
    p = _problem()
    npr = len(p.expo)
    whole, wl, offs = ez.ez_lattice_sums([ez.Lattice(p.A)], [ez.sum_spec(p.nu, p.expo)], [ez.quadrature(p.quad)],
                                         lines=True)
    wl = wl[offs[0]: offs[1], :npr]
    assert np.all(np.abs(np.asarray(tot0) - whole[0, :npr]) <= 1e-14 * np.abs(whole[0, :npr]))
    covered = np.zeros(len(wl), dtype=int)
    for lk in (np.asarray(l0), np.asarray(l1)):
        nz = np.any(lk != 0.0, axis=1)
        assert np.array_equal(lk[nz], wl[nz])
        covered += nz
    assert np.all(covered[np.any(wl != 0.0, axis=1)] == 1)
