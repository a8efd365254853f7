"""Scheduler of the serving loop (ez_server_*) without a GPU: EZ_SERVER_DRYRUN plans
and admits requests exactly as the real server does and accounts the device memory a
tick would hold, but launches nothing (values are NaN)."""
import math
from collections import Counter

import numpy as np
import pytest

from paper_2504_11989_gb300 import workloads as W


@pytest.fixture(scope="module")
def ez():
    from paper_2504_11989_gb300 import build, ezeta

    build.build()
    return ezeta


def _req(ez, p, prec=1, tag=0):
    return ez.make_request(p.A, p.nu, p.expo, ez.quadrature(p.quad, prec=prec), tag)


def test_dryrun_admits_every_request_in_fifo_ticks(ez):
    reqs = W.serving_mix(400, 11, 1000.0)
    srv = ez.Server(96 << 20, n_streams=3, max_batch=12, dryrun=True)
    tickets = [srv.submit(_req(ez, W.request_problem(r), tag=r.rid)) for r in reqs]
    res = [srv.wait(t, 10000) for t in tickets]
    st = srv.stats()
    assert st.submitted == st.completed == 400 and st.failed == 0
    assert 1 <= st.max_batch_seen <= 12
    assert st.ticks >= math.ceil(400 / 12)
    assert 0 < st.peak_device_bytes <= 96 << 20
    assert all(r.status == 0 and math.isnan(r.value[0]) for r in res)
    assert [r.tag for r in res] == [r.rid for r in reqs]
    # FIFO: tickets start in submission order
    starts = [r.t_start for r in res]
    assert all(b >= a for a, b in zip(starts, starts[1:]))
    assert all(r.t_submit <= r.t_start <= r.t_done for r in res)
    srv.close()


def test_memory_budget_bounds_what_runs_at_once(ez):
    p = W.nbody_problem("fcc", 6.0, 3, W.serve_quad(3, 64, False))
    one = ez.Server(1 << 40, n_streams=1, max_batch=1, dryrun=True)
    t = one.submit(_req(ez, p))
    one.wait(t)
    per_req = one.stats().peak_device_bytes
    one.close()
    budget = int(2.5 * per_req)
    srv = ez.Server(budget, n_streams=4, max_batch=64, dryrun=True)
    tickets = [srv.submit(_req(ez, p)) for _ in range(20)]
    for t in tickets:
        srv.wait(t, 10000)
    st = srv.stats()
    assert st.peak_device_bytes <= budget
    assert st.max_batch_seen <= 2
    srv.close()


def test_per_request_errors_come_back_as_results(ez):
    srv = ez.Server(64 << 20, n_streams=2, max_batch=8, dryrun=True)
    good = W.nbody_problem("square", 3.0, 3, W.config2(16))
    bad_nu = W.Problem("bad", W.lattice("square"), [float("nan")], [[3]], W.config2(16))
    pole = W.Problem("pole", W.lattice("square"), [-2.0], [[3]], W.config2(16))
    huge = W.nbody_problem("hexagonal", 3.0, 3, W.config2(256))
    small = ez.Server(1 << 16, n_streams=1, max_batch=1, dryrun=True)  # 64 KiB: too small for a 256^2 sum
    t_huge = small.submit(_req(ez, huge))
    assert small.wait(t_huge).status == ez.EZ_ENOMEM
    small.close()
    ts = [srv.submit(_req(ez, q)) for q in (good, bad_nu, pole, good)]
    codes = [srv.wait(t).status for t in ts]
    assert codes == [0, ez.EZ_EINVAL, ez.EZ_EDOMAIN, 0]
    st = srv.stats()
    assert st.failed == 2 and st.completed == 4
    with pytest.raises(ez.EzError) as e:  # unknown ticket
        srv.wait(10 ** 9, 10)
    assert e.value.code == ez.EZ_EINVAL
    with pytest.raises(ez.EzError) as e:  # already collected
        srv.wait(ts[0], 10)
    assert e.value.code == ez.EZ_EINVAL
    srv.close()


def test_poll_and_queue_limits(ez):
    with pytest.raises(ez.EzError) as e:
        ez.Server(0, n_streams=1, max_batch=1, dryrun=True)
    assert e.value.code == ez.EZ_EINVAL
    srv = ez.Server(64 << 20, n_streams=1, max_batch=4, dryrun=True)
    p = W.nbody_problem("Z", 4.0, 3, W.config1(64))
    tickets = {srv.submit(_req(ez, p, tag=i)) for i in range(50)}
    got = []
    for _ in range(2000):
        got += srv.poll(16)
        if len(got) == 50:
            break
        import time

        time.sleep(0.001)
    assert {r.ticket for r in got} == tickets
    assert Counter(r.status for r in got) == Counter({0: 50})
    srv.close()


def test_error_estimate_flag_is_planned_with_its_coarse_rule(ez):
    # EZ_REQ_ERR_EST adds the embedded coarse-rule sum to the request's tick: the tick holds
    # more device memory; unknown flags are refused at submission
    A = W.lattice("square")
    q = ez.quadrature(W.Quad(n_u=16, n_v=16, u_rule=1, lam=1.0, r_real=6.0, r_recip=6.0))
    peaks = []
    for flag in (False, True):
        srv = ez.Server(1 << 30, n_streams=1, max_batch=1, dryrun=True)
        t = srv.submit(ez.make_request(A, [3.0], [[3]], q, err_est=flag))
        r = srv.wait(t, 10000)
        assert r.status == 0
        peaks.append(srv.stats().peak_device_bytes)
        srv.close()
    assert peaks[1] > peaks[0]
    bad = ez.make_request(A, [3.0], [[3]], q)
    bad.flags = 6
    srv = ez.Server(1 << 30, n_streams=1, max_batch=1, dryrun=True)
    with pytest.raises(ez.EzError) as e:
        srv.submit(bad)
    assert e.value.code == ez.EZ_EINVAL
    srv.close()
