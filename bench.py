#!/usr/bin/env python
"""Throughput of the Epstein zeta method on GB300: lattice sums/s (and Epstein zeta
evaluations/s) of the three-body zeta function zeta^(3)(3,3,3) on the square and
hexagonal lattices (unit density times a seeded lattice constant in [0.9, 1.3]),
256 x 256 Brillouin-zone grid mapped to 4 Duffy sectors x 128 u x 128 v nodes,
cutoff radius 6 in real and reciprocal space, FP64.

One step = one pass of the whole path (table setup, per-node Epstein zeta, product,
quadrature reduction) over a batch of 128 sums (64 per lattice).  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Epstein zeta evals/sec and lattice sums/sec at stated rel. error; p50/p99 latency"
PER_LATTICE = 64
LATTICES = ("square", "hexagonal")
GRID = 256
R_CUT = 6.0
NU = 3.0
N_BODY = 3
# DRAM bytes (read + write) of one far_kernel_d2 launch of the default 128-sum step, from the
# full-size ncu capture summarised in profiles/far_kernel_d2_config2.md.  Set to None whenever
# that kernel changes until re-captured (other batch sizes report null: the shared phase
# table makes the traffic not proportional to the number of sums).
FAR_DRAM_BYTES_PER_LAUNCH = 8673536


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--per-lattice", type=int, default=PER_LATTICE, help="sums per lattice per step (profiling)")
    ap.add_argument("--workload", default="config2",
                    choices=["config2", "serve", "config1", "config3", "config4", "epstein"])
    ap.add_argument("--requests", type=int, default=10000, help="serve: number of requests")
    return ap.parse_args()


def workload(rank: int, per_lattice: int = PER_LATTICE):
    """[(lattice name, lattice constant)] of the sums of one step."""
    from paper_2504_11989_gb300 import workloads as W

    items = []
    for li, name in enumerate(LATTICES):
        for s in W.lattice_constants(per_lattice, W.SEED_BASE + 1 + 100 * rank + li):
            items.append((name, float(s)))
    return items


def job_rate(local_ms: float, sums_per_rank: int, steps: int, dist=None, device: str = "cpu"):
    """Whole-job lattice sums/s: every rank ran sums_per_rank * steps sums (weak scaling, no
    data exchange between ranks); the job took as long as its slowest rank.  Returns the
    rate and that time (ms)."""
    import torch

    ms = float(local_ms)
    world = 1
    if dist is not None:
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        world = dist.get_world_size()
    return world * sums_per_rank * steps / (ms / 1e3), ms


def quad_for(scale: float):
    from paper_2504_11989_gb300 import workloads as W

    # lattice constant s scales lambda = V^{1/d} = s and the cutoffs (6 spacings)
    return W.Quad(n_u=GRID // 2, n_v=GRID // 2, u_rule=1, lam=scale, r_real=R_CUT * scale, r_recip=R_CUT / scale)


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "100"], stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        os.unlink(self.path)
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].strip().replace(".", "").isdigit()]
        if not sm:
            return None
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": float(rows[0][2]), "samples": len(sm),
                "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------- CPU oracle
def oracle_sums(items, seconds: float, threads: int):
    """Oracle on the first sums of the workload until `seconds` have elapsed."""
    import oracle
    from paper_2504_11989_gb300 import workloads as W

    oracle.build()
    vals, t0 = [], time.perf_counter()
    for name, s in items:
        prob = W.nbody_problem(name, NU, N_BODY, quad_for(s), scale=s)
        vals.append(float(oracle.nbody(prob, threads=threads)[0]))
        if time.perf_counter() - t0 >= seconds:
            break
    return vals, time.perf_counter() - t0


def run_reference(args, rank, world):
    if rank != 0:
        return
    threads = os.cpu_count() or 1
    items = workload(0)
    per_step = max(1, int(args.cpu_seconds / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_sums(items[:1], 0.0, threads)
    times, n_done = [], 0
    for k in range(args.steps):
        sub = items[(k * per_step) % len(items):][:per_step]
        vals, dt = oracle_sums(sub, 1e9, threads)
        times.append(dt)
        n_done += len(vals)
    total = sum(times)
    value = n_done / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "lattice_sums/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic lattices (seeded lattice constants)",
            "config": config_dict(),
            "cpu_baseline": {"value": value, "unit": "lattice_sums/s", "cores": threads, "kind": "oracle",
                             "sample": f"{per_step} full sum(s) per step of the same workload"},
            "e2e": {"value": value, "unit": "lattice_sums/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def config_dict(per_lattice: int = PER_LATTICE):
    return {"workload": "zeta^(3)(3,3,3) on square+hexagonal lattices, 256^2 BZ grid (4x128x128 Duffy nodes), "
                        f"cutoff radius 6, {per_lattice} lattice constants per lattice per step",
            "global_batch": len(LATTICES) * per_lattice, "nodes_per_sum": 4 * (GRID // 2) ** 2,
            "parallelism": "independent sums per GPU", "l2": "flushed (256 MiB write) between timed steps"}


# ----------------------------------------------------------------------------- serving
def run_serve(args):
    """Served stability scan: `--requests` lattice sums with random d, lattice, lattice
    constant, exponent (or the ATM form), n and BZ resolution, mixed precision.  The same
    requests run saturated in the plain FP64 form first (reference rate and values), then
    saturated in the mixed form (sums/s, error against FP64), then on Poisson arrivals at
    0.8x the mixed saturated rate (latency percentiles)."""
    import threading

    import numpy as np
    import torch

    from paper_2504_11989_gb300 import build, ezeta
    from paper_2504_11989_gb300 import workloads as W

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    build.build()
    reqs = W.serving_mix(args.requests, W.SEED_BASE + 5, 1.0)
    made, made64 = [], []
    for r in reqs:
        p = W.request_problem(r)
        made.append(ezeta.make_request(p.A, p.nu, p.expo, ezeta.quadrature(p.quad, prec=ezeta.EZ_MIXED), r.rid))
        made64.append(ezeta.make_request(p.A, p.nu, p.expo, ezeta.quadrature(p.quad, prec=ezeta.EZ_FP64), r.rid))
    budget = 16 << 30

    def run(arrivals, made=made):
        srv = ezeta.Server(budget, n_streams=4, max_batch=256)
        warm = [srv.submit(made[i]) for i in range(16)]
        for t in warm:
            srv.wait(t, 600000)
        tickets = [None] * len(made)
        t0 = time.perf_counter()

        def submitter():
            for i, req in enumerate(made):
                if arrivals is not None:
                    dt = arrivals[i] - (time.perf_counter() - t0)
                    if dt > 0:
                        time.sleep(dt)
                tickets[i] = srv.submit(req)

        th = threading.Thread(target=submitter)
        th.start()
        th.join()
        res = [srv.wait(t, 600000) for t in tickets]
        wall = time.perf_counter() - t0
        st = srv.stats()
        srv.close()
        return res, wall, st

    res64, wall64, _ = run(None, made64)  # the plain FP64 form, saturated, same requests
    res_sat, wall_sat, st_sat = run(None)
    sat_rate = len(made) / wall_sat
    rel = []
    for a, b in zip(res_sat, res64):
        va, vb = np.asarray(a.value, dtype=float), np.asarray(b.value, dtype=float)
        ok = np.isfinite(vb) & (vb != 0)
        rel.append(float(np.max(np.abs(va[ok] - vb[ok]) / np.abs(vb[ok]))) if ok.any() else 0.0)
    rate = 0.8 * sat_rate
    arrivals = np.cumsum(np.random.default_rng(W.SEED_BASE + 6).exponential(1.0 / rate, size=len(made)))
    res, wall, st = run(arrivals)
    lat = np.array([r.t_done - r.t_submit for r in res]) * 1e3
    failed = sum(1 for r in res + res_sat if r.status != 0)
    line = {"metric": METRIC, "workload": "served stability scan (config 5)", "value": len(made) / wall,
            "unit": "lattice_sums/s", "saturated_value": sat_rate, "offered_rate": rate,
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "max": float(lat.max())},
            "fp64_saturated_value": len(made64) / wall64, "speedup_vs_fp64_saturated": wall64 / wall_sat,
            "max_rel_err_vs_fp64": max(rel), "median_rel_err_vs_fp64": float(np.median(rel)),
            "n_requests": len(made), "failed": failed, "dtype": "f32 tails + float-float heads", "n_gpus": 1,
            "higher_is_better": True, "data": "synthetic request stream (seeded)",
            "server": {"streams": 4, "max_batch": 256, "budget_bytes": budget, "ticks": st.ticks,
                       "max_batch_seen": st.max_batch_seen, "gpu_busy_fraction": st.busy_seconds / wall,
                       "peak_device_bytes": st.peak_device_bytes, "saturated_ticks": st_sat.ticks}}
    print(json.dumps(line))


# ----------------------------------------------------------------------------- other configs
def _time_batch(ezeta, torch, lats, specs, quads, steps, warmup, stream, flush):
    batch = ezeta.Batch(lats, specs, quads, stream=stream)
    out = torch.zeros(len(lats) * ezeta.EZ_MAX_PROD, dtype=torch.float64, device="cuda")
    for _ in range(max(3, warmup)):
        batch.run(out, stream)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    batch.timing(True)
    far = []
    with torch.cuda.stream(stream):
        for k in range(steps):
            flush.fill_(k & 0xFF)
            ev[k][0].record(stream)
            batch.run(out, stream)
            ev[k][1].record(stream)
            far.append(batch.timing(True)[0])
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in ev]
    vals = out.view(len(lats), ezeta.EZ_MAX_PROD).cpu().numpy().copy()
    flops = batch.far_flops()[0]
    lines, offs = batch.lines()
    return vals, sum(ms) / steps, sum(far) / steps, flops, lines, offs


def run_config(args):
    """Configs 1, 3, 4 of the workload list, FP64 and mixed form, one JSON line each."""
    import numpy as np
    import torch

    import oracle
    from paper_2504_11989_gb300 import build, ezeta
    from paper_2504_11989_gb300 import workloads as W

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    build.build()
    oracle.build()
    stream = torch.cuda.Stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    auto = dict(lam=0.0, r_real=0.0, r_recip=0.0)
    if args.workload == "config1":
        probs = []
        for s in W.lattice_constants(1024, W.SEED_BASE + 11):
            probs.append(W.nbody_problem("Z", 4.0, 3, W.Quad(n_u=4096, n_v=1, u_rule=1, lam=s, r_real=8 * s,
                                                            r_recip=8 / s), scale=s))
        label = "zeta^(3)_Z(4,4,4), 4096 GL nodes on [0,1/2], 8 shells, 1024 lattice constants per step"
    elif args.workload == "config3":
        probs = [W.atm_problem(n, W.Quad(n_u=8, n_v=64, u_rule=2, **auto)) for n in ("sc", "fcc", "bcc")]
        label = "ATM energy on sc, fcc, bcc (unit density), 12 sectors x 48 u x 64^2 v nodes + eps-split near part"
    else:
        probs = [W.nbody_problem("fcc", 6.0, n, W.Quad(n_u=32, n_v=48, u_rule=1, **auto)) for n in (3, 4, 5, 6, 8)]
        label = "zeta^(n)(6,..,6) on fcc, n = 3,4,5,6,8, 12 sectors x 32 u x 48^2 v nodes"
    lats = [ezeta.Lattice(p.A) for p in probs]
    specs = [ezeta.sum_spec(p.nu, p.expo) for p in probs]
    res = {}
    for prec, tag in ((ezeta.EZ_FP64, "f64"), (ezeta.EZ_MIXED, "mixed")):
        quads = [ezeta.quadrature(p.quad, prec=prec) for p in probs]
        res[tag] = _time_batch(ezeta, torch, lats, specs, quads, args.steps, args.warmup, stream, flush)
    per_factor = None
    if args.workload == "config4":
        quads = [ezeta.quadrature(p.quad, dedupe=0) for p in probs]
        specs_pf = [ezeta.sum_spec([6.0] * p.expo[0][0], [[1] * p.expo[0][0]]) for p in probs]
        per_factor = []
        for i in range(len(probs)):
            _, ms1, _, _, _, _ = _time_batch(ezeta, torch, [lats[i]], [specs_pf[i]], [quads[i]], 3, 3, stream, flush)
            per_factor.append({"n": probs[i].expo[0][0], "ms": ms1})
    # sampled oracle lines (full-size sums): first product, a few far lines of each sum
    rng = np.random.default_rng(4)
    worst = {"f64": 0.0, "mixed": 0.0}
    t0 = time.perf_counter()
    for i, p in enumerate(W.explicit_splitting(p) for p in probs[:3]):
        ns, nu_t = oracle.n_sectors(p), oracle.n_u_total(p)
        for _ in range(2 if args.workload != "config1" else 8):
            sct, iu = int(rng.integers(ns)), int(rng.integers(nu_t))
            ref = oracle.nbody_line(p, sct, iu)
            for tag in worst:
                _, _, _, _, lines, offs = res[tag]
                row = lines[offs[i] + sct * nu_t + iu, : len(ref)]
                scale = np.max(np.abs(lines[offs[i]: offs[i + 1], : len(ref)]), axis=0)
                worst[tag] = max(worst[tag], float(np.max(np.abs(row - ref) / np.maximum(np.abs(ref), scale))))
    cpu_s = time.perf_counter() - t0
    for tag in ("f64", "mixed"):
        vals, ms, far_ms, flops, _, _ = res[tag]
        line = {"metric": METRIC, "workload": args.workload, "config": label, "dtype": tag, "sums_per_step": len(probs),
                "value": len(probs) / (ms / 1e3), "unit": "lattice_sums/s", "ms_per_step": ms,
                "far_ms_per_step": far_ms, "far_tflops_algorithmic": flops / (far_ms * 1e-3) / 1e12,
                "max_line_rel_err_vs_oracle": worst[tag], "oracle_lines_seconds": cpu_s,
                "values": [list(map(float, v[: len(p.expo)])) for v, p in zip(vals, probs)][:6]}
        if args.workload == "config3":
            line["atm_energy"] = [float(v[0] / 24 - 3 * v[1] / 16 + 3 * v[2] / 8) for v in vals]
        if tag == "mixed":
            line["speedup_vs_f64"] = res["f64"][1] / ms
        if per_factor is not None and tag == "f64":
            line["per_factor_ms_vs_n"] = per_factor
        print(json.dumps(line))


# ----------------------------------------------------------------------------- Epstein zeta
def run_epstein(args):
    """ez_epstein_zeta alone: 2^20 points y uniform in the Brillouin zone per call (device
    buffers), x = 0 and x uniform in the unit cell, d = 1, 2, 3; evaluations/s, and the
    largest error of 256 sampled points against the oracle relative to max(1, |Z|)."""
    import numpy as np
    import torch

    import oracle
    from paper_2504_11989_gb300 import build, ezeta
    from paper_2504_11989_gb300 import workloads as W

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    build.build()
    oracle.build()
    m = 1 << 20
    stream = torch.cuda.Stream()
    rng = np.random.default_rng(W.SEED_BASE + 21)
    cases = [("Z", 4.0), ("hexagonal", 3.0), ("fcc", 6.0), ("sc", 4.0)]
    for lat_name, nu in cases:
        A = W.lattice(lat_name)
        d = A.shape[0]
        L = ezeta.Lattice(A)
        Ait = np.linalg.inv(A).T
        for xkind in ("x=0", "x in cell"):
            kt = rng.uniform(-0.5, 0.5, size=(m, d))
            y = kt @ Ait.T  # y = A^{-T} k~
            x = np.zeros(d) if xkind == "x=0" else A @ rng.uniform(0.0, 1.0, size=d)
            yd = torch.tensor(y, dtype=torch.float64, device="cuda")
            re = torch.empty(m, dtype=torch.float64, device="cuda")
            im = torch.empty(m, dtype=torch.float64, device="cuda")
            with torch.cuda.stream(stream):
                for _ in range(max(3, args.warmup)):
                    ezeta.ez_epstein_zeta(L, nu, x, yd, re, im, stream=stream)
            torch.cuda.synchronize()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
            with torch.cuda.stream(stream):
                for k in range(args.steps):
                    ev[k][0].record(stream)
                    ezeta.ez_epstein_zeta(L, nu, x, yd, re, im, stream=stream)
                    ev[k][1].record(stream)
            torch.cuda.synchronize()
            ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
            idx = rng.choice(m, size=256, replace=False)
            got = re.cpu().numpy()[idx] + 1j * im.cpu().numpy()[idx]
            lam = abs(np.linalg.det(A)) ** (1.0 / d)
            ref = np.array([oracle.epstein_zeta(A, nu, x, y[i], lam, 9.0 * lam, 9.0 / lam) for i in idx])
            # relative to max(1, |Z|), as the parity tests (Z crosses zero inside the zone)
            err = float(np.max(np.abs(got - ref) / np.maximum(np.abs(ref), 1.0)))
            print(json.dumps({"metric": METRIC, "workload": "epstein", "lattice": lat_name, "d": d, "nu": nu,
                              "x": xkind, "points_per_call": m, "value": m / (ms * 1e-3) / 1e6, "unit": "M evals/s",
                              "ms_per_call": ms, "dtype": "f64", "max_err_vs_oracle_256_rel_to_max_1_absZ": err}))


# ----------------------------------------------------------------------------- main
def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "serve":
        if rank == 0:
            run_serve(args)
        return
    if args.workload in ("config1", "config3", "config4"):
        if rank == 0:
            run_config(args)
        return
    if args.workload == "epstein":
        if rank == 0:
            run_epstein(args)
        return
    import numpy as np
    import torch

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2504_11989_gb300 import build, ezeta
    from paper_2504_11989_gb300 import workloads as W

    build.build()
    items = workload(rank, args.per_lattice)
    lats = [ezeta.Lattice(W.lattice(n, scale=s)) for n, s in items]
    spec = ezeta.sum_spec([NU], [[N_BODY]])
    quads = [ezeta.quadrature(quad_for(s)) for _, s in items]
    stream = torch.cuda.Stream()
    batch = ezeta.Batch(lats, [spec] * len(items), quads, stream=stream)
    out = torch.zeros(len(items) * ezeta.EZ_MAX_PROD, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(max(3, args.warmup)):
        batch.run(out, stream)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    batch.timing(True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches0 = ezeta.ez_launch_count()
    far_ms = []
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            ev[k][0].record(stream)
            batch.run(out, stream)
            ev[k][1].record(stream)
            f, _ = batch.timing(True)
            far_ms.append(f)
    torch.cuda.synchronize()
    launches = ezeta.ez_launch_count() - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    n_sums = len(items)
    value, total_ms = job_rate(sum(step_ms), n_sums, args.steps, dist, "cuda")
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    res = out.view(n_sums, ezeta.EZ_MAX_PROD)[:, 0].cpu().numpy()

    # mixed form (binary32 tails, binary64 heads), same workload and timing rules
    quads_m = [ezeta.quadrature(quad_for(s), prec=ezeta.EZ_MIXED) for _, s in items]
    batch_m = ezeta.Batch(lats, [spec] * len(items), quads_m, stream=stream)
    out_m = torch.zeros_like(out)
    for _ in range(max(3, args.warmup)):
        batch_m.run(out_m, stream)
    torch.cuda.synchronize()
    evm = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            evm[k][0].record(stream)
            batch_m.run(out_m, stream)
            evm[k][1].record(stream)
    torch.cuda.synchronize()
    mixed_value, mixed_ms = job_rate(sum(a.elapsed_time(b) for a, b in evm), n_sums, args.steps, dist, "cuda")
    res_m = out_m.view(n_sums, ezeta.EZ_MAX_PROD)[:, 0].cpu().numpy()

    # end to end through the C ABI with host buffers (planning, upload, kernels, download)
    host_out = np.zeros((n_sums, ezeta.EZ_MAX_PROD))
    e2e_steps = max(2, min(args.steps, 5))
    ezeta.ez_lattice_sums(lats, [spec] * n_sums, quads, out=host_out)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ezeta.ez_lattice_sums(lats, [spec] * n_sums, quads, out=host_out)
    e2e_value, _ = job_rate(1e3 * (time.perf_counter() - t0), n_sums, e2e_steps, dist, "cuda")
    assert np.array_equal(host_out[:, 0], res), "batch and one-shot paths disagree"
    _, staging = batch.sizes()

    # roofline of the far-field kernel (one launch per step): algorithmic FP64 flops counted
    # by the library for the last run (same work every step)
    flops, n_terms, n_coefs = batch.far_flops()
    nodes_total = n_sums * 4 * (GRID // 2) ** 2
    far_mean_ms = float(np.mean(far_ms))
    achieved = flops / (far_mean_ms * 1e-3) / 1e12
    peak_nominal = 152 * 2 * 2 * 2.07e9 / 1e12  # SMs x DFMA/clk x flops x max clock
    probe = ezeta.ez_diag_fp64_peak(stream)
    line = {
        "metric": METRIC, "value": value, "unit": "lattice_sums/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic lattices (seeded lattice constants)",
        "config": config_dict(args.per_lattice),
        "zeta_evals_per_s": {"per_factor": value * nodes_total / n_sums * N_BODY, "distinct_nu": value * nodes_total / n_sums},
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99)),
                       "unit": f"per step of {n_sums} sums"},
        "e2e": {"value": e2e_value, "unit": "lattice_sums/s", "h2d_bytes_per_step": int(staging),
                "d2h_bytes_per_step": int(n_sums * ezeta.EZ_MAX_PROD * 8)},
        "gpu_launches": int(launches),
        "roofline": {"bound": "alu", "kernel": "far_kernel_d2", "achieved": achieved, "peak": peak_nominal,
                     "unit": "TFLOP/s", "frac": achieved / peak_nominal,
                     "traffic": FAR_DRAM_BYTES_PER_LAUNCH if args.per_lattice == PER_LATTICE else None,
                     "peak_source": "FP64 pipe: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (nominal); "
                                    f"DFMA probe measured {probe:.3f} TFLOP/s in this run",
                     "far_ms_per_launch": far_mean_ms, "flops_per_launch": flops,
                     "recip_terms_per_launch": n_terms, "mean_poly_len": n_coefs / max(1, n_terms)},
        "clocks": clocks,
        "mixed_precision": {"value": mixed_value, "unit": "lattice_sums/s", "speedup_vs_fp64": mixed_value / value,
                            "dtype": "f32 tails + float-float heads", "ms_per_step": mixed_ms / args.steps,
                            "max_rel_err_vs_fp64": float(np.max(np.abs(res_m - res) / np.abs(res)))},
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        vals, dt = oracle_sums(items, args.cpu_seconds, threads)
        rel = [abs(res[i] - v) / abs(v) for i, v in enumerate(vals)]
        line["cpu_baseline"] = {"value": len(vals) / dt, "unit": "lattice_sums/s", "cores": threads, "kind": "oracle",
                                "sample": f"first {len(vals)} sums of the step's batch, full size"}
        line["rel_err_vs_oracle"] = float(max(rel))
        line["mixed_precision"]["max_rel_err_vs_oracle"] = float(max(abs(res_m[i] - v) / abs(v) for i, v in enumerate(vals)))
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
