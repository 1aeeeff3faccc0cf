#!/usr/bin/env python3
"""Benchmark: batched FP64 tile-Cholesky factorizations on GB300.

Workload (default): symmetric banded SPD matrix, n = 200,000, half-bandwidth 200,
off-diagonals U(-1,1)*0.5/200, diagonal 1 + absolute row sum, semisparse route with
active-column tiles of n_b = 128, natural ordering; a batch of 64 value sets of the same
pattern (seeds 0..63) per GPU.  One step = value scatter + task-DAG factorization +
log-determinant + one solve per item (RHS ~ N(0,1)), i.e. every row of the hot path.
The plain (one factorization per launch, batch 1) rate is reported beside the batched
one.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Prints ONE JSON line (rank 0).  Under torchrun each rank factorizes its own batch
(independent value sets, no data-path collective): weak scaling.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2609_29765_gb300 import inputs as I  # noqa: E402

METRIC = "FP64 factorizations/s per pattern (batched vs plain) and % of FP64/HBM roofline"
UNIT = "factorizations/s"
N, BW, NB = 200_000, 200, 128
SMS, DFMA_PER_CLK, MAX_MHZ = 152, 2, 2070.0
# nominal FP64 ALU peak from unit counts and the maximum SM clock (TFLOP/s)
PEAK_FP64_NOMINAL = SMS * DFMA_PER_CLK * 2 * MAX_MHZ * 1e6 / 1e12


def _hbm_peak():
    """Measured copy bandwidth of the GB300s (MEASURED_PEAKS.json, written by the
    pool's driver), else the recipe's fallback figure."""
    try:
        v = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
        return v, "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, ValueError, KeyError, TypeError):
        return 6800.0, "fallback 6.8 TB/s"


HBM_GBS, HBM_SOURCE = _hbm_peak()


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--batch", type=int, default=64)
    p.add_argument("--n", type=int, default=N)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--row-slices", type=int, default=0,
                   help="row slices per off-diagonal tile (0: the library's choice)")
    p.add_argument("--workloads", default="c1,c3,c4,c5",
                   help="other workloads measured after the headline, comma list or 'none' "
                        "('forced': the selector's route against every forced route)")
    p.add_argument("--small-workloads", action="store_true",
                   help="the other workloads at reduced batch sizes (a quick check, not the configured sizes)")
    p.add_argument("--c3-grid", default="60,60,50",
                   help="grid nx,ny,nt of the spatio-temporal workloads (configs 3 and 5); a smaller one "
                        "is for profiling captures only")
    return p.parse_args()


def workload_config(args, batch):
    return {"workload": "banded SPD n=%d half-bandwidth %d, active-column tiles n_b=%d, batch %d value sets"
                        % (args.n, BW, NB, batch),
            "n": args.n, "half_bandwidth": BW, "nb": NB, "batch_per_gpu": batch,
            "route": "semisparse", "ordering": "natural",
            "step": "scatter+factorize(with the forward substitution in its launch)+logdet+backward "
                    "substitution (1 rhs)",
            "l2": "inputs larger than L2 (values %.1f GB, factor %.1f GB per step)"}


def replay_traffic(n, batch):
    """DRAM bytes per replay launch from the committed ncu capture (profiles/), scaled to
    this launch; None when the kernel source changed since the capture."""
    import hashlib
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "replay_kernel_traffic.json")))
        src = open(os.path.join(ROOT, "paper_2609_29765_gb300", "csrc", "replay.cu"), "rb").read()
    except OSError:
        return None
    if hashlib.sha256(src).hexdigest()[:16] != rec["source_sha256_prefix"]:
        return None
    cap = rec["captured"]
    per = (cap["dram_bytes_read"] + cap["dram_bytes_write"]) / (cap["n"] * cap["batch"])
    return per * n * batch


# ------------------------------------------------------------------ clocks
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        pw = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(pw) if pw else None}


# ------------------------------------------------------------------ oracle (CPU baseline)
def oracle_sample(n, items, seed0=0):
    """Time the CPU oracle (single thread) on `items` value sets of the workload."""
    from oracle import oracle as O
    Ap, Ai = I.band_pattern(n, BW)
    F = O.OracleFactor(n, Ap, Ai)
    times = []
    for s in range(items):
        Ax = I.band_values(n, BW, seed0 + s, Ap, Ai)
        b = I.rhs(n, 1000 + s)[0]
        t0 = time.perf_counter()
        Lx, info = F.factor(Ax)
        F.logdet(Lx)
        F.solve(Lx, b)
        times.append(time.perf_counter() - t0)
    return times


def _oracle_worker(n, seed, rounds, barrier, results):
    from oracle import oracle as O
    Ap, Ai = I.band_pattern(n, BW)
    F = O.OracleFactor(n, Ap, Ai)
    Ax = I.band_values(n, BW, seed, Ap, Ai)
    b = I.rhs(n, 1000 + seed)[0]
    for r in range(rounds):
        barrier.wait()
        t0 = time.time()
        Lx, info = F.factor(Ax)
        F.logdet(Lx)
        F.solve(Lx, b)
        results.put((r, t0, time.time()))


def oracle_parallel(n, procs, rounds=1):
    """The oracle on `procs` value sets at once, one single-threaded process per host core
    (spawned, so safe before or after CUDA use), `rounds` times; returns the wall time of
    each round (all processes start a round together)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    barrier, results = ctx.Barrier(procs), ctx.Queue()
    ps = [ctx.Process(target=_oracle_worker, args=(n, s, rounds, barrier, results)) for s in range(procs)]
    for p in ps:
        p.start()
    try:
        spans = [results.get(timeout=900) for _ in range(procs * rounds)]
    finally:
        for p in ps:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    walls = []
    for r in range(rounds):
        sp = [(a, b) for q, a, b in spans if q == r]
        walls.append(max(b for _, b in sp) - min(a for a, _ in sp))
    return walls


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    steps, warm = args.steps, args.warmup
    cores = host_cores()
    # each step: `cores` value sets factorized (+logdet+solve) at once, one oracle process per
    # host core -- a bounded sample of the 64-set batch
    walls = oracle_parallel(args.n, cores, warm + steps)[warm:]
    ms = 1e3 * sum(walls) / len(walls)
    value = cores * 1e3 / ms
    cfg = workload_config(args, args.batch)
    cfg["l2"] = "host run"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": steps, "warmup": warm, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d value sets per step (factor+logdet+solve), one single-threaded "
                                       "oracle process per host core" % cores},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ ranks
def rank_seeds(rank, batch):
    """Value-set seeds of one rank: ranks factorize disjoint, contiguous seed ranges."""
    return list(range(rank * batch, (rank + 1) * batch))


def max_over_ranks(values, dist, device):
    """Element-wise maximum of per-rank timings (ms) on every rank."""
    import torch
    t = torch.tensor(values, dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


# ------------------------------------------------------------------ other workloads
def _events_ms(fn, reps, warm):
    """Mean CUDA-event time (ms) of fn() on the current stream after `warm` untimed calls."""
    import torch
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def _fp64(flops, ms):
    t = flops / (ms * 1e-3) / 1e12
    return {"achieved_tflops": t, "frac": t / PEAK_FP64_NOMINAL}


def _distinct_values(gen, count, distinct):
    """[count, nnzA] host values cycling through `distinct` generated value sets."""
    sets = [gen(s) for s in range(distinct)]
    return np.stack([sets[i % distinct] for i in range(count)])


def measure_workloads(args):
    """Factorizations/s (plain per call vs batched) and adjoint gradients/s on the other
    workloads, each timed with CUDA events after a warm-up; not part of the headline step."""
    import torch
    from paper_2609_29765_gb300 import _lib as L
    from paper_2609_29765_gb300.api import Group, Plan

    want = [] if args.workloads == "none" else args.workloads.split(",")
    small = args.small_workloads
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    out = {}

    def plain_and_batched(P, vals, reps_b, reps_p, with_solve, warm_b=1):
        batch = vals.shape[0]
        fac = torch.empty(P.factor_bytes(batch) // 8, dtype=torch.float64, device="cuda")
        info = torch.empty(batch, dtype=torch.int32, device="cuda")
        ld = torch.empty(batch, dtype=torch.float64, device="cuda")
        ws = P.workspace(batch)
        b = torch.ones(batch, 1, P.n, dtype=torch.float64, device="cuda")
        x = torch.empty_like(b)

        def run(bt):
            L.check(L.stc_factorize(P.h, vals[:bt], bt, fac, ws, info), "factorize")
            L.check(L.stc_logdet(P.h, fac, bt, ld), "logdet")
            if with_solve:
                L.check(L.stc_solve(P.h, fac, bt, 1, b[:bt], x[:bt], ws), "solve")
        ms_p = _events_ms(lambda: run(1), reps_p, 1)
        # the batched launch is warmed up on a few items (same kernels, same plan upload)
        _events_ms(lambda: run(min(batch, 8)), warm_b, 0)
        ms_b = _events_ms(lambda: run(batch), reps_b, 0)
        L.check(L.stc_sync_status(ws), "device status")
        assert int(info.abs().sum()) == 0 and bool(torch.isfinite(ld[:batch]).all())
        ms_f = _events_ms(lambda: L.check(L.stc_factorize(P.h, vals, batch, fac, ws, info)), reps_b, 0)
        L.check(L.stc_sync_status(ws), "device status")
        del fac, b, x
        return ms_b, ms_f, ms_p

    if "c1" in want:
        Ap, Ai, _, coords = I.laplace2d_bordered(seed=0)
        n = len(Ap) - 1
        batch = 1024
        vals = dev(_distinct_values(lambda s: I.laplace2d_bordered(seed=s)[2], batch, 16))
        out["c1"] = {"workload": "n=1,026 32x32 Laplacian + 0.1 I + 2 border rows, ND, n_b=64; factor+logdet+solve",
                     "note": "latency-bound: roofline fraction not meaningful",
                     "values": "16 distinct value sets (seeds 0..15) cycled"}
        for route in ("semisparse", "supernodal"):
            P = Plan(n, Ap, Ai, coords=coords, nb=64, route=route)
            ms_b, ms_f, ms_p = plain_and_batched(P, vals, 5, 50, True)
            out["c1"][route] = {"route_selected": P.route_selected,
                                "plain": {"value": 1e3 / ms_p, "unit": UNIT, "us_per_call": 1e3 * ms_p},
                                "batched": {"value": batch * 1e3 / ms_b, "unit": UNIT, "batch": batch}}
        del vals
    gx, gy, gt = (int(v) for v in args.c3_grid.split(","))
    if "c3" in want:
        Ap, Ai, coords = I.stcov_pattern(gx, gy, gt)
        n = len(Ap) - 1
        batch = 16 if small else 256
        th = I.stcov_thetas(batch, 0)
        distinct = 4 if small else 16
        vals = dev(_distinct_values(lambda s: I.stcov_values(th[s], gx, gy, gt), batch, distinct))
        out["c3"] = {"workload": "tau AR1(rho) x SPDE 9-point %dx%d, %d steps, + 20 border rows, n=%d, "
                                 "ND; factor+logdet" % (gx, gy, gt, n), "values": "%d distinct theta draws cycled" % distinct}
        # the supernodal route (the selector's choice) holds all 256 theta sets in one launch
        P = Plan(n, Ap, Ai, coords=coords, nb=64, route="supernodal")
        ms_b, ms_f, ms_p = plain_and_batched(P, vals, 1, 2, False)
        fa, fx = P.info["flops_alg"], P.info["flops_tile"]
        out["c3"]["supernodal"] = {
            "route_selected": P.route_selected,
            "plain": {"value": 1e3 / ms_p, "unit": UNIT, "ms_per_call": ms_p},
            "batched": {"value": batch * 1e3 / ms_b, "unit": UNIT, "batch": batch,
                        "note": "one persistent launch of all %d theta sets (factors: %.0f GB)"
                                % (batch, P.factor_bytes(batch) / 1e9)},
            "roofline_replay": dict(_fp64(fa * batch, ms_f), bound="alu", peak=PEAK_FP64_NOMINAL,
                                    work="sum_j c_j^2 = %.4g flops per factorization (executed %.4g)" % (fa, fx),
                                    ms=ms_f),
            "analyze_seconds": P.info["analyze_seconds"]}
        del P
        torch.cuda.empty_cache()
        # the semisparse tile route on the same pattern (its factors take 1.8 GB per set)
        P = Plan(n, Ap, Ai, coords=coords, nb=64, route="semisparse")
        bt = 16
        ms_b, ms_f, ms_p = plain_and_batched(P, vals[:bt], 1, 2, False)
        out["c3"]["semisparse"] = {
            "plain": {"value": 1e3 / ms_p, "unit": UNIT, "ms_per_call": ms_p},
            "batched": {"value": bt * 1e3 / ms_b, "unit": UNIT, "batch": bt},
            "roofline_replay": dict(_fp64(fa * bt, ms_f), bound="alu", peak=PEAK_FP64_NOMINAL, ms=ms_f,
                                    work="sum_j c_j^2 = %.4g flops per factorization (executed %.4g)"
                                         % (fa, P.info["flops_tile"]))}
        del vals, P
        torch.cuda.empty_cache()
    if "c5" in want:
        Ap, Ai, coords = I.stcov_pattern(gx, gy, gt)
        batch = 8 if small else 64
        th = I.stcov_thetas(batch, 0)
        distinct = 4 if small else 16
        vals = dev(_distinct_values(lambda s: I.stcov_values(th[s], gx, gy, gt), batch, distinct))
        xs = dev(np.stack([I.rhs(len(Ap) - 1, s)[0] for s in range(batch)]))
        out["c5"] = {"workload": "d/dQ [logdet Q(theta) - x^T Q(theta) x] on the spatio-temporal pattern of config 3 "
                                 "(%dx%dx%d + 20 border rows)" % (gx, gy, gt),
                     "step": "factorize+logdet+selected inverse+gather+quad form+outer product",
                     "values": "%d distinct theta draws cycled" % distinct,
                     "gradient_w_r_t": "the nnzA values of Q; the 3-parameter theta chain is a host-side "
                                       "contraction outside the step"}
        for route in ("supernodal", "semisparse"):
            P = Plan(len(Ap) - 1, Ap, Ai, coords=coords, nb=64, route=route)
            fac = torch.empty(P.factor_bytes(batch) // 8, dtype=torch.float64, device="cuda")
            sig = torch.empty_like(fac)
            info = torch.empty(batch, dtype=torch.int32, device="cuda")
            ld = torch.empty(batch, dtype=torch.float64, device="cuda")
            q = torch.empty_like(ld)
            g = torch.empty(batch, P.nnzA, dtype=torch.float64, device="cuda")
            neg = torch.full((batch,), -1.0, dtype=torch.float64, device="cuda")
            ws = P.workspace(batch)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]

            def grad_step(bt, rec=False):
                if rec:
                    ev[0].record()
                L.check(L.stc_factorize(P.h, vals[:bt], bt, fac, ws, info), "factorize")
                L.check(L.stc_logdet(P.h, fac, bt, ld), "logdet")
                if rec:
                    ev[1].record()
                L.check(L.stc_logdet_backward(P.h, fac, bt, None, g[:bt], 0, sig, ws), "logdet_backward")
                if rec:
                    ev[2].record()
                L.check(L.stc_quad_form(P.h, bt, vals[:bt], xs[:bt], q), "quad_form")
                L.check(L.stc_sym_outer_backward(P.h, bt, xs[:bt], xs[:bt], neg, g[:bt], 1), "outer_backward")
                if rec:
                    ev[3].record()
            grad_step(min(batch, 4))       # warm-up on a few items (same kernels and plan upload)
            torch.cuda.synchronize()
            grad_step(batch, True)
            torch.cuda.synchronize()
            L.check(L.stc_sync_status(ws), "device status")
            assert int(info.abs().sum()) == 0
            ms_tot = ev[0].elapsed_time(ev[3])
            ms_bwd = ev[1].elapsed_time(ev[2])
            fa = P.info["flops_alg"]
            out["c5"][route] = {
                "gradients": {"value": batch * 1e3 / ms_tot, "unit": "gradients/s", "batch": batch, "ms": ms_tot},
                "roofline_selinv": dict(_fp64(2 * fa * batch, ms_bwd), bound="alu", peak=PEAK_FP64_NOMINAL,
                                        work="2 sum_j c_j^2 = %.4g flops per item (Takahashi)" % (2 * fa),
                                        ms=ms_bwd)}
            del fac, sig, g, P
            torch.cuda.empty_cache()
        del vals
    if "c4" in want:
        plans, vals = [], []
        per = 2 if small else 8
        for m in (32, 48, 64):
            vs = [I.fem3d(m, m, m, seed=s)[2] for s in range(per)]
            Ap, Ai, _, coords = I.fem3d(m, m, m, seed=0)
            P = Plan(len(Ap) - 1, Ap, Ai, coords=coords, nb=64, route="dense")
            plans.append(P)
            vals.append(dev(np.stack(vs)))
        P64 = plans[2]
        fac = torch.empty(P64.factor_bytes(1) // 8, dtype=torch.float64, device="cuda")
        info = torch.empty(1, dtype=torch.int32, device="cuda")
        ws = P64.workspace(1)
        ms_p = _events_ms(lambda: L.check(L.stc_factorize(P64.h, vals[2][:1], 1, fac, ws, info)), 1, 1)
        L.check(L.stc_sync_status(ws), "device status")
        del fac
        Ap, Ai, _, coords = I.fem3d(64, 64, 64, seed=0)
        Psn = Plan(len(Ap) - 1, Ap, Ai, coords=coords, nb=64, route="supernodal")
        fac = torch.empty(Psn.factor_bytes(1) // 8, dtype=torch.float64, device="cuda")
        ws = Psn.workspace(1)
        ms_sn = _events_ms(lambda: L.check(L.stc_factorize(Psn.h, vals[2][:1], 1, fac, ws, info)), 1, 1)
        L.check(L.stc_sync_status(ws), "device status")
        del fac
        G = Group(plans, [per] * 3)
        ms_g = _events_ms(lambda: G.factorize(vals), 1, 1)
        L.check(G.status(), "group status")
        fl = sum(P.info["flops_alg"] for P in plans) * per
        ft = sum(P.info["flops_tile"] for P in plans) * per
        out["c4"] = {"workload": "7-point lognormal-conductance FEM + 1e-3 I, ND, n_b=64",
                     "route_selected": P64.route_selected,
                     "plain_64cubed_dense": {"value": 1e3 / ms_p, "unit": UNIT, "ms_per_call": ms_p, "n": P64.n,
                                             **_fp64(P64.info["flops_alg"], ms_p),
                                             "tile_tflops": P64.info["flops_tile"] / (ms_p * 1e-3) / 1e12},
                     "plain_64cubed_supernodal": {"value": 1e3 / ms_sn, "unit": UNIT, "ms_per_call": ms_sn,
                                                  **_fp64(Psn.info["flops_alg"], ms_sn),
                                                  "executed_tflops": Psn.info["flops_tile"] / (ms_sn * 1e-3) / 1e12},
                     "mixed_batch_dense": {"value": 3 * per * 1e3 / ms_g, "unit": UNIT,
                                           "items": "32^3, 48^3, 64^3 x %d each, one persistent launch" % per,
                                           "ms": ms_g, **_fp64(fl, ms_g),
                                           "tile_tflops": ft / (ms_g * 1e-3) / 1e12}}
        del G, vals
    if "forced" in want:
        # the selector's choice against each forced route (Table 4's comparison on the
        # synthetic classes): factorize (scatter + task-DAG kernel), best of 3 after a warm-up
        cases = []
        Ap, Ai, _, coords = I.laplace2d_bordered(seed=0)
        cases.append(("config 1, 64 copies", Ap, Ai, coords, 64,
                      np.stack([I.laplace2d_bordered(seed=s % 16)[2] for s in range(64)])))
        Ap, Ai = I.band_pattern(N, BW)
        cases.append(("config 2, 8 value sets", Ap, Ai, None, 128,
                      np.stack([I.band_values(N, BW, s, Ap, Ai) for s in range(8)])))
        Ap, Ai, coords = I.stcov_pattern(gx, gy, gt)
        th = I.stcov_thetas(4, 0)
        cases.append(("config 3, 4 theta sets", Ap, Ai, coords, 64,
                      np.stack([I.stcov_values(t, gx, gy, gt) for t in th])))
        Ap, Ai, Ax, coords = I.fem3d(64, 64, 64, seed=0)
        cases.append(("config 4 64^3, 1 value set", Ap, Ai, coords, 64, Ax[None]))
        out["forced"] = {"note": "factorize (scatter + task-DAG kernel) per route, best of 3 after a warm-up; "
                                 "ms per launch"}
        for name, Ap, Ai, coords, nb, vals in cases:
            v = dev(vals)
            row = {}
            for route in ("auto", "semisparse", "dense", "supernodal"):
                P = Plan(len(Ap) - 1, Ap, Ai, coords=coords, nb=nb, route=route,
                         ordering="natural" if coords is None else "auto")
                bt = vals.shape[0]
                fac = torch.empty(P.factor_bytes(bt) // 8, dtype=torch.float64, device="cuda")
                info = torch.empty(bt, dtype=torch.int32, device="cuda")
                ws = P.workspace(bt)
                run = lambda: L.check(L.stc_factorize(P.h, v, bt, fac, ws, info), "factorize")
                run()
                torch.cuda.synchronize()
                best = min(_events_ms(run, 1, 0) for _ in range(3))
                L.check(L.stc_sync_status(ws), "device status")
                row[route] = {"ms": best, "route_executed": P.route, "factor_GB": P.factor_bytes(bt) / 1e9}
                if route == "auto":
                    row["selected"] = P.route_selected
                del fac, P
                torch.cuda.empty_cache()
            out["forced"][name] = row
            del v
    torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------------ ours
def run_ours(args):
    import torch
    from paper_2609_29765_gb300 import _lib as L
    from paper_2609_29765_gb300.api import Plan

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    # the CPU baseline runs first, before any GPU work of this process (rank 0, N=1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = host_cores()
        walls = oracle_parallel(args.n, cores, rounds=4)
        wall = min(walls[1:])          # minimum of 3 after a warm-up round, as the paper times
        rate = cores / wall
        t = oracle_sample(args.n, 4, seed0=0)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "%d value sets of the workload at once (factor+logdet+solve), one single-threaded "
                         "oracle process per host core; minimum of 3 rounds after a warm-up round, %.1f s wall"
                         % (cores, wall),
               "single_thread": {"value": 1.0 / min(t[1:]), "unit": UNIT, "cores": 1,
                                 "sample": "one value set, minimum of 3 after a warm-up, %.2f s" % min(t[1:])}}

    n, batch = args.n, args.batch
    Ap, Ai = I.band_pattern(n, BW)
    P = Plan(n, Ap, Ai, nb=NB, ordering="natural", route="semisparse", row_slices=args.row_slices)
    P.upload()
    nnz = P.nnzA
    # host (pinned) values for the e2e leg; device copies for the resident leg
    hv = torch.empty(batch, nnz, dtype=torch.float64, pin_memory=True)
    hb = torch.empty(batch, 1, n, dtype=torch.float64, pin_memory=True)
    for b, seed in enumerate(rank_seeds(rank, batch)):
        hv[b].numpy()[:] = I.band_values(n, BW, seed, Ap, Ai)
        hb[b, 0].numpy()[:] = I.rhs(n, 1000 + seed)[0]
    dv = hv.to("cuda")
    db = hb.to("cuda")
    fac = torch.empty(P.factor_bytes(batch) // 8, dtype=torch.float64, device="cuda")
    ws = torch.empty(max(P.workspace_bytes(batch), L.stc_factorize_solve_workspace_bytes(P.h, batch, 1), 64),
                     dtype=torch.uint8, device="cuda")
    info = torch.empty(batch, dtype=torch.int32, device="cuda")
    ld = torch.empty(batch, dtype=torch.float64, device="cuda")
    dx = torch.empty_like(db)
    hld = torch.empty(batch, dtype=torch.float64, pin_memory=True)
    hx = torch.empty_like(hb, pin_memory=True)
    st = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def step(vals, bvec, xout, rp=None):
        if rp is not None:
            rp[0].record(st)
            rp[1].record(st)
        # the value upload, the factorization and the forward substitution in one launch,
        # then the backward substitution (stc_factorize_solve's two halves)
        L.check(L.stc_factorize_forward(P.h, vals, batch, 1, bvec, fac, ws, info), "factorize+forward")
        if rp is not None:
            rp[2].record(st)
        L.check(L.stc_logdet(P.h, fac, batch, ld), "logdet")
        if rp is not None:
            rp[3].record(st)
        L.check(L.stc_solve_backward(P.h, fac, batch, 1, xout, ws), "backward solve")
        if rp is not None:
            rp[4].record(st)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # measured DFMA peak of this GPU (outside the timed region)
    scratch = torch.empty(SMS * 4 * 256, dtype=torch.float64, device="cuda")
    rc, dfma_gflops = L.stc_fp64_peak_probe(scratch, 8192)
    L.check(rc)
    for _ in range(args.warmup):
        step(dv, db, dx)
    torch.cuda.synchronize()
    status = L.stc_sync_status(ws)
    L.check(status, "device status")
    assert int(info.abs().sum()) == 0 and bool(torch.isfinite(ld).all())
    # ---- timed, inputs resident in HBM
    clocks = Clocks(local) if rank == 0 else None
    rps = [tuple(ev() for _ in range(5)) for _ in range(args.steps)]
    barrier()
    e0, e1 = ev(), ev()
    e0.record(st)
    for k in range(args.steps):
        step(dv, db, dx, rps[k])
    e1.record(st)
    barrier()
    ck = clocks.stop() if clocks else None
    ms_step = e0.elapsed_time(e1) / args.steps
    fill_inside = L.lib().stc_factorize_forward_fills(P.h, batch) == 1
    ms_replay = sum(r[1].elapsed_time(r[2]) for r in rps) / args.steps
    ms_logdet = sum(r[2].elapsed_time(r[3]) for r in rps) / args.steps
    ms_solve = sum(r[3].elapsed_time(r[4]) for r in rps) / args.steps
    L.check(L.stc_sync_status(ws), "device status")
    # the scatter kernel on its own (outside the timed region): in the step the value
    # upload runs inside the factorization's launch when the task set hosts it
    ms_scatter = _events_ms(lambda: L.check(L.stc_scatter_values(P.h, dv, batch, fac), "scatter"), 3, 1)
    # ---- e2e: inputs in pinned host memory, logdet + x back out, every step.  (1) the
    # kernels read the values and right-hand sides in place from pinned host memory (the
    # value upload runs inside the factorization's launch, over NVLink-C2C); (2) the same
    # with explicit copies on a second stream, double-buffered: step k+1's inputs go up
    # while step k factorizes.  Both copy logdet and x back on a second stream while the
    # next step runs.
    e2e_ms = e2e_copy_ms = 0.0
    if not args.no_e2e:
        cs = torch.cuda.Stream()
        xb = [dx, torch.empty_like(dx)]
        lb = [ld, torch.empty_like(ld)]
        zdone = [ev(), ev()]
        zout = [ev(), ev()]

        def run_zc(steps):
            for k in range(steps):
                j = k % 2
                if k >= 2:
                    st.wait_event(zout[j])        # step k-2's results have left this buffer
                L.check(L.stc_factorize_forward(P.h, hv, batch, 1, hb, fac, ws, info), "factorize+forward")
                L.check(L.stc_logdet(P.h, fac, batch, lb[j]), "logdet")
                L.check(L.stc_solve_backward(P.h, fac, batch, 1, xb[j], ws), "backward solve")
                zdone[j].record(st)
                with torch.cuda.stream(cs):
                    cs.wait_event(zdone[j])
                    hld.copy_(lb[j], non_blocking=True)
                    hx.copy_(xb[j], non_blocking=True)
                    zout[j].record(cs)
            st.wait_stream(cs)

        run_zc(2)
        barrier()
        t0, t1 = ev(), ev()
        t0.record(st)
        cs.wait_stream(st)
        run_zc(args.steps)
        t1.record(st)
        barrier()
        e2e_ms = t0.elapsed_time(t1) / args.steps
        L.check(L.stc_sync_status(ws), "device status")
        del xb, lb
        bufs = [(dv, db, dx, ld),
                (torch.empty_like(dv), torch.empty_like(db), torch.empty_like(dx), torch.empty_like(ld))]
        ev_in = [ev(), ev()]
        ev_done = [ev(), ev()]
        ev_out = [ev(), ev()]

        def step_io(vals, bvec, xout, ldout):
            L.check(L.stc_factorize_forward(P.h, vals, batch, 1, bvec, fac, ws, info), "factorize+forward")
            L.check(L.stc_logdet(P.h, fac, batch, ldout), "logdet")
            L.check(L.stc_solve_backward(P.h, fac, batch, 1, xout, ws), "backward solve")

        def run_e2e(steps):
            with torch.cuda.stream(cs):
                bufs[0][0].copy_(hv, non_blocking=True)
                bufs[0][1].copy_(hb, non_blocking=True)
                ev_in[0].record(cs)
            for k in range(steps):
                j = k % 2
                vals, bvec, xout, ldout = bufs[j]
                st.wait_event(ev_in[j])
                if k >= 2:
                    st.wait_event(ev_out[j])      # step k-2's results have left this buffer
                step_io(vals, bvec, xout, ldout)
                ev_done[j].record(st)
                with torch.cuda.stream(cs):
                    if k + 1 < steps:
                        jn = (k + 1) % 2
                        if k >= 1:
                            cs.wait_event(ev_done[jn])  # step k-1 no longer reads that buffer
                        bufs[jn][0].copy_(hv, non_blocking=True)
                        bufs[jn][1].copy_(hb, non_blocking=True)
                        ev_in[jn].record(cs)
                    cs.wait_event(ev_done[j])
                    hld.copy_(ldout, non_blocking=True)
                    hx.copy_(xout, non_blocking=True)
                    ev_out[j].record(cs)
            st.wait_stream(cs)

        run_e2e(2)
        barrier()
        t0, t1 = ev(), ev()
        t0.record(st)
        cs.wait_stream(st)
        run_e2e(args.steps)
        t1.record(st)
        barrier()
        e2e_copy_ms = t0.elapsed_time(t1) / args.steps
        del bufs
    # ---- plain: one factorization per launch (batch 1)
    fac1 = torch.empty(P.factor_bytes(1) // 8, dtype=torch.float64, device="cuda")
    info1 = torch.empty(1, dtype=torch.int32, device="cuda")
    ld1 = torch.empty(1, dtype=torch.float64, device="cuda")
    x1 = torch.empty(1, 1, n, dtype=torch.float64, device="cuda")

    def step1():
        L.check(L.stc_factorize_solve(P.h, dv[0:1], 1, 1, db[0:1], fac1, x1, ws, info1), "factorize+solve1")
        L.check(L.stc_logdet(P.h, fac1, 1, ld1), "logdet1")

    for _ in range(2):
        step1()
    torch.cuda.synchronize()
    p0, p1 = ev(), ev()
    p0.record(st)
    for _ in range(args.steps):
        step1()
    p1.record(st)
    torch.cuda.synchronize()
    ms_plain = p0.elapsed_time(p1) / args.steps
    L.check(L.stc_sync_status(ws), "device status")

    # ---- max over ranks
    ms_step, ms_replay, e2e_ms, e2e_copy_ms, ms_plain = max_over_ranks(
        [ms_step, ms_replay, e2e_ms, e2e_copy_ms, ms_plain], dist, "cuda")
    # ---- the other workloads (rank 0, after the headline; free the headline's buffers first)
    workloads = None
    if rank == 0 and args.workloads != "none":
        del dv, db, fac, dx, fac1
        torch.cuda.empty_cache()
        workloads = measure_workloads(args)
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    stored = P.info["stored_entries"]
    scat_bytes = P.factor_bytes(batch) + batch * nnz * 8 + P.factor_bytes(1) // 2
    solve_bytes = batch * (stored * 8 + 2 * n * 8)
    total_items = batch * world
    value = total_items / (ms_step * 1e-3)
    flops_alg = P.info["flops_alg"]
    achieved = flops_alg * batch / (ms_replay * 1e-3) / 1e12
    peak = PEAK_FP64_NOMINAL
    cfg = workload_config(args, batch)
    cfg["l2"] = cfg["l2"] % (batch * nnz * 8 / 1e9, P.factor_bytes(batch) / 1e9)
    cfg["parallelism"] = "independent value sets per GPU (replicas)" if world > 1 else "1 GPU"
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
        "plain": {"value": 1e3 / ms_plain, "unit": UNIT, "ms_per_factorization": ms_plain,
                  "note": "batch 1, one stc_factorize_solve per factorization (+logdet)"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": replay_traffic(args.n, batch),
                     "kernel": "replay_kernel (persistent task-DAG factorization, with the forward "
                               "substitution's steps%s)" % (" and the value upload" if fill_inside else ""),
                     "work": "algorithmic flops sum_j c_j^2 = %.4g per factorization x %d (the forward "
                             "substitution's 2 flops per stored entry not counted)" % (flops_alg, batch),
                     "peak_source": "nominal FP64 ALU: 152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz",
                     "peak_measured_dfma_tflops": dfma_gflops / 1e3,
                     "frac_of_measured_dfma": achieved / (dfma_gflops / 1e3),
                     "tile_flops_per_factorization": P.info["flops_tile"],
                     "ms_replay": ms_replay},
        "kernels": {
            "fill_kernel": {"ms": ms_scatter, "bound": "hbm", "unit": "GB/s",
                            "in_step": not fill_inside,
                            "note": ("timed on its own; in the step each block column's values are placed "
                                     "inside the factorization's launch" if fill_inside else
                                     "timed on its own; run by stc_factorize_forward before the factorization"),
                               "achieved": scat_bytes / (ms_scatter * 1e-3) / 1e9,
                               "peak": HBM_GBS, "peak_source": HBM_SOURCE,
                               "frac": scat_bytes / (ms_scatter * 1e-3) / 1e9 / HBM_GBS,
                               "work": "value scatter in gather form: every factor double written once + "
                                       "values read + int32 source map read once for the batch"},
            "solve_kernel": {"ms": ms_solve, "bound": "hbm", "unit": "GB/s",
                             "achieved": solve_bytes / (ms_solve * 1e-3) / 1e9,
                             "peak": HBM_GBS, "peak_source": HBM_SOURCE,
                             "frac": solve_bytes / (ms_solve * 1e-3) / 1e9 / HBM_GBS,
                             "work": "backward substitution: factor tiles read once + y, x"},
            "logdet_kernel": {"ms": ms_logdet},
        },
        "gpu_launches": (3 if fill_inside else 4) * args.steps,
        "clocks": ck,
        "analyze_seconds": P.info["analyze_seconds"],
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if not args.no_e2e:
        line["e2e"] = {"value": total_items / (e2e_ms * 1e-3), "unit": UNIT,
                       "h2d_bytes_per_step": batch * (nnz + n) * 8,
                       "d2h_bytes_per_step": batch * (1 + n) * 8,
                       "note": "every step's values and RHS start in pinned host memory and are read in place "
                               "by the kernels (the value upload runs inside the factorization's launch, over "
                               "NVLink-C2C; stc_factorize_forward given the host buffers); logdet + x copied "
                               "out on a second stream while the next step runs"}
        line["e2e_copies"] = {"value": total_items / (e2e_copy_ms * 1e-3), "unit": UNIT,
                              "h2d_bytes_per_step": batch * (nnz + n) * 8,
                              "d2h_bytes_per_step": batch * (1 + n) * 8,
                              "note": "the same with explicit copies: every step's values and RHS copied in "
                                      "(cudaMemcpyAsync from pinned memory) on a second stream, double-buffered "
                                      "against the factorization; the first step's copy is not hidden"}
    if workloads:
        line["workloads"] = workloads
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
