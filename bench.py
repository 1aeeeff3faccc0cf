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
HBM_GBS = 6678.5  # measured copy bandwidth of the GB300s (MEASURED_PEAKS.json)


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
    return p.parse_args()


def workload_config(args, batch):
    return {"workload": "banded SPD n=%d half-bandwidth %d, active-column tiles n_b=%d, batch %d value sets"
                        % (args.n, BW, NB, batch),
            "n": args.n, "half_bandwidth": BW, "nb": NB, "batch_per_gpu": batch,
            "route": "semisparse", "ordering": "natural",
            "step": "scatter+factorize+logdet+solve(1 rhs)",
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


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    steps, warm = args.steps, args.warmup
    # each step is one factorization (+logdet+solve) of one value set: a bounded sample
    times = oracle_sample(args.n, warm + steps)[warm:]
    ms = 1e3 * sum(times) / len(times)
    value = 1e3 / ms
    cfg = workload_config(args, args.batch)
    cfg["l2"] = "host run"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": steps, "warmup": warm, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "one value set per step (factor+logdet+solve), single thread"},
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
        t = oracle_sample(args.n, 2, seed0=0)
        cpu = {"value": len(t) / sum(t), "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "2 value sets of the workload, factor+logdet+solve each, single thread, %.1f s"
                         % sum(t)}

    n, batch = args.n, args.batch
    Ap, Ai = I.band_pattern(n, BW)
    P = Plan(n, Ap, Ai, nb=NB, ordering="natural", route="semisparse")
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
    ws = torch.empty(max(P.workspace_bytes(batch), 64), dtype=torch.uint8, device="cuda")
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
        L.check(L.stc_scatter_values(P.h, vals, batch, fac), "scatter")
        if rp is not None:
            rp[1].record(st)
        L.check(L.stc_factorize_scattered(P.h, batch, fac, ws, info), "factorize")
        if rp is not None:
            rp[2].record(st)
        L.check(L.stc_logdet(P.h, fac, batch, ld), "logdet")
        if rp is not None:
            rp[3].record(st)
        L.check(L.stc_solve(P.h, fac, batch, 1, bvec, xout, ws), "solve")
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
    ms_scatter = sum(r[0].elapsed_time(r[1]) for r in rps) / args.steps
    ms_replay = sum(r[1].elapsed_time(r[2]) for r in rps) / args.steps
    ms_logdet = sum(r[2].elapsed_time(r[3]) for r in rps) / args.steps
    ms_solve = sum(r[3].elapsed_time(r[4]) for r in rps) / args.steps
    L.check(L.stc_sync_status(ws), "device status")
    # ---- e2e: host buffers in, logdet + x back out, every step
    e2e_ms = 0.0
    if not args.no_e2e:
        for _ in range(1):
            dv.copy_(hv, non_blocking=True)
            step(dv, db, dx)
        barrier()
        t0, t1 = ev(), ev()
        t0.record(st)
        for k in range(args.steps):
            dv.copy_(hv, non_blocking=True)
            db.copy_(hb, non_blocking=True)
            step(dv, db, dx)
            hld.copy_(ld, non_blocking=True)
            hx.copy_(dx, non_blocking=True)
        t1.record(st)
        barrier()
        e2e_ms = t0.elapsed_time(t1) / args.steps
    # ---- plain: one factorization per launch (batch 1)
    fac1 = torch.empty(P.factor_bytes(1) // 8, dtype=torch.float64, device="cuda")
    info1 = torch.empty(1, dtype=torch.int32, device="cuda")
    ld1 = torch.empty(1, dtype=torch.float64, device="cuda")
    x1 = torch.empty(1, 1, n, dtype=torch.float64, device="cuda")

    def step1():
        L.check(L.stc_factorize(P.h, dv[0:1], 1, fac1, ws, info1), "factorize1")
        L.check(L.stc_logdet(P.h, fac1, 1, ld1), "logdet1")
        L.check(L.stc_solve(P.h, fac1, 1, 1, db[0:1], x1, ws), "solve1")

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
    ms_step, ms_replay, e2e_ms, ms_plain = max_over_ranks([ms_step, ms_replay, e2e_ms, ms_plain], dist, "cuda")
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    stored = P.info["stored_entries"]
    scat_bytes = P.factor_bytes(batch) + batch * nnz * 16 + nnz * 8
    solve_bytes = batch * (2 * stored * 8 + 2 * n * 8)
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
                  "note": "batch 1, one launch per factorization (+logdet+solve)"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": replay_traffic(args.n, batch),
                     "kernel": "replay_kernel (persistent task-DAG factorization)",
                     "work": "algorithmic flops sum_j c_j^2 = %.4g per factorization x %d" % (flops_alg, batch),
                     "peak_source": "nominal FP64 ALU: 152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz",
                     "peak_measured_dfma_tflops": dfma_gflops / 1e3,
                     "frac_of_measured_dfma": achieved / (dfma_gflops / 1e3),
                     "tile_flops_per_factorization": P.info["flops_tile"],
                     "ms_replay": ms_replay},
        "kernels": {
            "scatter_kernel": {"ms": ms_scatter, "bound": "hbm", "unit": "GB/s",
                               "achieved": scat_bytes / (ms_scatter * 1e-3) / 1e9,
                               "peak": HBM_GBS, "frac": scat_bytes / (ms_scatter * 1e-3) / 1e9 / HBM_GBS,
                               "work": "zero-fill of the factor + values read + map read + scattered writes"},
            "solve_kernel": {"ms": ms_solve, "bound": "hbm", "unit": "GB/s",
                             "achieved": solve_bytes / (ms_solve * 1e-3) / 1e9,
                             "peak": HBM_GBS, "frac": solve_bytes / (ms_solve * 1e-3) / 1e9 / HBM_GBS,
                             "work": "factor tiles read twice (forward + backward) + b, x"},
            "logdet_kernel": {"ms": ms_logdet},
        },
        "gpu_launches": 4 * args.steps,
        "clocks": ck,
        "analyze_seconds": P.info["analyze_seconds"],
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if not args.no_e2e:
        line["e2e"] = {"value": total_items / (e2e_ms * 1e-3), "unit": UNIT,
                       "h2d_bytes_per_step": batch * (nnz + n) * 8,
                       "d2h_bytes_per_step": batch * (1 + n) * 8}
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
