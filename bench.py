#!/usr/bin/env python
"""Benchmark of exact k-nearest-neighbour search (dual-tree, kd-tree, B(N_q) bound).

Default workload (synthetic, seeded; --workload powerlaw64): bichromatic kNN
with N_r = N_q = 2,000,000 points in d = 64 drawn from a Gaussian with a
power-law covariance spectrum (eigenvalue i proportional to i^-1.5, random
rotation), k = 50, leaf size 32.  The headline arm is the learned proposal
(trained once, before the timed region, on the method's own answers for
200,000 disjoint training queries) with split-BF16 tensor-core BaseCase tiles
and the float64 re-rank; the same run times the same precision without the
proposal and the plain FP32 GPU dual-tree (CUDA-core tiles) on the same
inputs, and reports value / plain as `vs_plain_fp32`.  --workload latent3
(10M x 1M, d = 8, k = 10) and gmm16 (4M x 1M, d = 16, k = 10) run the same
contract.

One step = the whole path: build the reference kd-tree, build the query
kd-tree, run the exact kNN search (seed, per-query caps, bounds, pruning
dual-tree traversal, BaseCase tiles, float64 re-rank, output).  `value` =
queries/s of the whole job (all ranks' queries / the slowest rank's time).
The inputs exceed the 129 MB L2, so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload powerlaw64|latent3|gmm16] [--op knn|kfn|range|emst]

Under torchrun each rank searches its own query shard against the same
reference set (weak scaling, no collective on the data path).
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1304_4327_gb300 import inputs  # noqa: E402

METRIC = "exact kNN queries/s (oracle-identical neighbors)"
UNIT = "queries/s"
WORKLOAD = ("gmm16: bichromatic exact kNN, N_r=4,000,000, N_q=1,000,000, d=16, k=10, "
            "32-component isotropic Gaussian mixture (centres U[-10,10]^16, sigma=1)")


def parse():
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--op", choices=["knn", "kfn", "range", "emst"], default="knn",
                   help="knn (the headline), k-furthest neighbours, range search, or the "
                        "Euclidean minimum spanning tree")
    p.add_argument("--workload", choices=["powerlaw64", "latent3", "gmm16", "batched"], default="powerlaw64",
                   help="kNN workload (--op knn)")
    p.add_argument("--precision", choices=["fp32", "tf32", "bf16"], default=None,
                   help="BaseCase arithmetic (default: the workload's)")
    p.add_argument("--bound", choices=["box", "ball", "both"], default="box",
                   help="Score's node lower bound d_min: boxes (kd-tree), balls (ball tree over the "
                        "same splits) or the larger of the two")
    p.add_argument("--proposal", type=int, default=None,
                   help="learned-proposal cells per query block, 0 = none (default: the workload's)")
    p.add_argument("--train-queries", type=int, default=200_000)
    p.add_argument("--arm-steps", type=int, default=2,
                   help="timed steps of the same precision without the proposal")
    p.add_argument("--plain-steps", type=int, default=1,
                   help="timed steps of the plain FP32 dual-tree (0 skips it)")
    p.add_argument("--leaf", type=int, default=32)
    p.add_argument("--query-block", type=int, default=0)
    p.add_argument("--e2e-steps", type=int, default=3)
    p.add_argument("--n-ref", type=int, default=0, help="override the workload's reference count")
    p.add_argument("--n-query", type=int, default=0, help="override the workload's query count")
    p.add_argument("--cpu-queries", type=int, default=0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--ref-queries", type=int, default=0,
                   help="queries per step of the reference arm (default: the workload's)")
    p.add_argument("--range", type=float, nargs=2, default=[0.0, 2.5], metavar=("D_LO", "D_HI"))
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_uuid):
        self.proc = None
        self.path = None
        self.uuid = device_uuid

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        cmd = ["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
               "-lms", "100"]
        if self.uuid:
            cmd += ["-i", self.uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 8:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[2]) for r in rows
                                                        if r[2].replace(".", "").isdigit())
                if any(r[2].replace(".", "").isdigit() for r in rows) else None}


# ---------------------------------------------------------------------------
# the reference arm: the oracle on the host cores
# ---------------------------------------------------------------------------

def run_reference(args, rank, world):
    """The oracle on the host cores: each step answers a fresh sample of
    queries of the same workload against its full reference set by brute
    force (the definition of the result)."""
    if rank != 0:
        return
    import oracle
    if args.workload == "batched":
        run_reference_batched(args, world)
        return
    spec = WORKLOADS[args.workload]
    a = argparse.Namespace(**vars(args))
    a.train_queries = 0
    W = spec["make"](a, 0)
    cores = oracle.set_threads(os.cpu_count() or 1)
    nq = args.ref_queries or max(8, min(512, int(2e9 / (len(W.ref) * W.d * 3))))
    times = []
    for step in range(args.warmup + args.steps):
        lo = (step * nq) % max(1, len(W.query) - nq)
        t0 = time.perf_counter()
        oracle.knn_brute(W.ref, W.query[lo:lo + nq], W.k)
        if step >= args.warmup:
            times.append(time.perf_counter() - t0)
    t = sum(times) / len(times)
    value = nq / t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": spec["desc"], "step": f"{nq}-query sample per step, brute force"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{nq} queries per step vs all {len(W.ref):,} references, "
                                   "float64 brute force (oracle_knn_brute)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_reference_batched(args, world):
    """The batched workload's reference arm: each step answers a sample of
    queries of one of the 256 problems (in turn) by brute force."""
    import oracle
    cores = oracle.set_threads(os.cpu_count() or 1)
    specs = inputs.batched_specs()
    nq = args.ref_queries or 256
    times, done = [], 0
    for step in range(args.warmup + args.steps):
        W = inputs.batched_problem(specs[step % len(specs)])
        m = min(nq, len(W.ref))
        t0 = time.perf_counter()
        oracle.knn_brute(W.ref, W.ref[:m], W.k, self_idx=np.arange(m, dtype=np.int64))
        if step >= args.warmup:
            times.append(time.perf_counter() - t0)
            done += m
    t = sum(times)
    value = done / t
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t / len(times) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_BATCHED,
                   "step": f"up to {nq} queries of one problem (in turn) per step, brute force"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"up to {nq} queries per step of problem (step mod 256) against "
                                   "its own points, float64 brute force (oracle_knn_brute)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ---------------------------------------------------------------------------
# multi-process helpers (query shards; the slowest rank sets the time)
# ---------------------------------------------------------------------------

def shard_workload(args, rank):
    """Rank r searches its own query shard (an independent seeded stream)
    against the same reference set: the problem splits by queries with no
    exchange step."""
    return inputs.gmm16(n_ref=args.n_ref or 4_000_000, n_query=args.n_query or 1_000_000,
                        leaf_size=args.leaf, shard=rank)


def max_over_ranks(x, world, device):
    """The maximum of a per-rank float over all ranks (identity at world 1)."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, n_per_rank, ms_max):
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return world * n_per_rank / (ms_max / 1e3)


# ---------------------------------------------------------------------------
# the CUDA path
# ---------------------------------------------------------------------------

# ---------------------------------------------------------------------------
# exact kNN (--op knn): the workloads and their arms
# ---------------------------------------------------------------------------

WORKLOADS = {
    # the combined configuration: learned proposal + BF16 tensor-core tiles +
    # exact re-rank, against the plain FP32 GPU dual-tree
    "powerlaw64": {
        "desc": ("powerlaw64: bichromatic exact kNN, N_r=2,000,000, N_q=2,000,000, d=64, k=50, "
                 "Gaussian with power-law covariance spectrum (eigenvalue i ~ i^-1.5, random rotation)"),
        "make": lambda a, rank: inputs.powerlaw64(n_ref=a.n_ref or 2_000_000, n_query=a.n_query or 2_000_000,
                                                  n_train=a.train_queries, shard=rank),
        "precision": "bf16", "proposal": 1, "cpu_queries": 256,
        # blocks of 512 queries (4 chunks of 128 sharing their candidate
        # leaves): at d = 64 the bound prunes almost nothing, and the
        # traversal over 4x fewer blocks takes 94 ms instead of 344
        "query_block": 512,
        # a per-query cap search of 16 leaves (the library's default is 8):
        # its 41 ms more buy 63 ms of the main pass
        "cap_leaves": 16,
    },
    # the learned-proposal configuration at d = 8.  FP32 tiles: at this point
    # density the k-th neighbour's squared distance (~1e-5) is no larger than
    # BF16's rounding band, so about half the queries overflow their lists
    # and are recomputed exactly (--precision bf16 shows it)
    "latent3": {
        "desc": ("latent3: bichromatic exact kNN, N_r=10,000,000, N_q=1,000,000, d=8, k=10, "
                 "3-dim latent U[0,1]^3 mapped by a seeded 8x3 linear map plus N(0,0.01^2) noise"),
        "make": lambda a, rank: inputs.latent3(n_ref=a.n_ref or 10_000_000, n_query=a.n_query or 1_000_000,
                                               n_train=a.train_queries, shard=rank),
        "precision": "fp32", "proposal": 4, "cpu_queries": 8192,
    },
    # the 16-dimensional mixture at BF16 (no training set: no proposal)
    "gmm16": {
        "desc": WORKLOAD,
        "make": lambda a, rank: inputs.gmm16(n_ref=a.n_ref or 4_000_000, n_query=a.n_query or 1_000_000,
                                             leaf_size=a.leaf, shard=rank),
        "precision": "bf16", "proposal": 0, "cpu_queries": 8192,
        # blocks of 256 queries: the traversal 7.7 -> 4.7 ms, the main pass
        # 42.9 -> 43.8 ms
        "query_block": 256,
    },
}

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one main
# BaseCase launch from a one-pass ncu capture, with the point pairs that launch
# evaluated, per (workload, precision); a run's traffic is that capture's
# bytes per pair times its own pairs.  Absent where no capture of the current
# kernel exists.
TRAFFIC_CAPTURE = {
    # k_tile_tc<3, 64, 64, 1>, 2M x 2M, 512-query blocks, no proposal:
    # 6,941,407,034,112 B read + 1,359,624,448 B written over
    # 3,867,716,373,340 point pairs
    ("powerlaw64", "bf16"): (6_941_407_034_112 + 1_359_624_448, 3_867_716_373_340),
}


def traffic_of(workload, precision, pairs):
    cap = TRAFFIC_CAPTURE.get((workload, precision))
    return None if cap is None else cap[0] * pairs / cap[1]


def roofline(precision, d, pairs, ns_tile, sms, traffic):
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
        src = "of measured"
    except (OSError, ValueError):
        src = "of fallback"
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    secs = ns_tile * 1e-9
    if precision == "fp32":
        flops = 3.0 * d * pairs                  # d subtractions + d FMAs (2 flops each)
        peak = 2.0 * 128 * sms * sm_max * 1e6 / 1e12
        bound, kernel = "alu", "k_tile main launch (BaseCase, CUDA-core float32)"
        psrc = f"2 x 128 FP32 lanes x {sms} SMs x {sm_max:.0f} MHz"
    else:
        flops = 2.0 * d * pairs                  # one multiply-add per coordinate and pair
        bf16 = float(peaks.get("bf16_tflops_sustained", 1700.0))
        peak = bf16 if precision == "bf16" else bf16 * 1.1 / 2.25
        bound, kernel = "tensor", f"k_tile_tc main launch (BaseCase, tcgen05 {precision})"
        psrc = (f"sustained BF16 dense {bf16:.1f} TFLOP/s ({src})"
                + ("" if precision == "bf16" else " x 1.1/2.25 (nominal TF32:BF16)"))
    achieved = flops / secs / 1e12 if secs > 0 else 0.0
    return {"bound": bound, "kernel": kernel, "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak if peak else None, "traffic": traffic,
            "peak_source": psrc, "algorithmic_flops_per_step": flops,
            "point_pairs_per_step": pairs, "kernel_ms": ns_tile / 1e6}


def cpu_baseline(W, n_queries, desc):
    import oracle
    cores = oracle.set_threads(os.cpu_count() or 1)
    q = W.query[:n_queries]
    t0 = time.perf_counter()
    oracle.knn_dualtree(W.ref, q, W.k, W.leaf_size, par_depth=8)
    dt = time.perf_counter() - t0
    return {"value": n_queries / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": (f"float64 kd-tree dual-tree (Alg 1-3, sound B; the oracle) on the full "
                       f"{len(W.ref):,}-point reference set and the first {n_queries} queries "
                       f"(an i.i.d. sample of the {len(W.query):,}) of {desc.split(':')[0]}; both "
                       f"tree builds included; {dt:.1f} s wall")}


def run_knn(args, rank, world, local):
    import torch
    import torch.distributed as dist

    spec = WORKLOADS[args.workload]
    precision = args.precision or spec["precision"]
    M = spec["proposal"] if args.proposal is None else args.proposal
    qblock = args.query_block or spec.get("query_block", 128)
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1304_4327_gb300 import dtree

    W = spec["make"](args, rank)
    d, k = W.d, W.k
    ref_d = torch.from_numpy(W.ref).cuda()
    q_d = torch.from_numpy(W.query).cuda()
    nq = q_d.shape[0]
    out_idx = torch.empty((nq, k), dtype=torch.int64, device="cuda")
    out_dist = torch.empty((nq, k), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()

    # the learned proposal, trained once on the method's own answers for a
    # disjoint training query set (outside the timed region); a tree rebuilt
    # from the same points has the same cells, so each step attaches it
    model, train_s, train_info = None, None, None
    if M > 0:
        if "train" not in W.extra:
            raise SystemExit(f"workload {args.workload} has no training queries for a proposal")
        t0 = time.perf_counter()
        tr0 = dtree.dtree_build(ref_d, W.leaf_size)
        tt0 = dtree.dtree_build(torch.from_numpy(W.extra["train"]).cuda(), W.leaf_size)
        try:
            model = dtree.dtree_proposal_train(tr0, tt0, k, precision=precision)
        finally:
            tr0.free()
            tt0.free()
        torch.cuda.synchronize()
        train_s = time.perf_counter() - t0
        train_info = {"train_queries": int(len(W.extra["train"])), "cells": model.classes,
                      "epochs": len(model.losses), "loss_first": model.losses[0],
                      "loss_last": model.losses[-1], "seconds": train_s}

    def step(ref, qry, prec=precision, nprop=M):
        tr = dtree.dtree_build(ref, W.leaf_size)
        tq = dtree.dtree_build(qry, W.leaf_size)
        try:
            if nprop > 0:
                dtree.dtree_attach_proposal(tr, model)
            _, _, st = dtree.dtree_knn(tq, tr, k, precision=prec, query_block=qblock,
                                       out_idx=out_idx, out_dist=out_dist, with_stats=True,
                                       proposal=nprop, bound=args.bound,
                                       cap_leaves=spec.get("cap_leaves", 0))
        finally:
            tr.free()
            tq.free()
        return st

    def timed(n, warm, **kw):
        for _ in range(warm):
            step(ref_d, q_d, **kw)
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = [step(ref_d, q_d, **kw) for _ in range(n)]
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        return max_over_ranks(e0.elapsed_time(e1) / n, world, "cuda"), st

    # the headline arm: W warm-up steps, then exactly K timed steps
    for _ in range(args.warmup):
        step(ref_d, q_d)
    props = torch.cuda.get_device_properties(local)
    uuid = getattr(props, "uuid", None)
    clocks = ClockSampler(f"GPU-{uuid}" if uuid else None)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = dtree.launch_count()
    ms_max, stats = timed(args.steps, 0)
    clock_info = clocks.stop()
    launches = dtree.launch_count() - launches0
    value = job_rate(world, nq, ms_max)

    # end to end through the public API: pinned host inputs in, host results out
    ref_h = torch.from_numpy(W.ref).pin_memory()
    q_h = torch.from_numpy(W.query).pin_memory()
    idx_h = torch.empty((nq, k), dtype=torch.int64).pin_memory()
    dist_h = torch.empty((nq, k), dtype=torch.float32).pin_memory()
    ref_e, q_e = torch.empty_like(ref_d), torch.empty_like(q_d)

    def e2e_step():
        ref_e.copy_(ref_h, non_blocking=True)
        q_e.copy_(q_h, non_blocking=True)
        step(ref_e, q_e)
        idx_h.copy_(out_idx, non_blocking=True)
        dist_h.copy_(out_dist, non_blocking=True)

    e2e_step()  # untimed: the first copies through freshly pinned buffers
    barrier()
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(args.e2e_steps):
        e2e_step()
    f1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(f0.elapsed_time(f1) / args.e2e_steps, world, "cuda")
    e2e_value = job_rate(world, nq, e2e_ms)

    # the comparison arms on the same inputs: the same precision without the
    # proposal, and the plain FP32 GPU dual-tree (CUDA-core tiles, no proposal)
    arms = {}
    if M > 0 and args.arm_steps > 0:
        ms_tc, st_tc = timed(args.arm_steps, 1, nprop=0)
        arms[f"{precision}_no_proposal"] = {"value": job_rate(world, nq, ms_tc), "ms_per_step": ms_tc,
                                            "basecase_ms": st_tc[-1]["ns_basecase"] / 1e6,
                                            "seed_ms": st_tc[-1]["ns_seed"] / 1e6,
                                            "traverse_ms": st_tc[-1]["ns_traverse"] / 1e6}
    if args.plain_steps > 0 and precision != "fp32":
        ms_pl, st_pl = timed(args.plain_steps, 0, prec="fp32", nprop=0)
        arms["plain_fp32"] = {"value": job_rate(world, nq, ms_pl), "ms_per_step": ms_pl,
                              "basecase_ms": st_pl[-1]["ns_basecase"] / 1e6,
                              "steps": args.plain_steps, "warmup": 0}

    # roofline of the dominant kernel: the main BaseCase tile launch, timed per
    # call with CUDA events on the launching stream
    mean = lambda key: sum(s[key] for s in stats) / len(stats)
    ns_tile, ns_seed, ns_fb, ns_trav = mean("ns_basecase"), mean("ns_seed"), mean("ns_fallback"), mean("ns_traverse")
    pairs = mean("point_pairs")
    sms = props.multi_processor_count
    roof = roofline(precision, d, pairs, ns_tile, sms, traffic_of(args.workload, precision, pairs))
    s0 = stats[-1]
    arm_name = ("learned proposal (M=%d) + " % M if M else "") + precision.upper() + (
        " tensor-core tiles + float64 re-rank" if precision != "fp32" else " CUDA-core tiles")
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if precision == "fp32" else precision,
        "data": "synthetic",
        "config": {"workload": spec["desc"], "arm": arm_name, "precision": precision,
                   "proposal": M, "bound": args.bound, "leaf_size": W.leaf_size,
                   "query_block": qblock, "cap_leaves": spec.get("cap_leaves", 8),
                   "step": "build ref tree + build query tree + dtree_knn",
                   "l2": (f"inputs ({(W.ref.nbytes + W.query.nbytes) / 1e6:.0f} MB) larger than the "
                          "129 MB L2; no flush"),
                   "parallelism": f"{world} GPU(s), one query shard each, reference replicated"},
        "roofline": roof,
        "phases_ms": {"seed": ns_seed / 1e6, "basecase_main": ns_tile / 1e6,
                      "fallback": ns_fb / 1e6, "traverse": ns_trav / 1e6,
                      "build_and_rest": ms_max - (ns_seed + ns_tile + ns_fb + ns_trav) / 1e6},
        "counters": {k2: s0[k2] for k2 in ("node_pairs_scored", "node_pairs_pruned",
                                          "leaf_pairs_emitted", "leaf_pairs_skipped",
                                          "leaf_pairs_evaluated", "point_pairs",
                                          "rerank_candidates", "fallback_queries",
                                          "seed_point_pairs")},
        "arms": arms,
        "e2e": {"value": e2e_value, "unit": UNIT,
                "h2d_bytes_per_step": int(W.ref.nbytes + W.query.nbytes),
                "d2h_bytes_per_step": int(nq * k * (8 + 4))},
        "gpu_launches": int(launches),
        "clocks": clock_info,
    }
    if "plain_fp32" in arms:
        line["vs_plain_fp32"] = value / arms["plain_fp32"]["value"]
    if train_info:
        line["proposal_training"] = train_info
    if model is not None:
        model.free()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(W, args.cpu_queries or spec["cpu_queries"], spec["desc"])
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# the batched workload (--workload batched): 256 problems, one call
# ---------------------------------------------------------------------------

WORKLOAD_BATCHED = ("batched: 256 independent monochromatic exact kNN problems, N log-normal "
                    "between 1,000 and 200,000 (6.68 M points in all), d from {3, 8, 32}, k from "
                    "{1, 10}, uniform or Gaussian by seed, autotuned leaf size and queries per block")


def run_batched(args, rank, world, local):
    """One step = build every problem's tree (its tuned leaf size) + one
    dtree_knn_batch call over all 256 problems (their tuned block sizes).
    The tuner measures each problem class once, before the timed region.
    The same invocation times one dtree_knn call per problem on the same
    trees' inputs.  Under torchrun every rank solves its own copy of the
    batch (weak scaling)."""
    import torch
    import torch.distributed as dist
    from paper_1304_4327_gb300 import autotune

    precision = args.precision or "bf16"
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1304_4327_gb300 import dtree

    specs = inputs.batched_specs()
    probs = [inputs.batched_problem(sp) for sp in specs]
    pts = [torch.from_numpy(W.ref).cuda() for W in probs]
    nq = sum(len(W.ref) for W in probs)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()

    t0 = time.perf_counter()
    tuner = autotune.Autotuner(repeats=1)
    choice = tuner.choose_batch([(p, None, W.k) for p, W in zip(pts, probs)], precision)
    torch.cuda.synchronize()
    tune_s = time.perf_counter() - t0

    def step(points, batched=True):
        trees = [dtree.dtree_build(p, leaf) for p, (leaf, _) in zip(points, choice)]
        try:
            if batched:
                outs, st = dtree.dtree_knn_batch(
                    [(None, tr, W.k, qb) for tr, W, (_, qb) in zip(trees, probs, choice)],
                    precision=precision, with_stats=True)
            else:
                outs, st = [], None
                for tr, W, (_, qb) in zip(trees, probs, choice):
                    i, d = dtree.dtree_knn(None, tr, W.k, precision=precision, query_block=qb)
                    outs.append((i, d))
        finally:
            for tr in trees:
                tr.free()
        return outs, st

    # the batch's inputs (80 MB) fit the 129 MB L2: before every timed step a
    # 256 MB buffer is written, outside the step's events, so no step finds
    # the previous one's data in L2
    l2_flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    def timed(n, batched=True):
        barrier()
        torch.cuda.synchronize()
        total, res = 0.0, []
        for _ in range(n):
            l2_flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res.append(step(pts, batched))
            e1.record(stream)
            torch.cuda.synchronize()
            total += e0.elapsed_time(e1)
        barrier()
        return max_over_ranks(total / n, world, "cuda"), res

    for _ in range(args.warmup):
        step(pts)
    props = torch.cuda.get_device_properties(local)
    uuid = getattr(props, "uuid", None)
    clocks = ClockSampler(f"GPU-{uuid}" if uuid else None)
    clocks.start()
    launches0 = dtree.launch_count()
    ms_max, res = timed(args.steps)
    clock_info = clocks.stop()
    launches = dtree.launch_count() - launches0
    value = job_rate(world, nq, ms_max)
    stats = [r[1] for r in res]

    # end to end: every problem's points from pinned host memory, the lists back
    host = [torch.from_numpy(W.ref).pin_memory() for W in probs]
    dev = [torch.empty_like(p) for p in pts]
    barrier()
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    d2h = 0
    # one untimed iteration first: the first copies through freshly pinned buffers
    for it in range(args.e2e_steps + 1):
        if it == 1:
            f0.record(stream)
        for h, dv in zip(host, dev):
            dv.copy_(h, non_blocking=True)
        outs, _ = step(dev)
        back = [(i.to("cpu", non_blocking=True), d.to("cpu", non_blocking=True)) for i, d in outs]
        d2h = sum(i.numel() * 8 + d.numel() * 4 for i, d in outs)
    f1.record(stream)
    torch.cuda.synchronize()
    e2e_value = job_rate(world, nq, max_over_ranks(f0.elapsed_time(f1) / args.e2e_steps, world, "cuda"))
    del back

    # one call per problem, the same trees and parameters
    arms = {}
    if args.arm_steps > 0:
        ms_one, _ = timed(args.arm_steps, batched=False)
        arms["one_call_per_problem"] = {"value": job_rate(world, nq, ms_one), "ms_per_step": ms_one}

    # roofline of the main BaseCase launches (CUDA-core float32 tiles at
    # 3 d flops per pair), per width bucket from an untimed pass
    flops, pairs_all = 0.0, 0
    for dd in sorted({W.d for W in probs}):
        sel = [i for i, W in enumerate(probs) if W.d == dd]
        trees = [dtree.dtree_build(pts[i], choice[i][0]) for i in sel]
        try:
            _, stb = dtree.dtree_knn_batch([(None, tr, probs[i].k, choice[i][1]) for tr, i in zip(trees, sel)],
                                           precision=precision, with_stats=True)
        finally:
            for tr in trees:
                tr.free()
        flops += (3.0 if precision == "fp32" else 2.0) * dd * stb["point_pairs"]
        pairs_all += stb["point_pairs"]
    ns_tile = sum(s["ns_basecase"] for s in stats) / len(stats)
    sms = props.multi_processor_count
    roof = roofline(precision, 1, 1.0, ns_tile, sms, None)
    roof["algorithmic_flops_per_step"] = flops
    roof["point_pairs_per_step"] = pairs_all
    roof["achieved"] = flops / (ns_tile * 1e-9) / 1e12 if ns_tile else 0.0
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["kernel"] = (f"main BaseCase launches of the batch ({precision}), all width buckets"
                      if precision == "fp32" else roof["kernel"])
    s0 = stats[-1]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if precision == "fp32" else precision,
        "data": "synthetic",
        "config": {"workload": WORKLOAD_BATCHED, "precision": precision,
                   "step": "build 256 trees + one dtree_knn_batch",
                   "l2": "inputs (80 MB) fit the 129 MB L2: a 256 MB buffer is written before each timed step, outside its events",
                   "parallelism": f"{world} GPU(s), every rank its own copy of the batch",
                   "autotune_s": tune_s, "classes": len(tuner.table)},
        "roofline": roof,
        "phases_ms": {"seed": s0["ns_seed"] / 1e6, "basecase_main": ns_tile / 1e6,
                      "traverse": s0["ns_traverse"] / 1e6, "fallback": s0["ns_fallback"] / 1e6,
                      "build_and_rest": ms_max - (s0["ns_seed"] + ns_tile + s0["ns_traverse"] + s0["ns_fallback"]) / 1e6},
        "counters": {k2: s0[k2] for k2 in ("leaf_pairs_emitted", "point_pairs", "fallback_queries",
                                          "kernel_launches")},
        "arms": arms,
        "e2e": {"value": e2e_value, "unit": UNIT,
                "h2d_bytes_per_step": int(sum(W.ref.nbytes for W in probs)),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
        "clocks": clock_info,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.op in ("kfn", "range"):
        run_kfn(args, rank, world, local)
        return
    if args.op == "emst":
        run_emst(args, rank, world, local)
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "batched":
        run_batched(args, rank, world, local)
        return
    run_knn(args, rank, world, local)


# ---------------------------------------------------------------------------
# k-furthest neighbours (--op kfn): the same workload, the same contract
# ---------------------------------------------------------------------------

METRIC_KFN = "exact k-furthest-neighbour queries/s (oracle-identical)"
WORKLOAD_KFN = WORKLOAD.replace("exact kNN", "exact k-furthest neighbours")
METRIC_RANGE = "exact range-search queries/s (oracle-identical)"


def run_kfn(args, rank, world, local):
    """--op kfn: one step = build the reference tree + build the query tree +
    dtree_kfn (one warp per query: the single-tree depth-first search with the
    inverted Score and BaseCase, float32 keys, float64 re-rank and fallback).
    --op range: the same with dtree_range (count, scan, fill) over --range."""
    from oracle import kfn as okfn
    from oracle import rangesearch as orange
    is_range = args.op == "range"
    d_lo, d_hi = args.range
    metric = METRIC_RANGE if is_range else METRIC_KFN
    workload = (WORKLOAD.replace("exact kNN", f"exact range search [{d_lo:g}, {d_hi:g}]")
                .replace(", k=10", "") if is_range else WORKLOAD_KFN)

    def oracle_call(ref, qry, k):
        if is_range:
            orange.range_brute(ref, qry, d_lo, d_hi)
        else:
            okfn.kfn_brute(ref, qry, k)

    if args.impl == "reference":
        if rank != 0:
            return
        W = inputs.gmm16(n_ref=args.n_ref or 4_000_000, n_query=args.n_query or 1_000_000)
        nq = min(args.ref_queries or 16, 16)
        times = []
        for step in range(args.warmup + args.steps):
            lo = (step * nq) % max(1, len(W.query) - nq)
            t0 = time.perf_counter()
            oracle_call(W.ref, W.query[lo:lo + nq], W.k)
            if step >= args.warmup:
                times.append(time.perf_counter() - t0)
        t = sum(times) / len(times)
        value = nq / t
        print(json.dumps({
            "impl": "reference", "metric": metric, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload, "step": f"{nq}-query sample per step, brute force"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{nq} queries per step vs all {len(W.ref)} references, "
                                       "float64 brute force (numpy, one thread)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }), flush=True)
        return
    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1304_4327_gb300 import dtree
    W = shard_workload(args, rank)
    d, k = W.d, W.k
    ref_d = torch.from_numpy(W.ref).cuda()
    q_d = torch.from_numpy(W.query).cuda()
    nq = q_d.shape[0]
    out_idx = torch.empty((nq, k), dtype=torch.int64, device="cuda")
    out_dist = torch.empty((nq, k), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    res = {}

    def step(ref, qry):
        tr = dtree.dtree_build(ref, args.leaf)
        tq = dtree.dtree_build(qry, args.leaf)
        try:
            if is_range:
                res["off"], res["idx"], res["dist"], st = dtree.dtree_range(
                    tq, tr, d_lo, d_hi, with_stats=True)
            else:
                _, _, st = dtree.dtree_kfn(tq, tr, k, out_idx=out_idx, out_dist=out_dist,
                                           with_stats=True)
        finally:
            tr.free()
            tq.free()
        return st

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(args.warmup):
        step(ref_d, q_d)
    props = torch.cuda.get_device_properties(local)
    uuid = getattr(props, "uuid", None)
    clocks = ClockSampler(f"GPU-{uuid}" if uuid else None)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = dtree.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    stats = [step(ref_d, q_d) for _ in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clock_info = clocks.stop()
    launches = dtree.launch_count() - launches0
    ms_max = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, "cuda")
    value = job_rate(world, nq, ms_max)
    # end to end: pinned host inputs in, host results out
    ref_h = torch.from_numpy(W.ref).pin_memory()
    q_h = torch.from_numpy(W.query).pin_memory()
    idx_h = torch.empty((nq, k), dtype=torch.int64).pin_memory()
    dist_h = torch.empty((nq, k), dtype=torch.float32).pin_memory()
    ref_e, q_e = torch.empty_like(ref_d), torch.empty_like(q_d)
    barrier()
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    d2h = 0
    # one untimed iteration first: the first copies through freshly pinned buffers
    for it in range(args.e2e_steps + 1):
        if it == 1:
            f0.record(stream)
        ref_e.copy_(ref_h, non_blocking=True)
        q_e.copy_(q_h, non_blocking=True)
        step(ref_e, q_e)
        if is_range:
            outs = [res["off"].to("cpu", non_blocking=True), res["idx"].to("cpu", non_blocking=True),
                    res["dist"].to("cpu", non_blocking=True)]
            d2h = sum(int(t.numel() * t.element_size()) for t in outs)
        else:
            idx_h.copy_(out_idx, non_blocking=True)
            dist_h.copy_(out_dist, non_blocking=True)
            d2h = int(nq * k * (8 + 4))
    f1.record(stream)
    torch.cuda.synchronize()
    e2e_value = job_rate(world, nq, max_over_ranks(f0.elapsed_time(f1) / args.e2e_steps, world, "cuda"))
    ns = sum(s["ns_basecase"] for s in stats) / len(stats)
    pairs = sum(s["point_pairs"] for s in stats) / len(stats)
    sms = props.multi_processor_count
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except (OSError, ValueError):
        pass
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    flops = 3.0 * d * pairs  # d subtractions + d FMAs per point distance
    peak = 2.0 * 128 * sms * sm_max * 1e6 / 1e12
    achieved = flops / (ns * 1e-9) / 1e12 if ns > 0 else 0.0
    s0 = stats[-1]
    line = {
        "metric": metric, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload, "precision": "fp32 keys, f64 decisions", "leaf_size": args.leaf,
                   "step": "build ref tree + build query tree + "
                           + ("dtree_range (count, scan, fill)" if is_range else "dtree_kfn"),
                   "l2": "inputs (320 MB) larger than the 129 MB L2; no flush",
                   "parallelism": f"{world} GPU(s), one query shard each, reference replicated"},
        "roofline": {"bound": "alu",
                     "kernel": ("k_range count launch" if is_range else "k_kfn")
                     + " (one warp per query, float32 keys)",
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak if peak else None, "traffic": None,
                     "peak_source": f"2 x 128 FP32 lanes x {sms} SMs x {sm_max:.0f} MHz",
                     "algorithmic_flops_per_step": flops, "point_pairs_per_step": pairs,
                     "kernel_ms": ns / 1e6},
        "phases_ms": {("range_count" if is_range else "kfn"): ns / 1e6,
                      "build_and_rest": ms_max - ns / 1e6},
        "counters": {k2: s0[k2] for k2 in ("point_pairs", "leaf_pairs_evaluated",
                                          "node_pairs_pruned", "fallback_queries",
                                          "rerank_candidates")},
        "e2e": {"value": e2e_value, "unit": UNIT,
                "h2d_bytes_per_step": int(W.ref.nbytes + W.query.nbytes),
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "clocks": clock_info,
    }
    if is_range:
        line["counters"]["results"] = int(res["off"][-1].item())
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        nb = 16
        t0 = time.perf_counter()
        oracle_call(W.ref, W.query[:nb], k)
        dt_ = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": nb / dt_, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"float64 brute force (numpy, one thread) for the first {nb} "
                                          f"queries against all {len(W.ref)} references; {dt_:.1f} s"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# the Euclidean minimum spanning tree (--op emst)
# ---------------------------------------------------------------------------

METRIC_EMST = "exact Euclidean MST points/s (oracle-identical edges)"


def run_emst(args, rank, world, local):
    """One step = build the tree + dtree_emst (Boruvka rounds) on --n-ref
    uniform points in d = 3 (the mixture of the kNN workload at d = 16 takes
    seconds per round; see the design notes).  One problem per GPU: under
    torchrun every rank solves its own point set."""
    from oracle import emst as oemst
    n = args.n_ref or 1_000_000
    P = inputs.uniform(n, 3, 7 + rank)
    workload = f"emst: uniform U[0,1]^3, N={n:,}, leaf {args.leaf}"
    if args.impl == "reference":
        if rank != 0:
            return
        m = 2000
        times = []
        for step in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            oemst.emst_kruskal(P[:m])
            if step >= args.warmup:
                times.append(time.perf_counter() - t0)
        t = sum(times) / len(times)
        print(json.dumps({"impl": "reference", "metric": METRIC_EMST, "value": m / t, "unit": "points/s",
                          "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
                          "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                          "config": {"workload": workload, "step": f"Kruskal on the first {m} points"},
                          "cpu_baseline": {"value": m / t, "unit": "points/s", "cores": 1, "kind": "oracle",
                                           "sample": f"float64 Kruskal over all pairs of the first {m} points"},
                          "e2e": {"value": m / t, "unit": "points/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}), flush=True)
        return
    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1304_4327_gb300 import dtree
    p_d = torch.from_numpy(P).cuda()
    stream = torch.cuda.current_stream()
    res = {}

    def step(pts):
        t = dtree.dtree_build(pts, args.leaf)
        try:
            res["e"], res["d"], st = dtree.dtree_emst(t, with_stats=True)
        finally:
            t.free()
        return st

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(args.warmup):
        step(p_d)
    props = torch.cuda.get_device_properties(local)
    uuid = getattr(props, "uuid", None)
    clocks = ClockSampler(f"GPU-{uuid}" if uuid else None)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = dtree.launch_count()
    # the points (12 MB) fit the 129 MB L2: before every timed step a 256 MB
    # buffer is written, outside the step's events
    l2_flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    total, stats = 0.0, []
    for _ in range(args.steps):
        l2_flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        stats.append(step(p_d))
        e1.record(stream)
        torch.cuda.synchronize()
        total += e0.elapsed_time(e1)
    barrier()
    clock_info = clocks.stop()
    launches = dtree.launch_count() - launches0
    ms_max = max_over_ranks(total / args.steps, world, "cuda")
    value = job_rate(world, n, ms_max)
    p_h = torch.from_numpy(P).pin_memory()
    p_e = torch.empty_like(p_d)
    barrier()
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # one untimed iteration first: the first copies through freshly pinned buffers
    for it in range(args.e2e_steps + 1):
        if it == 1:
            f0.record(stream)
        p_e.copy_(p_h, non_blocking=True)
        step(p_e)
        res["e"].to("cpu", non_blocking=True)
        res["d"].to("cpu", non_blocking=True)
    f1.record(stream)
    torch.cuda.synchronize()
    e2e_value = job_rate(world, n, max_over_ranks(f0.elapsed_time(f1) / args.e2e_steps, world, "cuda"))
    ns = sum(s["ns_basecase"] for s in stats) / len(stats)
    pairs = sum(s["point_pairs"] for s in stats) / len(stats)
    line = {
        "metric": METRIC_EMST, "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload, "step": "build tree + dtree_emst (Boruvka rounds)",
                   "l2": "inputs (12 MB) fit the 129 MB L2: a 256 MB buffer is written before each timed step, outside its events",
                   "parallelism": f"{world} GPU(s), one problem each"},
        "roofline": {"bound": "fp64", "kernel": "k_emst_nn (one warp per point, float64 distances)",
                     "achieved": None, "peak": None, "unit": None, "frac": None, "traffic": None,
                     "note": "the float64 pipe is the limit (about 80% busy in the ncu capture, "
                             "profiles/k_emst_nn_uniform3.md); no algorithmic-flop count is claimed"},
        "phases_ms": {"emst": ns / 1e6, "build_and_rest": ms_max - ns / 1e6},
        "counters": {"point_pairs": pairs, "leaf_pairs_evaluated": stats[-1]["leaf_pairs_evaluated"]},
        "e2e": {"value": e2e_value, "unit": "points/s", "h2d_bytes_per_step": int(P.nbytes),
                "d2h_bytes_per_step": int((n - 1) * (16 + 4))},
        "gpu_launches": int(launches),
        "clocks": clock_info,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        m = 2000
        t0 = time.perf_counter()
        oemst.emst_kruskal(P[:m])
        dt_ = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": m / dt_, "unit": "points/s", "cores": 1, "kind": "oracle",
                                "sample": f"float64 Kruskal over all pairs of the first {m} points; {dt_:.1f} s"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
