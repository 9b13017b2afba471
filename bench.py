#!/usr/bin/env python
"""Benchmark of the GOSMA branch-and-bound hot path on GB300.

Metric: pair-bound evaluations per second, counting (sub-cube, model
component i, image component j) cross pairs, each bounded from below and
evaluated at the centre (Theorem 1).  A step is one full iteration of
Algorithm 1 on the device: radix-select pop of 8,192 parents, branching into
65,536 children, the bound kernel, pruning/appending by scan, the smallest
live key, and the FP64 incumbent refinement (SMA) when a child improves d*.

Workload: one 128 x 64 component problem (10 x 10 x 3 m room, sigma in
U[0.03, 0.1], Dirichlet weights, 48 noisy inliers + 16 outliers, kappa in
U[20, 200], translation domain [-2, 2]^3, eps = 1e-4), seeded synthetic.
Steps are taken after the queue holds at least 8,192 live sub-cubes, so
every timed step bounds exactly 65,536 children.  L2 is flushed (a 512 MB
write) between timed steps, outside the timed region.

e2e: the same metric through gosma_eval_bounds with host buffers: every step
copies a batch of 65,536 sub-cubes of the same tree depths from host memory
and reads back their lower and upper bounds.

--batch-only (with --batch-budget and --batch-queue): just the batched
measurement, autotuned shape only (a long documented run of the 256 uneven
problems with large queues).

--impl reference: the FP64 CPU oracle, as it stands, on the host cores, on a
bounded sample of the same workload per step (sub-cubes of the same problem
at tree depths 2-12, Theorem 1 bounds; --ref-seconds of host time spread over
the warm-up and timed steps, 150 s by default, at least 0.25 s a step).

Multi-GPU (torchrun): every rank solves its own independent problem (seed +
rank); no data-path collective; value = pairs of all ranks / max rank time.

Two more measurements ride on the same line (rank 0, N = 1, unless
--no-extra):
* "batched": 256 independent problems of uneven sizes (model components
  U{16..256}, image U{8..128} with 20% outliers, tiny-problem generator,
  eps 1e-3) in one batched solve (one captured CUDA graph per iteration)
  under a time budget: aggregate pair-bound evals/s and per-problem time to
  the certified optimum (p50/p99 over the problems certified in the budget,
  with the count), with the bound kernel's shape picked by the autotuner and,
  on the same problems and budget, with the fixed default shape (128
  threads, one sub-cube per block);
* "time_to_certified": tiny problems (10 x 8 components, eps 1e-3) solved
  to the certified optimum by the plain single-problem solver (one after the
  other), the plain batched solver and the learned batched solver (network
  weights from paper_1812_01232_gb300/weights, scoring during the first 8
  iterations, about the first 10% of the nodes, where the incumbent is
  found), on the same problems, each with its automatic pop, three times
  each (median wall time; the iteration of the final incumbent shows what
  the network's seeds change);
* "psi_r_point": the same tiny problems solved by the single-problem solver
  with the point-independent and the point-dependent rotation uncertainty
  angle (Lemma 2): nodes and wall time (median of three) to the certified
  optima;
* "sma": the batched device refinement (SMA, Sec. 5) of many seed poses of
  the 128 x 64 paper-scale problem (half near the true pose, half uniform),
  seeds refined per second with the FP32 and the FP64 search (CUDA events
  around the whole call, the FP64 f of the results included), beside the
  oracle's L-BFGS on one host core;
* "mixgen": mixture generation (Sec. 6) for a synthetic indoor scene at the
  size the paper downsamples to: DP-means of 100k points (lambda 2 m^2) and
  DP-vMF-means of 100k bearing vectors (12-degree threshold), scales that
  give 60-100 components as the paper's real-data runs choose them, 30
  passes each, through the host-buffer C-ABI calls, beside the oracle on one
  core; and at the paper's default scales (0.25 m, 2 degrees: thousands of
  clusters), the oracle timed over the first two passes.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pair-bound evals/s (cube*i*j/s)"
UNIT = "pairs/s"
POP = 8192
SEED = 2000
# FP32-pipe lane operations per pair the bound kernel executes, counted from
# the source of cross_pair2 / self_pair2 (packed FP32x2 instructions count
# as two): geometry 12, centre term 15 (cross) or 16 (self), bound term 36
# (cross) or 58 (self), and 1.5 per pair for the chunked compensated
# accumulation.
OPS_CROSS = 65
OPS_SELF = 88
FP32_LANES_PER_SM = 128
# Algorithmic work per pair bound, counted from the kernel's closed forms of
# Theorem 1 (the bound) and Lemma 1 (the centre term) without its
# outward-rounding allowances, double-float low parts and compensated sums:
# |v -+ u|^2 12, centre term 14, bound term 31 FP32 operations; 5 sqrt
# (sin and cos of theta/2, K at the centre, the largest and the smallest K),
# 2 rcp and 2 ex2 on the multi-function unit.  The self pairs are counted
# alike (their four-corner K maximum makes them dearer, so this undercounts).
ALG_FP32_PER_PAIR = 57
ALG_MUFU_MIX = {"sqrt": 5, "rcp": 2, "ex2": 2}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons (every 50 ms)
    from the pipe-rate probes through the warm-up to the end of the timed
    region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.p = None
        self.path = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "50"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def lines(self):
        """Samples written so far."""
        if self.p is None:
            return 1 << 30
        self.f.flush()
        try:
            with open(self.path) as f:
                return sum(1 for _ in f)
        except OSError:
            return 0

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.p is None:
            return out
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if sm:
            out = {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                   "samples": len(sm), "window": "every 50 ms from the pipe-rate probes through the warm-up "
                                                 "to the end of the timed steps"}
        return out


def _code_only(text):
    """Source text without comments and blank lines (the fingerprint follows
    the code, not its commentary)."""
    import re
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(line.rstrip() for line in text.split("\n") if line.strip())


def kernel_source_sha256():
    """Fingerprint of the bound kernel's device code: the bound core, the
    double-float helpers, the queue-node helpers and the kernel function,
    comments left out."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_1812_01232_gb300", "csrc")
    h = hashlib.sha256()
    for f in ("bounds_core.cuh", "dfloat.cuh", "bnb_common.cuh"):
        h.update(_code_only(open(os.path.join(csrc, f)).read()).encode())
    src = open(os.path.join(csrc, "bnb.cu")).read()
    i = src.index("bound_children(MixDev mx")
    j = src.index("\n}\n", i)
    h.update(_code_only(src[i:j]).encode())
    return h.hexdigest()


def kernel_traffic():
    """DRAM bytes per launch of the bound kernel from the committed ncu capture,
    or None when the kernel's device code changed since the capture."""
    prof = os.path.join(ROOT, "profiles", "bound_children_traffic.txt")
    if not os.path.exists(prof):
        return None
    rec = json.load(open(prof))
    return rec.get("bytes_per_launch") if rec.get("source_sha256") == kernel_source_sha256() else None


def reduce_over_ranks(t_local, pairs_local, dist, device):
    """Whole-job aggregation over the ranks: the slowest rank's time and the
    pairs of all ranks (every rank works on its own problem)."""
    if dist is None:
        return t_local, float(pairs_local)
    import torch
    tt = torch.tensor([t_local], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    pp = torch.tensor([float(pairs_local)], dtype=torch.float64, device=device)
    dist.all_reduce(pp)
    return float(tt.item()), float(pp.item())


def workload_config(n1, n2):
    """The workload both arms are quoted on (the `config` of either JSON line)."""
    return {"workload": "paper_scale: one problem per GPU, 128 model x 64 image components, "
                        "branch-and-bound step of %d parents -> %d children, eps 1e-4" % (POP, 8 * POP),
            "n1": n1, "n2": n2, "children_per_step": 8 * POP, "l2": "flushed between steps (512 MB write)"}


def make_problem(rank):
    from paper_1812_01232_gb300 import synth
    return synth.paper_scale_problem(SEED + rank)


def cube_pool(prob, seed):
    """65,536 sub-cubes of the problem at tree depths 2-12 (drawn once; the
    samples below take windows of it)."""
    from paper_1812_01232_gb300 import synth
    return synth.tree_cubes(seed, 65536, prob["t_lo"], prob["t_hi"], 2, 12)


def cpu_sample(prob, target_s, pool, start=0):
    """Time the FP64 oracle's Theorem 1 bounds on a bounded sample of cubes:
    about `target_s` seconds of consecutive cubes of `pool` from `start`
    (wrapping around)."""
    import oracle
    mix = oracle.Mixtures.from_problem(prob)
    n1, n2 = len(prob["sigma1"]), len(prob["kappa2"])

    def window(n):
        return np.ascontiguousarray(pool[(start + np.arange(n)) % len(pool)])

    n = 16
    t0 = time.perf_counter()
    oracle.bounds(mix, window(n), prob["zeta"])
    dt = time.perf_counter() - t0
    n = int(min(len(pool), max(16, n * target_s / max(dt, 1e-6))))
    cubes = window(n)
    t0 = time.perf_counter()
    oracle.bounds(mix, cubes, prob["zeta"])
    dt = time.perf_counter() - t0
    return n, dt, n * n1 * n2 / dt, oracle.max_threads()


# Counting rule shared by both arms.  `value` counts cross pairs (cube, i, j)
# only, the metric's unit.  Both arms also bound self pairs, in different
# amounts: the oracle bounds every self pair of every sub-cube, the device
# step only those of sub-cubes whose translation cuboid changed (a rotation
# split keeps the parent's cached self sums).  `all_pairs_per_s` counts the
# work each arm did: cross pairs plus the distinct off-diagonal self pairs
# (i < m) it bounded, n1 (n1 - 1) / 2 per sub-cube that computed its self sums.
COUNTING_RULE = ("value counts cross pairs (cube*i*j); all_pairs_per_s adds the distinct self pairs i < m the arm "
                 "bounded: the oracle bounds n1(n1-1)/2 for every sub-cube, the device step only for sub-cubes "
                 "whose translation cuboid changed")


def oracle_all_pairs(n, n1, n2):
    """Cross plus distinct off-diagonal self pairs the oracle bounds for n sub-cubes."""
    return n * (n1 * n2 + n1 * (n1 - 1) // 2)


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    prob = make_problem(0)
    n1, n2 = len(prob["sigma1"]), len(prob["kappa2"])
    per_step = max(0.25, args.ref_seconds / max(1, args.steps + args.warmup))
    pool = cube_pool(prob, 100)
    for k in range(args.warmup):
        cpu_sample(prob, min(per_step, 2.0), pool, 7919 * k)
    tot_pairs, tot_t, cubes = 0.0, 0.0, 0
    for k in range(args.steps):
        n, dt, _, cores = cpu_sample(prob, per_step, pool, cubes)
        tot_pairs += n * n1 * n2
        tot_t += dt
        cubes += n
    value = tot_pairs / tot_t
    all_rate = oracle_all_pairs(cubes, n1, n2) / tot_t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(n1, n2),
        "all_pairs_per_s": all_rate, "counting_rule": COUNTING_RULE,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "all_pairs_per_s": all_rate,
                         "sample": "%d sub-cubes over %d steps, Theorem 1 lb+ub in FP64, every sub-cube's self "
                                   "pairs bounded too (%s)" % (cubes, args.steps, COUNTING_RULE)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1812_01232_gb300 import synth
    from paper_1812_01232_gb300.gosma import Gosma
    prob = make_problem(rank)
    ctx = Gosma(local)
    # clock sampling from here to the end of the timed steps: the pipe-rate
    # probes, the warm-up and the timed steps all keep the GPU busy
    clocks = Clocks(local)
    clocks.start()
    rates = ctx.selftest_pipe_rates()  # measured pipe throughputs (lanes per SM per clock)
    ctx.set_problem(prob)
    n1, n2 = ctx.n1, ctx.n2
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    # ---------------- warm-up: grow the queue until a full pop is possible, then W steps
    ctx.bnb_start(eps=prob["eps"], pop=POP, queue_capacity=args.queue_capacity)
    r = ctx.bnb_step(1)
    while r["queue_size"] < POP and r["status_name"] == "running":
        r = ctx.bnb_step(1)
    for _ in range(args.warmup):
        r = ctx.bnb_step(1)
    if r["status_name"] != "running":
        raise RuntimeError("branch-and-bound stopped during warm-up: %s" % r["status_name"])

    # the sampler's first samples before the timed steps: L2-flush writes keep
    # the GPU busy meanwhile (at most 3 s), without stepping the solver
    t_wait = time.perf_counter()
    while clocks.lines() < 2 and time.perf_counter() - t_wait < 3.0:
        flush.zero_()
        torch.cuda.synchronize()

    # ---------------- timed steps
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    times = []
    pairs = 0
    self_pairs = 0
    b0, l0 = r["bound_ms"], r["launches"]
    bound_ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        prev = r
        r = ctx.bnb_step(1)
        e1.record(stream)
        torch.cuda.synchronize()
        if r["iterations"] != prev["iterations"] + 1 or r["cross_pairs"] - prev["cross_pairs"] != 8 * POP * n1 * n2:
            raise RuntimeError("a timed step did not bound a full batch")
        times.append(e0.elapsed_time(e1))
        pairs += r["cross_pairs"] - prev["cross_pairs"]
        self_pairs += r["self_pairs"] - prev["self_pairs"]
    bound_ms = r["bound_ms"] - b0
    launches = r["launches"] - l0
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ck = clocks.stop()
    t_total, pairs_all = reduce_over_ranks(sum(times) / 1e3, pairs, dist, "cuda")
    _, self_all = reduce_over_ranks(0.0, self_pairs, dist, "cuda")
    value = pairs_all / t_total

    # ---------------- e2e through the host-buffer C-ABI call
    cubes = synth.tree_cubes(SEED + 17 + rank, 8 * POP, prob["t_lo"], prob["t_hi"], 2, 12)
    n_cuboids = int(len(np.unique(np.ascontiguousarray(cubes[:, 4:10]), axis=0)))
    ctx.eval_bounds(cubes)  # warm the staging buffers
    e2e_t = []
    for _ in range(max(3, args.steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lb, ub = ctx.eval_bounds(cubes)
        e2e_t.append(time.perf_counter() - t0)
    e2e_value = 8 * POP * n1 * n2 / float(np.mean(e2e_t))

    # ---------------- roofline of the bound kernel: algorithmic operations against the measured
    # rates of the FP32 pipe (packed FMA) and the multi-function unit; the binding pipe is the roofline
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count
    max_mhz = ck["sm_max_mhz"] or rates["clock_mhz"]
    sec = bound_ms / 1e3
    alg_pairs = pairs + self_pairs
    fp32_peak = sm_count * rates["ffma2"] * max_mhz * 1e6 / 1e9  # Gop/s
    # effective MUFU rate of the mix (harmonic: the cycles of a pair's operations add up)
    mufu_n = sum(ALG_MUFU_MIX.values())
    mufu_rate = mufu_n / sum(k / rates[op] for op, k in ALG_MUFU_MIX.items())
    mufu_peak = sm_count * mufu_rate * max_mhz * 1e6 / 1e9  # Gop/s
    alg_fp32 = ALG_FP32_PER_PAIR * alg_pairs / sec / 1e9
    alg_mufu = mufu_n * alg_pairs / sec / 1e9
    binding = "mufu" if alg_mufu / mufu_peak >= alg_fp32 / fp32_peak else "fp32"
    unit_peak = sm_count * FP32_LANES_PER_SM * max_mhz * 1e6 / 1e9
    executed = (OPS_CROSS * pairs + OPS_SELF * self_pairs) / sec / 1e9
    traffic = kernel_traffic()
    roof = {
        "bound": "alu", "binding_pipe": binding,
        "achieved": alg_mufu if binding == "mufu" else alg_fp32,
        "peak": mufu_peak if binding == "mufu" else fp32_peak,
        "unit": "Gop/s (%s, algorithmic)" % ("MUFU" if binding == "mufu" else "FP32"),
        "traffic": traffic, "kernel": "bound_children", "kernel_ms_per_step": bound_ms / args.steps,
        "pairs_per_step": alg_pairs / args.steps,
        "algorithmic": {"fp32_ops_per_pair": ALG_FP32_PER_PAIR, "mufu_ops_per_pair": mufu_n,
                        "mufu_mix": ALG_MUFU_MIX, "fp32_achieved": alg_fp32, "fp32_peak": fp32_peak,
                        "fp32_frac": alg_fp32 / fp32_peak, "mufu_achieved": alg_mufu, "mufu_peak": mufu_peak,
                        "mufu_frac": alg_mufu / mufu_peak, "unit": "Gop/s"},
        "peak_basis": "%d SMs x the measured lanes per SM per clock x %.0f MHz: FP32 %.1f (packed FMA), MUFU "
                      "%.1f (the sqrt/rcp/ex2 rates weighted by the mix %s); gosma_selftest_pipe_rates, 8 "
                      "independent chains per thread, 2048 threads per SM, CUDA events"
                      % (sm_count, max_mhz, rates["ffma2"], mufu_rate, ALG_MUFU_MIX),
        "fp32_executed": {"ops_per_cross_pair": OPS_CROSS, "ops_per_self_pair": OPS_SELF, "achieved": executed,
                          "peak": unit_peak, "frac": executed / unit_peak, "unit": "Gop/s",
                          "peak_basis": "%d SMs x %d FP32 lanes x %.0f MHz (unit count)"
                                        % (sm_count, FP32_LANES_PER_SM, max_mhz)},
        "measured_pipe_rates": rates,
    }
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["frac_algorithmic"] = roof["frac"]

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    # ---------------- CPU baseline: the oracle on a bounded sample (rank 0, N = 1 only)
    cpu = None
    if world == 1 and not args.no_cpu:
        import oracle
        oracle.build()
        n, dt, v, cores = cpu_sample(prob, args.cpu_seconds, cube_pool(prob, 99))
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "all_pairs_per_s": oracle_all_pairs(n, n1, n2) / dt,
               "sample": "%d sub-cubes of the same workload (depths 2-12), Theorem 1 lb+ub in FP64, every "
                         "sub-cube's self pairs bounded too, %.1f s (%s)" % (n, dt, COUNTING_RULE)}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 pair terms, f64 per-cube sums", "data": "synthetic",
        "config": dict(workload_config(n1, n2), self_pairs_per_step=self_pairs / args.steps,
                       queue_size_end=r["queue_size"]),
        "all_pairs_per_s": (pairs_all + self_all) / t_total, "counting_rule": COUNTING_RULE,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(cubes.nbytes),
                "d2h_bytes_per_step": int(2 * 8 * len(cubes)),
                "call": "gosma_eval_bounds on host buffers, %d sub-cubes per step (self sums computed once per "
                        "distinct translation cuboid; %d distinct)" % (len(cubes), n_cuboids)},
        "roofline": roof,
        "cpu_baseline": cpu,
        "clocks": ck,
        "gpu_launches": launches,
    }
    if world == 1 and not args.no_extra:
        ctx.close()
        line["batched"] = run_batched(args.batch_budget, args.batch_queue)
        line["time_to_certified"] = run_time_to_certified(8)
        line["psi_r_point"] = run_psi_r_point(8)
        line["sma"] = run_sma()
        line["mixgen"] = run_mixgen()
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_batched(budget_s, queue=1 << 20, compare_fixed=True):
    """Config of 256 uneven problems in one batched solve (see module doc):
    the autotuned bound-kernel shape, and the fixed default shape (128
    threads, one sub-cube per block) on the same problems and budget."""
    from paper_1812_01232_gb300 import synth
    from paper_1812_01232_gb300.gosma import Gosma
    ctx = Gosma(0)
    probs = synth.uneven_problems(3000, count=256)
    out = {"workload": "256 problems, n1 ~ U{16..256}, n2 ~ U{8..128}, 20%% outliers, eps 1e-3, pop 64 per problem, "
                       "queue %d per problem, budget %.0f s" % (queue, budget_s)}
    for name, shape in (("tuned", None), ("fixed_128x1", (128, 1))) if compare_fixed else (("tuned", None),):
        t0 = time.perf_counter()
        res = ctx.bnb_solve_batch(probs, eps=1e-3, pop=64, max_seconds=budget_s, queue_capacity=queue, shape=shape)
        wall = time.perf_counter() - t0
        dev_s = res[0]["iteration_ms"] / 1e3
        pairs = float(sum(r["cross_pairs"] for r in res))
        cert = [r["seconds"] for r in res if r["status_name"] == "optimal"]
        st = [r["status_name"] for r in res]
        row = {"pairs_per_s": pairs / dev_s, "device_s": dev_s, "wall_s": wall,
               "certified": len(cert), "statuses": {k: st.count(k) for k in sorted(set(st))},
               "p50_s": float(np.percentile(cert, 50)) if cert else None,
               "p99_s": float(np.percentile(cert, 99)) if cert else None,
               "queue_peak_max": int(max(r["queue_peak"] for r in res)),
               "shape": [res[0]["block_size"], res[0]["cubes_per_block"]], "tunings": res[0]["tunings"]}
        if name == "tuned":
            out.update(row)
        else:
            out[name] = row
    if compare_fixed:
        out["tuned_over_fixed"] = out["pairs_per_s"] / out["fixed_128x1"]["pairs_per_s"]
    ctx.close()
    return out


def run_sma():
    """Seeds refined per second by gosma_sma_batch (see module doc)."""
    import torch
    from paper_1812_01232_gb300 import synth
    from paper_1812_01232_gb300.gosma import Gosma
    import oracle
    prob = synth.paper_scale_problem(7)
    ctx = Gosma(0)
    ctx.set_problem(prob)
    out = {"workload": "128 x 64 paper-scale problem, seeds half near the true pose, half uniform, up to 100 L-BFGS "
                       "iterations each"}
    for prec, n in ((32, 152 * 32), (64, 152 * 4)):
        xs = torch.from_numpy(synth.pose_seeds(prob, n, 8)).cuda()
        xo = torch.empty_like(xs)
        f = torch.empty(n, dtype=torch.float64, device="cuda")
        it = torch.empty(n, dtype=torch.int32, device="cuda")
        ctx.sma_batch(xs[:152], 100, prec, xo[:152], f[:152], None, it[:152])  # warm-up
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        ctx.sma_batch(xs, 100, prec, xo, f, None, it)
        e1.record()
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) / 1e3
        out["fp%d" % prec] = {"seeds": n, "seconds": sec, "seeds_per_s": n / sec,
                              "median_iterations": int(it.median().item())}
    ctx.close()
    mix = oracle.Mixtures.from_problem(prob)
    x0 = synth.pose_seeds(prob, 8, 8)
    t0 = time.perf_counter()
    for x in x0:
        oracle.sma(mix, x, prob["t_lo"], prob["t_hi"], prob["zeta"], max_iter=100, memory=8, gtol=1e-10)
    sec = time.perf_counter() - t0
    out["oracle"] = {"seeds": len(x0), "seconds": sec, "seeds_per_s": len(x0) / sec, "cores": 1, "kind": "oracle"}
    return out


def run_mixgen():
    """Mixture generation of a 100k-point scene (see module doc)."""
    from paper_1812_01232_gb300 import synth
    from paper_1812_01232_gb300.gosma import Gosma
    import oracle
    sc = synth.scene_points(11)
    ctx = Gosma(0)
    lam_v = float(np.cos(np.radians(12.0)))
    ctx.dp_means(sc["points"][:1000], 2.0, max_iter=2)  # warm-up
    out = {"workload": "100k scene points (lambda 2 m^2) and 100k bearing vectors (cosine threshold cos 12 deg), "
                       "30 passes each, host buffers"}
    for name, call in (("dp_means", lambda: ctx.dp_means(sc["points"], 2.0, max_iter=30)),
                       ("dp_vmf_means", lambda: ctx.dp_vmf_means(sc["bearings"], lam_v, max_iter=30))):
        t0 = time.perf_counter()
        r = call()
        sec = time.perf_counter() - t0
        out[name] = {"seconds": sec, "clusters": r["k"], "passes": r["passes"]}
    # the paper's default scale parameters (lambda_p = 0.25 m, lambda_f = 2 deg): thousands of clusters
    lam_f = float(np.cos(np.radians(2.0)))
    dflt = {"workload": "the same scene at lambda_p 0.25 m (0.0625 m^2 penalty) and lambda_f 2 deg, 30 passes "
                        "at most; the oracle runs the first 2 passes"}
    for name, call in (("dp_means", lambda: ctx.dp_means(sc["points"], 0.0625, max_iter=30, kmax=8192)),
                       ("dp_vmf_means", lambda: ctx.dp_vmf_means(sc["bearings"], lam_f, max_iter=30, kmax=8192))):
        t0 = time.perf_counter()
        r = call()
        sec = time.perf_counter() - t0
        dflt[name] = {"seconds": sec, "clusters": r["k"], "passes": r["passes"]}
    ctx.close()
    t0 = time.perf_counter()
    oracle.dp_cluster(sc["points"], 2.0, max_iter=30)
    t1 = time.perf_counter()
    oracle.dp_cluster(sc["bearings"], lam_v, vmf=True, max_iter=30)
    t2 = time.perf_counter()
    out["oracle"] = {"dp_means_seconds": t1 - t0, "dp_vmf_means_seconds": t2 - t1, "cores": 1, "kind": "oracle"}
    t0 = time.perf_counter()
    oracle.dp_cluster(sc["points"], 0.0625, max_iter=2, kmax=8192)
    t1 = time.perf_counter()
    oracle.dp_cluster(sc["bearings"], lam_f, vmf=True, max_iter=2, kmax=8192)
    t2 = time.perf_counter()
    dflt["oracle_2_passes"] = {"dp_means_seconds": t1 - t0, "dp_vmf_means_seconds": t2 - t1, "cores": 1,
                               "kind": "oracle"}
    out["paper_defaults"] = dflt
    return out


def run_time_to_certified(n_prob, repeats=3):
    """Plain single, plain batched and learned batched solves of the same tiny
    problems, `repeats` times each (the arms interleaved); wall_s is the
    median over the repeats."""
    from paper_1812_01232_gb300 import learn, synth
    from paper_1812_01232_gb300.gosma import Gosma
    ctx = Gosma(0)
    eps = 1e-3
    probs = [synth.tiny_problem(200000 + s) for s in range(n_prob)]
    out = {"workload": "%d tiny problems (10 x 8 components), eps 1e-3, queue 2^26 per problem; every solver "
                       "with its automatic pop (65536 sub-cubes per iteration and problem for 10 x 8 mixtures); "
                       "%d repeats, wall_s the median" % (n_prob, repeats)}
    ctx.mlp_set_params(learn.load(os.path.join(ROOT, "paper_1812_01232_gb300", "weights", "gosma_mlp.npz")))
    walls = {"plain_single": [], "plain_batched": [], "learned_batched": []}
    last = {}
    for _ in range(repeats):
        single = []
        t0 = time.perf_counter()
        for p in probs:
            ctx.set_problem(p)
            single.append(ctx.bnb_solve(eps=eps, max_seconds=60, queue_capacity=1 << 26))
        walls["plain_single"].append(time.perf_counter() - t0)
        last["plain_single"] = single
        for name, learned in (("plain_batched", None),
                              ("learned_batched", {"beta": 1e-4, "seed": True, "active_iters": 8})):
            t0 = time.perf_counter()
            last[name] = ctx.bnb_solve_batch(probs, eps=eps, max_seconds=120, queue_capacity=1 << 26,
                                             learned=learned)
            walls[name].append(time.perf_counter() - t0)
    single = last["plain_single"]
    for name, res in last.items():
        out[name] = {"wall_s": float(np.median(walls[name])), "wall_s_runs": [round(w, 4) for w in walls[name]],
                     "nodes": int(sum(r["nodes"] for r in res)),
                     "certified": int(sum(r["status_name"] == "optimal" for r in res)),
                     "median_dstar_iteration": float(np.median([r["dstar_iteration"] for r in res]))}
        if name != "plain_single":
            out[name].update({
                "agree_with_single": int(sum(abs(r["f"] - q["f"]) <= eps * q["c22"] for r, q in zip(res, single))),
                "p50_s": float(np.median([r["seconds"] for r in res])),
                "shape": [res[0]["block_size"], res[0]["cubes_per_block"]], "tunings": res[0]["tunings"]})
    ctx.close()
    return out


def run_psi_r_point(n_prob, repeats=3):
    """The same tiny problems solved to the certified optimum with the
    point-independent and the point-dependent rotation uncertainty angle
    (Lemma 2; gosma_set_psi_r_mode), single-problem solver, automatic pop,
    `repeats` times each (wall_s the median)."""
    from paper_1812_01232_gb300 import synth
    from paper_1812_01232_gb300.gosma import Gosma
    ctx = Gosma(0)
    probs = [synth.tiny_problem(200000 + s) for s in range(n_prob)]
    out = {"workload": "%d tiny problems (10 x 8 components), eps 1e-3, queue 2^26, automatic pop, single-problem "
                       "solver; %d repeats, wall_s the median" % (n_prob, repeats)}
    walls = {"cube": [], "point": []}
    for _ in range(repeats):
        for name, point in (("cube", False), ("point", True)):
            ctx.set_psi_r_mode(point)
            res = []
            t0 = time.perf_counter()
            for p in probs:
                ctx.set_problem(p)
                res.append(ctx.bnb_solve(eps=1e-3, max_seconds=60, queue_capacity=1 << 26))
            walls[name].append(time.perf_counter() - t0)
            out[name] = {"nodes": int(sum(r["nodes"] for r in res)),
                         "certified": int(sum(r["status_name"] == "optimal" for r in res)),
                         "f": [r["f"] for r in res]}
    ctx.set_psi_r_mode(False)
    for name in walls:
        out[name]["wall_s"] = float(np.median(walls[name]))
        out[name]["wall_s_runs"] = [round(w, 4) for w in walls[name]]
    ctx.close()
    out["node_ratio"] = out["point"]["nodes"] / max(1, out["cube"]["nodes"])
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-seconds", type=float, default=150.0,
                    help="--impl reference: host-core seconds spread over the warm-up and timed steps")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the batched and time-to-certificate measurements")
    ap.add_argument("--batch-budget", type=float, default=15.0, help="seconds for each 256-problem batched solve")
    ap.add_argument("--batch-queue", type=int, default=1 << 20, help="queue capacity per problem of the batched solve")
    ap.add_argument("--batch-only", action="store_true",
                    help="print only the batched measurement (one JSON line), autotuned shape only")
    ap.add_argument("--queue-capacity", type=int, default=1 << 27,
                    help="device queue capacity in sub-cubes (64 bytes each, twice)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.batch_only:
        print(json.dumps({"batched": run_batched(args.batch_budget, args.batch_queue, compare_fixed=False)}),
              flush=True)
        return 0
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
