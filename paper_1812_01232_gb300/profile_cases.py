"""Small, fixed GPU workloads for profiler captures (ncu), one per kernel family.

    python -m paper_1812_01232_gb300.profile_cases stress --cubes 4096 --reps 2
    python -m paper_1812_01232_gb300.profile_cases mlp --steps 4
    python -m paper_1812_01232_gb300.profile_cases batch --problems 64 --max-nodes 100000
    python -m paper_1812_01232_gb300.profile_cases sma --seeds 1216 --precision 32
    python -m paper_1812_01232_gb300.profile_cases mixgen --points 100000 --passes 30
    python -m paper_1812_01232_gb300.profile_cases tiny --problems 8 --reps 1

stress  Theorem 1 bounds of `cubes` sub-cubes of the 2048 x 512 stress problem
        (device buffers), `reps` launches of the bound kernel.
mlp     `steps` training steps of the queue-ordering network on 65,536 random
        rows (batch 4,096): forward, backward and Adam on the tensor cores.
batch   one batched solve of `problems` uneven problems (tiny generator,
        n1 ~ U{16..256}, n2 ~ U{8..128}) with a per-problem node limit.
sma     SMA from `seeds` seed poses of the 128 x 64 paper-scale problem
        (half near the true pose, half uniform over the domain), `reps`
        launches of the batched refinement at the given precision.
mixgen  DP-means of `points` points of the synthetic indoor scene
        (lambda 2 m^2) with at most `passes` passes, then DP-vMF-means of as
        many bearing vectors (12-degree threshold).
tiny    the tiny problems 200000.. (10 x 8 components) solved one after the
        other to the certificate by the single-problem solver (eps 1e-3,
        automatic pop, 2^26-node queue), `reps` times.
Each prints one line of timing so that the plain run can be compared.
"""
from __future__ import annotations

import argparse
import sys
import time

import numpy as np

from . import learn, synth
from .gosma import Gosma


def stress(a):
    import torch
    prob = synth.stress_problem(4000)
    ctx = Gosma(0)
    ctx.set_problem(prob)
    cubes = synth.tree_cubes(4001, a.cubes, prob["t_lo"], prob["t_hi"], 2, 12,
                             near=(prob["r_gt"], prob["t_gt"]), near_frac=0.3)
    dc = torch.from_numpy(cubes).cuda()
    lb = torch.empty(len(cubes), dtype=torch.float64, device="cuda")
    ub = torch.empty_like(lb)
    ctx.eval_bounds(dc, lb, ub)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(a.reps):
        ctx.eval_bounds(dc, lb, ub)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / a.reps
    n1, n2 = len(prob["sigma1"]), len(prob["kappa2"])
    # self sums are computed once per distinct translation cuboid of the call
    cuboids = len(np.unique(np.ascontiguousarray(cubes[:, 4:10]), axis=0))
    print("stress: %d cubes (%d distinct translation cuboids), %.3f ms per call, %.3e cross pairs/s, "
          "%.3e self pairs computed/s" % (len(cubes), cuboids, 1e3 * dt, len(cubes) * n1 * n2 / dt,
                                         cuboids * n1 * (n1 - 1) / 2 / dt))


def mlp(a):
    ctx = Gosma(0)
    rng = np.random.default_rng(0)
    n = 65536
    x = rng.standard_normal((n, 16)).astype(np.float32)
    label = (rng.random(n) < 0.2).astype(np.float32)
    target = rng.uniform(-1, 1, (n, 6)).astype(np.float32)
    ctx.mlp_set_params(learn.init_params(0))
    t0 = time.perf_counter()
    losses = ctx.mlp_train(x, label, target, batch=4096, steps=a.steps, lr=1e-3)
    dt = time.perf_counter() - t0
    y = ctx.mlp_forward(x)
    print("mlp: %d steps in %.3f s, loss %.4f -> %.4f, forward %d rows ok=%s" % (
        a.steps, dt, losses[0], losses[-1], n, bool(np.isfinite(y).all())))


def batch(a):
    ctx = Gosma(0)
    probs = synth.uneven_problems(3000, count=a.problems)
    t0 = time.perf_counter()
    res = ctx.bnb_solve_batch(probs, eps=1e-3, pop=64, max_nodes=a.max_nodes, queue_capacity=1 << 20)
    dt = time.perf_counter() - t0
    pairs = sum(r["cross_pairs"] for r in res)
    print("batch: %d problems, %.3f s wall, %.3f s device, %.3e pairs/s, block %d" % (
        len(res), dt, res[0]["iteration_ms"] / 1e3, pairs / (res[0]["iteration_ms"] / 1e3), res[0]["block_size"]))


def sma(a):
    import torch
    prob = synth.paper_scale_problem(7)
    ctx = Gosma(0)
    ctx.set_problem(prob)
    xs = torch.from_numpy(synth.pose_seeds(prob, a.seeds, 8)).cuda()
    xo = torch.empty_like(xs)
    f = torch.empty(a.seeds, dtype=torch.float64, device="cuda")
    it = torch.empty(a.seeds, dtype=torch.int32, device="cuda")
    ctx.sma_batch(xs, 100, a.precision, xo, f, None, it)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(a.reps):
        ctx.sma_batch(xs, 100, a.precision, xo, f, None, it)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / a.reps
    print("sma: %d seeds, precision %d, %.3f ms per call, %.0f seeds/s, median iterations %d" % (
        a.seeds, a.precision, 1e3 * dt, a.seeds / dt, int(it.median().item())))


def mixgen(a):
    prob = synth.scene_points(11, n=a.points, n_bear=a.points)
    ctx = Gosma(0)
    t0 = time.perf_counter()
    r = ctx.dp_means(prob["points"], 2.0, max_iter=a.passes)
    t1 = time.perf_counter()
    v = ctx.dp_vmf_means(prob["bearings"], float(np.cos(np.radians(12.0))), max_iter=a.passes)
    t2 = time.perf_counter()
    print("mixgen: %d points -> %d clusters in %d passes, %.3f s; %d vectors -> %d clusters in %d passes, %.3f s" % (
        a.points, r["k"], r["passes"], t1 - t0, a.points, v["k"], v["passes"], t2 - t1))


def tiny(a):
    probs = [synth.tiny_problem(200000 + s) for s in range(a.problems)]
    ctx = Gosma(0)
    for _ in range(a.reps):
        t0 = time.perf_counter()
        nodes = 0
        for p in probs:
            ctx.set_problem(p)
            nodes += ctx.bnb_solve(eps=1e-3, max_seconds=60, queue_capacity=1 << 26)["nodes"]
        print("tiny: %d problems, %d nodes, %.3f s" % (a.problems, nodes, time.perf_counter() - t0))


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    sub = ap.add_subparsers(dest="case", required=True)
    s = sub.add_parser("stress")
    s.add_argument("--cubes", type=int, default=4096)
    s.add_argument("--reps", type=int, default=2)
    m = sub.add_parser("mlp")
    m.add_argument("--steps", type=int, default=4)
    b = sub.add_parser("batch")
    b.add_argument("--problems", type=int, default=64)
    b.add_argument("--max-nodes", type=int, default=100000)
    q = sub.add_parser("sma")
    q.add_argument("--seeds", type=int, default=1216)
    q.add_argument("--precision", type=int, default=32)
    q.add_argument("--reps", type=int, default=2)
    g = sub.add_parser("mixgen")
    g.add_argument("--points", type=int, default=100000)
    g.add_argument("--passes", type=int, default=30)
    t = sub.add_parser("tiny")
    t.add_argument("--problems", type=int, default=8)
    t.add_argument("--reps", type=int, default=1)
    a = ap.parse_args(argv)
    {"stress": stress, "mlp": mlp, "batch": batch, "sma": sma, "mixgen": mixgen, "tiny": tiny}[a.case](a)
    return 0


if __name__ == "__main__":
    sys.exit(main())
