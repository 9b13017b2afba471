"""Train the queue-ordering network on branch-and-bound traces and evaluate it.

    python -m paper_1812_01232_gb300.train_mlp --out weights.npz --report report.json

1. Traces: the plain batched solver runs on `--train` seeded paper-scale-style
   problems (128 x 64 components, synth.paper_scale_problem) with a node
   budget per problem; every popped sub-cube is recorded with its features
   and labelled against the best pose the run ended with (learn.py).
2. Training: Adam on the device's tensor-core kernels, positives
   oversampled.
3. Evaluation on `--held` held-out seeds (never traced):
   a. paper-scale-style problems at equal node budgets, plain vs learned
      batched solver: incumbent f / C22 + 1 and lower bound reached;
   b. tiny problems (synth.tiny_problem), which the method certifies:
      nodes and time to the eps-certified optimum for the plain
      single-problem solver, the plain batched solver and the learned
      batched solver, on the same problems.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import learn, synth
from .gosma import Gosma


def _collect(ctx, seeds, chunk, eps, pop, max_nodes, trace_cap, cap):
    F, L, T = [], [], []
    for i in range(0, len(seeds), chunk):
        probs = [synth.paper_scale_problem(int(s)) for s in seeds[i:i + chunk]]
        f, l, t, _ = learn.collect(ctx, probs, eps=eps, pop=pop, max_nodes=max_nodes, trace_cap=trace_cap,
                                   queue_capacity=cap, max_seconds=600)
        F.append(f)
        L.append(l)
        T.append(t)
    return np.concatenate(F), np.concatenate(L), np.concatenate(T)


def _auc(score, label, rng, n_neg=20000):
    pos, neg = score[label > 0.5], score[label <= 0.5]
    if len(pos) == 0 or len(neg) == 0:
        return float("nan")
    neg = rng.choice(neg, min(n_neg, len(neg)), replace=False)
    return float((pos[:, None] > neg[None, :]).mean() + 0.5 * (pos[:, None] == neg[None, :]).mean())


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--train", type=int, default=2000, help="training problems (seeds 0..)")
    ap.add_argument("--held", type=int, default=200, help="held-out problems")
    ap.add_argument("--node-budget", type=int, default=200_000, help="nodes per traced problem")
    ap.add_argument("--trace-cap", type=int, default=2048)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--beta", type=float, default=1e-4, help="priority weight (f / C22 units)")
    ap.add_argument("--eval-budgets", type=str, default="50000,200000")
    ap.add_argument("--tiny", type=int, default=24, help="tiny held-out problems for time to certificate")
    ap.add_argument("--out", required=True)
    ap.add_argument("--report", default=None)
    a = ap.parse_args(argv)
    ctx = Gosma(0)
    rng = np.random.default_rng(0)
    rep = dict(args=vars(a))
    eps2 = 1e-4

    t0 = time.time()
    F, L, T = _collect(ctx, np.arange(a.train), 250, eps2, 256, a.node_budget, a.trace_cap, 1 << 19)
    rep["traces"] = dict(rows=int(len(F)), positives=int(L.sum()), seconds=time.time() - t0)
    print("traces", rep["traces"], flush=True)

    t0 = time.time()
    params, losses = learn.train(ctx, F, L, T, steps=a.steps, batch=a.batch, lr=a.lr)
    rep["training"] = dict(loss_first=float(losses[:20].mean()), loss_last=float(losses[-20:].mean()),
                           seconds=time.time() - t0, steps=a.steps, batch=a.batch)
    print("training", rep["training"], flush=True)
    learn.save(a.out, params, train=a.train, node_budget=a.node_budget)

    held = np.arange(100000, 100000 + a.held)
    Fh, Lh, Th = _collect(ctx, held, 200, eps2, 256, a.node_budget, a.trace_cap, 1 << 19)
    ctx.mlp_set_params(params)
    y = ctx.mlp_forward(Fh)
    pos = Lh > 0.5
    rep["held_out"] = dict(rows=int(len(Fh)), positives=int(pos.sum()), auc=_auc(y[:, 0], Lh, rng),
                           seed_abs_err=float(np.abs(y[pos, 1:7] - Th[pos]).mean()) if pos.any() else None,
                           seed_abs_err_centre=float(np.abs(Th[pos]).mean()) if pos.any() else None)
    print("held-out", rep["held_out"], flush=True)

    # a. equal node budgets on held-out paper-scale-style problems
    probs = [synth.paper_scale_problem(int(s)) for s in held]
    rep["budget"] = []
    for nb in [int(x) for x in a.eval_budgets.split(",")]:
        row = dict(nodes=nb)
        for name, learned in (("plain", None), ("learned", dict(beta=a.beta, seed=True))):
            t0 = time.time()
            res = ctx.bnb_solve_batch(probs, eps=eps2, pop=256, max_nodes=nb, queue_capacity=1 << 19,
                                      max_seconds=900, learned=learned)
            row[name] = dict(wall=time.time() - t0, f_norm=float(np.mean([r["f_norm"] for r in res])),
                             gap_norm=float(np.mean([r["gap_norm"] for r in res])))
        row["learned_minus_plain_f_norm"] = row["learned"]["f_norm"] - row["plain"]["f_norm"]
        rep["budget"].append(row)
        print("budget", row, flush=True)

    # b. time to the certified optimum on tiny problems
    eps1 = 1e-3
    tiny = [synth.tiny_problem(200000 + s) for s in range(a.tiny)]
    single = []
    t0 = time.time()
    for p in tiny:
        ctx.set_problem(p)
        single.append(ctx.bnb_solve(eps=eps1, pop=1024, max_seconds=120, queue_capacity=1 << 25))
    rep["tiny"] = dict(single=dict(wall=time.time() - t0, nodes=int(sum(r["nodes"] for r in single)),
                                   optimal=int(sum(r["status_name"] == "optimal" for r in single))))
    for name, learned in (("batch_plain", None), ("batch_learned", dict(beta=a.beta, seed=True))):
        t0 = time.time()
        res = ctx.bnb_solve_batch(tiny, eps=eps1, pop=1024, max_seconds=600, queue_capacity=1 << 25,
                                  learned=learned)
        agree = sum(abs(r["f"] - s["f"]) <= eps1 * s["c22"] for r, s in zip(res, single))
        rep["tiny"][name] = dict(wall=time.time() - t0, nodes=int(sum(r["nodes"] for r in res)),
                                 optimal=int(sum(r["status_name"] == "optimal" for r in res)), agree=int(agree),
                                 p50=float(np.median([r["seconds"] for r in res])),
                                 p99=float(np.percentile([r["seconds"] for r in res], 99)))
    print("tiny", rep["tiny"], flush=True)
    if a.report:
        with open(a.report, "w") as f:
            json.dump(rep, f, indent=1)
    ctx.close()


if __name__ == "__main__":
    main()
