"""Train the queue-ordering network on branch-and-bound traces and evaluate it.

    python -m paper_1812_01232_gb300.train_mlp --out weights.npz --report report.json
    python -m paper_1812_01232_gb300.train_mlp --mode certified --train 512 --held 64 --repeats 3 \
        --out weights.npz --report report.json

Certified mode (the labels a certificate stands behind): the plain batched
solver runs `--train` tiny problems (seeds 300000..) to their eps-certified
optima, the popped sub-cubes of the runs that certify are labelled against
the certified optimum, the network is trained on the device, and the plain
and learned batched solvers run the same `--held` held-out tiny problems
(seeds 400000..) `--repeats` times each: device time to each certificate,
nodes, and the iteration of the final incumbent (what the seed head can
bring forward), compared problem by problem.

Budget mode:

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


def _bootstrap_median(x, rng, n=2000):
    """Median of x and a 95% bootstrap interval of it."""
    x = np.asarray(x, float)
    meds = np.median(rng.choice(x, (n, len(x)), replace=True), axis=1)
    return float(np.median(x)), float(np.percentile(meds, 2.5)), float(np.percentile(meds, 97.5))


def collect_certified(ctx, seeds, eps, trace_cap, cap, chunk=64):
    """Traces of plain batched runs (automatic pop) on tiny problems; only runs
    that certify are kept, and their popped sub-cubes are labelled against the
    certified optimum (learn.label_trace)."""
    F, L, T = [], [], []
    kept = 0
    for i in range(0, len(seeds), chunk):
        probs = [synth.tiny_problem(int(s)) for s in seeds[i:i + chunk]]
        res, traces = ctx.bnb_solve_batch(probs, eps=eps, max_seconds=600, queue_capacity=cap, trace_cap=trace_cap)
        for r, tr in zip(res, traces):
            if r["status_name"] != "optimal" or len(tr) == 0:
                continue
            kept += 1
            lab, tgt = learn.label_trace(tr, r["r"], r["t"])
            F.append(tr["feat"])
            L.append(lab)
            T.append(tgt)
    return np.concatenate(F), np.concatenate(L), np.concatenate(T), kept


def evaluate_certified(ctx, params, seeds, eps, beta, active_iters, repeats, cap, rng, chunk=32):
    """Plain and learned batched solves of the same held-out tiny problems,
    `repeats` times each, in batches of `chunk` problems (the queues of a
    batch are allocated together): per problem and repeat the device time to
    its certificate, its nodes and the iteration of its final incumbent;
    paired learned / plain ratios with bootstrap intervals of their medians."""
    probs = [synth.tiny_problem(int(s)) for s in seeds]
    ctx.mlp_set_params(params)
    runs = {"plain": [], "learned": []}
    for _ in range(repeats):
        for name, learned in (("plain", None), ("learned", dict(beta=beta, seed=True, active_iters=active_iters))):
            t0 = time.time()
            res = []
            for i in range(0, len(probs), chunk):
                res += ctx.bnb_solve_batch(probs[i:i + chunk], eps=eps, max_seconds=600, queue_capacity=cap,
                                           learned=learned)
            runs[name].append(dict(wall=time.time() - t0, res=res))
    out = {"problems": len(probs), "repeats": repeats, "beta": beta, "active_iters": active_iters}
    both = [k for k in range(len(probs))
            if all(r["res"][k]["status_name"] == "optimal" for n in runs for r in runs[n])]
    out["certified_in_every_run"] = len(both)
    agree = all(abs(a["res"][k]["f"] - b["res"][k]["f"]) <= eps * a["res"][k]["c22"]
                for a, b in zip(runs["plain"], runs["learned"]) for k in both)
    out["same_optima"] = bool(agree)
    for name in runs:
        sec = [r["res"][k]["seconds"] for r in runs[name] for k in both]
        nod = [r["res"][k]["nodes"] for r in runs[name] for k in both]
        it = [r["res"][k]["dstar_iteration"] for r in runs[name] for k in both]
        out[name] = {"median_seconds": float(np.median(sec)), "total_nodes": int(np.sum(nod)) // repeats,
                     "median_dstar_iteration": float(np.median(it)),
                     "wall_s": [round(r["wall"], 3) for r in runs[name]]}
    ratio_t = [l["res"][k]["seconds"] / p["res"][k]["seconds"]
               for p, l in zip(runs["plain"], runs["learned"]) for k in both]
    ratio_n = [l["res"][k]["nodes"] / p["res"][k]["nodes"] for p, l in zip(runs["plain"], runs["learned"]) for k in both]
    diff_it = [l["res"][k]["dstar_iteration"] - p["res"][k]["dstar_iteration"]
               for p, l in zip(runs["plain"], runs["learned"]) for k in both]
    out["time_ratio_median_ci"] = _bootstrap_median(ratio_t, rng)
    out["node_ratio_median_ci"] = _bootstrap_median(ratio_n, rng)
    out["dstar_iteration_diff_median_ci"] = _bootstrap_median(diff_it, rng)
    return out


def main_certified(a):
    """Training on traces of runs that certify, and the paired evaluation."""
    ctx = Gosma(0)
    rng = np.random.default_rng(0)
    eps = 1e-3
    rep = dict(args=vars(a), mode="certified")
    t0 = time.time()
    F, L, T, kept = collect_certified(ctx, np.arange(300000, 300000 + a.train), eps, a.trace_cap, 1 << 24)
    rep["traces"] = dict(problems=a.train, certified=kept, rows=int(len(F)), positives=int(L.sum()),
                         seconds=time.time() - t0)
    print("traces", rep["traces"], flush=True)
    t0 = time.time()
    params, losses = learn.train(ctx, F, L, T, steps=a.steps, batch=a.batch, lr=a.lr)
    rep["training"] = dict(loss_first=float(losses[:20].mean()), loss_last=float(losses[-20:].mean()),
                           seconds=time.time() - t0, steps=a.steps, batch=a.batch)
    print("training", rep["training"], flush=True)
    learn.save(a.out, params, train=a.train, mode="certified")
    held = np.arange(400000, 400000 + a.held)
    Fh, Lh, Th, kh = collect_certified(ctx, held, eps, a.trace_cap, 1 << 24)
    ctx.mlp_set_params(params)
    y = ctx.mlp_forward(Fh)
    pos = Lh > 0.5
    rep["held_out"] = dict(problems=a.held, certified=kh, rows=int(len(Fh)), positives=int(pos.sum()),
                           auc=_auc(y[:, 0], Lh, rng),
                           seed_abs_err=float(np.abs(y[pos, 1:7] - Th[pos]).mean()) if pos.any() else None,
                           seed_abs_err_centre=float(np.abs(Th[pos]).mean()) if pos.any() else None)
    print("held-out", rep["held_out"], flush=True)
    rep["evaluation"] = evaluate_certified(ctx, params, held, eps, a.beta, a.active_iters, a.repeats, 1 << 24, rng)
    print("evaluation", rep["evaluation"], flush=True)
    if a.report:
        with open(a.report, "w") as f:
            json.dump(rep, f, indent=1)
    ctx.close()


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--mode", choices=["budget", "certified"], default="budget",
                    help="budget: paper-scale traces at node budgets; certified: traces of tiny problems that "
                         "certify, labelled against the certified optimum, and a paired evaluation")
    ap.add_argument("--repeats", type=int, default=3, help="certified mode: repeats of each evaluation")
    ap.add_argument("--active-iters", type=int, default=8, help="certified mode: iterations the network scores")
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
    if a.mode == "certified":
        return main_certified(a)
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
