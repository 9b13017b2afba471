"""One alignment problem solved by several ranks (GPUs, or contexts of one GPU).

Algorithm 1 shards over the translation domain: rank k searches slab k of
Omega_t (the domain cut into equal slabs along its longest axis) with every
rotation, so the ranks' sub-cubes are disjoint and together cover the
domain.  Between `steps` iterations the ranks exchange a record of ten
doubles: their incumbent d*_k with its pose, the lower bound L_k of their
slab (the smallest lower bound left in their queue, their d* once the queue
is empty), a status code (running, certified, or the limit that stopped
them) and their node count.  Every rank
then takes d* = min_k d*_k as its incumbent (gosma_bnb_set_incumbent), so it
prunes against the best pose found anywhere, and the run stops when
d* - min_k L_k <= eps C22 (the certificate of Algorithm 1 over the whole
domain: each L_k bounds f from below on slab k) or when no rank is running.
A rank whose own stopping test fired has L_k >= d*_k - eps C22 >= d* - eps C22,
so it needs no further steps.

The exchange is one all-gather per round (`solve_distributed`, through
torch.distributed), or a loop over the contexts of one process
(`solve_local`).
"""
from __future__ import annotations

import numpy as np

_FIELDS = 10  # d*, L, status code, nodes, r (3), t (3)
_CODES = {"running": 0, "optimal": 1, "node_limit": 2, "time_limit": 3, "queue_full": 4}
_NAMES = {v: k for k, v in _CODES.items()}


def slab(t_lo, t_hi, rank: int, world: int):
    """Translation slab of `rank`: the domain cut along its longest axis into
    `world` equal slabs; neighbours share their boundary value exactly."""
    lo, hi = np.array(t_lo, dtype=np.float64), np.array(t_hi, dtype=np.float64)
    ax = int(np.argmax(hi - lo))
    w = (hi[ax] - lo[ax]) / world
    a, b = lo.copy(), hi.copy()
    a[ax] = lo[ax] + rank * w
    b[ax] = hi[ax] if rank == world - 1 else lo[ax] + (rank + 1) * w
    return a, b


def _record(res) -> np.ndarray:
    rec = np.zeros(_FIELDS)
    rec[0] = res["f"]
    rec[1] = res["lb"]
    rec[2] = _CODES.get(res["status_name"], 2)
    rec[3] = float(res["nodes"])
    rec[4:7] = res["r"]
    rec[7:10] = res["t"]
    return rec


def _merge(recs: np.ndarray, c22: float, eps: float, rounds: int):
    """Global incumbent and lower bound; the result dict when the run is over, else None."""
    k = int(np.argmin(recs[:, 0]))
    dstar, x, lb = float(recs[k, 0]), recs[k, 4:10].copy(), float(np.min(recs[:, 1]))
    codes = [int(c) for c in recs[:, 2]]
    certified = dstar - lb <= eps * c22
    if not certified and 0 in codes:
        return dstar, x, None
    stops = [_NAMES[c] for c in codes if c > 1]
    return dstar, x, {"f": dstar, "lb": lb, "gap_norm": (dstar - lb) / c22, "c22": c22, "f_norm": dstar / c22 + 1.0,
                      "r": x[:3], "t": x[3:], "status_name": "optimal" if certified or not stops else stops[0],
                      "nodes": int(np.sum(recs[:, 3])), "rounds": rounds}


def solve_local(ctxs, prob, eps=0.1, steps=8, max_rounds=100000, **opts):
    """Shards of one problem on the contexts `ctxs` of this process (one per
    rank), stepped in turn; returns the global certificate and pose."""
    world = len(ctxs)
    for k, c in enumerate(ctxs):
        lo, hi = slab(prob["t_lo"], prob["t_hi"], k, world)
        c.set_problem(dict(prob, t_lo=lo, t_hi=hi))
        c.bnb_start(eps=eps, **opts)
    results = [None] * world
    for rounds in range(1, max_rounds + 1):
        for k, c in enumerate(ctxs):
            if results[k] is None or results[k]["status_name"] == "running":
                results[k] = c.bnb_step(steps)
        c22 = results[0]["c22"]
        dstar, x, out = _merge(np.stack([_record(r) for r in results]), c22, eps, rounds)
        if out is not None:
            return out
        for k, c in enumerate(ctxs):
            if results[k]["status_name"] == "running" and dstar < results[k]["f"]:
                c.bnb_set_incumbent(dstar, x)
    raise RuntimeError("sharded solve: max_rounds reached")


def solve_distributed(ctx, prob, eps=0.1, steps=8, group=None, max_rounds=100000, **opts):
    """This process's shard of one problem (rank and world size from
    torch.distributed); every rank returns the same global result."""
    import torch
    import torch.distributed as dist
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    lo, hi = slab(prob["t_lo"], prob["t_hi"], rank, world)
    ctx.set_problem(dict(prob, t_lo=lo, t_hi=hi))
    ctx.bnb_start(eps=eps, **opts)
    res = None
    for rounds in range(1, max_rounds + 1):
        if res is None or res["status_name"] == "running":
            res = ctx.bnb_step(steps)
        mine = torch.tensor(_record(res), dtype=torch.float64, device=dev)
        parts = [torch.zeros_like(mine) for _ in range(world)]
        dist.all_gather(parts, mine, group=group)
        dstar, x, out = _merge(torch.stack(parts).cpu().numpy(), res["c22"], eps, rounds)
        if out is not None:
            return out
        if res["status_name"] == "running" and dstar < res["f"]:
            ctx.bnb_set_incumbent(dstar, x)
    raise RuntimeError("sharded solve: max_rounds reached")
