"""One alignment problem solved by several ranks (GPUs, or contexts of one GPU).

Algorithm 1 over several solvers: their queues together hold the live
sub-cubes, so d* = min_k d*_k is the incumbent and L = min_k L_k (each rank's
smallest queued lower bound, its d* once its queue is empty) bounds f from
below over the whole domain; the run is certified when d* - L <= eps C22.

* Deal: every rank starts a run of the whole problem (the same domain, so
  queue records mean the same sub-cube on every rank).  Rank 0 runs the first
  `deal_iters` iterations alone and deals its queue: rank k keeps records
  k, k + world, ... (the others empty their queue and import their share).
* Rounds: every rank runs `steps` iterations, then the ranks exchange a
  record of eleven doubles: d*_k with its pose, L_k, a status code (running,
  certified, or the limit that stopped it), the node count and the number of
  queued sub-cubes.  Every rank offers d* to its run
  (gosma_bnb_set_incumbent), so it prunes against the best pose found
  anywhere; the run stops when the global gap closes or no rank runs.
* Rebalancing: after the exchange the ranks with queued work are sorted by
  their queue sizes; the largest hands half of its surplus over the smallest
  (a rank that has certified its own queue counts as empty) to it, the second
  largest to the second smallest, and so on, while the donor holds at least
  twice the receiver's work and at least `min_move` sub-cubes
  (gosma_bnb_export / gosma_bnb_import).  No record is outside a queue when
  the next round's records are taken, so the certificate is that of
  Algorithm 1.  A rank whose run was stopped by a limit neither gives nor
  takes work.

The exchange is an all-gather and point-to-point transfers through
torch.distributed (`solve_distributed`), or direct calls between the contexts
of one process (`solve_local`).
"""
from __future__ import annotations

import numpy as np

_FIELDS = 11  # d*, L, status code, nodes, r (3), t (3), queued sub-cubes
_CODES = {"running": 0, "optimal": 1, "node_limit": 2, "time_limit": 3, "queue_full": 4}
_NAMES = {v: k for k, v in _CODES.items()}
MAX_MOVE = 1 << 20  # sub-cubes handed over per transfer


def _record(res) -> np.ndarray:
    rec = np.zeros(_FIELDS)
    rec[0] = res["f"]
    rec[1] = res["lb"]
    rec[2] = _CODES.get(res["status_name"], 2)
    rec[3] = float(res["nodes"])
    rec[4:7] = res["r"]
    rec[7:10] = res["t"]
    rec[10] = float(res.get("queue_size", 0))
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


def plan_moves(recs: np.ndarray, min_move: int = 64):
    """Transfers (donor, receiver, count) of one rebalancing round, the same on
    every rank (a function of the exchanged records only)."""
    codes = recs[:, 2].astype(int)
    work = np.where(codes == 0, recs[:, 10], 0.0)  # a rank that certified its queue is idle
    open_ranks = [k for k in range(len(recs)) if codes[k] <= 1]  # running or idle, not stopped by a limit
    order = sorted(open_ranks, key=lambda k: (-work[k], k))
    moves = []
    lo, hi = 0, len(order) - 1
    while lo < hi:
        d, r = order[lo], order[hi]
        if work[d] < max(2.0 * work[r], float(min_move)):
            break
        m = int(min((work[d] - work[r]) // 2, MAX_MOVE))
        if m < min_move // 2:
            break
        moves.append((d, r, m))
        lo, hi = lo + 1, hi - 1
    return moves


def _deal(nodes, rank: int, world: int):
    return nodes[rank::world]


def solve_local(ctxs, prob, eps=0.1, steps=8, max_rounds=100000, deal_iters=2, rebalance=True, min_move=64,
                deal=_deal, **opts):
    """Shards of one problem on the contexts `ctxs` of this process (one per
    rank), stepped in turn; returns the global certificate and pose, with the
    sub-cubes each rank bounded ("nodes_per_rank") and the transfers made."""
    world = len(ctxs)
    for c in ctxs:
        c.set_problem(prob)
        c.bnb_start(eps=eps, **opts)
    ctxs[0].bnb_step(deal_iters)
    dealt = ctxs[0].bnb_export(1 << 30)
    for k, c in enumerate(ctxs):
        if k:
            c.bnb_export(1 << 30)  # the root: rank 0 dealt its children
        c.bnb_import(deal(dealt, k, world))
    results = [None] * world
    moved = 0
    for rounds in range(1, max_rounds + 1):
        for k, c in enumerate(ctxs):
            if results[k] is None or results[k]["status_name"] == "running":
                results[k] = c.bnb_step(steps)
        recs = np.stack([_record(r) for r in results])
        dstar, x, out = _merge(recs, results[0]["c22"], eps, rounds)
        if out is not None:
            out["nodes_per_rank"] = [int(r["nodes"]) for r in results]
            out["moved"] = moved
            return out
        for k, c in enumerate(ctxs):
            if results[k]["status_name"] in ("running", "optimal") and dstar < results[k]["f"]:
                c.bnb_set_incumbent(dstar, x)
        if rebalance:
            for d, r, m in plan_moves(recs, min_move):
                nodes = ctxs[d].bnb_export(m)
                ctxs[r].bnb_import(nodes)
                moved += len(nodes)
                results[r] = None  # it has work again: step it in the next round
    raise RuntimeError("sharded solve: max_rounds reached")


def _send_nodes(dist, nodes, dst, dev, group):
    import torch
    n = torch.tensor([len(nodes)], dtype=torch.int64, device=dev)
    dist.send(n, dst, group=group)
    if len(nodes):
        buf = torch.from_numpy(np.ascontiguousarray(nodes).view(np.uint8).copy()).to(dev)
        dist.send(buf, dst, group=group)


def _recv_nodes(dist, dtype, src, dev, group):
    import torch
    n = torch.zeros(1, dtype=torch.int64, device=dev)
    dist.recv(n, src, group=group)
    if int(n.item()) == 0:
        return np.zeros(0, dtype=dtype)
    buf = torch.zeros(int(n.item()) * dtype.itemsize, dtype=torch.uint8, device=dev)
    dist.recv(buf, src, group=group)
    return buf.cpu().numpy().view(dtype)


def solve_distributed(ctx, prob, eps=0.1, steps=8, group=None, max_rounds=100000, deal_iters=2, rebalance=True,
                      min_move=64, deal=_deal, **opts):
    """This process's share of one problem (rank and world size from
    torch.distributed); every rank returns the same global result.  `ctx`
    needs the stepping interface and node_dtype (the record type of
    bnb_export / bnb_import)."""
    import torch
    import torch.distributed as dist
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    ranks = [dist.get_global_rank(group, k) for k in range(world)] if group is not None else list(range(world))
    ctx.set_problem(prob)
    ctx.bnb_start(eps=eps, **opts)
    if rank == 0:
        ctx.bnb_step(deal_iters)
        dealt = ctx.bnb_export(1 << 30)
        for k in range(1, world):
            _send_nodes(dist, deal(dealt, k, world), ranks[k], dev, group)
        ctx.bnb_import(deal(dealt, 0, world))
    else:
        ctx.bnb_export(1 << 30)  # the root: rank 0 deals its children
        ctx.bnb_import(_recv_nodes(dist, ctx.node_dtype, ranks[0], dev, group))
    res = None
    moved = 0
    for rounds in range(1, max_rounds + 1):
        if res is None or res["status_name"] == "running":
            res = ctx.bnb_step(steps)
        mine = torch.tensor(_record(res), dtype=torch.float64, device=dev)
        parts = [torch.zeros_like(mine) for _ in range(world)]
        dist.all_gather(parts, mine, group=group)
        recs = torch.stack(parts).cpu().numpy()
        dstar, x, out = _merge(recs, res["c22"], eps, rounds)
        if out is not None:
            out["nodes_per_rank"] = [int(v) for v in recs[:, 3]]
            out["moved"] = moved
            return out
        if res["status_name"] in ("running", "optimal") and dstar < res["f"]:
            ctx.bnb_set_incumbent(dstar, x)
        if rebalance:
            for d, r, m in plan_moves(recs, min_move):
                if rank == d:
                    _send_nodes(dist, ctx.bnb_export(m), ranks[r], dev, group)
                elif rank == r:
                    nodes = _recv_nodes(dist, ctx.node_dtype, ranks[d], dev, group)
                    ctx.bnb_import(nodes)
                    res = None
                moved += m  # planned; the donor may hand over fewer (its queue drops pruned ones first)
    raise RuntimeError("sharded solve: max_rounds reached")
