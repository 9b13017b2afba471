"""The sharded solve of one problem across ranks (paper_1812_01232_gb300/sharded.py)
on CPU: two gloo ranks, and the same ranks stepped in one process.  The
ranks run a small branch-and-bound with the stepping interface of the
library (start, step, offer an incumbent, export and import queue records)
on a toy objective over the translation box, so the test covers the deal of
the first sub-cubes, the exchange of (d*, lower bound), the rebalancing of
queued work and the global stopping test without a GPU."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1812_01232_gb300 import sharded  # noqa: E402


class ToySolver:
    """Best-first interval branch-and-bound of f(t) = |t - c|^2 + 0.3 sin(7 t0)
    over a box, bounded by f(mid) - L(box) |half-widths| with L an upper bound
    of |grad f| on the box; the interface of Gosma's stepping solver, queue
    records (lb, box corners) included."""

    node_dtype = np.dtype([("lb", "<f8"), ("lo", "<f8", (3,)), ("hi", "<f8", (3,))])

    def set_problem(self, p):
        self.lo, self.hi, self.c = np.array(p["t_lo"], float), np.array(p["t_hi"], float), np.array(p["c"], float)
        self.max_nodes = p.get("max_nodes", 0)

    def _f(self, t):
        return float(np.sum((t - self.c) ** 2) + 0.3 * np.sin(7.0 * t[0]))

    def _box(self, lo, hi):
        mid, hw = 0.5 * (lo + hi), 0.5 * (hi - lo)
        L = 2.0 * (np.linalg.norm(mid - self.c) + np.linalg.norm(hw)) + 2.1
        fm = self._f(mid)
        return fm - L * np.linalg.norm(hw), fm, mid

    def bnb_start(self, eps, **opts):
        self.eps = eps
        lb, fm, mid = self._box(self.lo, self.hi)
        self.q = [(lb, self.lo, self.hi)]
        self.dstar, self.best, self.nodes, self.status = fm, mid, 1, "running"

    def bnb_set_incumbent(self, f, x):
        if f < self.dstar:
            self.dstar, self.best = f, np.array(x[3:], float)

    def _result(self):
        lb = min([b[0] for b in self.q], default=self.dstar)
        return {"f": self.dstar, "lb": min(lb, self.dstar), "status_name": self.status, "nodes": self.nodes,
                "r": np.zeros(3), "t": self.best.copy(), "c22": 1.0, "queue_size": len(self.q)}

    def bnb_export(self, m):
        self.q = [b for b in self.q if b[0] < self.dstar]
        m = min(m, len(self.q))
        out = np.zeros(m, dtype=self.node_dtype)
        for k, (lb, lo, hi) in enumerate(self.q[len(self.q) - m:]):
            out[k] = (lb, lo, hi)
        self.q = self.q[:len(self.q) - m]
        return out

    def bnb_import(self, nodes):
        for rec in nodes:
            self.q.append((float(rec["lb"]), np.array(rec["lo"], float), np.array(rec["hi"], float)))
        if len(nodes) and self.status == "optimal":
            self.status = "running"

    def bnb_step(self, n):
        for _ in range(n):
            self.q = [b for b in self.q if b[0] < self.dstar]
            if not self.q:
                self.status = "optimal"
                break
            lbmin = min(b[0] for b in self.q)
            if self.dstar - lbmin <= self.eps:
                self.status = "optimal"
                break
            if self.max_nodes and self.nodes >= self.max_nodes:
                self.status = "node_limit"
                break
            k = int(np.argmin([b[0] for b in self.q]))
            _, lo, hi = self.q.pop(k)
            ax = int(np.argmax(hi - lo))
            m = 0.5 * (lo[ax] + hi[ax])
            for a, b in ((lo, np.where(np.arange(3) == ax, m, hi)), (np.where(np.arange(3) == ax, m, lo), hi)):
                lb, fm, mid = self._box(a, b)
                self.nodes += 1
                if fm < self.dstar:
                    self.dstar, self.best = fm, mid
                self.q.append((lb, a, b))
        return self._result()


PROB = {"t_lo": [-1.0, -1.0, -0.5], "t_hi": [1.0, 1.0, 0.5], "c": [0.6, -0.2, 0.1]}


def _single(eps):
    s = ToySolver()
    s.set_problem(PROB)
    s.bnb_start(eps)
    r = s.bnb_step(10 ** 6)
    assert r["status_name"] == "optimal"
    return r


def test_the_deal_covers_the_queue():
    nodes = np.arange(11)
    for world in (1, 2, 3, 8):
        parts = [sharded._deal(nodes, k, world) for k in range(world)]
        assert sorted(np.concatenate(parts).tolist()) == nodes.tolist()


def test_rebalancing_plan():
    """The largest queues hand half of their surplus to the smallest; ranks
    stopped by a limit take no part; a certified rank counts as idle."""
    def recs(codes, work):
        r = np.zeros((len(codes), sharded._FIELDS))
        r[:, 2] = codes
        r[:, 10] = work
        return r
    assert sharded.plan_moves(recs([0, 0], [1000, 0])) == [(0, 1, 500)]
    assert sharded.plan_moves(recs([0, 1], [1000, 7])) == [(0, 1, 500)]       # certified: idle
    assert sharded.plan_moves(recs([0, 2], [1000, 0])) == []                  # stopped by a limit
    assert sharded.plan_moves(recs([0, 0], [1000, 600])) == []                # within a factor 2
    assert sharded.plan_moves(recs([0, 0], [100, 0]), min_move=256) == []      # too little to move
    assert sharded.plan_moves(recs([0, 0, 0, 0], [0, 4000, 10, 2000])) == [(1, 0, 2000), (3, 2, 995)]


EPS = 0.05


def test_local_shards_certify_the_global_optimum():
    eps = EPS
    one = _single(eps)
    r = sharded.solve_local([ToySolver(), ToySolver(), ToySolver()], PROB, eps=eps, steps=5, min_move=4)
    assert r["status_name"] == "optimal"
    assert r["f"] - r["lb"] <= eps
    assert abs(r["f"] - one["f"]) <= eps and r["lb"] <= one["f"] + 1e-12
    assert r["rounds"] > 1


def _all_to_rank0(nodes, rank, world):
    return nodes if rank == 0 else nodes[:0]


def test_rebalancing_spreads_work_dealt_to_one_rank():
    """All the dealt work on rank 0: with rebalancing the idle ranks receive
    queued sub-cubes and bound a share of the nodes, the certificate is the
    same, and the run needs fewer rounds than without."""
    one = _single(EPS)
    out = {}
    for rb in (False, True):
        r = sharded.solve_local([ToySolver(), ToySolver(), ToySolver()], PROB, eps=EPS, steps=3, min_move=4,
                                deal=_all_to_rank0, rebalance=rb)
        assert r["status_name"] == "optimal" and r["f"] - r["lb"] <= EPS
        assert abs(r["f"] - one["f"]) <= EPS and r["lb"] <= one["f"] + 1e-12
        out[rb] = r
    assert out[False]["moved"] == 0 and out[False]["nodes_per_rank"][1:] == [1, 1]
    assert out[True]["moved"] > 0 and min(out[True]["nodes_per_rank"][1:]) > 10
    assert out[True]["rounds"] < out[False]["rounds"]


def test_local_shards_report_a_limit():
    r = sharded.solve_local([ToySolver(), ToySolver()], dict(PROB, max_nodes=40), eps=1e-9, steps=5)
    assert r["status_name"] == "node_limit" and r["lb"] <= r["f"]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q, unbalanced):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_1812_01232_gb300 import sharded as sh
    dist.init_process_group("gloo", rank=rank, world_size=world)
    deal = _all_to_rank0 if unbalanced else sh._deal
    r = sh.solve_distributed(ToySolver(), PROB, eps=EPS, steps=3, min_move=4, deal=deal)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, r["f"], r["lb"], r["status_name"], r["nodes"], list(r["t"]), r["nodes_per_rank"], r["moved"]))


@pytest.mark.parametrize("unbalanced", [False, True])
def test_two_gloo_ranks_certify_the_global_optimum(unbalanced):
    """Two gloo ranks; with unbalanced=True rank 0 is dealt all the work and
    the rebalancing hands queued sub-cubes to rank 1 (point-to-point)."""
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q, unbalanced)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    one = _single(EPS)
    # every rank returns the same global result, which certifies the optimum
    assert out[0][1:] == out[1][1:]
    _, f, lb, status, nodes, t, per_rank, moved = out[0]
    assert status == "optimal" and f - lb <= EPS
    assert abs(f - one["f"]) <= EPS and lb <= one["f"] + 1e-12
    assert t[0] > 0  # the optimum lies at t0 > 0 (c0 = 0.6)
    if unbalanced:
        assert moved > 0 and per_rank[1] > 10


def _rec(f, lb, status, nodes=10, t=(0.0, 0.0, 0.0)):
    return sharded._record({"f": f, "lb": lb, "status_name": status, "nodes": nodes, "r": np.zeros(3),
                            "t": np.array(t, float), "queue_size": 0})


def test_merge_rules():
    c22, eps = 2.0, 0.01
    # a running rank and an uncertified gap: keep going, incumbent = smallest d*
    d, x, out = sharded._merge(np.stack([_rec(1.0, 0.5, "running", t=(1, 0, 0)), _rec(0.9, 0.85, "optimal",
                                                                                      t=(2, 0, 0))]), c22, eps, 3)
    assert out is None and d == 0.9 and x[3] == 2.0
    # the global gap closes while a rank still runs: certified
    d, x, out = sharded._merge(np.stack([_rec(1.0, 0.895, "running"), _rec(0.9, 0.89, "optimal")]), c22, eps, 4)
    assert out["status_name"] == "optimal" and out["lb"] == 0.89 and out["f"] == 0.9 and out["nodes"] == 20
    # nobody runs and a rank hit a limit: the gap stays open, the limit is reported
    d, x, out = sharded._merge(np.stack([_rec(1.0, 0.5, "node_limit"), _rec(0.9, 0.89, "optimal")]), c22, eps, 5)
    assert out["status_name"] == "node_limit" and out["gap_norm"] == pytest.approx((0.9 - 0.5) / c22)
    # every rank certified its own slab: the global certificate holds
    d, x, out = sharded._merge(np.stack([_rec(1.0, 0.995, "optimal"), _rec(0.9, 0.895, "optimal")]), c22, eps, 6)
    assert out["status_name"] == "optimal" and out["f"] - out["lb"] <= eps * c22
