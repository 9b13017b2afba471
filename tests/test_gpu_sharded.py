"""One problem shared by two and three contexts of one GPU
(paper_1812_01232_gb300/sharded.py): the first sub-cubes dealt from one run,
then stepped in turn, exchanging (d*, lower bound) through
gosma_bnb_set_incumbent and rebalancing queued sub-cubes through
gosma_bnb_export / gosma_bnb_import.  The global certificate must agree with
a single-context solve and with the stored oracle optimum."""
import json
import os

import numpy as np
import pytest

from paper_1812_01232_gb300 import sharded, synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "bnb_tiny_oracle.json")


@pytest.fixture(scope="module")
def ctxs():
    from paper_1812_01232_gb300 import build
    build.build()
    from paper_1812_01232_gb300.gosma import Gosma
    cs = [Gosma(0) for _ in range(3)]
    yield cs
    for c in cs:
        c.close()


@pytest.mark.parametrize("world", [2, 3])
def test_shards_certify_like_a_single_solve(ctxs, oracle_mod, world):
    p = synth.tiny_problem(1000)
    gold = json.load(open(GOLDEN))["1000"]
    eps = 1e-3
    ctxs[0].set_problem(p)
    one = ctxs[0].bnb_solve(eps=eps, queue_capacity=1 << 26)
    r = sharded.solve_local(ctxs[:world], p, eps=eps, steps=8, queue_capacity=1 << 26)
    epsf = eps * one["c22"]
    assert r["status_name"] == "optimal" and r["c22"] == one["c22"]
    assert r["f"] - r["lb"] <= epsf
    # the two certificates cover each other, and the oracle's optimum
    assert r["lb"] <= one["f"] + 1e-9 and one["lb"] <= r["f"] + 1e-9
    assert abs(r["f"] - gold["f"]) <= epsf and r["lb"] <= gold["f"] + 1e-9
    mix = oracle_mod.Mixtures.from_problem(p)
    assert oracle_mod.objective_r(mix, r["r"], r["t"]) == pytest.approx(r["f"], rel=1e-10)
    assert r["rounds"] > 1


def test_incumbent_offer(ctxs):
    from paper_1812_01232_gb300.gosma import GosmaError
    p = synth.tiny_problem(1001)
    c = ctxs[0]
    c.set_problem(p)
    with pytest.raises(GosmaError):
        c.bnb_set_incumbent(0.0, np.zeros(6))  # no run in progress yet
    c.bnb_start(eps=1e-3, queue_capacity=1 << 24)
    r = c.bnb_step(2)
    c.bnb_set_incumbent(r["f"] + 1.0, np.zeros(6))  # worse: ignored
    assert c.bnb_step(1)["f"] <= r["f"]
    x = np.concatenate([r["r"], r["t"]])
    c.bnb_set_incumbent(r["f"] - 1e-9, x)  # better: taken
    s = c.bnb_step(1)
    assert s["f"] <= r["f"] - 1e-9


def test_export_import_round_trip(ctxs, oracle_mod):
    """Sub-cubes exported from one run and imported into another run of the
    same problem: the exporting run's lower bound never falls, nothing is
    lost (the two runs together certify the stored oracle optimum), and the
    records are the queue's own."""
    from paper_1812_01232_gb300.gosma import GosmaError
    p = synth.tiny_problem(1000)
    gold = json.load(open(GOLDEN))["1000"]
    a, b = ctxs[0], ctxs[1]
    for c in (a, b):
        c.set_problem(p)
        c.bnb_start(eps=1e-3, queue_capacity=1 << 26)
    ra = a.bnb_step(6)
    b.bnb_export(1 << 20)  # b gives away its root: its queue is empty
    nodes = a.bnb_export(ra["queue_size"] // 2)
    assert 0 < len(nodes) <= ra["queue_size"] // 2
    assert np.all(nodes["lb"] < ra["f"]) and np.all(nodes["lr"] <= 30) and np.all(nodes["flags"] & 1)
    bad = nodes[:1].copy()
    bad["lb"] = np.nan
    with pytest.raises(GosmaError):
        b.bnb_import(bad)  # not a record of this library
    b.bnb_import(nodes)
    b.bnb_set_incumbent(ra["f"], np.concatenate([ra["r"], ra["t"]]))
    ra2, rb = a.bnb_step(0), b.bnb_step(0)
    assert ra2["status_name"] == rb["status_name"] == "optimal"
    f, lb = min(ra2["f"], rb["f"]), min(ra2["lb"], rb["lb"])
    epsf = 1e-3 * gold["c22"]
    assert abs(f - gold["f"]) <= epsf and lb <= gold["f"] + 1e-9 and gold["lb"] <= f + 1e-9


def test_rebalancing_on_one_gpu(ctxs):
    """All the dealt sub-cubes on one context: rebalancing moves work to the
    others, and the certificate equals the balanced run's within eps."""
    p = synth.tiny_problem(1002)
    eps = 1e-3

    def all_to_rank0(nodes, rank, world):
        return nodes if rank == 0 else nodes[:0]

    a = sharded.solve_local(ctxs[:2], p, eps=eps, steps=8, queue_capacity=1 << 26)
    b = sharded.solve_local(ctxs[:2], p, eps=eps, steps=8, queue_capacity=1 << 26, deal=all_to_rank0)
    assert a["status_name"] == b["status_name"] == "optimal"
    assert abs(a["f"] - b["f"]) <= eps * a["c22"]
    assert b["moved"] > 0 and min(b["nodes_per_rank"]) > 0.1 * max(b["nodes_per_rank"])
