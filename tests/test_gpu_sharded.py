"""One problem split over translation slabs (paper_1812_01232_gb300/sharded.py)
and solved by two and three contexts of one GPU, stepped in turn and
exchanging (d*, lower bound) through gosma_bnb_set_incumbent: the global
certificate must agree with a single-context solve and with the stored
oracle optimum."""
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
