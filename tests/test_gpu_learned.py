"""The shipped queue-ordering weights against the plain solver on held-out
tiny problems (seeds 400000.., never used in training, which draws from
300000..).

The network reorders pops and proposes SMA seeds (Sec. 5); it never changes a
bound, so both forms certify the same optima.  The stated bound on its cost:
over the problems that certify in every run, the learned form bounds at most
1% more sub-cubes in total, its median per-problem device time to the
certificate is at most 10% above the plain form's (median of per-problem
ratios over two repeats), and its final incumbent is found no later (median
difference of the iteration of the final incumbent at most one iteration).
"""
import os

import numpy as np
import pytest

from paper_1812_01232_gb300 import learn, synth

pytestmark = pytest.mark.gpu

WEIGHTS = os.path.join(os.path.dirname(__file__), "..", "paper_1812_01232_gb300", "weights", "gosma_mlp.npz")
SEEDS = range(400000, 400016)
EPS = 1e-3
NODE_BOUND = 1.01
TIME_BOUND = 1.10
ITER_BOUND = 1.0


@pytest.fixture(scope="module")
def ctx():
    from paper_1812_01232_gb300.gosma import Gosma
    c = Gosma(0)
    yield c
    c.close()


def test_shipped_weights_cost_no_more_than_the_stated_bound(ctx):
    probs = [synth.tiny_problem(s) for s in SEEDS]
    ctx.mlp_set_params(learn.load(WEIGHTS))
    runs = {"plain": [], "learned": []}
    for _ in range(2):
        for name, kw in (("plain", {}), ("learned", dict(learned=dict(beta=1e-4, seed=True, active_iters=8)))):
            runs[name].append(ctx.bnb_solve_batch(probs, eps=EPS, max_seconds=300, queue_capacity=1 << 24, **kw))
    both = [k for k in range(len(probs)) if all(r[k]["status_name"] == "optimal" for n in runs for r in runs[n])]
    assert len(both) >= 8, len(both)
    for p, l in zip(runs["plain"], runs["learned"]):
        for k in both:
            assert abs(p[k]["f"] - l[k]["f"]) <= EPS * p[k]["c22"]
            # each certificate covers the other's incumbent
            assert l[k]["lb"] <= p[k]["f"] + 1e-9 and p[k]["lb"] <= l[k]["f"] + 1e-9
    nodes_p = sum(r[k]["nodes"] for r in runs["plain"] for k in both)
    nodes_l = sum(r[k]["nodes"] for r in runs["learned"] for k in both)
    assert nodes_l <= NODE_BOUND * nodes_p, (nodes_l, nodes_p)
    ratio = [l[k]["seconds"] / p[k]["seconds"] for p, l in zip(runs["plain"], runs["learned"]) for k in both]
    assert np.median(ratio) <= TIME_BOUND, ratio
    diff = [l[k]["dstar_iteration"] - p[k]["dstar_iteration"]
            for p, l in zip(runs["plain"], runs["learned"]) for k in both]
    assert np.median(diff) <= ITER_BOUND, diff
