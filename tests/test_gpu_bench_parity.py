"""Parity where the benchmark runs: one branch-and-bound step of the
benchmark's workload (the 128 x 64 paper-scale problem, 8,192 parents popped,
65,536 children bounded by the children kernel in the benchmark's launch
configuration), every child compared element by element with the FP64
oracle's Theorem 1 bounds of the same sub-cube.

The children come from the step's own buffers (gosma_bnb_last_children), so
the comparison covers the children kernel's branching, its pre-pass and the
cached self sums that children of a rotation split take from their parent
(Algorithm 1; Sec. 4.1).  The step must hold children of both split types.
Tolerances are those of parity_util.py; over the children whose oracle lower
bound is within eps C22 of the incumbent (the only ones whose pruning or
stopping-test decision a deficit can change) the deficit is also held below
CERT_BAR eps C22: every such decision the oracle takes with a margin of
eps C22 the device takes too.
"""
import numpy as np
import pytest

from paper_1812_01232_gb300 import synth
from parity_util import compare

pytestmark = pytest.mark.gpu

POP = 8192      # the benchmark's parents per step
SEED = 2000     # the benchmark's problem
CERT_BAR = 1.0  # largest deficit near the incumbent, in units of eps * C22


def _bench_like_run(steps_after_fill):
    from paper_1812_01232_gb300 import build
    build.build()
    from paper_1812_01232_gb300.gosma import Gosma
    prob = synth.paper_scale_problem(SEED)
    ctx = Gosma(0)
    ctx.set_problem(prob)
    ctx.bnb_start(eps=prob["eps"], pop=POP, queue_capacity=1 << 22)
    r = ctx.bnb_step(1)
    while r["queue_size"] < POP and r["status_name"] == "running":
        r = ctx.bnb_step(1)
    for _ in range(steps_after_fill):
        r = ctx.bnb_step(1)
    assert r["status_name"] == "running"
    return prob, ctx, r


@pytest.mark.parametrize("steps_after_fill", [3, 12])
def test_bench_step_children_match_the_oracle(oracle_mod, steps_after_fill):
    prob, ctx, prev = _bench_like_run(steps_after_fill)
    n1 = ctx.n1
    r = ctx.bnb_step(1)
    cubes, got = ctx.bnb_last_children()
    ctx.close()
    assert len(cubes) == 8 * POP and r["iterations"] == prev["iterations"] + 1
    # children of both split types: some compute their self sums, others reuse the parent's
    fresh = (r["self_pairs"] - prev["self_pairs"]) // (n1 * (n1 - 1) // 2)
    assert 0 < fresh < 8 * POP, fresh
    # the children tile their parents: 8 per parent, halving one half-width
    rhw = cubes[:, 3].reshape(POP, 8)
    thw = cubes[:, 4:10][:, 3:].reshape(POP, 8, 3)
    assert np.all(rhw == rhw[:, :1]) and np.all(thw == thw[:, :1])
    mix = oracle_mod.Mixtures.from_problem(prob)
    ref = oracle_mod.bounds(mix, cubes, prob["zeta"])
    st = compare(got, ref, "bench step children (+%d)" % steps_after_fill,
                 eps_c22=prob["eps"] * oracle_mod.c22(mix), dstar=r["f"], cubes=cubes)
    assert st["near_deficit_over_eps_c22"] < CERT_BAR, st


def test_last_children_before_and_between_runs():
    from paper_1812_01232_gb300 import build
    build.build()
    from paper_1812_01232_gb300.gosma import Gosma, GosmaError
    prob = synth.tiny_problem(1000)
    ctx = Gosma(0)
    ctx.set_problem(prob)
    with pytest.raises(GosmaError):
        ctx.bnb_last_children()  # no run
    ctx.bnb_start(eps=1e-3, pop=64, queue_capacity=1 << 16)
    cubes, rec = ctx.bnb_last_children()
    assert len(cubes) == 0  # no iteration yet
    ctx.bnb_step(1)
    cubes, rec = ctx.bnb_last_children()
    assert len(cubes) == 8  # the root's children
    assert np.allclose(cubes[:, 3], np.pi / 2)  # the root's first split halves the rotation cube
    ctx.bnb_step(2)
    c2, _ = ctx.bnb_last_children()
    assert 0 < len(c2) <= 8 * 64 and len(c2) % 8 == 0
    ctx.close()


@pytest.mark.parametrize("seed,steps", [(1000, 4), (1003, 9)])
def test_small_mixture_step_children_match_the_oracle(oracle_mod, seed, steps):
    """The same element-by-element comparison for a 10 x 8 tiny problem, whose
    children kernel runs two sub-cubes per warp (half-warp groups: model rows
    on 16 lanes, the sums reduced within the half), at the solver's automatic
    pop (65,536 parents, 524,288 children per step)."""
    from paper_1812_01232_gb300 import build
    build.build()
    from paper_1812_01232_gb300.gosma import Gosma
    prob = synth.tiny_problem(seed)
    ctx = Gosma(0)
    ctx.set_problem(prob)
    ctx.bnb_start(eps=1e-3, queue_capacity=1 << 24)
    n1 = ctx.n1
    prev = ctx.bnb_step(steps)
    for _ in range(16):  # the first later step with children of both split types
        r = ctx.bnb_step(1)
        cubes, got = ctx.bnb_last_children()
        fresh = (r["self_pairs"] - prev["self_pairs"]) // (n1 * (n1 - 1) // 2)
        if r["status_name"] != "running" or 0 < fresh < len(cubes):
            break
        prev = r
    ctx.close()
    assert r["status_name"] == "running" and len(cubes) >= 8 * 512, (r["status_name"], len(cubes))
    assert 0 < fresh < len(cubes), fresh
    mix = oracle_mod.Mixtures.from_problem(prob)
    ref = oracle_mod.bounds(mix, cubes, prob["zeta"])
    st = compare(got, ref, "tiny step children (seed %d, +%d)" % (seed, steps),
                 eps_c22=1e-3 * oracle_mod.c22(mix), dstar=r["f"], cubes=cubes, kappa2_max=prob["kappa2"].max())
    assert st["near_deficit_over_eps_c22"] < CERT_BAR, st
