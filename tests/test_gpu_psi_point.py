"""The point-dependent rotation uncertainty of Lemma 2 (gosma_set_psi_r_mode,
GOSMA_PSI_R_POINT; reading R16) on the GPU.

* bounds: element by element against the oracle's bounds in the same mode
  (parity_util tolerances), and never looser than the point-independent
  bounds of the same cubes;
* branch-and-bound: certificates against the stored oracle optima, and the
  nodes the solver expands with and without it on the same problems.
"""
import json
import os

import numpy as np
import pytest

from paper_1812_01232_gb300 import synth
from parity_util import compare

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "bnb_tiny_oracle.json")


@pytest.fixture(scope="module")
def ctx():
    from paper_1812_01232_gb300 import build
    build.build()
    from paper_1812_01232_gb300.gosma import Gosma
    c = Gosma(0)
    yield c
    c.close()


def _both_modes(ctx, cubes):
    ctx.set_psi_r_mode(False)
    cube_mode = ctx.eval_bounds_detail(cubes)
    ctx.set_psi_r_mode(True)
    point = ctx.eval_bounds_detail(cubes)
    ctx.set_psi_r_mode(False)
    return cube_mode, point


@pytest.mark.parametrize("seed", [1000, 1001, 1002])
def test_tiny_parity_point_mode(ctx, oracle_mod, seed):
    prob = synth.tiny_problem(seed)
    ctx.set_problem(prob)
    cubes = synth.tree_cubes(seed + 7, 1024, prob["t_lo"], prob["t_hi"], 0, 16, near=(prob["r_gt"], prob["t_gt"]),
                             near_frac=0.5)
    g0, g1 = _both_modes(ctx, cubes)
    mix = oracle_mod.Mixtures.from_problem(prob)
    compare(g0, oracle_mod.bounds(mix, cubes, prob["zeta"]), "tiny %d cube-psi_r" % seed, cubes=cubes,
            kappa2_max=prob["kappa2"].max())
    compare(g1, oracle_mod.bounds(mix, cubes, prob["zeta"], psi_mode=1), "tiny %d point-psi_r" % seed, cubes=cubes,
            kappa2_max=prob["kappa2"].max())
    fin = np.isfinite(g0[:, 0])
    assert np.array_equal(g0[:, 1], g1[:, 1], equal_nan=True)  # the centre term does not use psi_r
    assert np.array_equal(g0[:, 2], g1[:, 2], equal_nan=True)  # nor do the self pairs
    assert np.all(g1[fin, 0] >= g0[fin, 0])                     # the cross sums only shrink
    assert np.mean(g1[fin, 0] > g0[fin, 0]) > 0.5


@pytest.mark.parametrize("n1,n2", [(1, 1), (33, 17), (257, 40)])
def test_ragged_parity_point_mode(ctx, oracle_mod, n1, n2):
    rng = np.random.default_rng(n1 * 7 + n2)
    n_in = min(n1, max(1, n2 - 1))
    prob = synth.tiny_problem(int(rng.integers(1 << 30)), n1=n1, n_in=n_in, n_out=n2 - n_in)
    ctx.set_problem(prob)
    cubes = synth.tree_cubes(int(rng.integers(1 << 30)), 97, prob["t_lo"], prob["t_hi"], 1, 14,
                             near=(prob["r_gt"], prob["t_gt"]), near_frac=0.5)
    g0, g1 = _both_modes(ctx, cubes)
    mix = oracle_mod.Mixtures.from_problem(prob)
    compare(g0, oracle_mod.bounds(mix, cubes, prob["zeta"]), "%dx%d cube-psi_r" % (n1, n2), cubes=cubes,
            kappa2_max=prob["kappa2"].max())
    compare(g1, oracle_mod.bounds(mix, cubes, prob["zeta"], psi_mode=1), "%dx%d point-psi_r" % (n1, n2), cubes=cubes,
            kappa2_max=prob["kappa2"].max())


def test_paper_scale_parity_point_mode(ctx, oracle_mod):
    """128 x 64 components, 8,192 sub-cubes at depths 2-12, every one
    against the oracle."""
    prob = synth.paper_scale_problem(2000)
    ctx.set_problem(prob)
    cubes = synth.tree_cubes(2011, 8192, prob["t_lo"], prob["t_hi"], 2, 12, near=(prob["r_gt"], prob["t_gt"]),
                             near_frac=0.3)
    g0, g1 = _both_modes(ctx, cubes)
    mix = oracle_mod.Mixtures.from_problem(prob)
    compare(g1, oracle_mod.bounds(mix, cubes, prob["zeta"], psi_mode=1), "paper-scale point-psi_r",
            eps_c22=prob["eps"] * oracle_mod.c22(mix), cubes=cubes)
    fin = np.isfinite(g0[:, 0])
    assert np.all(g1[fin, 0] >= g0[fin, 0])


def test_invalid_mode_rejected(ctx):
    from paper_1812_01232_gb300.gosma import GosmaError
    with pytest.raises(GosmaError):
        ctx._check(ctx.L.gosma_set_psi_r_mode(ctx.h, 2), "set_psi_r_mode")


@pytest.mark.parametrize("seed", [1000, 1001, 1002])
def test_tiny_certificate_point_mode(ctx, oracle_mod, seed):
    """The certified optimum with the point-dependent angle and the stored
    oracle optimum certify each other, and it expands no more nodes than the
    point-independent run of the same problem (1% for the different pop
    order)."""
    gold = json.load(open(GOLDEN))[str(seed)]
    p = synth.tiny_problem(seed)
    ctx.set_problem(p)
    ctx.set_psi_r_mode(False)
    r0 = ctx.bnb_solve(eps=p["eps"], pop=1024, max_seconds=300, queue_capacity=1 << 27)
    ctx.set_psi_r_mode(True)
    r1 = ctx.bnb_solve(eps=p["eps"], pop=1024, max_seconds=300, queue_capacity=1 << 27)
    ctx.set_psi_r_mode(False)
    assert r0["status_name"] == r1["status_name"] == "optimal"
    epsf = p["eps"] * gold["c22"]
    assert abs(r1["f"] - gold["f"]) <= epsf
    assert r1["lb"] <= gold["f"] + 1e-9 and gold["lb"] <= r1["f"] + 1e-9
    mix = oracle_mod.Mixtures.from_problem(p)
    assert oracle_mod.objective_r(mix, r1["r"], r1["t"]) == pytest.approx(r1["f"], rel=1e-10)
    # tighter bounds prune at least as much; the pop order differs, so allow 1%
    assert r1["nodes"] <= 1.01 * r0["nodes"], (r1["nodes"], r0["nodes"])


def test_batched_solver_point_mode(ctx):
    """The batched solver takes the context's mode: the same optima as the
    point-independent batch, with no more nodes in total (1% for the
    different pop order)."""
    probs = [synth.tiny_problem(200000 + s) for s in range(4)]
    ctx.set_psi_r_mode(False)
    a = ctx.bnb_solve_batch(probs, eps=1e-3, max_seconds=120, queue_capacity=1 << 24)
    ctx.set_psi_r_mode(True)
    b = ctx.bnb_solve_batch(probs, eps=1e-3, max_seconds=120, queue_capacity=1 << 24)
    ctx.set_psi_r_mode(False)
    for x, y in zip(a, b):
        if x["status_name"] == y["status_name"] == "optimal":
            assert abs(x["f"] - y["f"]) <= 1e-3 * x["c22"]
    assert sum(y["nodes"] for y in b) <= 1.01 * sum(x["nodes"] for x in a)
