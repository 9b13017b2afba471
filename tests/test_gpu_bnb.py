"""GPU branch-and-bound (Algorithm 1) against the FP64 oracle.

* the certified optimum agrees with the oracle's within eps (normalised,
  times C22), and each side's lower bound stays below the other's optimum;
* on noise-free data the true pose is recovered (Sec. 6 success criterion);
* the stepping interface, limits and queue overflow behave as documented.
"""
import json
import os

import numpy as np
import pytest

from paper_1812_01232_gb300 import synth

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


def _rot_err(R, Rgt):
    return np.arccos(np.clip((np.trace(R.T @ Rgt) - 1) / 2, -1, 1))


def _noise_free(seed, n1, sigma):
    p = synth.noise_free_problem(seed, n1=n1)
    p["sigma1"] = np.full(n1, sigma)
    p["kappa2"] = (np.linalg.norm(p["mu1"] - p["t_gt"], axis=1) / sigma) ** 2 + 1
    return p


@pytest.mark.parametrize("seed", [2, 3])
def test_noise_free_recovery(ctx, oracle_mod, seed):
    p = _noise_free(seed, 4, 0.1)
    ctx.set_problem(p)
    r = ctx.bnb_solve(eps=1e-2, pop=64, max_seconds=120)
    c22 = oracle_mod.c22(oracle_mod.Mixtures.from_problem(p))
    assert r["status_name"] == "optimal"
    assert r["c22"] == pytest.approx(c22, rel=1e-12)
    assert r["gap_norm"] <= 1e-2
    assert r["f"] == pytest.approx(-c22, abs=1e-2 * c22)
    assert r["lb"] <= -c22 + 1e-9
    assert _rot_err(r["R"], p["R_gt"]) < 0.1
    assert np.linalg.norm(r["t"] - p["t_gt"]) < 0.05 * np.linalg.norm(p["t_gt"]) + 1e-3
    # the reported objective is f at the reported pose (FP64, checked by the oracle)
    f = oracle_mod.objective_r(oracle_mod.Mixtures.from_problem(p), r["r"], r["t"])
    assert f == pytest.approx(r["f"], rel=1e-10, abs=1e-12)


@pytest.mark.parametrize("seed", [1000, 1001, 1002])
def test_tiny_problem_matches_oracle_certificate(ctx, oracle_mod, seed):
    """10 x 8 components, eps = 1e-3: the GPU optimum and the stored oracle
    optimum (tests/golden/make_bnb_golden.py) certify each other."""
    gold = json.load(open(GOLDEN))[str(seed)]
    p = synth.tiny_problem(seed)
    ctx.set_problem(p)
    r = ctx.bnb_solve(eps=p["eps"], pop=1024, max_seconds=300, queue_capacity=1 << 27)
    assert r["status_name"] == "optimal"
    epsf = p["eps"] * gold["c22"]
    assert r["c22"] == pytest.approx(gold["c22"], rel=1e-12)
    assert abs(r["f"] - gold["f"]) <= epsf
    assert r["lb"] <= gold["f"] + 1e-9 and gold["lb"] <= r["f"] + 1e-9
    mix = oracle_mod.Mixtures.from_problem(p)
    assert oracle_mod.objective_r(mix, r["r"], r["t"]) == pytest.approx(r["f"], rel=1e-10)
    # both poses are optimal to within eps of each other's certificate
    assert oracle_mod.objective_r(mix, gold["r"], gold["t"]) - epsf <= r["f"]


def test_step_interface_matches_solve(ctx):
    p = _noise_free(2, 4, 0.1)
    ctx.set_problem(p)
    a = ctx.bnb_solve(eps=2e-2, pop=128, max_seconds=120)
    ctx.bnb_start(eps=2e-2, pop=128, max_seconds=120)
    r = ctx.bnb_step(3)
    assert r["status_name"] == "running" and r["iterations"] == 3
    while r["status_name"] == "running":
        r = ctx.bnb_step(50)
    for k in ("f", "lb", "nodes", "iterations", "sma_calls"):
        assert r[k] == a[k], k
    assert r["bound_ms"] > 0 and r["iteration_ms"] >= r["bound_ms"]


def test_automatic_pop(ctx):
    """pop = 0 takes 2^23 / (n1 n2) sub-cubes per iteration, clamped to
    [8192, 65536]: 65536 for 10 x 8 mixtures, 8192 for 128 x 64; the run is
    the same as with that pop given explicitly."""
    p = synth.tiny_problem(1000)
    ctx.set_problem(p)
    a = ctx.bnb_solve(eps=p["eps"], queue_capacity=1 << 26)
    b = ctx.bnb_solve(eps=p["eps"], pop=65536, queue_capacity=1 << 26)
    assert a["status_name"] == "optimal"
    for k in ("f", "lb", "nodes", "iterations"):
        assert a[k] == b[k], k
    q = synth.paper_scale_problem(2000)
    ctx.set_problem(q)
    a = ctx.bnb_solve(eps=q["eps"], max_nodes=200000)
    b = ctx.bnb_solve(eps=q["eps"], pop=8192, max_nodes=200000)
    for k in ("f", "lb", "nodes", "iterations"):
        assert a[k] == b[k], k


def test_limits_and_queue_capacity(ctx):
    p = synth.paper_scale_problem(2000)
    ctx.set_problem(p)
    r = ctx.bnb_solve(eps=p["eps"], pop=512, max_nodes=20000)
    assert r["status_name"] == "node_limit" and r["nodes"] >= 20000
    assert r["lb"] <= r["f"]
    r = ctx.bnb_solve(eps=p["eps"], pop=512, queue_capacity=16 * 512)
    assert r["status_name"] == "queue_full"
    assert r["lb"] <= r["f"]
    r = ctx.bnb_solve(eps=p["eps"], pop=512, max_seconds=0.5)
    assert r["status_name"] == "time_limit"


def test_step_before_start_is_an_error():
    from paper_1812_01232_gb300.gosma import Gosma, GosmaError
    c = Gosma(0)
    c.set_problem(synth.tiny_problem(3))
    with pytest.raises(GosmaError):
        c.bnb_step(1)
    c.close()


# ---------------------------------------------------------------- batched problems (one launch, CUDA graph)
def test_batch_matches_oracle_certificates(ctx, oracle_mod):
    """Two stored oracle certificates and a third problem of other sizes
    solved together in one batch: each result certifies against the oracle's
    optimum exactly as a single-problem solve does."""
    gold = json.load(open(GOLDEN))
    probs = [synth.tiny_problem(1000), synth.tiny_problem(11, n1=20, n_in=8, n_out=2), synth.tiny_problem(1001)]
    res = ctx.bnb_solve_batch(probs, eps=1e-3, pop=1024, max_seconds=300, queue_capacity=1 << 26)
    assert [r["status_name"] for r in res] == ["optimal"] * 3
    for p, r, seed in ((probs[0], res[0], 1000), (probs[2], res[2], 1001)):
        g = gold[str(seed)]
        epsf = 1e-3 * g["c22"]
        assert r["c22"] == pytest.approx(g["c22"], rel=1e-12)
        assert abs(r["f"] - g["f"]) <= epsf
        assert r["lb"] <= g["f"] + 1e-9 and g["lb"] <= r["f"] + 1e-9
        assert r["gap_norm"] <= 1e-3
    for p, r in zip(probs, res):
        mix = oracle_mod.Mixtures.from_problem(p)
        assert oracle_mod.objective_r(mix, r["r"], r["t"]) == pytest.approx(r["f"], rel=1e-10)
        assert r["sma_calls"] >= 1
    assert res[0]["block_size"] in (32, 64, 128, 256, 512, 1024)


def test_batch_noise_free_recovery(ctx, oracle_mod):
    probs = [_noise_free(2, 4, 0.1), _noise_free(3, 4, 0.1)]
    res = ctx.bnb_solve_batch(probs, eps=1e-2, pop=64, max_seconds=120, queue_capacity=1 << 24)
    for p, r in zip(probs, res):
        c22 = oracle_mod.c22(oracle_mod.Mixtures.from_problem(p))
        assert r["status_name"] == "optimal"
        assert r["f"] == pytest.approx(-c22, abs=1e-2 * c22)
        assert _rot_err(r["R"], p["R_gt"]) < 0.1
        assert np.linalg.norm(r["t"] - p["t_gt"]) < 0.05 * np.linalg.norm(p["t_gt"]) + 1e-3


@pytest.mark.parametrize("learned", [False, True])
def test_tiled_append_matches_the_oracle(ctx, oracle_mod, learned):
    """With pop 4096 (32,768 children per problem) the batch appends children
    in 4,096-child tiles (count, scan, scatter in child order): the
    certificates still cover the stored oracle optima, plain and learned."""
    gold = json.load(open(GOLDEN))
    probs = [synth.tiny_problem(1000), synth.tiny_problem(1001)]
    kw = dict(learned=dict(beta=1e-4, seed=True, active_iters=1000)) if learned else {}
    if learned:
        ctx.mlp_set_params(_params(5))
    res = ctx.bnb_solve_batch(probs, eps=1e-3, pop=4096, max_seconds=300, queue_capacity=1 << 26, **kw)
    for p, r, seed in zip(probs, res, (1000, 1001)):
        g = gold[str(seed)]
        epsf = 1e-3 * g["c22"]
        assert r["status_name"] == "optimal"
        assert abs(r["f"] - g["f"]) <= epsf
        assert r["lb"] <= g["f"] + 1e-9 and g["lb"] <= r["f"] + 1e-9
        mix = oracle_mod.Mixtures.from_problem(p)
        assert oracle_mod.objective_r(mix, r["r"], r["t"]) == pytest.approx(r["f"], rel=1e-10)


def test_batch_member_agrees_with_single_solve(ctx):
    """A problem solved alone, in a batch with a neighbour of other sizes, and
    by the single-problem solver reaches the same certified optimum."""
    a = synth.tiny_problem(1000)
    b = _noise_free(2, 4, 0.1)
    alone = ctx.bnb_solve_batch([a], eps=1e-2, pop=256, max_seconds=120, queue_capacity=1 << 24)[0]
    both = ctx.bnb_solve_batch([b, a], eps=1e-2, pop=256, max_seconds=120, queue_capacity=1 << 24)
    ctx.set_problem(a)
    single = ctx.bnb_solve(eps=1e-2, pop=256, max_seconds=120, queue_capacity=1 << 24)
    epsf = 1e-2 * single["c22"]
    for r in (alone, both[1]):
        assert r["status_name"] == "optimal"
        assert abs(r["f"] - single["f"]) <= epsf
        assert r["lb"] <= single["f"] + 1e-9 and single["lb"] <= r["f"] + 1e-9
    assert both[0]["status_name"] == "optimal" and both[0]["gap_norm"] <= 1e-2


def test_batch_limits_and_errors(ctx):
    from paper_1812_01232_gb300.gosma import GosmaError
    probs = [synth.tiny_problem(1000), synth.tiny_problem(1001)]
    res = ctx.bnb_solve_batch(probs, eps=1e-3, pop=64, max_nodes=4096)
    assert [r["status_name"] for r in res] == ["node_limit"] * 2
    assert all(r["nodes"] >= 4096 and r["lb"] <= r["f"] for r in res)
    res = ctx.bnb_solve_batch(probs, eps=1e-3, pop=64, queue_capacity=16 * 64)
    assert [r["status_name"] for r in res] == ["queue_full"] * 2
    assert ctx.bnb_solve_batch([], eps=1e-3) == []
    bad = dict(probs[0])
    bad["phi1"] = bad["phi1"] * 2.0
    with pytest.raises(GosmaError):
        ctx.bnb_solve_batch([probs[1], bad], eps=1e-3)
    with pytest.raises(GosmaError):
        ctx.bnb_solve_batch(probs, eps=1e-3, pop=-1)
    with pytest.raises(GosmaError):
        ctx.bnb_solve_batch(probs, eps=1e-3, pop=65537)
    with pytest.raises(GosmaError):  # 8 x pop x problems must stay below 2^31 (32-bit child offsets)
        ctx.bnb_solve_batch([probs[0]] * 4097, eps=1e-3, pop=65536, queue_capacity=1 << 20)


# ---------------------------------------------------------------- learned form (network-ordered queue, seeds, traces)
def _params(seed):
    from paper_1812_01232_gb300 import learn
    return learn.init_params(seed)


@pytest.mark.parametrize("beta,active", [(0.0, 0), (1e-4, 0), (1e-3, 8)])
def test_learned_form_keeps_the_certificate(ctx, oracle_mod, beta, active):
    """The network only reorders pops and proposes seeds: with any weights the
    certified optimum is the oracle's."""
    gold = json.load(open(GOLDEN))["1000"]
    ctx.mlp_set_params(_params(3))
    p = synth.tiny_problem(1000)
    r = ctx.bnb_solve_batch([p], eps=1e-3, pop=1024, max_seconds=120, queue_capacity=1 << 26,
                            learned=dict(beta=beta, seed=True, active_iters=active))[0]
    assert r["status_name"] == "optimal"
    assert abs(r["f"] - gold["f"]) <= 1e-3 * gold["c22"]
    assert r["lb"] <= gold["f"] + 1e-9 and gold["lb"] <= r["f"] + 1e-9
    mix = oracle_mod.Mixtures.from_problem(p)
    assert oracle_mod.objective_r(mix, r["r"], r["t"]) == pytest.approx(r["f"], rel=1e-10)


def test_learned_form_needs_parameters():
    from paper_1812_01232_gb300.gosma import Gosma, GosmaError
    c = Gosma(0)
    with pytest.raises(GosmaError):
        c.bnb_solve_batch([synth.tiny_problem(1)], eps=1e-2, learned=dict(beta=0.0))
    c.close()


def test_traces(ctx):
    """Trace records: pop order, the root first, features as documented and
    cubes inside the search domain."""
    probs = [synth.tiny_problem(1000), synth.tiny_problem(7, n1=14, n_in=6, n_out=2)]
    res, tr = ctx.bnb_solve_batch(probs, eps=1e-3, pop=64, max_nodes=20000, trace_cap=256)
    for k, (p, t) in enumerate(zip(probs, tr)):
        assert 0 < len(t) <= 256
        assert np.all(t["problem"] == k) and np.all(np.diff(t["iteration"]) >= 0)
        assert t["iteration"][0] == 0 and t["lb"][0] == -np.inf
        f = t["feat"]
        assert np.all(np.isfinite(f)) and np.all(np.abs(f) <= 8.0) and np.all(f[:, 15] == 1.0)
        assert f[0, 10] == -8.0 and f[0, 6] == pytest.approx(0.0, abs=1e-6)
        c = t["cube"]
        assert np.all(c[:, 4:7] - c[:, 7:10] >= p["t_lo"] - 1e-12) and np.all(c[:, 4:7] + c[:, 7:10] <= p["t_hi"] + 1e-12)
        assert np.all(np.abs(c[:, 0:3]) + c[:, 3:4] <= np.pi + 1e-12)
        # features carry the cube: rotation centre / pi and log2 half-width / 16
        assert np.allclose(f[:, 0:3], c[:, 0:3] / np.pi, atol=1e-2)
        assert np.allclose(f[:, 6], np.log2(c[:, 3] / np.pi) / 16, atol=1e-2)
        finite = np.isfinite(t["lb"])
        assert np.all(t["lb"][finite] <= t["ub"][finite] + 1e-6 * np.abs(t["ub"][finite]))


def test_history_follows_the_run(ctx):
    """Per-iteration history (the quantities of Fig. 5): d* never rises, the
    node count grows by 8 per popped cube, the last point is the result."""
    p = synth.tiny_problem(1000)
    ctx.set_problem(p)
    r = ctx.bnb_solve(eps=1e-3, pop=1024, max_seconds=120, queue_capacity=1 << 26)
    h = ctx.bnb_history()
    assert len(h) == r["iterations"]
    assert np.all(np.diff(h["dstar"]) <= 0) and np.all(np.diff(h["nodes"]) > 0)
    assert np.all(np.diff(h["seconds"]) >= 0) and np.array_equal(h["iteration"], np.arange(1, len(h) + 1))
    assert h["dstar"][-1] == r["f"] and h["lower_bound"][-1] == pytest.approx(r["lb"], abs=1e-12)
    assert h["nodes"][-1] == r["nodes"]
    # the incumbent reaches its final value early; most of the run raises the lower bound
    first = np.flatnonzero(h["dstar"] - r["f"] <= 1e-3 * r["c22"])[0]
    assert first < 0.5 * len(h)


def test_batch_bound_shapes_agree(ctx):
    """The bound kernel's shapes (threads per block x sub-cubes per block,
    32 x 2 in half-warp groups): every fixed shape and the autotuned run
    certify the same optima, the
    result reports the shape used, the autotuner timed the shapes at least
    once, and an unsupported shape is refused."""
    from paper_1812_01232_gb300.gosma import GosmaError
    probs = [synth.tiny_problem(200000 + s) for s in range(4)]
    tuned = ctx.bnb_solve_batch(probs, eps=1e-3, max_seconds=120, queue_capacity=1 << 24)
    assert all(r["tunings"] >= 1 for r in tuned)
    assert (tuned[0]["block_size"], tuned[0]["cubes_per_block"]) in [
        (32, 1), (32, 2), (64, 1), (64, 2), (128, 1), (128, 2), (128, 4), (256, 1), (256, 2), (256, 4)]
    for shape in ((32, 1), (32, 2), (64, 2), (128, 4), (256, 1)):
        res = ctx.bnb_solve_batch(probs, eps=1e-3, max_seconds=120, queue_capacity=1 << 24, shape=shape)
        for a, b in zip(res, tuned):
            assert a["block_size"] == shape[0] and a["cubes_per_block"] == shape[1] and a["tunings"] == 0
            if a["status_name"] == b["status_name"] == "optimal":
                assert abs(a["f"] - b["f"]) <= 1e-3 * a["c22"]
                assert a["lb"] <= b["f"] + 1e-9 and b["lb"] <= a["f"] + 1e-9
    with pytest.raises(GosmaError):
        ctx.bnb_solve_batch(probs, eps=1e-3, max_seconds=10, shape=(128, 3))
