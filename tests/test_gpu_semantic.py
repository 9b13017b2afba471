"""Semantic form (Sec. 4.2): f = sum_l w_l f_l over classes, each class with
its own mixtures.  The reference is the FP64 oracle applied class by class
and summed with the weights (the objective, C22 and Theorem 1 bounds are
all linear in the class terms); the GPU evaluates the whole sum in one pass
with pairs restricted to within-class pairs."""
import numpy as np
import pytest

from paper_1812_01232_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1812_01232_gb300 import build
    build.build()
    from paper_1812_01232_gb300.gosma import Gosma
    c = Gosma(0)
    yield c
    c.close()


def _mixes(oracle_mod, p):
    return [oracle_mod.Mixtures.from_problem(dict(c, t_lo=p["t_lo"], t_hi=p["t_hi"], zeta=p["zeta"]))
            for c in p["classes"]]


def _ref_bounds(oracle_mod, p, cubes):
    """Weighted sum of the per-class oracle records (lb, ub, self_lb, cross_ub,
    self_c, cross_c, psi_r, psi_t_max)."""
    recs = [oracle_mod.bounds(m, cubes, p["zeta"]) for m in _mixes(oracle_mod, p)]
    out = np.zeros_like(recs[0])
    for w, r in zip(p["w"], recs):
        out[:, :6] += w * r[:, :6]
    out[:, 6] = recs[0][:, 6]
    out[:, 7] = np.max([r[:, 7] for r in recs], axis=0)
    return out


def test_objective_and_c22(ctx, oracle_mod):
    p = synth.semantic_problem(5, nclass=3)
    ctx.set_problem(p)
    mixes = _mixes(oracle_mod, p)
    rng = np.random.default_rng(0)
    for _ in range(8):
        r = rng.uniform(-2, 2, 3)
        t = rng.uniform(-1, 1, 3)
        f = ctx.eval_objective(r, t)
        ref = sum(w * oracle_mod.objective_r(m, r, t) for w, m in zip(p["w"], mixes))
        assert f == pytest.approx(ref, rel=1e-10, abs=1e-12)
    r = ctx.bnb_solve(eps=0.5, pop=64, max_nodes=64)
    c22 = sum(w * oracle_mod.c22(m) for w, m in zip(p["w"], mixes))
    assert r["c22"] == pytest.approx(c22, rel=1e-12)


@pytest.mark.parametrize("seed", [6, 7])
def test_bounds_parity(ctx, oracle_mod, seed):
    from test_gpu_bounds import compare
    p = synth.semantic_problem(seed, nclass=3, n1=5, n_in=3, n_out=2)
    ctx.set_problem(p)
    cubes = synth.tree_cubes(seed + 100, 777, p["t_lo"], p["t_hi"], 0, 14, near=(p["r_gt"], p["t_gt"]), near_frac=0.4)
    got = ctx.eval_bounds_detail(cubes)
    ref = _ref_bounds(oracle_mod, p, cubes)
    compare(got, ref, "semantic")


def test_one_class_equals_plain(ctx):
    p = synth.tiny_problem(1000)
    cubes = synth.tree_cubes(9, 300, p["t_lo"], p["t_hi"], 0, 12)
    ctx.set_problem(p)
    a = ctx.eval_bounds_detail(cubes)
    ctx.set_mixtures_classes([len(p["sigma1"])], [len(p["kappa2"])], [1.0], p["mu1"], p["sigma1"], p["phi1"],
                             p["mu2"], p["kappa2"], p["phi2"])
    b = ctx.eval_bounds_detail(cubes)
    assert np.array_equal(a, b)


def test_noise_free_recovery(ctx, oracle_mod):
    """Noise-free classes: the minimum is -C22 at the true pose."""
    p = synth.semantic_problem(3, nclass=2, n1=3, noise_free=True)
    ctx.set_problem(p)
    r = ctx.bnb_solve(eps=1e-2, pop=256, max_seconds=120, queue_capacity=1 << 25)
    assert r["status_name"] == "optimal"
    assert r["f"] == pytest.approx(-r["c22"], abs=1e-2 * r["c22"])
    ang = np.arccos(np.clip((np.trace(r["R"].T @ p["R_gt"]) - 1) / 2, -1, 1))
    assert ang < 0.1
    assert np.linalg.norm(r["t"] - p["t_gt"]) < 0.05 * np.linalg.norm(p["t_gt"]) + 1e-3


def test_certificate_against_the_oracle(ctx, oracle_mod):
    """A certified semantic optimum: the reported f is the oracle's f at the
    reported pose, and no sampled pose (nor the true one) lies below the
    certified lower bound."""
    p = synth.semantic_problem(11, nclass=2, n1=4, n_in=3, n_out=1)
    ctx.set_problem(p)
    r = ctx.bnb_solve(eps=1e-2, pop=256, max_seconds=120, queue_capacity=1 << 25)
    assert r["status_name"] == "optimal" and r["gap_norm"] <= 1e-2
    mixes = _mixes(oracle_mod, p)
    fo = lambda rr, tt: sum(w * oracle_mod.objective_r(m, rr, tt) for w, m in zip(p["w"], mixes))
    assert fo(r["r"], r["t"]) == pytest.approx(r["f"], rel=1e-10, abs=1e-12)
    rng = np.random.default_rng(1)
    zeta2 = p["zeta"] ** 2
    for _ in range(300):
        t = rng.uniform(-1, 1, 3)
        if np.min(np.sum((p["mu1"] - t) ** 2, axis=1)) < zeta2:
            continue
        assert fo(rng.uniform(-np.pi, np.pi, 3) / np.sqrt(3), t) >= r["lb"] - 1e-9
    assert fo(p["r_gt"], p["t_gt"]) >= r["lb"] - 1e-9


def test_invalid_classes(ctx):
    from paper_1812_01232_gb300.gosma import GosmaError
    p = synth.semantic_problem(5, nclass=2)
    with pytest.raises(GosmaError):   # class sizes that do not cover the arrays
        ctx.set_mixtures_classes([3, 3], p["n2c"], p["w"], p["mu1"], p["sigma1"], p["phi1"], p["mu2"], p["kappa2"],
                                 p["phi2"])
    bad = p["phi1"].copy()
    bad[0] += 0.1                     # class 0 weights no longer sum to 1
    with pytest.raises(GosmaError):
        ctx.set_mixtures_classes(p["n1c"], p["n2c"], p["w"], p["mu1"], p["sigma1"], bad, p["mu2"], p["kappa2"],
                                 p["phi2"])
    with pytest.raises(GosmaError):
        ctx.set_mixtures_classes([p["n1c"][0], 0], p["n2c"], p["w"], p["mu1"], p["sigma1"], p["phi1"], p["mu2"],
                                 p["kappa2"], p["phi2"])


def test_batched_semantic_problems(ctx, oracle_mod):
    """Semantic and plain problems in one batch reach the certificates of
    their single-problem solves."""
    probs = [synth.semantic_problem(11, nclass=2, n1=4, n_in=3, n_out=1), synth.tiny_problem(1000),
             synth.semantic_problem(3, nclass=2, n1=3, noise_free=True)]
    res = ctx.bnb_solve_batch(probs, eps=1e-2, pop=256, max_seconds=120, queue_capacity=1 << 25)
    for p, r in zip(probs, res):
        ctx.set_problem(p)
        s = ctx.bnb_solve(eps=1e-2, pop=256, max_seconds=120, queue_capacity=1 << 25)
        assert r["status_name"] == s["status_name"] == "optimal"
        assert r["c22"] == pytest.approx(s["c22"], rel=1e-12)
        assert abs(r["f"] - s["f"]) <= 1e-2 * s["c22"]
        assert r["lb"] <= s["f"] + 1e-9 and s["lb"] <= r["f"] + 1e-9
    p = probs[0]
    mixes = _mixes(oracle_mod, p)
    f = sum(w * oracle_mod.objective_r(m, res[0]["r"], res[0]["t"]) for w, m in zip(p["w"], mixes))
    assert f == pytest.approx(res[0]["f"], rel=1e-10, abs=1e-12)
