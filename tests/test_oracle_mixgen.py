"""Pins of the oracle's mixture generation (Sec. 6: DP-means for the point
set, DP-vMF-means for the bearing vectors, maximum-likelihood fits) against
hand-worked passes, closed forms, separable data and the sampling
distributions the fits estimate."""
import json
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "dp_means_worked.json")


def _q(x, scale=2.0 ** 32):
    return np.rint(np.asarray(x) * scale) / scale


def test_worked_examples(oracle_mod):
    for case in json.load(open(GOLDEN))["cases"]:
        r = oracle_mod.dp_cluster(np.array(case["points"], float), case["lambda"],
                                  sigma_min=case.get("sigma_min", 1e-3))
        assert r["k"] == case["k"] and r["passes"] == case["passes"]
        np.testing.assert_array_equal(r["labels"], case["labels"])
        np.testing.assert_allclose(r["mu"], case["mu"], atol=1e-15)
        np.testing.assert_allclose(r["phi"], case["phi"], rtol=1e-15)
        np.testing.assert_allclose(r["sigma"], case["sigma"], rtol=1e-14)


def test_huge_penalty_gives_the_sample_mean(oracle_mod):
    x = np.random.default_rng(1).normal(size=(500, 3)) * [1.0, 2.0, 0.5] + [3, -1, 2]
    r = oracle_mod.dp_cluster(x, 1e12)
    xq = _q(x)
    assert r["k"] == 1 and np.all(r["labels"] == 0) and r["passes"] == 1
    np.testing.assert_allclose(r["mu"][0], xq.mean(0), atol=1e-13)
    sig = np.sqrt(np.sum((xq - xq.mean(0)) ** 2) / (3 * len(x)))
    assert r["sigma"][0] == pytest.approx(sig, rel=1e-12)
    assert r["phi"][0] == 1.0


def test_tiny_penalty_gives_one_cluster_per_point(oracle_mod):
    x = np.random.default_rng(2).uniform(-1, 1, (60, 3))
    r = oracle_mod.dp_cluster(x, 1e-12, sigma_min=0.01)
    assert r["k"] == 60
    assert len(set(r["labels"].tolist())) == 60
    np.testing.assert_allclose(r["mu"][r["labels"]], _q(x), atol=1e-15)
    np.testing.assert_array_equal(r["sigma"], 0.01)


def _blobs(rng, centres, n_each, spread):
    x = np.concatenate([c + spread * rng.normal(size=(n_each, 3)) for c in centres])
    lab = np.repeat(np.arange(len(centres)), n_each)
    perm = rng.permutation(len(x))
    return x[perm], lab[perm]


def _same_partition(a, b):
    pairs = set(zip(a.tolist(), b.tolist()))
    return len(pairs) == len(set(a.tolist())) == len(set(b.tolist()))


def test_separated_blobs_are_recovered(oracle_mod):
    rng = np.random.default_rng(3)
    centres = rng.uniform(-20, 20, (6, 3))
    centres[:, 0] += 10 * np.arange(6)  # pairwise far apart
    x, lab = _blobs(rng, centres, 200, 0.05)
    r = oracle_mod.dp_cluster(x, 1.0)
    assert r["k"] == 6
    assert _same_partition(r["labels"], lab)


def test_converged_state_is_a_fixed_point(oracle_mod):
    """At convergence every point lies within lambda of its centre, that centre
    is the nearest (lowest index on ties), and each centre is its members' mean."""
    x = np.random.default_rng(4).uniform(-3, 3, (400, 3))
    lam = 1.5
    r = oracle_mod.dp_cluster(x, lam, max_iter=200)
    assert 0 < r["passes"] < 200
    xq = _q(x)
    d2 = np.sum((xq[:, None, :] - r["mu"][None, :, :]) ** 2, axis=2)
    np.testing.assert_array_equal(np.argmin(d2, axis=1), r["labels"])
    assert np.all(d2.min(axis=1) <= lam)
    for c in range(r["k"]):
        np.testing.assert_allclose(r["mu"][c], xq[r["labels"] == c].mean(0), atol=1e-13)
        assert r["phi"][c] == pytest.approx(np.mean(r["labels"] == c), rel=1e-15)


def test_gaussian_fit_estimates_sigma(oracle_mod):
    rng = np.random.default_rng(5)
    x = 0.1 * rng.normal(size=(20000, 3)) + [1, 2, 3]
    r = oracle_mod.dp_cluster(x, 1e6)
    assert r["k"] == 1
    assert r["sigma"][0] == pytest.approx(0.1, rel=0.02)
    np.testing.assert_allclose(r["mu"][0], [1, 2, 3], atol=0.005)


def test_overflow_reports_minus_one(oracle_mod):
    rng = np.random.default_rng(6)
    centres = np.array([[0, 0, 0], [50, 0, 0], [0, 50, 0], [0, 0, 50], [50, 50, 0], [50, 0, 50]], float)
    x, _ = _blobs(rng, centres, 20, 0.01)
    assert oracle_mod.dp_cluster(x, 1.0, kmax=3)["k"] == -1


# ---------------------------------------------------------------- DP-vMF-means
def _vmf_sample(rng, mu, kappa, n):
    """Textbook sampler of the vMF on S^2: w = 1 + log(u + (1 - u) e^{-2 kappa}) / kappa
    is the cosine with mu, the azimuth is uniform."""
    u = rng.random(n)
    w = 1.0 + np.log(u + (1.0 - u) * np.exp(-2.0 * kappa)) / kappa
    phi = rng.uniform(0, 2 * np.pi, n)
    s = np.sqrt(np.clip(1 - w * w, 0, None))
    mu = mu / np.linalg.norm(mu)
    a = np.array([1.0, 0, 0]) if abs(mu[0]) < 0.9 else np.array([0, 1.0, 0])
    e1 = np.cross(mu, a)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(mu, e1)
    return w[:, None] * mu + s[:, None] * (np.cos(phi)[:, None] * e1 + np.sin(phi)[:, None] * e2)


def test_vmf_low_threshold_gives_the_mean_direction(oracle_mod):
    x = _vmf_sample(np.random.default_rng(7), np.array([1.0, 2.0, 2.0]), 5.0, 3000)
    r = oracle_mod.dp_cluster(x, -1.5, vmf=True)
    assert r["k"] == 1
    s = _q(x, 2.0 ** 40).sum(0)
    np.testing.assert_allclose(r["mu"][0], s / np.linalg.norm(s), atol=1e-14)


def test_vmf_fit_estimates_kappa(oracle_mod):
    """kappa solves coth k - 1/k = |sum x| / n and estimates the sampler's kappa."""
    rng = np.random.default_rng(8)
    mu = np.array([0.3, -0.2, 0.9])
    x = _vmf_sample(rng, mu, 50.0, 20000)
    r = oracle_mod.dp_cluster(x, -1.5, vmf=True)
    k = r["kappa"][0]
    rbar = np.linalg.norm(_q(x, 2.0 ** 40).sum(0)) / len(x)
    assert 1 / np.tanh(k) - 1 / k == pytest.approx(rbar, rel=1e-12)
    assert k == pytest.approx(50.0, rel=0.03)
    assert np.arccos(np.clip(r["mu"][0] @ (mu / np.linalg.norm(mu)), -1, 1)) < 0.01


def test_vmf_separated_directions_are_recovered(oracle_mod):
    rng = np.random.default_rng(9)
    dirs = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [-1, 0, 0], [0, -1, 0]], float)
    x = np.concatenate([_vmf_sample(rng, d, 500.0, 150) for d in dirs])
    lab = np.repeat(np.arange(5), 150)
    perm = rng.permutation(len(x))
    r = oracle_mod.dp_cluster(x[perm], np.cos(np.radians(25)), vmf=True)
    assert r["k"] == 5
    assert _same_partition(r["labels"], lab[perm])


def test_vmf_cluster_with_zero_direction_sum(oracle_mod):
    """Reading M2: a cluster whose direction sum is exactly zero is centred
    on its lowest-index point.  Antipodal unit vectors with a threshold
    below -1 share one cluster whose sum is zero; its centre is the first
    vector in either order, and a zero resultant length gives the smallest
    concentration the fit returns."""
    for x in (np.array([[0.0, 0.0, 1.0], [0.0, 0.0, -1.0]]),
              np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [-1.0, 0.0, 0.0]])):
        for order in (x, x[::-1].copy()):
            r = oracle_mod.dp_cluster(order, -1.5, vmf=True, max_iter=10, kappa_max=1e4)
            assert r["k"] == 1 and r["passes"] == 1
            np.testing.assert_array_equal(r["labels"], np.zeros(len(order), int))
            np.testing.assert_array_equal(r["mu"][0], order[0])
            assert r["kappa"][0] < 1e-6 and r["phi"][0] == 1.0


def test_vmf_fit_capped_at_kappa_max(oracle_mod):
    """Reading M3: identical directions have mean resultant length 1, whose
    maximum-likelihood concentration is unbounded; the fit returns the cap.
    A spread-out cluster stays below it."""
    x = np.tile([[0.6, 0.0, 0.8]], (5, 1))
    r = oracle_mod.dp_cluster(x, 0.5, vmf=True, max_iter=10, kappa_max=1234.0)
    assert r["k"] == 1 and r["kappa"][0] == 1234.0
    y = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    r = oracle_mod.dp_cluster(y, -0.5, vmf=True, max_iter=10, kappa_max=1234.0)
    assert r["k"] == 1 and 0.0 < r["kappa"][0] < 10.0
