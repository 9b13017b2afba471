"""The seeded input generators shared by the oracle tests and the GPU path
(paper_1812_01232_gb300/synth.py) produce well-formed problems: mixture
weights summing to 1 (per class for semantic problems), unit image means,
positive spreads, a true camera inside the translation domain and at least
zeta from every model mean, a rotation in the pi-ball whose matrix is the
Rodrigues matrix of the angle-axis vector, and deterministic output per seed."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from paper_1812_01232_gb300 import synth

GENERATORS = {
    "tiny": lambda s: synth.tiny_problem(s),
    "noise_free": lambda s: synth.noise_free_problem(s),
    "paper_scale": lambda s: synth.paper_scale_problem(s),
    "uneven": lambda s: synth.uneven_problems(s, count=3)[2],
    "stress": lambda s: synth.stress_problem(s, n1=256, n2=64),
}


def _check(p):
    n1, n2 = len(p["sigma1"]), len(p["kappa2"])
    assert p["mu1"].shape == (n1, 3) and p["mu2"].shape == (n2, 3)
    assert np.all(p["sigma1"] > 0) and np.all(p["kappa2"] > 0)
    assert np.all(p["phi1"] >= 0) and np.all(p["phi2"] >= 0)
    np.testing.assert_allclose(np.linalg.norm(p["mu2"], axis=1), 1.0, atol=1e-12)
    t = p["t_gt"]
    assert np.all(t >= p["t_lo"]) and np.all(t <= p["t_hi"])
    assert np.min(np.linalg.norm(p["mu1"] - t, axis=1)) >= p["zeta"]
    assert np.linalg.norm(p["r_gt"]) <= np.pi + 1e-12
    np.testing.assert_allclose(p["R_gt"], Rotation.from_rotvec(p["r_gt"]).as_matrix(), atol=1e-12)


@pytest.mark.parametrize("name", sorted(GENERATORS))
def test_problems_are_well_formed_and_deterministic(name):
    for seed in (0, 1, 1000):
        p = GENERATORS[name](seed)
        _check(p)
        assert np.sum(p["phi1"]) == pytest.approx(1.0, abs=1e-12)
        assert np.sum(p["phi2"]) == pytest.approx(1.0, abs=1e-12)
        q = GENERATORS[name](seed)
        for k in ("mu1", "sigma1", "phi1", "mu2", "kappa2", "phi2", "t_gt", "r_gt"):
            np.testing.assert_array_equal(p[k], q[k])


def test_semantic_problems_sum_to_one_per_class():
    p = synth.semantic_problem(5, nclass=3)
    _check(p)
    i0 = j0 = 0
    for a, b in zip(p["n1c"], p["n2c"]):
        assert np.sum(p["phi1"][i0:i0 + a]) == pytest.approx(1.0, abs=1e-12)
        assert np.sum(p["phi2"][j0:j0 + b]) == pytest.approx(1.0, abs=1e-12)
        i0, j0 = i0 + a, j0 + b
    assert i0 == len(p["phi1"]) and j0 == len(p["phi2"])
    assert np.sum(p["w"]) == pytest.approx(1.0)


def test_pose_seeds_and_scene():
    p = synth.tiny_problem(3)
    x = synth.pose_seeds(p, 64, 1)
    assert x.shape == (64, 6)
    assert np.all(np.linalg.norm(x[1::2, :3], axis=1) <= np.pi)      # uniform half: inside the pi-ball
    assert np.all(x[1::2, 3:] >= p["t_lo"]) and np.all(x[1::2, 3:] <= p["t_hi"])
    np.testing.assert_array_equal(x, synth.pose_seeds(p, 64, 1))
    sc = synth.scene_points(2, n=2000, n_bear=500)
    assert sc["points"].shape == (2000, 3) and sc["bearings"].shape == (500, 3)
    np.testing.assert_allclose(np.linalg.norm(sc["bearings"], axis=1), 1.0, atol=1e-12)
    assert np.all(sc["bearings"][:, 2] > np.cos(np.radians(60)) - 1e-12)  # inside the camera's 60-degree cone
    assert np.all(np.abs(sc["points"][:, :2]) <= 5.1) and np.all(sc["points"][:, 2] >= -0.1)
