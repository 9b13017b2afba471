"""Pins of the FP64 oracle against facts fixed outside it.

Each test checks the oracle against something it does not compute itself:
numerical quadrature on the sphere, a closed form, the values printed in
the paper's Figure 3(b), a library routine (scipy's rotation), or dense
sampling of the cube that a bound must dominate.
"""
import os

import numpy as np
import pytest
from scipy import integrate
from scipy.spatial.transform import Rotation
from scipy.stats import norm

from paper_1812_01232_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Eq. (Z)
@pytest.mark.parametrize("kappa", [1e-6, 1e-3, 0.1, 1.0, 7.5, 60.0, 700.0])
def test_logZ_is_log_of_vmf_normaliser(oracle_mod, kappa):
    # 2 pi Z(k) = integral over S^2 of exp(k mu.f) = 2 pi * integral_{-1}^{1} exp(k x) dx;
    # integrate exp(k (x - 1)) to stay in range and add k back.
    val, _ = integrate.quad(lambda x: np.exp(kappa * (x - 1.0)), -1.0, 1.0, epsabs=0, epsrel=1e-13, limit=200)
    assert oracle_mod.logZ(kappa) == pytest.approx(kappa + np.log(val), rel=1e-11, abs=1e-12)


def test_logZ_limits(oracle_mod):
    assert oracle_mod.logZ(0.0) == pytest.approx(np.log(2.0), abs=1e-15)
    x = 1e-3
    assert oracle_mod.logZ(x) == pytest.approx(np.log(2.0) + x * x / 6 - x ** 4 / 180, rel=1e-14)
    assert oracle_mod.phiZ(40.0) == pytest.approx(-np.log(40.0), rel=1e-14)
    # near 0, phiZ(x) = log((1 - e^{-2x}) / x) = log 2 - x + x^2 / 6 + O(x^3):
    # below and above any switch to a series the value follows it to rounding
    for x in (1e-16, 3e-14, 9.9e-13, 1e-12, 1.01e-12, 1e-11, 1e-9):
        assert abs(oracle_mod.phiZ(x) - (np.log(2.0) - x + x * x / 6)) <= 2e-16, x


# ------------------------------------------------- vMF inner product (Lemma 1 proof)
def _sphere_quadrature(n_theta=240, n_phi=480):
    """Gauss-Legendre in cos(theta) times the periodic trapezoid rule in phi."""
    x, w = np.polynomial.legendre.leggauss(n_theta)
    ph = np.arange(n_phi) * (2 * np.pi / n_phi)
    st = np.sqrt(1 - x * x)
    F = np.stack([np.outer(st, np.cos(ph)), np.outer(st, np.sin(ph)), np.outer(x, np.ones(n_phi))], axis=-1)
    W = np.outer(w, np.full(n_phi, 2 * np.pi / n_phi))
    return F.reshape(-1, 3), W.reshape(-1)


def _vmf_density(F, mu, kappa):
    # Eq. (vMF) written directly: exp(k mu.f) / (2 pi Z(k)), Z(k) = (e^k - e^-k)/k
    return kappa * np.exp(kappa * (F @ mu - 1.0)) / (2 * np.pi * (1 - np.exp(-2 * kappa)))


@pytest.mark.parametrize("ka,kb,ang", [(3.0, 5.0, 0.3), (20.0, 8.0, 1.2), (0.5, 12.0, 2.9), (15.0, 15.0, 0.0)])
def test_pair_log_matches_quadrature(oracle_mod, ka, kb, ang):
    F, W = _sphere_quadrature()
    rng = np.random.default_rng(7)
    R = Rotation.random(random_state=rng).as_matrix()
    ua = R @ np.array([0.0, 0.0, 1.0])
    ub = R @ np.array([np.sin(ang), 0.0, np.cos(ang)])
    integral = np.sum(W * _vmf_density(F, ua, ka) * _vmf_density(F, ub, kb))
    # integral of vMF_a vMF_b = Z(K) / (2 pi Z_a Z_b)
    assert np.exp(oracle_mod.pair_log(ka, ua, kb, ub)) / (2 * np.pi) == pytest.approx(integral, rel=1e-9)


@pytest.mark.parametrize("k", [1e-4, 0.3, 2.0, 50.0, 3000.0])
def test_aligned_pair_closed_form(oracle_mod, k):
    u = np.array([0.0, 0.6, 0.8])
    # Z(2k) / Z(k)^2 = k coth(k) / 2
    assert np.exp(oracle_mod.pair_log(k, u, k, u)) == pytest.approx(0.5 * k / np.tanh(k), rel=1e-12)


# ------------------------------------------------- qPN mapping (Eq. qPN), Figure 3(b)
def _pn_density(alpha_angle, rho):
    # Eq. (PN), isotropic projected normal, written directly (Phi from scipy)
    a = rho * np.cos(alpha_angle)
    return np.exp(-rho ** 2 / 2) / (2 * np.pi) * (a / np.sqrt(2 * np.pi) + norm.cdf(a) * np.exp(a ** 2 / 2) * (1 + a ** 2))


def test_qpn_mae_reproduces_figure_3b(oracle_mod):
    """The MAE of Figure 3(b) is the mean over the integer angles 0..180
    degrees of |PN - qPN|; the oracle's qPN concentration and log Z must
    reproduce every printed value."""
    rows = np.loadtxt(os.path.join(GOLDEN, "qpn_mae_fig3b.txt"))
    ang = np.deg2rad(np.arange(181))
    sigma = 0.7
    for rho, mae in rows:
        kappa = oracle_mod.kappa_qpn(rho * sigma, sigma)
        qpn = np.exp(kappa * np.cos(ang) - oracle_mod.logZ(kappa)) / (2 * np.pi)
        got = np.mean(np.abs(_pn_density(ang, rho) - qpn))
        assert got == pytest.approx(mae, rel=1e-9), rho


# ------------------------------------------------- Lemma 1: objective = L2 distance
def _l2_by_quadrature(prob, R, t, F, W):
    mu1, s1, w1 = prob["mu1"], prob["sigma1"], prob["phi1"]
    p1 = np.zeros(len(W))
    for i in range(len(w1)):
        d = R @ (mu1[i] - t)  # transformed model T(theta_1, R, t)
        k = (np.linalg.norm(mu1[i] - t) / s1[i]) ** 2 + 1  # Eq. (qPN)
        p1 += w1[i] * _vmf_density(F, d / np.linalg.norm(d), k)
    p2 = np.zeros(len(W))
    for j in range(len(prob["phi2"])):
        p2 += prob["phi2"][j] * _vmf_density(F, prob["mu2"][j], prob["kappa2"][j])
    return np.sum(W * (p1 - p2) ** 2), np.sum(W * p2 ** 2)


def _small_prob(seed):
    rng = np.random.default_rng(seed)
    mu1 = rng.uniform(-2, 2, (3, 3))
    mu2 = rng.standard_normal((2, 3))
    mu2 /= np.linalg.norm(mu2, axis=1, keepdims=True)
    return dict(mu1=mu1, sigma1=rng.uniform(0.6, 1.2, 3), phi1=rng.dirichlet(np.ones(3)),
                mu2=mu2, kappa2=rng.uniform(1.0, 12.0, 2), phi2=rng.dirichlet(np.ones(2)))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_objective_equals_l2_distance(oracle_mod, seed):
    prob = _small_prob(seed)
    mix = oracle_mod.Mixtures.from_problem(prob)
    F, W = _sphere_quadrature(300, 600)
    rng = np.random.default_rng(100 + seed)
    R = Rotation.random(random_state=rng).as_matrix()
    t = rng.uniform(-0.3, 0.3, 3)
    d_l2, p2sq = _l2_by_quadrature(prob, R, t, F, W)
    f = oracle_mod.objective(mix, R, t)
    c22 = oracle_mod.c22(mix)
    # d_L2 = (f + C22) / (2 pi) and C22 = 2 pi * integral of p2^2
    assert c22 == pytest.approx(2 * np.pi * p2sq, rel=1e-9)
    assert (f + c22) / (2 * np.pi) == pytest.approx(d_l2, rel=1e-8, abs=1e-12)


def test_objective_parts_sum(oracle_mod):
    prob = _small_prob(5)
    mix = oracle_mod.Mixtures.from_problem(prob)
    R = Rotation.from_rotvec([0.3, -0.2, 1.0]).as_matrix()
    t = np.array([0.1, 0.2, -0.1])
    s, c = oracle_mod.objective_parts(mix, R, t)
    assert s - 2 * c == pytest.approx(oracle_mod.objective(mix, R, t), rel=1e-13)


# ------------------------------------------------- rotation parameterisation (Sec. 4.1)
def test_rodrigues_matches_scipy(oracle_mod):
    rng = np.random.default_rng(3)
    for _ in range(50):
        r = rng.uniform(-np.pi, np.pi, 3)
        assert np.allclose(oracle_mod.rodrigues(r), Rotation.from_rotvec(r).as_matrix(), atol=1e-14)
    assert np.allclose(oracle_mod.rodrigues([1e-10, 0, 0]), Rotation.from_rotvec([1e-10, 0, 0]).as_matrix())


# ------------------------------------------------- Lemma 2 / Lemma 3 by dense sampling
def test_psi_r_dominates_sampled_rotations(oracle_mod):
    rng = np.random.default_rng(11)
    for _ in range(40):
        hw = rng.uniform(0.01, 1.2)
        r0 = rng.uniform(-2, 2, 3)
        p = rng.standard_normal(3)
        R0p = Rotation.from_rotvec(r0).apply(p)
        rs = r0 + rng.uniform(-hw, hw, (400, 3))
        rs[:8] = r0 + hw * np.array([[(k >> a & 1) * 2 - 1 for a in range(3)] for k in range(8)])
        Rp = Rotation.from_rotvec(rs).apply(p)
        ang = np.arccos(np.clip(Rp @ R0p / np.linalg.norm(p) ** 2, -1, 1))
        assert ang.max() <= oracle_mod.psi_r(hw) + 1e-12


def _largest_rotation_angle(r0, hw, p, rng, n_inner=2000):
    """Largest angle between R_r p and R_r0 p (scipy rotations) over samples of
    the rotation cube: its 8 vertices, 20 points on each of its 12 edges,
    100 on each of its 6 faces and n_inner inside."""
    corners = np.array([[(k >> a & 1) * 2 - 1 for a in range(3)] for k in range(8)], float)
    pts = [corners]
    for a in range(3):  # edges along axis a
        for k in range(4):
            e = np.zeros((20, 3))
            e[:, a] = np.linspace(-1, 1, 20)
            o = [b for b in range(3) if b != a]
            e[:, o[0]] = 1.0 if k & 1 else -1.0
            e[:, o[1]] = 1.0 if k & 2 else -1.0
            pts.append(e)
    for a in range(3):  # faces normal to axis a
        for sgn in (-1.0, 1.0):
            f = rng.uniform(-1, 1, (100, 3))
            f[:, a] = sgn
            pts.append(f)
    pts.append(rng.uniform(-1, 1, (n_inner, 3)))
    rs = r0 + hw * np.concatenate(pts)
    a = Rotation.from_rotvec(rs).apply(p)
    b = Rotation.from_rotvec(r0).apply(p)
    return float(np.arctan2(np.linalg.norm(np.cross(a, b), axis=1), a @ b).max())


def _random_rotation_cube(rng, k):
    """Cube centres over the whole pi-ball, a third of them near its surface,
    where the exponential map's Jacobian contracts most."""
    d = rng.standard_normal(3)
    d /= np.linalg.norm(d)
    rad = rng.uniform(2.6, 3.1) if k % 3 == 0 else rng.uniform(0, 2.6)
    return rad * d


def test_point_psi_r_dominates_sampled_rotations(oracle_mod):
    """Lemma 2, point-dependent form (reading R16): the bound is never below
    the largest angle found by dense sampling of the rotation cube, and never
    above the point-independent sqrt(3) h."""
    rng = np.random.default_rng(13)
    for k in range(90):
        hw = [1e-3, 1e-2, 0.05, 0.2, 0.5, 1.0][k % 6]
        r0 = _random_rotation_cube(rng, k)
        p = rng.standard_normal(3)
        p /= np.linalg.norm(p)
        bound = oracle_mod.psi_r_point(r0, hw, p)
        assert _largest_rotation_angle(r0, hw, p, rng) <= bound + 1e-12, (k, r0, hw, p)
        assert bound <= oracle_mod.psi_r(hw) + 1e-15


def test_point_psi_r_is_tight_for_small_cubes(oracle_mod):
    """The bound's first-order term is attained at a vertex, so for small cubes
    it exceeds the sampled maximum by second-order terms only (at most 3 h^2 / 4
    of allowance and 3 h^2 / 4 of linearisation at the vertex)."""
    rng = np.random.default_rng(14)
    for k in range(60):
        hw = [1e-3, 3e-3][k % 2]
        r0 = _random_rotation_cube(rng, k)
        p = rng.standard_normal(3)
        p /= np.linalg.norm(p)
        bound = oracle_mod.psi_r_point(r0, hw, p)
        assert bound - _largest_rotation_angle(r0, hw, p, rng, 200) <= 2 * hw * hw, (k, r0, p)


@pytest.mark.parametrize("hw", [1e-3, 1e-2, 0.1])
def test_point_psi_r_closed_form_at_the_identity(oracle_mod, hw):
    """At r0 = 0 a unit vector p on a coordinate axis turns by at most sqrt(2) h
    over the cube (attained at r = (0, h, h) for p = e_x: the angle is
    2 asin(sin(|r|/2) |r x p| / |r|), largest where r is orthogonal to p), and
    the bound is that plus its second-order allowance."""
    for p in np.eye(3):
        b = oracle_mod.psi_r_point(np.zeros(3), hw, p)
        assert np.sqrt(2) * hw <= b <= np.sqrt(2) * hw + 0.8 * hw * hw
    # along the diagonal the largest turn is smaller: sqrt(8/3) h to first order
    d = np.ones(3) / np.sqrt(3)
    assert oracle_mod.psi_r_point(np.zeros(3), hw, d) <= np.sqrt(8 / 3) * hw + 0.8 * hw * hw


def test_psi_t_dominates_sampled_translations(oracle_mod):
    rng = np.random.default_rng(12)
    tight = 0
    for _ in range(200):
        t0 = rng.uniform(-1, 1, 3)
        thw = rng.uniform(0.01, 0.6, 3)
        p = t0 + rng.uniform(-3, 3, 3)
        psi = oracle_mod.psi_t(p, t0, thw)
        ts = t0 + rng.uniform(-1, 1, (2000, 3)) * thw
        a = p - ts
        c = p - t0
        ang = np.arccos(np.clip(a @ c / (np.linalg.norm(a, axis=1) * np.linalg.norm(c)), -1, 1))
        assert ang.max() <= psi + 1e-12
        if psi < np.pi / 2:
            tight += 1
            # the vertex maximum is attained by a vertex
            verts = t0 + thw * np.array([[(k >> q & 1) * 2 - 1 for q in range(3)] for k in range(8)])
            av = p - verts
            va = np.arccos(np.clip(av @ c / (np.linalg.norm(av, axis=1) * np.linalg.norm(c)), -1, 1))
            assert psi == pytest.approx(va.max(), rel=1e-12)
    assert tight > 50
    # a point inside the cuboid has psi_t = pi
    assert oracle_mod.psi_t([0.1, 0.1, 0.1], [0, 0, 0], [0.2, 0.2, 0.2]) == pytest.approx(np.pi)


def test_kappa_interval_contains_sampled_kappas(oracle_mod):
    rng = np.random.default_rng(13)
    zeta = 0.5
    for _ in range(200):
        t0 = rng.uniform(-1, 1, 3)
        thw = rng.uniform(0.05, 1.0, 3)
        p = t0 + rng.uniform(-2, 2, 3)
        sigma = rng.uniform(0.03, 0.3)
        ab = oracle_mod.kappa_interval(p, sigma, t0, thw, zeta)
        ts = t0 + rng.uniform(-1, 1, (3000, 3)) * thw
        d = np.linalg.norm(p - ts, axis=1)
        feas = d >= zeta
        if ab is None:
            assert not feas.any()
            continue
        k = (d[feas] / sigma) ** 2 + 1
        assert k.min() >= ab[0] * (1 - 1e-12) and k.max() <= ab[1] * (1 + 1e-12)


# ------------------------------------------------- Theorem 1 per pair, by brute force over its relaxation
def _term_grid(oracle_mod, k1s, k2s, angles):
    """Z(K)/(Z(k1)Z(k2)) from the pinned pair_log on a grid of concentrations
    and angles between the two mean directions."""
    u = np.array([1.0, 0.0, 0.0])
    out = np.empty((len(k1s), len(k2s), len(angles)))
    for c, ang in enumerate(angles):
        w = np.array([np.cos(ang), np.sin(ang), 0.0])
        for a, k1 in enumerate(k1s):
            for b, k2 in enumerate(k2s):
                out[a, b, c] = np.exp(oracle_mod.pair_log(k1, u, k2, w))
    return out


def _box_grid(lo, hi, n):
    """Both ends, evenly and geometrically spaced points of [lo, hi]."""
    return np.unique(np.concatenate([np.linspace(lo, hi, n), np.geomspace(lo, hi, n)]))


def test_self_pair_bound_below_the_term_over_its_relaxation(oracle_mod):
    """Theorem 1, self pairs: over the cuboid, kappa_1i and kappa_1j stay in
    their intervals and the angle between the two mean directions stays at
    most A (Eq. K1i1j_lb_A with Lemma 3), so the bound must not exceed the
    pair term anywhere on that box of (kappa_1i, kappa_1j, angle); broad
    components keep the concentrations small, where every factor matters."""
    rng = np.random.default_rng(14)
    zeta, checked, wide = 0.05, 0, 0
    for _ in range(120):
        mu1 = rng.uniform(-2, 2, (2, 3))
        prob = {"mu1": mu1, "sigma1": rng.uniform(0.1, 1.0, 2), "phi1": np.array([0.3, 0.7]),
                "mu2": np.array([[0.0, 0.0, 1.0]]), "kappa2": np.array([5.0]), "phi2": np.array([1.0])}
        mix = oracle_mod.Mixtures.from_problem(prob)
        cube = np.concatenate([[0.0, 0.0, 0.0, 0.1], rng.uniform(-1, 1, 3), rng.uniform(0.05, 1.0, 3)])
        t0, thw = cube[4:7], cube[7:10]
        ab = [oracle_mod.kappa_interval(mu1[i], prob["sigma1"][i], t0, thw, zeta) for i in range(2)]
        if ab[0] is None or ab[1] is None:
            continue
        v = (mu1 - t0) / np.linalg.norm(mu1 - t0, axis=1, keepdims=True)
        A = min(oracle_mod.angle(v[0], v[1]) + oracle_mod.psi_t(mu1[0], t0, thw) + oracle_mod.psi_t(mu1[1], t0, thw),
                np.pi)
        lb = oracle_mod.self_lb_term(mix, 0, 1, cube, zeta) / (0.3 * 0.7)
        T = _term_grid(oracle_mod, _box_grid(*ab[0], 10), _box_grid(*ab[1], 10), np.linspace(0.0, A, 5))
        assert lb <= T.min() * (1 + 1e-12)
        # the diagonal pair (i, i): the same direction at every t, only kappa varies
        lii = oracle_mod.self_lb_term(mix, 0, 0, cube, zeta) / 0.09
        assert lii <= _term_grid(oracle_mod, _box_grid(*ab[0], 20), _box_grid(*ab[0], 20), [0.0]).min() * (1 + 1e-12)
        checked += 1
        wide += A > np.pi / 2
    assert checked > 100 and wide > 10 and checked - wide > 10  # both sides of A = pi/2


def test_cross_pair_bound_above_the_term_over_its_relaxation(oracle_mod):
    """Theorem 1, cross pairs: over the cube, kappa_1i stays in its interval
    and the angle between R v_i and mu_2j stays at least B (Eq. K1i2j_ub_B
    with Lemmas 2 and 3), so the bound must not fall below the pair term
    anywhere on that box of (kappa_1i, angle)."""
    rng = np.random.default_rng(15)
    zeta, checked = 0.05, 0
    for _ in range(150):
        mu1 = rng.uniform(-2, 2, (1, 3))
        m2 = rng.standard_normal(3)
        k2 = rng.uniform(1.0, 60.0)
        prob = {"mu1": mu1, "sigma1": rng.uniform(0.1, 1.0, 1), "phi1": np.array([1.0]),
                "mu2": (m2 / np.linalg.norm(m2))[None], "kappa2": np.array([k2]), "phi2": np.array([1.0])}
        mix = oracle_mod.Mixtures.from_problem(prob)
        r_hw = rng.uniform(0.05, 1.0)
        cube = np.concatenate([rng.uniform(-1.5, 1.5, 3), [r_hw], rng.uniform(-1, 1, 3), rng.uniform(0.05, 1.0, 3)])
        t0, thw = cube[4:7], cube[7:10]
        ab = oracle_mod.kappa_interval(mu1[0], prob["sigma1"][0], t0, thw, zeta)
        if ab is None:
            continue
        v = (mu1[0] - t0) / np.linalg.norm(mu1[0] - t0)
        u = Rotation.from_rotvec(cube[0:3]).as_matrix().T @ prob["mu2"][0]
        B = max(oracle_mod.angle(v, u) - oracle_mod.psi_t(mu1[0], t0, thw) - oracle_mod.psi_r(r_hw), 0.0)
        ub = oracle_mod.cross_ub_term(mix, 0, 0, cube, zeta)
        T = _term_grid(oracle_mod, _box_grid(*ab, 30), [k2], np.linspace(B, np.pi, 6))
        assert ub >= T.max() * (1 - 1e-12)
        checked += 1
    assert checked > 100


# ------------------------------------------------- Theorem 1 by dense sampling
def _pose_pair_terms(oracle_mod, prob, R, t):
    """All self and cross pair terms of Eq. (objective_function) at one pose,
    from the pinned pair_log."""
    mu1 = prob["mu1"]
    v = (mu1 - t) / np.linalg.norm(mu1 - t, axis=1, keepdims=True)
    k = (np.linalg.norm(mu1 - t, axis=1) / prob["sigma1"]) ** 2 + 1
    n1, n2 = len(k), len(prob["kappa2"])
    S = np.array([[prob["phi1"][i] * prob["phi1"][j] * np.exp(oracle_mod.pair_log(k[i], v[i], k[j], v[j]))
                   for j in range(n1)] for i in range(n1)])
    Cx = np.array([[prob["phi1"][i] * prob["phi2"][j] *
                    np.exp(oracle_mod.pair_log(k[i], R @ v[i], prob["kappa2"][j], prob["mu2"][j]))
                    for j in range(n2)] for i in range(n1)])
    return S, Cx


def _sample_in_cube(rng, cube, prob, n):
    """Up to n feasible poses of the cube (at most 200 n draws, so that a cube
    with no feasible pose cannot stall the test)."""
    out = []
    for _ in range(200 * n):
        if len(out) == n:
            break
        r = cube[0:3] + rng.uniform(-1, 1, 3) * cube[3]
        t = cube[4:7] + rng.uniform(-1, 1, 3) * cube[7:10]
        if np.min(np.linalg.norm(prob["mu1"] - t, axis=1)) >= prob["zeta"]:
            out.append((r, t))
    return out


def test_pair_bounds_hold_on_samples(oracle_mod):
    prob = synth.tiny_problem(21, n1=6, n_in=4, n_out=1)
    prob["sigma1"] = np.full(6, 0.3)  # broad components: pair terms vary smoothly
    mix = oracle_mod.Mixtures.from_problem(prob)
    cubes = synth.tree_cubes(22, 12, prob["t_lo"], prob["t_hi"], 2, 9, near=(prob["r_gt"], prob["t_gt"]),
                             near_frac=0.5)
    rng = np.random.default_rng(23)
    n1, n2 = 6, 5
    checked = 0
    for cube in cubes:
        b = oracle_mod.bounds(mix, cube[None], prob["zeta"])[0]
        if not np.isfinite(b[0]):
            continue
        SL = np.array([[oracle_mod.self_lb_term(mix, i, j, cube, prob["zeta"]) for j in range(n1)] for i in range(n1)])
        CU = np.array([[oracle_mod.cross_ub_term(mix, i, j, cube, prob["zeta"]) for j in range(n2)] for i in range(n1)])
        assert SL.sum() == pytest.approx(b[2], rel=1e-12)
        assert CU.sum() == pytest.approx(b[3], rel=1e-12)
        for r, t in _sample_in_cube(rng, cube, prob, 25):
            S, Cx = _pose_pair_terms(oracle_mod, prob, Rotation.from_rotvec(r).as_matrix(), t)
            assert np.all(SL <= S * (1 + 1e-12) + 1e-300)
            assert np.all(CU >= Cx * (1 - 1e-12))
            checked += 1
    assert checked > 100


def test_bounds_sandwich_objective(oracle_mod):
    prob = synth.tiny_problem(31)
    mix = oracle_mod.Mixtures.from_problem(prob)
    cubes = synth.tree_cubes(32, 60, prob["t_lo"], prob["t_hi"], 3, 12, near=(prob["r_gt"], prob["t_gt"]),
                             near_frac=0.7)
    B = oracle_mod.bounds(mix, cubes, prob["zeta"])
    rng = np.random.default_rng(33)
    n = 0
    for cube, b in zip(cubes, B):
        if not np.isfinite(b[0]):
            continue
        if np.isfinite(b[1]):
            R0 = Rotation.from_rotvec(cube[0:3]).as_matrix()
            assert b[1] == pytest.approx(oracle_mod.objective(mix, R0, cube[4:7]), rel=1e-9)
        for r, t in _sample_in_cube(rng, cube, prob, 30):
            assert b[0] <= oracle_mod.objective_r(mix, r, t) + 1e-9
            n += 1
    assert n > 500


def test_point_psi_r_bounds_sandwich_objective(oracle_mod):
    """Theorem 1 with the point-dependent psi_r (reading R16): the lower bound
    stays below f at sampled poses of the cube, is at least the lower bound
    with the point-independent psi_r (never looser), and is strictly above it
    on most cubes; the upper bound is unchanged."""
    prob = synth.tiny_problem(34)
    mix = oracle_mod.Mixtures.from_problem(prob)
    cubes = synth.tree_cubes(35, 60, prob["t_lo"], prob["t_hi"], 3, 12, near=(prob["r_gt"], prob["t_gt"]),
                             near_frac=0.7)
    B0 = oracle_mod.bounds(mix, cubes, prob["zeta"])
    B1 = oracle_mod.bounds(mix, cubes, prob["zeta"], psi_mode=1)
    fin = np.isfinite(B0[:, 0])
    assert np.array_equal(fin, np.isfinite(B1[:, 0]))
    assert np.array_equal(B0[:, 1], B1[:, 1]) and np.array_equal(B0[:, 2], B1[:, 2])
    assert np.all(B1[fin, 0] >= B0[fin, 0] - 1e-12 * (B0[fin, 2] + 2 * B0[fin, 3]))
    assert np.mean(B1[fin, 0] > B0[fin, 0]) > 0.5
    rng = np.random.default_rng(36)
    n = 0
    for cube, b in zip(cubes, B1):
        if not np.isfinite(b[0]):
            continue
        for r, t in _sample_in_cube(rng, cube, prob, 30):
            assert b[0] <= oracle_mod.objective_r(mix, r, t) + 1e-9
            n += 1
    assert n > 500


def test_bound_gap_shrinks_to_zero(oracle_mod):
    """Bounds converge as the branch size tends to zero (Sec. 4)."""
    prob = synth.tiny_problem(41)
    mix = oracle_mod.Mixtures.from_problem(prob)
    r = prob["r_gt"] + 0.01
    t = prob["t_gt"] + 0.01
    gaps = []
    for k in range(2, 22, 2):
        h = 2.0 ** -k
        cube = np.concatenate([r, [h], t, [h, h, h]])
        b = oracle_mod.bounds(mix, cube[None], prob["zeta"])[0]
        gaps.append(b[1] - b[0])
    gaps = np.array(gaps)
    assert np.all(gaps >= -1e-9)
    assert np.all(np.diff(gaps[2:]) <= 1e-9)
    assert gaps[-1] < 1e-4 * abs(oracle_mod.c22(mix))


def test_infeasible_cubes(oracle_mod):
    prob = synth.tiny_problem(51)
    mix = oracle_mod.Mixtures.from_problem(prob)
    mu = prob["mu1"][0]
    inside_ball = np.concatenate([[0, 0, 0, 0.1], mu, [0.05, 0.05, 0.05]])
    outside_pi = np.concatenate([[3.0, 3.0, 3.0, 0.2], [0, 0, 0], [0.1, 0.1, 0.1]])
    B = oracle_mod.bounds(mix, np.stack([inside_ball, outside_pi]), prob["zeta"])
    assert np.all(np.isinf(B[:, 0])) and np.all(np.isinf(B[:, 1]))
    # reading R5: a centre within zeta of a mean is no pose, but the cuboid
    # around it still has feasible points: a finite lower bound, no upper bound
    wide = np.concatenate([[0, 0, 0, 0.1], mu + 0.1 * prob["zeta"], [2 * prob["zeta"]] * 3])
    b = oracle_mod.bounds(mix, wide[None], prob["zeta"])[0]
    assert np.isfinite(b[0]) and np.isinf(b[1])


# ------------------------------------------------- SMA gradient (Sec. 5)
def test_gradient_matches_central_differences(oracle_mod):
    prob = synth.tiny_problem(61)
    mix = oracle_mod.Mixtures.from_problem(prob)
    rng = np.random.default_rng(62)
    for _ in range(5):
        x = np.concatenate([prob["r_gt"] + rng.normal(0, 0.02, 3), prob["t_gt"] + rng.normal(0, 0.02, 3)])
        f, g = oracle_mod.objective_grad(mix, x)
        assert f == pytest.approx(oracle_mod.objective_r(mix, x[:3], x[3:]), rel=1e-13)
        h = 1e-6
        gn = np.zeros(6)
        for k in range(6):
            e = np.zeros(6)
            e[k] = h
            gn[k] = (oracle_mod.objective_r(mix, (x + e)[:3], (x + e)[3:]) -
                     oracle_mod.objective_r(mix, (x - e)[:3], (x - e)[3:])) / (2 * h)
        assert np.allclose(g, gn, rtol=1e-6, atol=1e-6 * np.abs(gn).max())


def test_gradient_near_the_identity_rotation(oracle_mod):
    """At tiny rotation vectors the left Jacobian of SO(3) is I + [r]x / 2 +
    O(|r|^2): its first-order term changes the rotation gradient by a
    relative ~|r|, which central differences with one Richardson step
    resolve at |r| = 1e-7 and 5e-7 (their own error there is about 1e-10
    of the gradient)."""
    prob = synth.tiny_problem(63)
    mix = oracle_mod.Mixtures.from_problem(prob)

    def central(r, t, k, h):
        e = np.zeros(3)
        e[k] = h
        return (oracle_mod.objective_r(mix, r + e, t) - oracle_mod.objective_r(mix, r - e, t)) / (2 * h)

    for r in (np.array([1e-7, -0.6e-7, 0.3e-7]), np.array([-4e-7, 2e-7, 2.5e-7])):
        x = np.concatenate([r, prob["t_gt"]])
        f, g = oracle_mod.objective_grad(mix, x)
        gn = np.array([(4 * central(r, x[3:], k, 1e-4) - central(r, x[3:], k, 2e-4)) / 3 for k in range(3)])
        assert np.allclose(g[:3], gn, rtol=0, atol=1e-9 * np.abs(gn).max()), (g[:3], gn)


def test_sma_reaches_true_pose_from_nearby(oracle_mod):
    prob = synth.noise_free_problem(71, n1=6)
    mix = oracle_mod.Mixtures.from_problem(prob)
    x0 = np.concatenate([prob["r_gt"] + 0.03, prob["t_gt"] - 0.03])
    f0 = oracle_mod.objective_r(mix, x0[:3], x0[3:])
    x1, f1, _ = oracle_mod.sma(mix, x0, prob["t_lo"], prob["t_hi"], prob["zeta"], max_iter=300)
    assert f1 <= f0
    assert f1 == pytest.approx(-oracle_mod.c22(mix), rel=1e-8)
    assert np.linalg.norm(x1[3:] - prob["t_gt"]) < 1e-4


def test_sma_results_are_local_minima(oracle_mod):
    """From seeds away from the optimum, an SMA result that stopped inside
    the feasible set (not on the domain box or a zeta-sphere) is a local
    minimum: no pose +-h along any of the 12 coordinate directions lowers f by
    more than a rounding-level amount (h = 1e-4 and 1e-3)."""
    prob = synth.tiny_problem(1003)
    mix = oracle_mod.Mixtures.from_problem(prob)
    x0s = synth.pose_seeds(prob, 24, 7)
    checked = 0
    for x0 in x0s:
        x1, f1, _ = oracle_mod.sma(mix, x0, prob["t_lo"], prob["t_hi"], prob["zeta"], max_iter=300, memory=8,
                                   gtol=1e-10)
        if not np.isfinite(f1):
            continue
        t = x1[3:]
        margin = min(np.min(t - prob["t_lo"]), np.min(prob["t_hi"] - t),
                     np.min(np.linalg.norm(prob["mu1"] - t, axis=1)) - prob["zeta"])
        if margin < 1e-2:
            continue  # stopped against the boundary of the feasible set
        assert f1 == pytest.approx(oracle_mod.objective_r(mix, x1[:3], x1[3:]), rel=1e-12)
        for h in (1e-4, 1e-3):
            for k in range(6):
                for sgn in (-1.0, 1.0):
                    x = x1.copy()
                    x[k] += sgn * h
                    assert oracle_mod.objective_r(mix, x[:3], x[3:]) >= f1 - 1e-9 * (1 + abs(f1)), (k, sgn, h)
        checked += 1
    assert checked >= 8
