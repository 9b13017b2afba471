"""The bound kernel's FP32 error budget, replayed on the CPU.

On the device the pair terms of Theorem 1 run in FP32 with the approximate
ex2 / rcp / sqrt instructions, and a slack is meant to keep every cross
upper bound at or above, and every self lower bound at or below, the exact
value (cross_pair2 and self_pair2 in csrc/bounds_core.cuh, per lane; the header states
the budget).  This test replays the bound part of those two functions in
numpy float32, operation by operation: plain operations rounded to nearest,
the fused multiply-adds the source writes rounded once, and every
approximate instruction off by its documented error bound (ex2 3u, rcp and
sqrt 2u, u = 2^-24) in either direction: all sign combinations for the
cross pair, random ones plus the all-low and all-high cases for the self
pair.  The inputs are what the kernel's first phase stores, at the edge of
that phase's own allowances: directions as double-floats, kappa interval
ends at a(1 - u) and b(1 + u), half-angle sines rounded up and cosines down,
kappa_2 and the column factor rounded to nearest.  The geometry (kappa
intervals, psi_t, psi_r, directions) comes from the FP64 oracle, and the
replayed bound must never cross the oracle's pair bound for the same cube.
On these 3,000 cubes the smallest margins are 25.4u (cross) and 39.9u (self):
a dropped angle allowance, the wrong end of a sine interval or clamp, or a
slack of the wrong sign crosses the oracle, while each few-u rounding
direction on its own stays inside the margin.
"""
import itertools

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

U = 2.0 ** -24
F = np.float32


def f32(x):
    return np.asarray(x, dtype=np.float64).astype(np.float32)


def fma(a, b, c):
    """fmaf: the exact product plus c, rounded once (through FP64: the product
    of two floats is exact there)."""
    return (np.float64(1) * a.astype(np.float64) * b.astype(np.float64) + np.asarray(c, np.float64)).astype(np.float32)


def ftz(x):
    return np.where(np.abs(x) < 2.0 ** -126, np.float32(0), x).astype(np.float32)


def toward(v, d):
    """v (FP64) to float32, rounded down where d < 0 and up where d > 0."""
    y = v.astype(np.float32)
    yd = y.astype(np.float64)
    y = np.where((d < 0) & (yd > v), np.nextafter(y, np.float32(-np.inf)), y)
    y = np.where((d > 0) & (yd < v), np.nextafter(y, np.float32(np.inf)), y)
    return y.astype(np.float32)


def approx(exact, s, rel):
    """An approximate instruction's result: exact (1 + s rel), rounded toward
    exact so that it stays within the bound; outputs flushed to zero."""
    v = exact * (1.0 + s * rel)
    return ftz(toward(v, -s * np.ones_like(v)))


def sqrta(x, s):
    return approx(np.sqrt(ftz(x).astype(np.float64)), s, 2 * U)


def rcpa(x, s):
    return approx(1.0 / ftz(x).astype(np.float64), s, 2 * U)


def ex2a(x, s):
    return approx(np.exp2(ftz(x).astype(np.float64)), s, 3 * U)


L2E = F(1.4426950408889634)
FU = F(U)
SLACK = F(15) * FU
CROSS_SLACK = F(20) * FU
# the absolute allowance on the half-angle sines for directions taken in
# their FP32 parts only (|v -+ u| within sqrt(3) u: sB within 1.23u)
HI_ALLOW = F(1.3) * FU


def c1(k):
    """The float32 constant 1 + k u as the source writes it, (1.f + k * U)."""
    return F(1) + F(k) * FU


def c1m(k):
    return F(1) - F(k) * FU


def gZ(x, s):
    return F(1) - ex2a(F(-2) * L2E * x, s)


def split(v):
    hi = f32(v)
    return hi, f32(v - hi.astype(np.float64))


def mul_rd(a, b):
    return toward(a.astype(np.float64) * b.astype(np.float64), -np.ones(np.shape(a)))


def mul_ru(a, b):
    return toward(a.astype(np.float64) * b.astype(np.float64), np.ones(np.shape(a)))


# ---------------------------------------------------------------- inputs from the oracle's geometry
def _cases(oracle_mod, rng, n):
    """Random two-component model, one image component and a cube, with the
    oracle's kappa intervals, psi_t, psi_r, directions and pair bounds."""
    out = []
    while len(out) < n:
        mu1 = rng.uniform(-3, 3, (2, 3))
        sig = np.exp(rng.uniform(np.log(0.02), np.log(0.5), 2))
        t0 = rng.uniform(-1, 1, 3)
        thw = np.exp(rng.uniform(np.log(1e-4), np.log(1.0), 3))
        if rng.random() < 0.2:  # row 0's mean next to or inside the cuboid: psi_t up to pi
            mu1[0] = t0 + rng.uniform(-2, 2, 3) * thw
        r0 = Rotation.random(random_state=rng).as_rotvec() * rng.uniform(0, 1)
        rhw = np.exp(rng.uniform(np.log(1e-4), np.log(1.0)))
        R0 = Rotation.from_rotvec(r0).as_matrix()
        v = (mu1 - t0) / np.linalg.norm(mu1 - t0, axis=1, keepdims=True)
        mode = rng.integers(3)  # image direction: anywhere, near R0 v_0, near -R0 v_0
        ang = rng.uniform(0, 3.0 * rhw + 1e-3)
        axis = np.cross(v[0], rng.standard_normal(3))
        near = Rotation.from_rotvec(axis / np.linalg.norm(axis) * ang).apply(v[0])
        m2 = [rng.standard_normal(3), R0 @ near, -(R0 @ near)][mode]
        m2 /= np.linalg.norm(m2)
        k2 = np.exp(rng.uniform(0, np.log(2000.0)))
        prob = {"mu1": mu1, "sigma1": sig, "phi1": np.array([0.4, 0.6]), "mu2": m2[None], "kappa2": np.array([k2]),
                "phi2": np.array([1.0])}
        mix = oracle_mod.Mixtures.from_problem(prob)
        zeta = 0.01
        ab = [oracle_mod.kappa_interval(mu1[i], sig[i], t0, thw, zeta) for i in range(2)]
        if ab[0] is None or ab[1] is None:
            continue
        cube = np.concatenate([r0, [rhw], t0, thw])
        out.append(dict(
            v=v, u=R0.T @ m2, k2=k2, phi1=prob["phi1"], phi2=1.0, a=np.array([ab[0][0], ab[1][0]]),
            b=np.array([ab[0][1], ab[1][1]]),
            psit=np.array([oracle_mod.psi_t(mu1[i], t0, thw) for i in range(2)]), psir=oracle_mod.psi_r(rhw),
            cross=oracle_mod.cross_ub_term(mix, 0, 0, cube, zeta),
            self2=oracle_mod.self_lb_term(mix, 0, 1, cube, zeta) + oracle_mod.self_lb_term(mix, 1, 0, cube, zeta),
            diag=oracle_mod.self_lb_term(mix, 0, 0, cube, zeta)))
    return {k: np.array([c[k] for c in out]) for k in out[0]}


def _hi_part_cases(oracle_mod, rng, n, pool=40):
    """Cross pairs where dropping the directions' low parts hurts most: fine
    cubes, concentrated components (kappa_1 and kappa_2 in the thousands),
    the image direction at an angle of s + 1/sqrt(kappa) or so from R0 v_0
    (where the term is most sensitive to sin(B/2)), and, of `pool` random
    directions each, the one whose FP32 parts lengthen |v - u| the most."""
    out = []
    while len(out) < n:
        t0 = rng.uniform(-1, 1, 3)
        thw = np.full(3, 10.0 ** rng.uniform(-5, -4))
        rhw = 10.0 ** rng.uniform(-5, -4)
        r0 = Rotation.random(random_state=rng).as_rotvec() * rng.uniform(0, 1)
        R0 = Rotation.from_rotvec(r0).as_matrix()
        sig = np.array([10.0 ** rng.uniform(-2, -1.3), 0.3])
        k2 = 10.0 ** rng.uniform(3, 4)
        best = None
        for _ in range(pool):
            mu1 = np.stack([t0 + rng.standard_normal(3) * rng.uniform(1, 3), rng.uniform(-3, 3, 3)])
            v = (mu1 - t0) / np.linalg.norm(mu1 - t0, axis=1, keepdims=True)
            ang = 2.2 * rhw + 2e-4 + rng.uniform(0.3, 3.0) / np.sqrt(k2)
            axis = np.cross(v[0], rng.standard_normal(3))
            u = Rotation.from_rotvec(axis / np.linalg.norm(axis) * ang).apply(v[0])
            d_hi = np.linalg.norm(f32(v[0]).astype(np.float64) - f32(u).astype(np.float64))
            gain = d_hi - np.linalg.norm(v[0] - u)
            if best is None or gain > best[0]:
                best = (gain, mu1, u)
        _, mu1, u = best
        m2 = R0 @ u
        prob = {"mu1": mu1, "sigma1": sig, "phi1": np.array([0.4, 0.6]), "mu2": m2[None], "kappa2": np.array([k2]),
                "phi2": np.array([1.0])}
        mix = oracle_mod.Mixtures.from_problem(prob)
        zeta = 0.01
        ab = [oracle_mod.kappa_interval(mu1[i], sig[i], t0, thw, zeta) for i in range(2)]
        if ab[0] is None or ab[1] is None:
            continue
        cube = np.concatenate([r0, [rhw], t0, thw])
        v = (mu1 - t0) / np.linalg.norm(mu1 - t0, axis=1, keepdims=True)
        out.append(dict(
            v=v, u=R0.T @ m2, k2=k2, phi1=prob["phi1"], phi2=1.0, a=np.array([ab[0][0], ab[1][0]]),
            b=np.array([ab[0][1], ab[1][1]]),
            psit=np.array([oracle_mod.psi_t(mu1[i], t0, thw) for i in range(2)]), psir=oracle_mod.psi_r(rhw),
            cross=oracle_mod.cross_ub_term(mix, 0, 0, cube, zeta)))
    return {k: np.array([c[k] for c in out]) for k in out[0]}


def _rows(c):
    """What the first phase stores for each model row (at the edge of its allowances)."""
    a = toward(c["a"] * (1 - U), -np.ones_like(c["a"]))
    b = toward(c["b"] * (1 + U), np.ones_like(c["b"]))
    wide = c["psit"] >= np.pi
    sp = np.where(wide, F(1), toward(np.sin(0.5 * c["psit"]), np.ones_like(c["psit"])))
    cp = np.where(wide, F(0), toward(np.cos(0.5 * c["psit"]), -np.ones_like(c["psit"])))
    return a, b, sp.astype(np.float32), cp.astype(np.float32)


# ---------------------------------------------------------------- cross pair
def _cross(c, s):
    """Upper bound of the cross pair (row 0, the image component) as the
    kernel forms it, times its row factor; s: signs of the 8 approximate
    instructions on the path."""
    e, wQ, Bw = _cross_parts(c, s)
    return fma(e, wQ, np.zeros_like(wQ)).astype(np.float64) * Bw.astype(np.float64)


def _cross_parts(c, s):
    """The exponential (the column factor inside, as its log2), the factor
    it multiplies and the row factor of the cross pair's upper bound."""
    a, b, sp, cp = _rows(c)
    a, b, sp, cp = a[:, 0], b[:, 0], sp[:, 0], cp[:, 0]
    vh, vl = split(c["v"][:, 0])
    uh, ul = split(c["u"])
    k2 = f32(c["k2"])
    # the column factor enters the exponent as its log2, from FP64, raised by
    # the cross slack and by the exponent's rounding of its own size, rounded up
    lq = np.log2(c["phi2"] * c["k2"] / -np.expm1(-2 * c["k2"]))
    lqb = toward(lq + np.float64(CROSS_SLACK) + U * (np.abs(lq) + 1.0), np.ones_like(lq))
    Sr = toward(np.sin(0.5 * c["psir"]), np.ones_like(c["psir"]))
    Cr = toward(np.cos(0.5 * c["psir"]), -np.ones_like(c["psir"]))
    Cs = f32(cp.astype(np.float64) * Cr - sp.astype(np.float64) * Sr)
    Ss = f32(sp.astype(np.float64) * Cr + cp.astype(np.float64) * Sr)
    Ss = np.where(Cs <= 0, F(1), Ss).astype(np.float32)
    Cs = np.where(Cs <= 0, F(0), Cs).astype(np.float32)
    # the directions' FP32 parts only: |v -+ u| within sqrt(3) u of the exact
    # value, so sin and cos of theta/2 within 0.87u and sB within 1.23u
    # absolute, which the row's allowance carries (1.3u)
    esS = fma(np.full_like(Ss, F(7.5) * FU), Ss, np.full_like(Ss, HI_ALLOW))
    d = [vh[:, k] - uh[:, k] for k in range(3)]
    p = [vh[:, k] + uh[:, k] for k in range(3)]
    x2 = fma(d[0], d[0], fma(d[1], d[1], d[2] * d[2]))
    y2 = fma(p[0], p[0], fma(p[1], p[1], p[2] * p[2]))
    sx, sy = sqrta(x2, s[0]), sqrta(y2, s[1])  # 2 sin, 2 cos of theta/2; the halves in the row constants
    sB = fma(sx, F(0.5) * Cs, -(sy * (F(0.5) * Ss)))
    es = fma(np.full_like(sx, F(3.75) * FU), sx, esS)
    slo = np.maximum(sB - es, F(0))
    shi = np.minimum(np.maximum(sB, F(0)) + es, F(1))
    # cos^2(B/2) = -(s^2 - 1), the fused s^2 - 1 rounded once; no outward factors
    q1 = fma(slo, slo, -np.ones_like(slo))
    q2 = fma(shi, shi, -np.ones_like(shi))
    assert np.all(q1 < 0) and np.all(q2 <= 0)
    nak4 = (-(F(4) * a)) * k2
    dka = a - k2
    Khi = sqrta(fma(nak4, q1, dka * dka), s[2])
    nkc = k2 * fma(np.full_like(q2, F(2)), q2, np.ones_like(q2))
    ks = np.minimum(np.maximum(nkc, a), b)
    dks = ks - k2
    Kmin = sqrta(fma(F(-4) * ks * k2, q2, dks * dks), s[3])
    den = (a + k2) + Khi
    Kc = np.maximum(Kmin, F(1e-20))
    r = rcpa(den * Kc, s[4])
    DL = nak4 * (slo * slo) * (Kc * r) * L2E
    w = np.minimum(den * r, F(2))
    e = ex2a(fma(DL, np.full_like(DL, F(1) - F(16) * FU), lqb), s[5])
    ph = f32(c["phi1"][:, 0])
    Bw = np.where(b < F(9), ph * b * rcpa(gZ(b, s[6]), s[7]) * c1(12), ph * b).astype(np.float32)
    Bw = mul_ru(Bw, np.full_like(Bw, c1(8 + 6)))
    return e, w.astype(np.float32), Bw


# ---------------------------------------------------------------- self pair
def _aw(a, ph, s0, s1):
    """phi a / g(a) from below (the row factor of the self lower bound)."""
    return np.where(a < F(9), ph * a * rcpa(gZ(a, s0), s1) * c1m(12), mul_rd(ph * a, np.full_like(a, c1m(3))))


def _self(c, s):
    """Lower bound of the self pair (0, 1), both orders, as the kernel forms
    it with its row factors; s: signs of the 11 approximate instructions."""
    e, wA, Awi = _self_parts(c, s)
    return fma(e, wA, np.zeros_like(wA)).astype(np.float64) * Awi.astype(np.float64)


def _self_parts(c, s):
    """The exponential, the factor it multiplies and the row factor of the
    self pair's lower bound."""
    a, b, sp, cp = _rows(c)
    vh, vl = split(c["v"][:, 0])
    mh, ml = split(c["v"][:, 1])
    ph = f32(c["phi1"])
    Am = _aw(a[:, 1], ph[:, 1], s[7], s[8]).astype(np.float32)
    Ai = _aw(a[:, 0], ph[:, 0], s[9], s[10]).astype(np.float32)
    d = [vh[:, k] - mh[:, k] for k in range(3)]
    p = [vh[:, k] + mh[:, k] for k in range(3)]
    x2 = fma(d[0], d[0], fma(d[1], d[1], d[2] * d[2]))
    y2 = fma(p[0], p[0], fma(p[1], p[1], p[2] * p[2]))
    sx, sy = sqrta(x2, s[0]), sqrta(y2, s[1])  # 2 sin, 2 cos of theta/2
    hcp, hsp = F(0.5) * cp, F(0.5) * sp       # the row's halved half-angle pair
    hC = fma(hcp[:, 0], cp[:, 1], -(hsp[:, 0] * sp[:, 1]))
    hS = fma(hsp[:, 0], cp[:, 1], hcp[:, 0] * sp[:, 1])
    cA = fma(sy, hC, -(sx * hS))
    sA = fma(sx, hC, sy * hS)
    es = fma(np.full_like(sx, F(5) * FU), sx, fma(np.full_like(hS, F(20) * FU), hS, np.full_like(hS, HI_ALLOW)))
    api = cA <= F(16) * FU
    shi = np.where(api, F(1), np.minimum(sA + es, F(1))).astype(np.float32)
    slo = np.maximum(sA - es, F(0))
    clo2 = fma(shi, shi, -np.ones_like(shi)) * (-c1m(2))
    chi2 = fma(slo, slo, -np.ones_like(slo)) * (-c1(2))
    ai, bi, am, bm = a[:, 0], b[:, 0], a[:, 1], b[:, 1]
    bb = bi * bm
    dbb = bi - bm
    Klo = sqrta(fma(dbb, dbb, F(4) * bb * clo2), s[2]) * c1m(4)
    c4 = F(4) * chi2
    q1, q2, q3 = ai - am, ai - bm, bi - am
    e1 = fma(q1, q1, c4 * ai * am)
    e2 = fma(q2, q2, c4 * ai * bm)
    e3 = fma(q3, q3, c4 * bi * am)
    e4 = fma(dbb, dbb, c4 * bb)
    Kmax = sqrta(np.maximum(np.maximum(e1, e2), np.maximum(e3, e4)), s[3]) * c1(5)
    den = (bi + bm) + Klo
    r = rcpa(den * Kmax, s[4])
    DL = bb * (shi * shi) * (Kmax * r) * (F(-4) * L2E)
    w = den * r
    small = Kmax < F(0.25)
    w = np.where(Kmax < F(9), np.where(small, np.maximum(F(2) - F(2) * Kmax, F(0)), gZ(Kmax, s[5]) * w * c1m(64)), w)
    w = w.astype(np.float32)
    e = ex2a(fma(DL, np.full_like(DL, F(1) + F(12) * FU), np.full_like(DL, -SLACK)), s[6])
    Awi = mul_rd(F(2) * Ai, np.full_like(Ai, c1m(8 + 3)))
    return e, (w * Am).astype(np.float32), Awi


# Terms below this leave FP32's normal range after the exponential and flush
# to zero; the per-cube allowance of 1e-12 S (S >= the diagonal self terms
# sum_i phi_i^2 a_i coth(a_i) / 2 >= 1 / (2 n1)) covers far more than all of
# them together, so the cross check starts here.
FLOOR = 1e-30


def _diag(c, s):
    """Diagonal self term phi^2 a coth(a) / 2 from below (half_kcothk at the
    row's a, its 16u allowance, and the 3u the row sums start with)."""
    a = _rows(c)[0][:, 0]
    ph = f32(c["phi1"][:, 0])
    e = ex2a(F(-2) * L2E * a, s[0])
    h = F(0.5) * a * (F(1) + e) * rcpa(F(1) - e, s[1])
    return (ph * ph * h * c1m(16)).astype(np.float64) * (1 - 3 * U)


@pytest.fixture(scope="module")
def cases(oracle_mod):
    return _cases(oracle_mod, np.random.default_rng(17), 3000)


def test_cross_upper_bound_never_below_the_oracle(cases):
    worst = np.inf
    for signs in itertools.product((-1.0, 1.0), repeat=8):
        ub = _cross(cases, signs)
        ref = cases["cross"]
        ok = ref > FLOOR
        ratio = ub[ok] / ref[ok]
        worst = min(worst, ratio.min())
        assert np.all(ub[ok] >= ref[ok]), (signs, ratio.min())
    assert worst >= 1.0


def test_cross_bound_covers_the_dropped_low_parts(oracle_mod):
    """The pair code takes the unit directions' FP32 parts only; the row's
    absolute allowance of 1.3u on sin(B/2) covers what the low parts would
    have changed.  On the pairs where that matters most the bound stays
    above the oracle's under every sign of the instruction errors, and
    without the allowance it does not."""
    global HI_ALLOW
    c = _hi_part_cases(oracle_mod, np.random.default_rng(23), 300)
    ok = c["cross"] > FLOOR
    assert ok.sum() > 200
    for signs in itertools.product((-1.0, 1.0), repeat=8):
        assert np.all(_cross(c, signs)[ok] >= c["cross"][ok]), signs
    keep, HI_ALLOW = HI_ALLOW, F(0)
    try:
        low = [np.any(_cross(c, signs)[ok] < c["cross"][ok]) for signs in ((-1.0,) * 8, (1.0,) * 8)]
    finally:
        HI_ALLOW = keep
    assert any(low)


def test_self_lower_bound_never_above_the_oracle(cases):
    rng = np.random.default_rng(18)
    combos = [(-1.0,) * 11, (1.0,) * 11] + [tuple(rng.choice([-1.0, 1.0], 11)) for _ in range(400)]
    for signs in combos:
        lb = _self(cases, signs)
        ref = cases["self2"]
        assert np.all(lb <= ref), (signs, np.max(lb / np.maximum(ref, 1e-300)))
        # and it stays close: the slack costs little where the term matters
        big = ref > FLOOR
        assert np.median(lb[big] / ref[big]) > 0.999


def test_diagonal_self_term_never_above_the_oracle(cases):
    for signs in itertools.product((-1.0, 1.0), repeat=2):
        assert np.all(_diag(cases, signs) <= cases["diag"])


def test_kappa_interval_rounded_outward(oracle_mod):
    """The first phase's kappa interval in FP32 (double-float differences,
    FP32 squares and sums, the end points multiplied by 1 -/+ 7u and rounded
    down / up): never inside the oracle's [a, b]; and a cuboid the kernel
    calls infeasible has no point at least zeta from the mean."""
    rng = np.random.default_rng(19)
    n = 20000
    mu = rng.uniform(-3, 3, (n, 3))
    t0 = rng.uniform(-1, 1, (n, 3))
    thw = np.exp(rng.uniform(np.log(1e-5), np.log(1.0), (n, 3)))
    near = rng.random(n) < 0.5
    mu[near] = t0[near] + rng.uniform(-1.5, 1.5, (near.sum(), 3)) * thw[near]
    sig = np.exp(rng.uniform(np.log(0.01), np.log(1.0), n))
    zeta = np.where(rng.random(n) < 0.5, 0.0, np.exp(rng.uniform(np.log(1e-4), np.log(2.0), n)))
    # the last quarter on the feasibility boundary: the farthest vertex at zeta (1 + delta), |delta| <= 30u
    m = n // 4
    zb = np.exp(rng.uniform(np.log(0.1), np.log(2.0), m))
    o = rng.uniform(-1, 1, (m, 3)) * rng.uniform(0, 0.25, (m, 1)) * zb[:, None]  # |o| < zeta / 2
    dirn = rng.uniform(0.2, 1.0, (m, 3))
    tgt = zb * (1 + rng.uniform(-30, 30, m) * U)
    # solve sum_k (|o_k| + lam d_k)^2 = tgt^2 for lam > 0
    qa, qb, qc = (dirn ** 2).sum(1), 2 * (np.abs(o) * dirn).sum(1), (o ** 2).sum(1) - tgt ** 2
    lam = (-qb + np.sqrt(qb * qb - 4 * qa * qc)) / (2 * qa)
    t0[-m:] = rng.uniform(-1, 1, (m, 3))
    mu[-m:] = t0[-m:] + o
    thw[-m:] = lam[:, None] * dirn
    zeta[-m:] = zb
    muh, mul = split(mu)
    th, tl = split(t0)
    wh, wl = split(thw)
    c = (muh.astype(np.float64) + mul) - (th.astype(np.float64) + tl)  # double-float difference, ~2^-44
    ac = np.abs(c)
    e = np.maximum(f32(ac - (wh.astype(np.float64) + wl)), F(0))
    f = f32(ac) + wh
    e2 = fma(e[:, 2], e[:, 2], fma(e[:, 1], e[:, 1], fma(e[:, 0], e[:, 0], np.zeros(n, np.float32))))
    f2 = fma(f[:, 2], f[:, 2], fma(f[:, 1], f[:, 1], fma(f[:, 0], f[:, 0], np.zeros(n, np.float32))))
    z2 = f32(zeta * zeta)
    is2 = f32(1.0 / (sig * sig))
    a = mul_rd(fma(np.maximum(e2, z2), is2, np.ones(n, np.float32)), np.full(n, c1m(7)))
    b = mul_ru(fma(f2, is2, np.ones(n, np.float32)), np.full(n, c1(7)))
    infeasible = f2 * c1(8) < z2
    checked = edge = 0
    for k in range(n):
        ab = oracle_mod.kappa_interval(mu[k], sig[k], t0[k], thw[k], zeta[k])
        if ab is None:
            continue
        assert not infeasible[k], k
        assert a[k] <= ab[0] and b[k] >= ab[1], (k, a[k], ab[0], b[k], ab[1])
        checked += 1
        edge += k >= n - m
    assert checked > n // 2 and edge > m // 4


def _sin_half_psi_t(mu, t0, thw, sg):
    """sin(psi_t / 2) as the first phase stores it (Lemma 3): FP32 angles to
    the eight vertices pick the largest, the double-float chord to that
    vertex gives it, the FP32 runner-up times (1 + 32u) covers a mis-chosen
    vertex, pi when the mean is inside or a vertex angle may reach pi/2.
    sg(shape) draws the signs of the approximate instructions.  The vertex
    loop runs for every case here and its results are masked afterwards
    where the mean is inside (the kernel skips it there)."""
    with np.errstate(divide="ignore", invalid="ignore"):
        return _sin_half_psi_t_all(mu, t0, thw, sg)


def _sin_half_psi_t_all(mu, t0, thw, sg):
    n = len(mu)
    muh, mul = split(mu)
    th, tl = split(t0)
    wh, wl = split(thw)
    c = (muh.astype(np.float64) + mul) - (th.astype(np.float64) + tl)
    w = wh.astype(np.float64) + wl
    inside = np.all(np.abs(c) - w <= 0, axis=1)
    ch, d2 = f32(c), f32((c * c).sum(1))
    m1 = np.full(n, F(-1))
    m2 = np.full(n, F(-1))
    best = np.zeros(n, int)
    wide = np.zeros(n, bool)
    for vtx in range(8):
        o = [np.where((vtx >> k) & 1, wh[:, k], -wh[:, k]).astype(np.float32) for k in range(3)]
        ax, ay, az = (ch[:, k] - o[k] for k in range(3))
        cx, cy, cz = ch[:, 0], ch[:, 1], ch[:, 2]
        crx, cry, crz = fma(o[1], cz, -(o[2] * cy)), fma(o[2], cx, -(o[0] * cz)), fma(o[0], cy, -(o[1] * cx))
        cr2 = fma(crx, crx, fma(cry, cry, crz * crz))
        ac = fma(ax, cx, fma(ay, cy, az * cz))
        a2 = fma(ax, ax, fma(ay, ay, az * az))
        nn = sqrta(a2 * d2, sg(n))
        wide |= ac <= (F(64) * FU) * nn
        s2 = cr2 * rcpa((F(2) * nn) * (nn + ac), sg(n))
        up = s2 > m1
        m2 = np.where(up, m1, np.maximum(m2, s2))
        best = np.where(up, vtx, best)
        m1 = np.where(up, s2, m1)
    # chord between the unit directions of mu - t_vertex and mu - t0 (double-float)
    sign = np.array([[1.0 if (b >> k) & 1 else -1.0 for k in range(3)] for b in range(8)])[best]
    q = c - sign * w
    qh, ql = split(q / np.linalg.norm(q, axis=1, keepdims=True))
    vh, vl = split(c / np.linalg.norm(c, axis=1, keepdims=True))
    dk = [(qh[:, k] - vh[:, k]) + (ql[:, k] - vl[:, k]) for k in range(3)]
    ch2 = fma(dk[2], dk[2], fma(dk[1], dk[1], fma(dk[0], dk[0], np.zeros(n, np.float32))))
    sp2 = np.minimum(np.maximum(F(0.25) * ch2 * c1(8), m2 * c1(32)), F(1))
    sp2 = np.where(inside | wide, F(1), sp2).astype(np.float32)
    return np.where(sp2 >= 1, F(1), np.minimum(sqrta(sp2, sg(n)) * c1(3), F(1)))


def test_psi_t_rounded_outward(oracle_mod):
    """The stored half-angle sine of psi_t is never below the oracle's (and
    reaches 1 wherever the oracle's psi_t is pi), under random error signs
    of the approximate instructions and under all-low and all-high ones."""
    rng = np.random.default_rng(20)
    n = 6000
    t0 = rng.uniform(-1, 1, (n, 3))
    thw = np.exp(rng.uniform(np.log(1e-5), np.log(1.0), (n, 3)))
    scale = np.exp(rng.uniform(np.log(0.5), np.log(200.0), (n, 1)))
    mu = t0 + rng.uniform(-1, 1, (n, 3)) * thw * scale
    # a third almost on a symmetry axis of the cuboid: vertex angles that
    # differ at FP32 precision, where the FP32 choice of vertex can be wrong
    m = n // 3
    ax = rng.integers(3, size=m)
    off = rng.uniform(-1, 1, (m, 3)) * thw[-m:] * 10.0 ** rng.uniform(-9, -5, (m, 1))
    off[np.arange(m), ax] = np.where(rng.random(m) < 0.5, -1, 1) * thw[-m:][np.arange(m), ax] * rng.uniform(1.5, 50, m)
    mu[-m:] = t0[-m:] + off
    psi = np.array([oracle_mod.psi_t(mu[k], t0[k], thw[k]) for k in range(n)])
    want = np.where(psi >= np.pi, 1.0, np.sin(0.5 * psi))
    for mode in ("low", "high", *range(30)):
        if mode == "low":
            sg = lambda m: -np.ones(m)  # noqa: E731
        elif mode == "high":
            sg = lambda m: np.ones(m)  # noqa: E731
        else:
            r = np.random.default_rng(100 + mode)
            sg = lambda m: r.choice([-1.0, 1.0], m)  # noqa: E731
        got = _sin_half_psi_t(mu, t0, thw, sg).astype(np.float64)
        assert np.all(got >= want), (mode, np.min(got - want))
    assert (psi >= np.pi).sum() > 300 and (psi < 1e-3).sum() > 300 and ((psi > 0.5) & (psi < np.pi)).sum() > 300


def _f(x):
    return np.float32(x)


def _fma1(a, b, c):
    """Scalar fmaf: the exact product plus c, rounded once (through FP64)."""
    return np.float32(np.float64(a) * np.float64(b) + np.float64(c))


def _two_sum(a, b):
    s_ = _f(a + b)
    bb = _f(s_ - a)
    return s_, _f(_f(a - _f(s_ - bb)) + _f(b - bb))


def _fast_two_sum(a, b):
    s_ = _f(a + b)
    return s_, _f(b - _f(s_ - a))


def _two_prod(a, b):
    p = _f(a * b)
    return p, _fma1(a, b, -p)


def _split(x):
    h = np.float32(x)
    return h, np.float32(x - np.float64(h))


def _df_dot3(a, b):
    """dfloat.cuh df_dot3 of double-float 3-vectors a, b (lists of (h, l))."""
    p = [_two_prod(a[k][0], b[k][0]) for k in range(3)]
    e = [_fma1(a[k][0], b[k][1], _fma1(a[k][1], b[k][0], p[k][1])) for k in range(3)]
    s1 = _two_sum(p[0][0], p[1][0])
    t = _two_sum(s1[0], p[2][0])
    return _fast_two_sum(t[0], _f(_f(s1[1] + t[1]) + _f(_f(e[0] + e[1]) + e[2])))


def _df_mul(a, b):
    p = _two_prod(a[0], b[0])
    return _fast_two_sum(p[0], _f(p[1] + _fma1(a[0], b[1], _f(a[1] * b[0]))))


def _df_sub(a, b):
    s_ = _two_sum(a[0], -b[0])
    return _fast_two_sum(s_[0], _f(s_[1] + _f(a[1] - b[1])))


def _up(x):
    return float(toward(np.array([x]), np.ones(1))[0])


def _down(x):
    return float(toward(np.array([x]), -np.ones(1))[0])


def _approx1(exact, sgn, rel):
    return float(approx(np.array([exact]), sgn, rel)[0])


def _newton_sqrt(w, sq, rc):
    """sqrt of a double-float w by one Newton step from the approximate FP32
    square root (sq, rc: the ends of the sqrt and rcp error bounds)."""
    r = _f(_approx1(np.sqrt(np.float64(w[0])), sq, 2 * U))
    rr = _two_prod(r, r)
    inv = _f(_approx1(1.0 / np.float64(r), rc, 2 * U))
    e = _f(_f(_f(_f(w[0] - rr[0]) - rr[1]) + w[1]) * _f(_f(0.5) * inv))
    return r, e


def _point_psi_r_device(r0, h, v, sq, rc):
    """The per-direction rotation uncertainty as the kernel forms it
    (point_psi_r in csrc/bounds_core.cuh): the pre-pass's FP64 vertex images
    J_r(r0) d / 2 and their squared norms split to double-floats, the
    double-float dot products, squared cross norms and Newton square roots,
    the approximate sqrt and rcp at the sq and rc ends of their error bounds,
    and the directed roundings.  Returns (sine, cosine, largest squared cross
    norm / largest squared image norm)."""
    th2 = float(r0 @ r0)
    th = np.sqrt(th2)
    A = 1 - th2 / 6 if th < 1e-8 else np.sin(th) / th
    B = 0.5 - th2 / 24 if th < 1e-8 else (1 - np.cos(th)) / th2
    Cc = 1 / 6 - th2 / 120 if th < 1e-6 else (th - A * th) / (th2 * th)
    x, y, z = r0
    S = np.array([[0, -z, y], [z, 0, -x], [-y, x, 0]])
    J = np.eye(3) - B * S + Cc * (S @ S)
    vd = [_split(c) for c in v]
    best, cmax, n2max = (_f(0), _f(0)), 0.0, 0.0
    for k in range(4):
        d = np.full(3, h)
        if k:
            d[k - 1] = -h
        c = 0.5 * (J @ d)
        n2 = float(c @ c)
        cmax = max(cmax, np.sqrt(n2))
        dot = _df_dot3([_split(ci) for ci in c], vd)
        n = _df_sub(_split(n2), _df_mul(dot, dot))
        n2max = max(n2max, float(n[0]) + float(n[1]))
        if n[0] > best[0] or (n[0] == best[0] and n[1] > best[1]):
            best = n
    ratio = n2max / cmax ** 2
    lh, ll = _f(0), _f(0)
    if best[0] > 0:
        r, e = _newton_sqrt(best, sq, rc)
        lh, ll = _fast_two_sum(r, e)
    s2 = _up(0.375 * h * h)
    al = _up(64.0 * 2.0 ** -48 * cmax)
    sn = _up(np.float64(lh) + np.float64(_up(np.float64(ll) + np.float64(_up(np.float64(s2) + np.float64(al))))))
    sf = _f(sn)
    p = _two_prod(sf, sf)
    t = _two_sum(_f(1), -p[0])
    w = _two_sum(t[0], _f(t[1] - p[1]))
    cs = 0.0
    if w[0] > 1 / 256:
        r, e = _newton_sqrt(w, sq, rc)
        lo = _down(-64.0 * U * U * np.float64(r) + np.float64(e))
        cs = _down(np.float64(r) + lo)
    return sn, cs, ratio


def test_point_psi_r_rounded_outward(oracle_mod):
    """The per-direction rotation uncertainty of Lemma 2 (reading R16) as the
    kernel computes it: its half-angle sine is never below and its cosine
    never above the oracle's, with the approximate sqrt and rcp at either
    end of their error bounds, over cubes all over the pi-ball (a third near
    its surface) from h = 1e-6 to 1; the sine is within 3u of the oracle's
    (one rounding up is up to 2u just above a power of two: the
    point-independent sine, rounded up once from FP64, is within 2u), and the
    largest squared cross
    norm is at least a quarter of the largest squared image norm (the
    cancellation the error budget allows)."""
    rng = np.random.default_rng(31)
    worst = 0.0
    for k in range(1500):
        h = float(np.exp(rng.uniform(np.log(1e-6), 0)))
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        r0 = d * (rng.uniform(2.6, 3.1) if k % 3 == 0 else rng.uniform(0, 2.6))
        v = rng.standard_normal(3)
        v /= np.linalg.norm(v)
        psi = oracle_mod.psi_r_point(r0, h, v)
        hk = min(np.sqrt(3) * h, np.pi)
        for sq in (-1.0, 1.0):
            for rc in (-1.0, 1.0):
                sn, cs, ratio = _point_psi_r_device(r0, h, v, sq, rc)
                assert ratio >= 0.25, (k, r0, h, v, ratio)
                if psi < hk:  # the kernel uses the point-dependent pair only where it is smaller
                    assert sn >= np.sin(0.5 * psi), (k, r0, h, v, sn / np.sin(0.5 * psi) - 1)
                    assert cs <= np.cos(0.5 * psi), (k, r0, h, v, cs / np.cos(0.5 * psi) - 1)
                    worst = max(worst, sn / np.sin(0.5 * psi) - 1)
    assert worst <= 3 * U, worst / U


def _row_cases(oracle_mod, rng, n2):
    """One model component against n2 image components in one cube: the
    pairs (0, j) of a row, with the oracle's pair bounds."""
    while True:
        mu1 = rng.uniform(-3, 3, (1, 3))
        t0 = rng.uniform(-1, 1, 3)
        thw = np.exp(rng.uniform(np.log(1e-3), np.log(0.3), 3))
        r0 = Rotation.random(random_state=rng).as_rotvec() * rng.uniform(0, 1)
        rhw = np.exp(rng.uniform(np.log(1e-3), np.log(0.3)))
        R0 = Rotation.from_rotvec(r0).as_matrix()
        v = (mu1[0] - t0) / np.linalg.norm(mu1[0] - t0)
        m2 = rng.standard_normal((n2, 3)) * 0.3 + R0 @ v  # mostly near the model direction: large terms
        m2 /= np.linalg.norm(m2, axis=1, keepdims=True)
        k2 = np.exp(rng.uniform(0, np.log(2000.0), n2))
        phi2 = rng.dirichlet(np.ones(n2))
        prob = {"mu1": mu1, "sigma1": np.array([np.exp(rng.uniform(np.log(0.02), np.log(0.5)))]),
                "phi1": np.array([1.0]), "mu2": m2, "kappa2": k2, "phi2": phi2}
        mix = oracle_mod.Mixtures.from_problem(prob)
        ab = oracle_mod.kappa_interval(mu1[0], prob["sigma1"][0], t0, thw, 0.01)
        if ab is None:
            continue
        cube = np.concatenate([r0, [rhw], t0, thw])
        ones = np.ones(n2)
        c = dict(v=np.repeat(np.array([[v, v]]), n2, 0), u=m2 @ R0, k2=k2, phi1=np.outer(ones, [1.0, 1.0]),
                 phi2=phi2, a=np.outer(ones, [ab[0], ab[0]]), b=np.outer(ones, [ab[1], ab[1]]),
                 psit=np.outer(ones, [oracle_mod.psi_t(mu1[0], t0, thw)] * 2), psir=oracle_mod.psi_r(rhw) * ones)
        ref = sum(oracle_mod.cross_ub_term(mix, 0, j, cube, 0.01) for j in range(n2))
        return c, ref


def _acc_add(s, c, x):
    """Compensated FP32 accumulation (TwoSum), as the kernel's Acc."""
    t = s + x
    z = t - s
    c = c + ((s - (t - z)) + (x - z))
    return t, c


def test_cross_row_sum_never_below_the_oracle(oracle_mod):
    """A whole row of cross pairs: terms fused into FP32 chunk sums of 8
    (one lane, or the packed loop's two lanes), chunks into a compensated
    sum, the row factor applied once (df_scale, exact product plus one
    rounding) -- the (8 + 6)u of the row factor has to cover the chunk and
    row sums."""
    rng = np.random.default_rng(21)
    for trial in range(40):
        n2 = int(rng.integers(8, 300))
        c, ref = _row_cases(oracle_mod, rng, n2)
        for signs in [(-1.0,) * 8] + [tuple(rng.choice([-1.0, 1.0], 8)) for _ in range(3)]:
            e, wQ, Bw = _cross_parts(c, signs)
            for paired in (False, True):  # any order of the pairs within a thread
                row = _row_sum(e, wQ, Bw[0], rng.permutation(n2), paired)
                assert row >= ref, (trial, n2, paired, row / ref - 1)


def _row_sum(e, wX, factor, order, paired=False):
    """A thread's row: FP32 chunk sums of 8 fused terms, a compensated sum
    of the chunks, and the row factor applied once (df_scale).  paired: the
    kernel's packed loop, which takes the terms two at a time into two lanes,
    each with its own chunk sum; after 8 steps both lanes go into the
    compensated sum (lane x first), and an odd last term joins lane x."""
    s_, c_ = F(0), F(0)

    def fused(j, acc):
        return F(np.float64(e[j]) * np.float64(wX[j]) + np.float64(acc))

    if not paired:
        pl, cnt = F(0), 0
        for j in order:
            pl = fused(j, pl)
            cnt += 1
            if cnt == 8:
                s_, c_ = _acc_add(s_, c_, pl)
                pl, cnt = F(0), 0
        s_, c_ = _acc_add(s_, c_, pl)
    else:
        px, py, cnt = F(0), F(0), 0
        n = len(order)
        for k in range(0, n - 1, 2):
            px, py = fused(order[k], px), fused(order[k + 1], py)
            cnt += 1
            if cnt == 8:
                s_, c_ = _acc_add(s_, c_, px)
                s_, c_ = _acc_add(s_, c_, py)
                px, py, cnt = F(0), F(0), 0
        if n % 2:
            px = fused(order[n - 1], px)
        s_, c_ = _acc_add(s_, c_, px)
        s_, c_ = _acc_add(s_, c_, py)
    h = F(np.float64(s_) * np.float64(factor))
    lo = F(np.float64(c_) * np.float64(factor) + (np.float64(s_) * np.float64(factor) - np.float64(h)))
    return np.float64(h) + np.float64(lo)


def test_self_row_sum_never_above_the_oracle(oracle_mod):
    """A row of self pairs (0, m), m = 1 .. n1 - 1, both orders, summed as
    the kernel sums them; the (8 + 3)u of the row factor covers the sums."""
    rng = np.random.default_rng(22)
    for trial in range(30):
        n1 = int(rng.integers(9, 120))
        t0 = rng.uniform(-1, 1, 3)
        thw = np.exp(rng.uniform(np.log(1e-3), np.log(0.3), 3))
        mu1 = t0 + rng.standard_normal((n1, 3)) * rng.uniform(0.3, 3.0)
        sig = np.exp(rng.uniform(np.log(0.05), np.log(1.0), n1))
        phi = rng.dirichlet(np.ones(n1))
        prob = {"mu1": mu1, "sigma1": sig, "phi1": phi, "mu2": np.array([[0.0, 0.0, 1.0]]),
                "kappa2": np.array([5.0]), "phi2": np.array([1.0])}
        ab = [oracle_mod.kappa_interval(mu1[i], sig[i], t0, thw, 0.01) for i in range(n1)]
        if any(x is None for x in ab):
            continue
        mix = oracle_mod.Mixtures.from_problem(prob)
        cube = np.concatenate([[0.0, 0.0, 0.0, 0.1], t0, thw])
        v = (mu1 - t0) / np.linalg.norm(mu1 - t0, axis=1, keepdims=True)
        psit = np.array([oracle_mod.psi_t(mu1[i], t0, thw) for i in range(n1)])
        m = np.arange(1, n1)
        c = dict(v=np.stack([np.repeat(v[:1], n1 - 1, 0), v[m]], 1), phi1=np.stack([np.full(n1 - 1, phi[0]), phi[m]], 1),
                 a=np.array([[ab[0][0], ab[k][0]] for k in m]), b=np.array([[ab[0][1], ab[k][1]] for k in m]),
                 psit=np.stack([np.full(n1 - 1, psit[0]), psit[m]], 1))
        ref = sum(oracle_mod.self_lb_term(mix, 0, k, cube, 0.01) + oracle_mod.self_lb_term(mix, k, 0, cube, 0.01)
                  for k in m)
        for signs in [(-1.0,) * 11, (1.0,) * 11] + [tuple(rng.choice([-1.0, 1.0], 11)) for _ in range(3)]:
            e, wA, Awi = _self_parts(c, signs)
            for paired in (False, True):
                row = _row_sum(e, wA, Awi[0], rng.permutation(n1 - 1), paired)
                assert row <= ref, (trial, n1, paired, row / ref - 1)


def test_the_cases_reach_every_regime(cases):
    """Near-aligned and near-antipodal pairs, tiny and pi-wide uncertainty
    angles, small and large concentrations."""
    ang = np.arccos(np.clip(np.sum(cases["v"][:, 0] * cases["u"], 1), -1, 1))
    assert (ang < 1e-2).sum() > 50 and (ang > np.pi - 1e-2).sum() > 50
    assert (cases["psit"][:, 0] >= np.pi).sum() > 100 and (cases["psit"][:, 0] < 1e-2).sum() > 100
    assert (cases["a"][:, 0] < 9).sum() > 100 and (cases["a"][:, 0] > 1e4).sum() > 100
    assert (cases["k2"] < 9).sum() > 100
