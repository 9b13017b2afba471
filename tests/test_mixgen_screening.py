"""The FP32 screening of mixture generation, replayed on the CPU.

The device's DP-means and DP-vMF-means (csrc/mixgen.cu) take every decision
in FP64 but first screen the centres in FP32: a squared distance of
quantized points is within E = 128 u A^2 of the FP64 one (A the largest
coordinate magnitude), a cosine of unit vectors within 8u.  A point's
nearest centre is searched among the centres whose FP32 value is within
2.25 E of the best FP32 value; a new centre is tested in FP64 against a
point's current best only when its FP32 value is within 1.25 E of beating
it.  This replays both steps as the kernel writes them (FP32 coordinates,
the same fused multiply-adds) on near-tie data and checks that the screened
decision always equals the exact FP64 one (lowest index on ties)."""
import numpy as np

U = 2.0 ** -24
F = np.float32


def fma(a, b, c):
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


def score32(x, m, vmf):
    """mg_score32 for points x (n, 3) against centres m (k, 3), float32."""
    x, m = x[:, None, :], m[None, :, :]
    if vmf:
        return fma(x[..., 2], m[..., 2], fma(x[..., 1], m[..., 1], x[..., 0] * m[..., 0]))
    d = x - m
    return fma(d[..., 2], d[..., 2], fma(d[..., 1], d[..., 1], d[..., 0] * d[..., 0]))


def score64(x, m, vmf):
    """The FP64 score with the stated order of operations, each rounded once."""
    x, m = x[:, None, :], m[None, :, :]
    if vmf:
        return (x[..., 0] * m[..., 0] + x[..., 1] * m[..., 1]) + x[..., 2] * m[..., 2]
    d = x - m
    return (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]


def quantize(x, vmf):
    s = 2.0 ** 40 if vmf else 2.0 ** 32
    return np.rint(x * s) / s


def bound(x, vmf):
    A = np.abs(x).max() + 2.0 ** -32
    return F(8.0 * U) if vmf else F(128.0 * U * A * A)


def _nearest(x, cen, vmf):
    """Step 1 of a pass: screened nearest centre (kernel) and the exact one."""
    xf, cf = x.astype(np.float32), cen.astype(np.float32)
    E = bound(np.concatenate([x, cen]), vmf)
    s32 = score32(xf, cf, vmf)
    b32 = s32.max(1) if vmf else s32.min(1)
    lim = (b32 - F(2.25) * E) if vmf else (b32 + F(2.25) * E)
    s64 = score64(x, cen, vmf)
    cand = (s32 >= lim[:, None]) if vmf else (s32 <= lim[:, None])
    masked = np.where(cand, s64, -np.inf if vmf else np.inf)
    screened = masked.argmax(1) if vmf else masked.argmin(1)  # first index on ties
    exact = s64.argmax(1) if vmf else s64.argmin(1)
    return screened, exact, cand.sum(1)


def _near_ties(rng, n, k, vmf, spread):
    """Centres on a sphere around each point's neighbourhood with tiny
    perturbations, so that several centres tie to FP32 precision."""
    if vmf:
        base = rng.standard_normal(3)
        base /= np.linalg.norm(base)
        ang = rng.uniform(0.01, 0.5)
        # centres on a cone of half-angle ang around base, points near base
        t = rng.standard_normal((k, 3))
        t -= (t @ base)[:, None] * base
        t /= np.linalg.norm(t, axis=1, keepdims=True)
        cen = np.cos(ang) * base + np.sin(ang) * t + rng.standard_normal((k, 3)) * spread
        cen /= np.linalg.norm(cen, axis=1, keepdims=True)
        x = base + rng.standard_normal((n, 3)) * spread
        x /= np.linalg.norm(x, axis=1, keepdims=True)
        return quantize(x, True), quantize(cen, True)
    c0 = rng.uniform(-50, 50, 3)
    r = rng.uniform(0.01, 5.0)
    dirs = rng.standard_normal((k, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    cen = c0 + r * dirs + rng.standard_normal((k, 3)) * spread * r
    x = c0 + rng.standard_normal((n, 3)) * spread * r
    return quantize(x, False), quantize(cen, False)


def test_screening_bound_holds():
    """|FP32 score - FP64 score| <= E on points and centres spread over
    [-A, A], near each other and far apart."""
    rng = np.random.default_rng(0)
    for vmf in (False, True):
        for _ in range(20):
            if vmf:
                x = rng.standard_normal((2000, 3))
                x /= np.linalg.norm(x, axis=1, keepdims=True)
                x = quantize(x, True)
            else:
                A = 10.0 ** rng.uniform(-2, 3)
                x = quantize(rng.uniform(-A, A, (2000, 3)), False)
            cen = x[rng.choice(len(x), 64, replace=False)] + (0 if vmf else rng.standard_normal((64, 3)) * 1e-3)
            if vmf:
                cen /= np.linalg.norm(cen, axis=1, keepdims=True)
            cen = quantize(cen, vmf)
            E = bound(np.concatenate([x, cen]), vmf)
            err = np.abs(score32(x.astype(np.float32), cen.astype(np.float32), vmf).astype(np.float64) -
                         score64(x, cen, vmf))
            assert err.max() <= E, (vmf, err.max() / E)


def test_nearest_centre_screen_keeps_the_exact_winner():
    rng = np.random.default_rng(1)
    total = multi = 0
    for vmf in (False, True):
        for trial in range(60):
            spread = 10.0 ** rng.uniform(-9, -3)
            x, cen = _near_ties(rng, 500, int(rng.integers(2, 40)), vmf, spread)
            screened, exact, ncand = _nearest(x, cen, vmf)
            np.testing.assert_array_equal(screened, exact)
            total += len(x)
            multi += (ncand > 1).sum()
    assert multi > total // 10  # the screen had real choices to make


def test_new_centre_screen_never_skips_a_winner():
    """Step 2: a new centre m replaces a point's best exactly when it is
    better in FP64; the FP32 test may skip the FP64 comparison only where m
    cannot win."""
    rng = np.random.default_rng(2)
    tested = skipped = 0
    for vmf in (False, True):
        for trial in range(60):
            spread = 10.0 ** rng.uniform(-9, -3)
            x, cen = _near_ties(rng, 500, 2, vmf, spread)
            E = bound(np.concatenate([x, cen]), vmf)
            best = score64(x, cen[:1], vmf)[:, 0]  # the current best, exact
            bf = best.astype(np.float32)
            s32 = score32(x.astype(np.float32), cen[1:].astype(np.float32), vmf)[:, 0]
            s64 = score64(x, cen[1:], vmf)[:, 0]
            skip = (s32 + F(1.25) * E <= bf) if vmf else (s32 - F(1.25) * E >= bf)
            wins = (s64 > best) if vmf else (s64 < best)
            assert not np.any(skip & wins), (vmf, trial)
            tested += len(x)
            skipped += skip.sum()
    assert 0 < skipped < tested  # both outcomes occur
