"""The pre-pass's Rodrigues' formula in double-float arithmetic, replayed on
the CPU (rodrigues_df in csrc/bounds_core.cuh, df_sincos and the other
double-float helpers in csrc/dfloat.cuh).

The constants are read from the source: pi/2 in three floats (the first two
of at most 20 significant bits, so that k times them is exact for the
quadrants used), 2/pi, and the double-float and FP32 coefficients of the
sin and cos series, each checked against the exact reciprocal factorial.
The algorithm is then replayed in numpy float32, operation by operation
(fused multiply-adds through FP64), and its rotations compared with the
oracle's FP64 Rodrigues' formula on the vectors the GPU test uses: cell
centres at every level, random vectors up to |r| = pi sqrt(3), vectors by
the range reduction's boundaries, the small-angle series and the zero
vector.  A wrong coefficient or reduction constant fails one of the two.
"""
import math
import os
import re
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1812_01232_gb300", "csrc")
F = np.float32
HEX = r"-?0x1\.[0-9a-f]+p[-+]?\d+f"


def _hex(s):
    return F(float.fromhex(s.rstrip("f")))


def _source_constants():
    src = open(os.path.join(CSRC, "dfloat.cuh")).read()
    body = src[src.index("__device__ inline void df_sincos"):]
    body = body[:body.index("\n}\n")]
    c = {}
    m = re.search(r"P1 = (%s), P2 = (%s), P3 = (%s);" % (HEX, HEX, HEX), body)
    c["P"] = [_hex(m.group(i)) for i in (1, 2, 3)]
    c["two_over_pi"] = _hex(re.search(r"rintf\(t\.h \* (%s)\)" % HEX, body).group(1))
    m = re.search(r"float ts = (%s), tc = (%s);" % (HEX, HEX), body)
    ts0, tc0 = _hex(m.group(1)), _hex(m.group(2))
    c["ts"] = [ts0] + [_hex(x) for x in re.findall(r"ts = fmaf\(ts, z\.h, (%s)\)" % HEX, body)]
    c["tc"] = [tc0] + [_hex(x) for x in re.findall(r"tc = fmaf\(tc, z\.h, (%s)\)" % HEX, body)]

    def pairs(name):
        block = body[body.index("const df %s[5]" % name):]
        block = block[:block.index("};")]
        out = [(F(1), F(0))] if "{1.f, 0.f}" in block.split("\n")[0] else []
        for a, b in re.findall(r"\{(%s|-?0\.5f), (%s|0\.f)\}" % (HEX, HEX), block):
            out.append((_hex(a) if a.startswith(("0x", "-0x")) else F(float(a.rstrip("f"))),
                        _hex(b) if b.startswith(("0x", "-0x")) else F(0)))
        return out

    c["cs"], c["cc"] = pairs("cs"), pairs("cc")
    return c


C = _source_constants()


def test_reduction_constants():
    P1, P2, P3 = (Fraction(float(p)) for p in C["P"])
    # the three parts sum to pi/2 within 2^-66 (a float P3 leaves ~2^-69)
    half_pi = Fraction("1.5707963267948966192313216916397514420985846996875529104875")
    assert abs(P1 + P2 + P3 - half_pi) < Fraction(1, 2 ** 66)
    for p in C["P"][:2]:  # at most 20 significant bits: k p exact for |k| <= 15
        m, e = math.frexp(float(p))
        assert (Fraction(abs(m)) * 2 ** 20).denominator == 1
    assert abs(Fraction(float(C["two_over_pi"])) - 1 / half_pi) <= Fraction(1, 2 ** 24)


def test_series_coefficients():
    """sin x / x = sum (-1)^n x^2n / (2n + 1)!, cos x = sum (-1)^n x^2n / (2n)!:
    the double-float leading terms to 2^-48 relative, the FP32 tail to 2^-24."""
    assert len(C["cs"]) == len(C["cc"]) == 5
    for n, (h, l) in enumerate(C["cs"]):
        exact = Fraction((-1) ** n, math.factorial(2 * n + 1))
        assert abs(Fraction(float(h)) + Fraction(float(l)) - exact) <= abs(exact) / 2 ** 48, n
    for n, (h, l) in enumerate(C["cc"]):
        exact = Fraction((-1) ** n, math.factorial(2 * n))
        assert abs(Fraction(float(h)) + Fraction(float(l)) - exact) <= abs(exact) / 2 ** 48, n
    # the tails run from the highest term down to n = 5
    for coeffs, off in ((C["ts"], 1), (C["tc"], 0)):
        top = 5 + len(coeffs) - 1
        for i, v in enumerate(coeffs):
            n = top - i
            exact = Fraction((-1) ** n, math.factorial(2 * n + off))
            assert abs(Fraction(float(v)) - exact) <= abs(exact) / 2 ** 24, (off, n)


# ---------------------------------------------------------------- the replay
def fmaf(a, b, c):
    return F(np.float64(a) * np.float64(b) + np.float64(c))


def two_sum(a, b):
    s = F(a + b)
    bb = F(s - a)
    return s, F(F(a - F(s - bb)) + F(b - bb))


def fast_two_sum(a, b):
    s = F(a + b)
    return s, F(b - F(s - a))


def two_prod(a, b):
    p = F(a * b)
    return p, fmaf(a, b, -p)


def df_mul(a, b):
    p = two_prod(a[0], b[0])
    return fast_two_sum(p[0], F(p[1] + fmaf(a[0], b[1], F(a[1] * b[0]))))


def df_add(a, b):
    s = two_sum(a[0], b[0])
    return fast_two_sum(s[0], F(s[1] + F(a[1] + b[1])))


def df_sub(a, b):
    s = two_sum(a[0], -b[0])
    return fast_two_sum(s[0], F(s[1] + F(a[1] - b[1])))


def df_rsqrt(d, r0):
    q = two_prod(r0, r0)
    hh = two_prod(d[0], q[0])
    hl = F(hh[1] + fmaf(d[0], q[1], F(d[1] * q[0])))
    return fast_two_sum(r0, F(F(F(0.5) * r0) * F(F(F(1) - hh[0]) - hl)))


def df_div(a, b):
    q0 = F(a[0] / b[0])
    p = two_prod(q0, b[0])
    r = F(F(F(F(a[0] - p[0]) - p[1]) + a[1]) - F(q0 * b[1]))
    return fast_two_sum(q0, F(r / b[0]))


def df_sincos(t):
    P1, P2, P3 = C["P"]
    k = F(np.rint(F(t[0] * C["two_over_pi"])))
    a = two_sum(F(t[0] - F(k * P1)), t[1])
    b = two_sum(a[0], F(-F(k * P2)))
    x = fast_two_sum(b[0], F(F(a[1] + b[1]) - F(k * P3)))
    z = df_mul(x, x)
    ts, tc = C["ts"][0], C["tc"][0]
    for c in C["ts"][1:]:
        ts = fmaf(ts, z[0], c)
    for c in C["tc"][1:]:
        tc = fmaf(tc, z[0], c)
    ps, pc = (ts, F(0)), (tc, F(0))
    for n in range(4, -1, -1):
        ps = df_add(df_mul(ps, z), C["cs"][n])
        pc = df_add(df_mul(pc, z), C["cc"][n])
    sx = df_mul(x, ps)
    nsx, npc = (-sx[0], -sx[1]), (-pc[0], -pc[1])
    q = int(k) & 3
    return [sx, pc, nsx, npc][q], [pc, nsx, npc, sx][q]


def _split(v):
    h = F(v)
    return h, F(v - np.float64(h))


def rodrigues_df(r0):
    x, y, z = _split(r0[0]), _split(r0[1]), _split(r0[2])
    xx, yy, zz = df_mul(x, x), df_mul(y, y), df_mul(z, z)
    th2 = df_add(df_add(xx, yy), zz)
    one = (F(1), F(0))
    if th2[0] < F(1e-6):
        A = df_add(one, df_mul(th2, (fmaf(th2[0], F(1) / F(120), F(-1) / F(6)), F(0))))
        B = df_add((F(0.5), F(0)), df_mul(th2, (fmaf(th2[0], F(1) / F(720), F(-1) / F(24)), F(0))))
    else:
        th = df_mul(th2, df_rsqrt(th2, F(1 / np.sqrt(np.float64(th2[0])))))
        sn, cs = df_sincos(th)
        A, B = df_div(sn, th), df_div(df_sub(one, cs), th2)
    xy, xz, yz = df_mul(x, y), df_mul(x, z), df_mul(y, z)
    Ax, Ay, Az = df_mul(A, x), df_mul(A, y), df_mul(A, z)
    Bxy, Bxz, Byz = df_mul(B, xy), df_mul(B, xz), df_mul(B, yz)
    R = [df_sub(one, df_mul(B, df_add(yy, zz))), df_sub(Bxy, Az), df_add(Bxz, Ay),
         df_add(Bxy, Az), df_sub(one, df_mul(B, df_add(xx, zz))), df_sub(Byz, Ax),
         df_sub(Bxz, Ay), df_add(Byz, Ax), df_sub(one, df_mul(B, df_add(xx, yy)))]
    return np.array([np.float64(h) + np.float64(l) for h, l in R]).reshape(3, 3)


def _vectors(rng):
    vecs = [np.zeros(3)]
    for lr in range(1, 31):
        h = np.pi * 2.0 ** -lr
        vecs += list(-np.pi + (2 * rng.integers(0, 2 ** lr, (4, 3)) + 1) * h)
    d = rng.standard_normal((1200, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    vecs += list(d[:500] * rng.uniform(0, np.pi * np.sqrt(3), 500)[:, None])
    near = np.concatenate([k * np.pi / 4 + rng.uniform(-1e-6, 1e-6, 50) for k in range(1, 7)])
    vecs += list(d[500:800] * near[:, None])
    small = np.concatenate([10.0 ** rng.uniform(-12, -3, 150), 1e-3 * (1 + rng.uniform(-1e-4, 1e-4, 50))])
    vecs += list(d[800:1000] * small[:, None])
    return vecs


def test_replayed_rotations_match_the_oracle(oracle_mod):
    vecs = _vectors(np.random.default_rng(5))
    err = np.array([np.abs(rodrigues_df(v) - oracle_mod.rodrigues(v)).max() for v in vecs])
    assert err.max() <= 2.0 ** -42, (err.max(), vecs[int(err.argmax())])


@pytest.mark.parametrize("which,index", [("cs", 2), ("cc", 3), ("P", 1), ("ts", 1)])
def test_a_wrong_constant_is_caught(oracle_mod, which, index):
    """One constant off in its last bits fails the replay (the leading
    terms, the reduction) or the coefficient check (the FP32 tail, whose
    terms are too small for the replay to see), so the tests above pin
    every constant."""
    global C
    keep = C
    C = {k: (list(v) if isinstance(v, list) else v) for k, v in keep.items()}
    try:
        if which in ("cs", "cc"):
            h, l = C[which][index]
            C[which][index] = (F(h * F(1 + 2 ** -20)), l)
        else:
            C[which][index] = F(C[which][index] * F(1 + 2 ** -20))
        if which == "ts":
            with pytest.raises(AssertionError):
                test_series_coefficients()
        else:
            vecs = _vectors(np.random.default_rng(6))
            err = max(np.abs(rodrigues_df(v) - oracle_mod.rodrigues(v)).max() for v in vecs)
            assert err > 2.0 ** -42
    finally:
        C = keep
