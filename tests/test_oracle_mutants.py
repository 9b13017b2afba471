"""The oracle's pins catch plausible mistakes.

Each case below plants one mistake in a copy of the oracle's source (a
dropped term or factor, a wrong sign, index or comparison, a transposed
operand, a missing clamp), builds that copy in a temporary directory and
runs the pin tests (test_oracle_pins, test_oracle_mixgen, test_oracle_mlp,
test_oracle_bnb) against it; the network's FP64 reference (an extension)
gets the same treatment.  At least one pin must fail for every mutant; the
oracle in the repository is not touched.  Mistakes that change only
efficiency (which of rotation or translation is split, the L-BFGS
direction's restart safeguard) or a documented reading (the scale of eps)
are not listed: no correctness pin can see them; nor is the global lower
bound left uncapped at d*, which differs only when a run ends with every
queued node stale.  Neither is phiZ of K at
the (b_i, b_j) corner in place of the largest corner K in the self-pair
bound: log Z(K) - k1 - k2 decreases in each concentration, so that form is a
valid (slightly tighter) bound too.  Nor are changes that double precision
cannot see: the second-order terms of the small-angle series of Rodrigues'
formula (below 1e-8 rad they round away against 1), of the right Jacobian
below 1e-6 rad (they multiply [r0]x, itself below 1e-6), or of d log Z / dx
below 1e-4 (no term of the objective reaches K < 1e-4 with any weight).
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = ["tests/test_oracle_pins.py", "tests/test_oracle_mixgen.py", "tests/test_oracle_mlp.py",
        "tests/test_oracle_bnb.py"]
G = "gosma_oracle.c"
M = "mixgen.c"
N = "mlp_oracle.py"

# (what the mistake is, file, text in the oracle, text with the mistake)
MUTANTS = [
    # Eq. (Z), the vMF inner product, Eq. (vMF_PN_map)
    ("log Z with e^-x for e^-2x", G, "return log(-expm1(-2.0 * x) / x);", "return log(-expm1(-x) / x);"),
    ("qPN concentration without the +1", G, "    return q * q + 1.0;", "    return q * q;"),
    ("log Z near 0: +x in place of -x", G, "if (x < 1e-12) return M_LN2 - x;", "if (x < 1e-12) return M_LN2 + x;"),
    ("pair term: difference in place of the sum in K", G, "w[k] = ka * ua[k] + kb * ub[k];",
     "w[k] = ka * ua[k] - kb * ub[k];"),
    ("pair term: normaliser of the wrong component", G, "return om_logZ(K) - om_logZ(ka) - om_logZ(kb);",
     "return om_logZ(K) - om_logZ(ka) - om_logZ(ka);"),
    # Rodrigues (Sec. 4.1)
    ("Rodrigues: sign of one skew term", G, "R[1] = -A * z + B * (x * y);", "R[1] = A * z + B * (x * y);"),
    ("Rodrigues: B over the angle, not its square", G, "B = (1.0 - cos(th)) / (th * th);",
     "B = (1.0 - cos(th)) / th;"),
    # Lemma 1
    ("objective: cross sum not doubled", G, "    return self - 2.0 * cross;", "    return self - cross;"),
    ("objective: model rotated by the transpose", G,
     "        matvec(R, v + 3 * i, Rv);\n        for (int j = 0; j < n2; ++j)\n            cross +=",
     "        matTvec(R, v + 3 * i, Rv);\n        for (int j = 0; j < n2; ++j)\n            cross +="),
    ("C22: both means of a pair from the same component", G, "m->kappa2[j], m->mu2 + 3 * j));\n    return s;",
     "m->kappa2[j], m->mu2 + 3 * i));\n    return s;"),
    # gradient for SMA (Sec. 5)
    ("gradient: sign of the rotation term", G, "gw[q] += -2.0 * term * gK * kap[i] * cr[q] / K;",
     "gw[q] += 2.0 * term * gK * kap[i] * cr[q] / K;"),
    ("gradient: sign of d kappa / dt", G, "dk[3 * i + q] = -2.0 * d[i] * v[3 * i + q] / s2;",
     "dk[3 * i + q] = 2.0 * d[i] * v[3 * i + q] / s2;"),
    ("gradient: right Jacobian of SO(3) in place of the left", G,
     "J[k] = (k % 4 == 0 ? 1.0 : 0.0) + a * S[k] + b * S2[k];",
     "J[k] = (k % 4 == 0 ? 1.0 : 0.0) - a * S[k] + b * S2[k];"),
    ("gradient: the left Jacobian's series at small angles", G, "a = 0.5 - th * th / 24.0;", "a = -0.5;"),
    ("gradient: d v / dt without the projection", G,
     "dv[9 * i + 3 * p + q] = -((p == q ? 1.0 : 0.0) - v[3 * i + p] * v[3 * i + q]) / d[i];",
     "dv[9 * i + 3 * p + q] = -((p == q ? 1.0 : 0.0)) / d[i];"),
    ("gradient: a self pair's kappa term of j dropped", G,
     "gt[q] += term * (gK * dK - gi * dk[3 * i + q] - gj * dk[3 * j + q]);",
     "gt[q] += term * (gK * dK - gi * dk[3 * i + q]);"),
    ("objective parts: a self pair with i twice", G,
     "self += m->phi1[i] * m->phi1[j] * exp(om_pair_log(ki, vi, kj, vj));",
     "self += m->phi1[i] * m->phi1[j] * exp(om_pair_log(ki, vi, ki, vi));"),
    ("gradient: sign of 1/x in d log Z / dx", G, "return 1.0 + 2.0 / expm1(2.0 * x) - 1.0 / x;",
     "return 1.0 + 2.0 / expm1(2.0 * x) + 1.0 / x;"),
    # Lemmas 2 and 3, the kappa interval
    ("Lemma 2: sqrt(2) in place of sqrt(3)", G, "double p = sqrt(3.0) * r_hw;", "double p = sqrt(2.0) * r_hw;"),
    ("Lemma 2 per direction: the left Jacobian in place of the right", G,
     "J[3 * p + q] = (p == q ? 1.0 : 0.0) - c1 * S[3 * p + q] + c2 * s2;",
     "J[3 * p + q] = (p == q ? 1.0 : 0.0) + c1 * S[3 * p + q] + c2 * s2;"),
    ("Lemma 2 per direction: the second-order allowance dropped", G, "double s = lin + 3.0 * r_hw * r_hw / 8.0;",
     "double s = lin;"),
    ("Lemma 2 per direction: one vertex only", G, "for (int k = 0; k < 4; ++k) { /* the 8 vertices",
     "for (int k = 0; k < 1; ++k) { /* the 8 vertices"),
    ("Lemma 2 per direction: the vertex images without the half", G, "double nx = 0.5 * norm3(x);",
     "double nx = norm3(x);"),
    ("Lemma 2 per direction: its bound unused by the cross pairs", G,
     "cp->psir_i[i] = mode == 1 ? om_psi_r_point(cube + CUBE_R0, cube[CUBE_RHW], cp->v + 3 * i) : cp->psir;",
     "cp->psir_i[i] = cp->psir;"),
    ("Lemma 3: half of the vertices", G, "for (int vtx = 0; vtx < 8; ++vtx) {", "for (int vtx = 0; vtx < 4; ++vtx) {"),
    ("Lemma 3: a point inside the cuboid gets 0", G, "if (inside) return M_PI;", "if (inside) return 0.0;"),
    ("kappa interval: nearest face in place of the farthest", G, "double f = f1 > f2 ? f1 : f2;",
     "double f = f1 < f2 ? f1 : f2;"),
    ("kappa interval: distance to the far face below the cuboid", G, "if (p[k] < lo) e = lo - p[k];",
     "if (p[k] < lo) e = hi - p[k];"),
    # Theorem 1, self pairs
    ("self pair i = j at the upper kappa", G, "        double k = a[i];\n        return w * 0.5 * k / tanh(k);",
     "        double k = b[i];\n        return w * 0.5 * k / tanh(k);"),
    ("self pair: one psi_t subtracted from A", G,
     "double A = om_angle(v + 3 * i, v + 3 * j) + psi[i] + psi[j];",
     "double A = om_angle(v + 3 * i, v + 3 * j) + psi[i] - psi[j];"),
    ("self pair: A not clamped to pi", G, "    if (A > M_PI) A = M_PI;\n", "\n"),
    ("self pair: exponent at the lower kappa ends", G, "double lg = (Kbb - b[i] - b[j]) + om_phiZ(Kmax)",
     "double lg = (Kbb - a[i] - a[j]) + om_phiZ(Kmax)"),
    # Theorem 1, cross pairs
    ("cross pair: psi_r left out of B", G, "double B = om_angle(v + 3 * i, u) - psi[i] - psir;",
     "double B = om_angle(v + 3 * i, u) - psi[i];"),
    ("cross pair: B not clamped at 0", G, "    if (B < 0.0) B = 0.0;\n", "\n"),
    ("cross pair: exponent at the upper kappa end", G, "double lg = (Ka - a[i] - k2)", "double lg = (Ka - b[i] - k2)"),
    ("cross pair: phiZ at the lower kappa end", G, "- om_phiZ(b[i]) - om_phiZ(k2);", "- om_phiZ(a[i]) - om_phiZ(k2);"),
    ("cross pair: image mean rotated by R0, not its inverse", G, "matTvec(R0, m->mu2 + 3 * j, u);",
     "matvec(R0, m->mu2 + 3 * j, u);"),
    # per-cube sums
    ("cube lower bound: cross sum not doubled", G, "out[0] = slb - 2.0 * cub;", "out[0] = slb - cub;"),
    ("cube upper bound: cross sum not doubled", G, "out[1] = cp.centre_feasible ? sc - 2.0 * cc : INFINITY;",
     "out[1] = cp.centre_feasible ? sc - cc : INFINITY;"),
    ("pi-ball test at radius 2 pi", G, "return sqrt(d2) > M_PI;", "return sqrt(d2) > 2.0 * M_PI;"),
    ("kappa interval: a cuboid wholly within zeta kept", G, "if (dmax < zeta) return 0;", "if (dmax < 0.0) return 0;"),
    ("a centre within zeta given an upper bound", G, "if (d < zeta) cp->centre_feasible = 0;",
     "if (d < 0.0) cp->centre_feasible = 0;"),
    # Algorithm 1
    ("queue: highest lower bound first", G, "if (x->lb != y->lb) return x->lb < y->lb;",
     "if (x->lb != y->lb) return x->lb > y->lb;"),
    ("Algorithm 1: global lower bound from the queue's last slot", G, "dlb = h.n > 0 ? h.a[0].lb : dstar;",
     "dlb = h.n > 0 ? h.a[h.n - 1].lb : dstar;"),
    ("Algorithm 1: children kept when above d*", G, "if (lb < dstar) heap_push(&h, &ch[c]);",
     "if (lb > dstar) heap_push(&h, &ch[c]);"),
    ("branching: both rotation halves on the same side", G,
     "c[CUBE_R0 + a] = p->cube[CUBE_R0 + a] + (((k >> a) & 1) ? h : -h);",
     "c[CUBE_R0 + a] = p->cube[CUBE_R0 + a] + (((k >> a) & 1) ? h : h);"),
    ("branching: both translation halves on the same side", G,
     "c[CUBE_T0 + a] = p->cube[CUBE_T0 + a] + (((k >> a) & 1) ? h : -h);",
     "c[CUBE_T0 + a] = p->cube[CUBE_T0 + a] + (((k >> a) & 1) ? -h : -h);"),
    # SMA
    ("SMA: Armijo test reversed", G, "if (fn <= f + 1e-4 * step * gd) {", "if (fn >= f + 1e-4 * step * gd) {"),
    ("SMA: two-loop correction with the wrong sign", G, "q[k] += S[6 * idx + k] * (alpha[h] - beta);",
     "q[k] += S[6 * idx + k] * (beta - alpha[h]);"),
    ("SMA: initial scaling inverted", G, "gamma = sy / yy;", "gamma = yy / sy;"),
    ("SMA: rho without the reciprocal", G, "rho[head] = 1.0 / sy;", "rho[head] = sy;"),
    ("SMA: gradient test on the smallest coordinate", G, "if (fabs(g[k]) > gmax) gmax = fabs(g[k]);",
     "if (fabs(g[k]) < gmax) gmax = fabs(g[k]);"),
    # mixture generation (Sec. 6)
    ("GMM fit: sigma^2 without the factor 3", M, "double s = sqrt(ss[c] / (3.0 * (double)cnt[c]));",
     "double s = sqrt(ss[c] / ((double)cnt[c]));"),
    ("vMF fit: sign of 1/kappa in the mean resultant length", M, "return 1.0 / tanh(k) - 1.0 / k;",
     "return 1.0 / tanh(k) + 1.0 / k;"),
    ("vMF fit: capped at 1, not at kappa_max", M, "                spread[c] = hi;\n", "                spread[c] = 1.0;\n"),
    ("vMF fit: mean length without the coordinate scale", M,
     "sqrt((s0 * s0 + s1 * s1) + s2 * s2) / (scale * (double)cnt[c]);",
     "sqrt((s0 * s0 + s1 * s1) + s2 * s2) / ((double)cnt[c]);"),
    ("cosine: wrong coordinate of the centre", M, "if (vmf) return (x[0] * m[0] + x[1] * m[1]) + x[2] * m[2];",
     "if (vmf) return (x[0] * m[0] + x[1] * m[1]) + x[2] * m[1];"),
    ("DP-means: a new cluster below lambda", M, "return vmf ? best < lambda : best > lambda;",
     "return vmf ? best < lambda : best < lambda;"),
    ("DP-vMF-means: a zero-sum cluster centred on its last point", M, "if (i < first[c]) first[c] = i;",
     "if (i > first[c] || first[c] == n) first[c] = i;"),
    ("GMM fit: the floor taken as a ceiling", M, "spread[c] = s > lo ? s : lo;", "spread[c] = s < lo ? s : lo;"),
    ("vMF fit: the bisection moves the wrong end", M, "if (mg_A3(exp(m)) < rbar) a = m;",
     "if (mg_A3(exp(m)) > rbar) a = m;"),
    ("DP-means: points compared with the first centre only", M, "for (int c = 1; c < K; ++c) {",
     "for (int c = 1; c < 1; ++c) {"),
    ("DP-means: the last pass not counted", M, "            ++pass;\n            break;", "            break;"),
    ("DP-means: points quantized at 2^-31", M, "#define MG_SCALE_PTS 4294967296.0       /* 2^32 */",
     "#define MG_SCALE_PTS 2147483648.0       /* 2^31 */"),
    ("DP-means: empty clusters kept", M, "            if (cnt[c] == 0) {\n                remap[c] = -1;",
     "            if (0) {\n                remap[c] = -1;"),
    ("DP-means: start at the first point, not the mean", M,
     "    mg_centre(vmf, S, n, xq, cen);\n    for (pass = 0;", "    memcpy(cen, xq, 3 * sizeof(double));\n    for (pass = 0;"),
    ("weights over the number of clusters", M, "phi[c] = (double)cnt[c] / (double)n;",
     "phi[c] = (double)cnt[c] / (double)K;"),
    # the queue-ordering network's reference (an extension)
    ("BF16: ties rounded up, not to even", N, "bias = 0x7FFF + ((u >> 16) & 1)", "bias = 0x8000 + 0 * u"),
    ("GELU: erf of z, not z / sqrt 2", N, "return 0.5 * z * (1.0 + _erf(z / SQRT2))",
     "return 0.5 * z * (1.0 + _erf(z))"),
    ("GELU derivative: sign of the density term", N, "+ z * np.exp(-0.5 * z * z)", "- z * np.exp(-0.5 * z * z)"),
    ("forward: second layer's weights transposed", N, 'z2 = h1 @ W2.T + p["b2"]', 'z2 = h1 @ W2 + p["b2"]'),
    ("backward: W2 gradient from the wrong activation", N, 'g["W2"] = dz2.T @ cache["h1"]',
     'g["W2"] = dz2.T @ cache["h2"]'),
    ("backward: first layer's GELU derivative at z2", N, 'gelu_grad(cache["z1"])', 'gelu_grad(cache["z2"])'),
    ("loss: sign in the logistic gradient", N, "dy[:, 0] = (1.0 / (1.0 + np.exp(-s)) - label) / n",
     "dy[:, 0] = (1.0 / (1.0 + np.exp(s)) - label) / n"),
    ("loss: seed gradient without the 2", N, "dy[:, 1:1 + N_SEED] = 2.0 * lam * label[:, None] * r / n",
     "dy[:, 1:1 + N_SEED] = lam * label[:, None] * r / n"),
    ("loss: seed term for negative labels too", N, "loss = (bce + lam * label * (r * r).sum(1)).mean()",
     "loss = (bce + lam * (r * r).sum(1)).mean()"),
    ("packing: biases and weights in another order", N,
     'for k in ("W1", "b1", "W2", "b2", "W3", "b3")])', 'for k in ("W1", "W2", "b1", "b2", "W3", "b3")])'),
]


def _workspace(tmp):
    """A copy of tests/ and oracle/ (sources only) beside a link to the package."""
    shutil.copytree(os.path.join(ROOT, "tests"), os.path.join(tmp, "tests"),
                    ignore=shutil.ignore_patterns("__pycache__", "test_oracle_mutants.py"))
    os.mkdir(os.path.join(tmp, "oracle"))
    for f in ("__init__.py", G, M, "mlp_oracle.py"):
        shutil.copy(os.path.join(ROOT, "oracle", f), os.path.join(tmp, "oracle", f))
    os.symlink(os.path.join(ROOT, "paper_1812_01232_gb300"), os.path.join(tmp, "paper_1812_01232_gb300"))


def _run(case):
    name, fname, old, new = case
    tmp = tempfile.mkdtemp(prefix="oracle_mutant_")
    try:
        _workspace(tmp)
        path = os.path.join(tmp, "oracle", fname)
        src = open(path).read()
        assert src.count(old) == 1, "%s: the text to change must occur exactly once" % name
        open(path, "w").write(src.replace(old, new))
        env = dict(os.environ, PYTHONDONTWRITEBYTECODE="1", OMP_NUM_THREADS="2")
        try:
            p = subprocess.run([sys.executable, "-m", "pytest", *PINS, "-x", "-q", "-p", "no:cacheprovider",
                                "-m", "not gpu"], cwd=tmp, env=env, capture_output=True, text=True, timeout=600)
        except subprocess.TimeoutExpired:
            return name, False, "timed out"
        failed = [ln.split(" ")[1] for ln in p.stdout.splitlines() if ln.startswith("FAILED ")]
        if p.returncode == 1 and failed:
            return name, True, failed[0]
        return name, False, "exit %d %s" % (p.returncode, p.stdout[-300:] + p.stderr[-300:])
    finally:
        shutil.rmtree(tmp, ignore_errors=True)


@pytest.mark.skipif(shutil.which("gcc") is None, reason="the oracle is built with gcc")
def test_every_planted_mistake_fails_a_pin():
    workers = max(1, min(8, (os.cpu_count() or 2) // 2))
    with cf.ThreadPoolExecutor(workers) as ex:
        results = list(ex.map(_run, MUTANTS))
    survivors = [(n, why) for n, caught, why in results if not caught]
    assert not survivors, "mistakes no pin catches: %s" % survivors
