"""Seeded synthetic GOSMA workloads (numpy only).

This module only draws inputs: mixtures, ground-truth poses and batches of
sub-cubes.  It holds none of the bound or objective arithmetic, so both the
CUDA path and the CPU oracle can be fed from it.

Workloads (sizes and distributions follow the evaluation set-up of the
method; the paper's own data sets are not used):

* ``tiny_problem``      10 Gaussian components in a 4 x 4 x 3 m room, 8 vMF
                        image components (7 projected + 1 outlier).
* ``paper_scale_problem`` 128 components in a 10 x 10 x 3 m room, 64 vMF
                        components (48 noisy inliers + 16 outliers in a 90
                        degree field of view).
* ``uneven_problems``   many independent tiny-style problems with component
                        counts drawn from U{16..256} x U{8..128}.
* ``stress_problem``    2048 x 512 components with kappa in U[5, 2000] and
                        near-antipodal image means.
* ``tree_cubes``        sub-cubes at given depths of the branch-and-bound
                        tree, reached by random root-to-leaf paths.

Conventions: a camera with rotation R (world to camera) and centre t sees
model point mu along R (mu - t) / |mu - t| (the transformation of the proof
of Lemma 1).  A cube row is ``[r0(3), r_half_width, t0(3), t_half_width(3)]``.
"""
from __future__ import annotations

import numpy as np

CUBE_LEN = 10


def _quat_to_matrix(q):
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
    ])


def random_rotation(rng):
    """Rotation uniform on SO(3) (normalised 4-D Gaussian quaternion).

    Returns (R, r) with r the angle-axis vector, |r| <= pi."""
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    if q[0] < 0:
        q = -q
    ang = 2.0 * np.arccos(min(1.0, q[0]))
    s = np.linalg.norm(q[1:])
    axis = q[1:] / s if s > 0 else np.array([1.0, 0.0, 0.0])
    return _quat_to_matrix(q), axis * ang


def _unit(v):
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def _uniform_sphere(rng, n):
    return _unit(rng.standard_normal((n, 3)))


def _uniform_cap(rng, n, half_angle):
    """Directions uniform (by area) on the cap of the given half-angle around +z."""
    cz = 1.0 - rng.random(n) * (1.0 - np.cos(half_angle))
    ph = rng.random(n) * 2 * np.pi
    sz = np.sqrt(np.maximum(0.0, 1 - cz * cz))
    return np.stack([sz * np.cos(ph), sz * np.sin(ph), cz], axis=1)


def _perturb(rng, d, sigma_ang):
    """Rotate each unit vector by a small random angle (isotropic, std sigma_ang per axis)."""
    out = d + sigma_ang * rng.standard_normal(d.shape)
    return _unit(out)


def _means_in_room(rng, n, half, t_gt, min_dist):
    mu = np.empty((n, 3))
    k = 0
    while k < n:
        p = (rng.random(3) * 2 - 1) * half
        if np.linalg.norm(p - t_gt) >= min_dist:
            mu[k] = p
            k += 1
    return mu


def _camera_dirs(R, mu, t):
    return _unit((mu - t) @ R.T)


def tiny_problem(seed: int, n1: int = 10, n_in: int = 7, n_out: int = 1, zeta: float = 0.5):
    """Small single problem: 4 x 4 x 3 m room, sigma = 0.05 m, equal weights,
    image = n_in projected components (qPN concentration) + n_out outliers
    (uniform direction, kappa = 50).  Translation domain [-1, 1]^3."""
    rng = np.random.default_rng(seed)
    R, r = random_rotation(rng)
    t_gt = rng.uniform(-0.5, 0.5, 3)
    half = np.array([2.0, 2.0, 1.5])
    mu1 = _means_in_room(rng, n1, half, t_gt, 1.2 * zeta)
    sigma1 = np.full(n1, 0.05)
    phi1 = np.full(n1, 1.0 / n1)
    idx = rng.permutation(n1)[:n_in]
    dirs_in = _camera_dirs(R, mu1[idx], t_gt)
    dist = np.linalg.norm(mu1[idx] - t_gt, axis=1)
    kap_in = (dist / sigma1[idx]) ** 2 + 1.0
    dirs_out = _uniform_sphere(rng, n_out)
    mu2 = np.concatenate([dirs_in, dirs_out])
    kappa2 = np.concatenate([kap_in, np.full(n_out, 50.0)])
    n2 = n_in + n_out
    phi2 = np.full(n2, 1.0 / n2)
    return dict(name="tiny", mu1=mu1, sigma1=sigma1, phi1=phi1, mu2=mu2, kappa2=kappa2, phi2=phi2,
                t_lo=np.full(3, -1.0), t_hi=np.full(3, 1.0), zeta=zeta, eps=1e-3,
                R_gt=R, r_gt=r, t_gt=t_gt)


def semantic_problem(seed: int, nclass: int = 3, n1: int = 4, n_in: int = 3, n_out: int = 1, zeta: float = 0.5,
                     noise_free: bool = False, sigma: float = None):
    """Semantic scene (Sec. 4.2): nclass classes sharing one true pose, each
    with its own model mixture (n1 components in the 4 x 4 x 3 m room,
    sigma = 0.05 m, or 0.1 m noise-free, unless given) and image mixture (n_in projected
    components with the qPN concentration + n_out outliers with kappa = 50;
    noise-free: every component projected, no outliers).  Equal weights
    within a class, class weights 1 / nclass.  Also returns the
    concatenation (class by class) with the class sizes n1c, n2c."""
    rng = np.random.default_rng(seed)
    R, r = random_rotation(rng)
    t_gt = rng.uniform(-0.5, 0.5, 3)
    half = np.array([2.0, 2.0, 1.5])
    classes = []
    for _ in range(nclass):
        mu1 = _means_in_room(rng, n1, half, t_gt, 1.2 * zeta)
        sig = sigma if sigma is not None else (0.1 if noise_free else 0.05)
        sigma1 = np.full(n1, sig)
        phi1 = np.full(n1, 1.0 / n1)
        idx = np.arange(n1) if noise_free else rng.permutation(n1)[:n_in]
        dirs = _camera_dirs(R, mu1[idx], t_gt)
        kap = (np.linalg.norm(mu1[idx] - t_gt, axis=1) / sigma1[idx]) ** 2 + 1.0
        no = 0 if noise_free else n_out
        mu2 = np.concatenate([dirs, _uniform_sphere(rng, no)]) if no else dirs
        kappa2 = np.concatenate([kap, np.full(no, 50.0)]) if no else kap
        phi2 = np.full(len(kappa2), 1.0 / len(kappa2))
        classes.append(dict(mu1=mu1, sigma1=sigma1, phi1=phi1, mu2=mu2, kappa2=kappa2, phi2=phi2))
    cat = {k: np.concatenate([c[k] for c in classes]) for k in ("mu1", "sigma1", "phi1", "mu2", "kappa2", "phi2")}
    return dict(name="semantic", classes=classes, w=np.full(nclass, 1.0 / nclass),
                n1c=np.array([len(c["sigma1"]) for c in classes]), n2c=np.array([len(c["kappa2"]) for c in classes]),
                t_lo=np.full(3, -1.0), t_hi=np.full(3, 1.0), zeta=zeta, eps=1e-3, R_gt=R, r_gt=r, t_gt=t_gt, **cat)


def noise_free_problem(seed: int, n1: int = 6, zeta: float = 0.5):
    """Every model component projected at the true pose with its own qPN
    concentration and weight: the image mixture equals the projected model
    mixture, so the L2 distance is zero at the true pose."""
    rng = np.random.default_rng(seed)
    R, r = random_rotation(rng)
    t_gt = rng.uniform(-0.5, 0.5, 3)
    half = np.array([2.0, 2.0, 1.5])
    mu1 = _means_in_room(rng, n1, half, t_gt, 1.2 * zeta)
    sigma1 = np.full(n1, 0.25)
    phi1 = np.full(n1, 1.0 / n1)
    mu2 = _camera_dirs(R, mu1, t_gt)
    kappa2 = (np.linalg.norm(mu1 - t_gt, axis=1) / sigma1) ** 2 + 1.0
    return dict(name="noise_free", mu1=mu1, sigma1=sigma1, phi1=phi1, mu2=mu2, kappa2=kappa2, phi2=phi1.copy(),
                t_lo=np.full(3, -1.0), t_hi=np.full(3, 1.0), zeta=zeta, eps=1e-3,
                R_gt=R, r_gt=r, t_gt=t_gt)


def paper_scale_problem(seed: int, n1: int = 128, n_in: int = 48, n_out: int = 16, zeta: float = 0.5):
    """10 x 10 x 3 m room, sigma in U[0.03, 0.1] m, Dirichlet(1) weights.
    Image: the n_in model components nearest the optical axis (+z of the
    camera), each direction perturbed by 1 degree of angular noise, plus
    n_out directions uniform on a 90 degree field-of-view cap; kappa in
    U[20, 200]; Dirichlet(1) weights.  Translation domain [-2, 2]^3."""
    rng = np.random.default_rng(seed)
    R, r = random_rotation(rng)
    t_gt = rng.uniform(-1.0, 1.0, 3)
    half = np.array([5.0, 5.0, 1.5])
    mu1 = _means_in_room(rng, n1, half, t_gt, 1.2 * zeta)
    sigma1 = rng.uniform(0.03, 0.1, n1)
    phi1 = rng.dirichlet(np.ones(n1))
    d = _camera_dirs(R, mu1, t_gt)
    idx = np.argsort(-d[:, 2])[:n_in]
    dirs_in = _perturb(rng, d[idx], np.deg2rad(1.0))
    dirs_out = _uniform_cap(rng, n_out, np.deg2rad(45.0))
    mu2 = np.concatenate([dirs_in, dirs_out])
    n2 = n_in + n_out
    kappa2 = rng.uniform(20.0, 200.0, n2)
    phi2 = rng.dirichlet(np.ones(n2))
    return dict(name="paper_scale", mu1=mu1, sigma1=sigma1, phi1=phi1, mu2=mu2, kappa2=kappa2, phi2=phi2,
                t_lo=np.full(3, -2.0), t_hi=np.full(3, 2.0), zeta=zeta, eps=1e-4,
                R_gt=R, r_gt=r, t_gt=t_gt)


def uneven_problems(seed: int, count: int = 256, outlier_frac: float = 0.2):
    """Independent tiny-style problems with n1 ~ U{16..256}, n2 ~ U{8..128},
    a fraction of the image components being outliers."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        n1 = int(rng.integers(16, 257))
        n2 = int(rng.integers(8, 129))
        n_out = int(round(outlier_frac * n2))
        n_in = min(n2 - n_out, n1)
        n_out = n2 - n_in
        p = tiny_problem(int(rng.integers(0, 2**31)), n1=n1, n_in=n_in, n_out=n_out)
        p["name"] = "uneven_%d" % k
        out.append(p)
    return out


def stress_problem(seed: int, n1: int = 2048, n2: int = 512, antipodal_frac: float = 0.1, zeta: float = 0.5):
    """Large precision stress: 10 x 10 x 3 m room, sigma in U[0.03, 0.1] m,
    kappa_2 in U[5, 2000]; at least ``antipodal_frac`` of the image means lie
    within 1 degree of the antipode of a projected model mean."""
    rng = np.random.default_rng(seed)
    R, r = random_rotation(rng)
    t_gt = rng.uniform(-1.0, 1.0, 3)
    half = np.array([5.0, 5.0, 1.5])
    mu1 = _means_in_room(rng, n1, half, t_gt, 1.2 * zeta)
    sigma1 = rng.uniform(0.03, 0.1, n1)
    phi1 = rng.dirichlet(np.ones(n1))
    d = _camera_dirs(R, mu1, t_gt)
    n_anti = int(np.ceil(antipodal_frac * n2))
    n_in = n2 // 2
    n_rand = n2 - n_in - n_anti
    pick = rng.permutation(n1)
    dirs_in = _perturb(rng, d[pick[:n_in]], np.deg2rad(0.5))
    anti = -d[pick[n_in:n_in + n_anti]]
    # move each antipode by an angle in [0, 1] degree
    dirs_anti = _unit(anti + np.tan(np.deg2rad(rng.uniform(0, 1.0, (n_anti, 1)))) *
                      _unit(np.cross(anti, rng.standard_normal((n_anti, 3)))))
    dirs_rand = _uniform_sphere(rng, n_rand)
    mu2 = np.concatenate([dirs_in, dirs_anti, dirs_rand])
    kappa2 = rng.uniform(5.0, 2000.0, n2)
    phi2 = rng.dirichlet(np.ones(n2))
    return dict(name="stress", mu1=mu1, sigma1=sigma1, phi1=phi1, mu2=mu2, kappa2=kappa2, phi2=phi2,
                t_lo=np.full(3, -2.0), t_hi=np.full(3, 2.0), zeta=zeta, eps=1e-4,
                R_gt=R, r_gt=r, t_gt=t_gt)


def pose_seeds(prob, n: int, seed: int):
    """n seed poses (r then t) for local refinement: every other one near the
    true pose (r, t perturbed by N(0, 0.1^2) per coordinate), the rest with
    r uniform in the pi-ball and t uniform over the translation domain."""
    rng = np.random.default_rng(seed)
    r = rng.normal(size=(n, 3))
    r /= np.linalg.norm(r, axis=1)[:, None]
    r *= (np.pi * rng.random(n) ** (1 / 3))[:, None]
    t = rng.uniform(prob["t_lo"], prob["t_hi"], (n, 3))
    near = np.arange(n) % 2 == 0
    r[near] = prob["r_gt"] + rng.normal(scale=0.1, size=(int(near.sum()), 3))
    t[near] = prob["t_gt"] + rng.normal(scale=0.1, size=(int(near.sum()), 3))
    return np.hstack([r, t])


def scene_points(seed: int, n: int = 100_000, n_bear: int = 100_000, noise: float = 0.01):
    """A synthetic indoor scene for mixture generation (Sec. 6 clusters a
    point set and an image's bearing vectors; the real-data runs downsample
    both to 100k).  Points lie on the floor, ceiling and walls of a
    10 x 10 x 3 m room and on 20 axis-aligned boxes, uniformly by area, with
    N(0, noise^2) jitter.  Bearing vectors are the unit directions
    R (p - t) / |p - t| of other surface points seen by a camera at t (random
    near the room centre, random rotation R) within a 60-degree half-angle
    cone.  Returns dict(points (n, 3), bearings (n_bear, 3), R, r, t)."""
    rng = np.random.default_rng(seed)
    L, W, H = 10.0, 10.0, 3.0
    faces = [  # (origin, edge u, edge v): rectangles of the room ...
        ((-L / 2, -W / 2, 0), (L, 0, 0), (0, W, 0)), ((-L / 2, -W / 2, H), (L, 0, 0), (0, W, 0)),
        ((-L / 2, -W / 2, 0), (L, 0, 0), (0, 0, H)), ((-L / 2, W / 2, 0), (L, 0, 0), (0, 0, H)),
        ((-L / 2, -W / 2, 0), (0, W, 0), (0, 0, H)), ((L / 2, -W / 2, 0), (0, W, 0), (0, 0, H))]
    for _ in range(20):  # ... and the five visible faces of each box
        c = rng.uniform([-4, -4, 0], [4, 4, 0])
        sx, sy, sz = rng.uniform([0.3, 0.3, 0.3], [1.5, 1.5, 1.2])
        o = c - [sx / 2, sy / 2, 0]
        faces += [(tuple(o + [0, 0, sz]), (sx, 0, 0), (0, sy, 0)), (tuple(o), (sx, 0, 0), (0, 0, sz)),
                  (tuple(o + [0, sy, 0]), (sx, 0, 0), (0, 0, sz)), (tuple(o), (0, sy, 0), (0, 0, sz)),
                  (tuple(o + [sx, 0, 0]), (0, sy, 0), (0, 0, sz))]
    O = np.array([f[0] for f in faces], float)
    U = np.array([f[1] for f in faces], float)
    V = np.array([f[2] for f in faces], float)
    area = np.linalg.norm(np.cross(U, V), axis=1)

    def sample(m):
        k = rng.choice(len(faces), size=m, p=area / area.sum())
        a, b = rng.random((2, m))
        return O[k] + a[:, None] * U[k] + b[:, None] * V[k] + noise * rng.normal(size=(m, 3))

    pts = sample(n)
    R, r = random_rotation(rng)
    t = rng.uniform([-1, -1, 1.2], [1, 1, 1.8])
    bear = np.zeros((0, 3))
    while len(bear) < n_bear:
        d = sample(4 * n_bear) - t
        d /= np.linalg.norm(d, axis=1)[:, None]
        d = d @ R.T
        bear = np.concatenate([bear, d[d[:, 2] > np.cos(np.radians(60))]])
    bear = bear[:n_bear]
    bear /= np.linalg.norm(bear, axis=1)[:, None]
    return {"points": pts, "bearings": bear, "R": R, "r": r, "t": t}


def root_cube(t_lo, t_hi):
    t_lo = np.asarray(t_lo, dtype=np.float64)
    t_hi = np.asarray(t_hi, dtype=np.float64)
    c = np.zeros(CUBE_LEN)
    c[3] = np.pi
    c[4:7] = 0.5 * (t_lo + t_hi)
    c[7:10] = 0.5 * (t_hi - t_lo)
    return c


def tree_cubes(seed: int, n: int, t_lo, t_hi, depth_lo: int = 2, depth_hi: int = 12, near=None, near_frac=0.0):
    """``n`` sub-cubes at depths uniform in [depth_lo, depth_hi], each reached
    from the root by a random path (at every level a random choice between
    splitting rotation and translation, then a random child of the eight).
    Cubes whose rotation part lies wholly outside the pi-ball are redrawn.
    With ``near=(r, t)``, a fraction ``near_frac`` of the paths follow the
    children that contain that pose, so the batch also holds cubes around
    the optimum.  (Scalar arithmetic per level, in the order of the
    vectorised statement c[a:b] + (2 bits - 1) h.)"""
    rng = np.random.default_rng(seed)
    root = [float(v) for v in root_cube(t_lo, t_hi)]
    nr = [float(v) for v in near[0]] if near is not None else None
    nt = [float(v) for v in near[1]] if near is not None else None
    out = np.empty((n, CUBE_LEN))
    depth = rng.integers(depth_lo, depth_hi + 1, n).tolist()
    k = 0
    while k < n:
        c = list(root)
        follow = near is not None and rng.random() < near_frac
        for _ in range(depth[k]):
            if rng.random() < 0.5:
                h = c[3] * 0.5
                if follow:
                    bits = [1.0 if nr[a] > c[a] else 0.0 for a in range(3)]
                else:
                    bits = rng.integers(0, 2, 3).tolist()
                for a in range(3):
                    c[a] = c[a] + (2.0 * bits[a] - 1.0) * h
                c[3] = h
            else:
                if follow:
                    bits = [1.0 if nt[a] > c[4 + a] else 0.0 for a in range(3)]
                else:
                    bits = rng.integers(0, 2, 3).tolist()
                for a in range(3):
                    h = c[7 + a] * 0.5
                    c[4 + a] = c[4 + a] + (2.0 * bits[a] - 1.0) * h
                    c[7 + a] = h
        gap = np.maximum(np.abs(np.array(c[0:3])) - c[3], 0.0)
        if np.linalg.norm(gap) > np.pi:
            continue
        out[k] = c
        k += 1
    return out
