"""FP64 CPU oracle for GOSMA: ctypes binding of ``gosma_oracle.c`` and
``mixgen.c`` (mixture generation, Sec. 6).

TEST INFRASTRUCTURE ONLY.  The test-suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` are the only callers.  The product
package never imports this module and the two share no code.

Every function maps one-to-one onto a C function whose comment cites the
passage of the paper it follows (Lemma 1, Lemmas 2-3, Theorem 1,
Algorithm 1).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gosma_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "mixgen.c")]
_LIB = os.path.join(_HERE, "liboracle_gosma.so")
_lock = threading.Lock()
_lib = None

D = C.POINTER(C.c_double)


class Mix(C.Structure):
    _fields_ = [("n1", C.c_int), ("mu1", D), ("sigma1", D), ("phi1", D),
                ("n2", C.c_int), ("mu2", D), ("kappa2", D), ("phi2", D)]


class Domain(C.Structure):
    _fields_ = [("t_lo", C.c_double * 3), ("t_hi", C.c_double * 3), ("zeta", C.c_double)]


class SmaOpts(C.Structure):
    _fields_ = [("max_iter", C.c_int), ("memory", C.c_int), ("gtol", C.c_double)]


class BnbOpts(C.Structure):
    _fields_ = [("eps", C.c_double), ("pop", C.c_int), ("max_nodes", C.c_longlong),
                ("max_seconds", C.c_double), ("use_sma", C.c_int), ("nthreads", C.c_int),
                ("sma", SmaOpts), ("psi_mode", C.c_int)]


class BnbResult(C.Structure):
    _fields_ = [("f", C.c_double), ("lb", C.c_double), ("f_norm", C.c_double),
                ("gap_norm", C.c_double), ("c22", C.c_double), ("r", C.c_double * 3),
                ("t", C.c_double * 3), ("R", C.c_double * 9), ("nodes", C.c_longlong),
                ("iterations", C.c_longlong), ("sma_calls", C.c_longlong),
                ("queue_peak", C.c_longlong), ("seconds", C.c_double), ("status", C.c_int)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP when available)."""
    with _lock:
        if not force and os.path.exists(_LIB) and all(os.path.getmtime(_LIB) >= os.path.getmtime(f) for f in _SRCS):
            return _LIB
        base = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared"] + _SRCS + ["-o", _LIB + ".tmp", "-lm"]
        r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True, text=True)
        if r.returncode != 0:
            r = subprocess.run(base, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError("oracle build failed:\n" + r.stderr)
        os.replace(_LIB + ".tmp", _LIB)
        return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        L.om_phiZ.restype = C.c_double
        L.om_phiZ.argtypes = [C.c_double]
        L.om_logZ.restype = C.c_double
        L.om_logZ.argtypes = [C.c_double]
        L.om_kappa_qpn.restype = C.c_double
        L.om_kappa_qpn.argtypes = [C.c_double, C.c_double]
        L.om_pair_log.restype = C.c_double
        L.om_pair_log.argtypes = [C.c_double, D, C.c_double, D]
        L.om_rodrigues.argtypes = [D, D]
        L.om_angle.restype = C.c_double
        L.om_angle.argtypes = [D, D]
        L.om_objective.restype = C.c_double
        L.om_objective.argtypes = [C.POINTER(Mix), D, D]
        L.om_objective_r.restype = C.c_double
        L.om_objective_r.argtypes = [C.POINTER(Mix), D, D]
        L.om_objective_parts.argtypes = [C.POINTER(Mix), D, D, D, D]
        L.om_objective_grad.argtypes = [C.POINTER(Mix), D, D, D]
        L.om_c22.restype = C.c_double
        L.om_c22.argtypes = [C.POINTER(Mix)]
        L.om_psi_r.restype = C.c_double
        L.om_psi_r.argtypes = [C.c_double]
        L.om_psi_t.restype = C.c_double
        L.om_psi_t.argtypes = [D, D, D]
        L.om_kappa_interval.restype = C.c_int
        L.om_kappa_interval.argtypes = [D, C.c_double, D, D, C.c_double, D, D]
        L.om_self_lb_term.restype = C.c_double
        L.om_self_lb_term.argtypes = [C.POINTER(Mix), C.c_int, C.c_int, D, C.c_double]
        L.om_cross_ub_term.restype = C.c_double
        L.om_cross_ub_term.argtypes = [C.POINTER(Mix), C.c_int, C.c_int, D, C.c_double]
        L.om_bounds.argtypes = [C.POINTER(Mix), D, C.c_double, D]
        L.om_bounds_batch.argtypes = [C.POINTER(Mix), C.c_int, D, C.c_double, D, C.c_int]
        L.om_bounds_batch_mode.argtypes = [C.POINTER(Mix), C.c_int, D, C.c_double, C.c_int, D, C.c_int]
        L.om_psi_r_point.restype = C.c_double
        L.om_psi_r_point.argtypes = [D, C.c_double, D]
        L.om_max_threads.restype = C.c_int
        L.om_sma.restype = C.c_int
        L.om_sma.argtypes = [C.POINTER(Mix), C.POINTER(Domain), C.POINTER(SmaOpts), D, D, D]
        L.om_bnb.restype = C.c_int
        L.om_bnb.argtypes = [C.POINTER(Mix), C.POINTER(Domain), C.POINTER(BnbOpts), C.POINTER(BnbResult)]
        L.om_dp_cluster.restype = C.c_int
        L.om_dp_cluster.argtypes = [C.c_int, C.c_int, D, C.c_double, C.c_int, C.c_int, C.c_double, C.c_double, D, D, D,
                                    C.POINTER(C.c_int), C.POINTER(C.c_int)]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(D)


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


class Mixtures:
    """Holds the GMM (theta_1) and vMFMM (theta_2) arrays for the oracle."""

    def __init__(self, mu1, sigma1, phi1, mu2, kappa2, phi2):
        self.mu1 = _f64(mu1, (-1, 3))
        self.sigma1 = _f64(sigma1, (-1,))
        self.phi1 = _f64(phi1, (-1,))
        self.mu2 = _f64(mu2, (-1, 3))
        self.kappa2 = _f64(kappa2, (-1,))
        self.phi2 = _f64(phi2, (-1,))
        self.c = Mix(len(self.sigma1), _p(self.mu1), _p(self.sigma1), _p(self.phi1),
                     len(self.kappa2), _p(self.mu2), _p(self.kappa2), _p(self.phi2))

    @classmethod
    def from_problem(cls, prob):
        return cls(prob["mu1"], prob["sigma1"], prob["phi1"], prob["mu2"], prob["kappa2"], prob["phi2"])

    @property
    def ref(self):
        return C.byref(self.c)


def phiZ(x):
    return lib().om_phiZ(float(x))


def logZ(x):
    return lib().om_logZ(float(x))


def kappa_qpn(dist, sigma):
    return lib().om_kappa_qpn(float(dist), float(sigma))


def pair_log(ka, ua, kb, ub):
    ua = _f64(ua)
    ub = _f64(ub)
    return lib().om_pair_log(float(ka), _p(ua), float(kb), _p(ub))


def rodrigues(r):
    r = _f64(r)
    R = np.zeros(9)
    lib().om_rodrigues(_p(r), _p(R))
    return R.reshape(3, 3)


def angle(a, b):
    a = _f64(a)
    b = _f64(b)
    return lib().om_angle(_p(a), _p(b))


def objective(mix: Mixtures, R, t):
    R = _f64(R, (9,))
    t = _f64(t)
    return lib().om_objective(mix.ref, _p(R), _p(t))


def objective_r(mix: Mixtures, r, t):
    r = _f64(r)
    t = _f64(t)
    return lib().om_objective_r(mix.ref, _p(r), _p(t))


def objective_parts(mix: Mixtures, R, t):
    R = _f64(R, (9,))
    t = _f64(t)
    s = C.c_double()
    c = C.c_double()
    lib().om_objective_parts(mix.ref, _p(R), _p(t), C.byref(s), C.byref(c))
    return s.value, c.value


def objective_grad(mix: Mixtures, x):
    x = _f64(x)
    f = C.c_double()
    g = np.zeros(6)
    lib().om_objective_grad(mix.ref, _p(x), C.byref(f), _p(g))
    return f.value, g


def c22(mix: Mixtures):
    return lib().om_c22(mix.ref)


def psi_r(r_hw):
    return lib().om_psi_r(float(r_hw))


def psi_r_point(r0, r_hw, p):
    """Lemma 2, point-dependent form (reading R16): bound of the angle
    between R_r p and R_r0 p over the rotation cube (r0, r_hw)."""
    r0, p = _f64(r0), _f64(p)
    return lib().om_psi_r_point(_p(r0), float(r_hw), _p(p))


def psi_t(p, t0, thw):
    p, t0, thw = _f64(p), _f64(t0), _f64(thw)
    return lib().om_psi_t(_p(p), _p(t0), _p(thw))


def kappa_interval(p, sigma, t0, thw, zeta):
    p, t0, thw = _f64(p), _f64(t0), _f64(thw)
    a = C.c_double()
    b = C.c_double()
    ok = lib().om_kappa_interval(_p(p), float(sigma), _p(t0), _p(thw), float(zeta), C.byref(a), C.byref(b))
    return (a.value, b.value) if ok else None


def self_lb_term(mix, i, j, cube, zeta):
    cube = _f64(cube)
    return lib().om_self_lb_term(mix.ref, int(i), int(j), _p(cube), float(zeta))


def cross_ub_term(mix, i, j, cube, zeta):
    cube = _f64(cube)
    return lib().om_cross_ub_term(mix.ref, int(i), int(j), _p(cube), float(zeta))


BOUND_FIELDS = ("lb", "ub", "self_lb", "cross_ub", "self_c", "cross_c", "psi_r", "psi_t_max")


def bounds(mix: Mixtures, cubes, zeta, nthreads: int = 0, psi_mode: int = 0):
    """Theorem 1 bounds of each cube; returns an (n, 8) array of BOUND_FIELDS.
    psi_mode 1 takes the point-dependent psi_r (reading R16) in the cross
    pairs."""
    cubes = _f64(cubes, (-1, 10))
    out = np.zeros((cubes.shape[0], 8))
    if cubes.shape[0]:
        lib().om_bounds_batch_mode(mix.ref, cubes.shape[0], _p(cubes), float(zeta), int(psi_mode), _p(out),
                                   int(nthreads))
    return out


def max_threads():
    return lib().om_max_threads()


def _domain(t_lo, t_hi, zeta):
    d = Domain()
    for k in range(3):
        d.t_lo[k] = float(t_lo[k])
        d.t_hi[k] = float(t_hi[k])
    d.zeta = float(zeta)
    return d


def sma(mix: Mixtures, x0, t_lo, t_hi, zeta, max_iter=100, memory=10, gtol=1e-9):
    x0 = _f64(x0)
    x1 = np.zeros(6)
    f = C.c_double()
    dom = _domain(t_lo, t_hi, zeta)
    o = SmaOpts(max_iter, memory, gtol)
    evals = lib().om_sma(mix.ref, C.byref(dom), C.byref(o), _p(x0), _p(x1), C.byref(f))
    return x1, f.value, evals


def bnb(mix: Mixtures, t_lo, t_hi, zeta, eps, pop=128, max_nodes=0, max_seconds=0.0, use_sma=True,
        nthreads=0, sma_max_iter=100, psi_mode=0):
    """Algorithm 1.  Returns a dict with the certificate and the pose.
    psi_mode 1 bounds with the point-dependent psi_r (reading R16)."""
    dom = _domain(t_lo, t_hi, zeta)
    o = BnbOpts(float(eps), int(pop), int(max_nodes), float(max_seconds), int(bool(use_sma)), int(nthreads),
                SmaOpts(sma_max_iter, 10, 1e-9), int(psi_mode))
    res = BnbResult()
    lib().om_bnb(mix.ref, C.byref(dom), C.byref(o), C.byref(res))
    return {
        "f": res.f, "lb": res.lb, "f_norm": res.f_norm, "gap_norm": res.gap_norm, "c22": res.c22,
        "r": np.array(res.r[:]), "t": np.array(res.t[:]), "R": np.array(res.R[:]).reshape(3, 3),
        "nodes": res.nodes, "iterations": res.iterations, "sma_calls": res.sma_calls,
        "queue_peak": res.queue_peak, "seconds": res.seconds, "status": res.status,
    }


def dp_cluster(x, lam, vmf=False, max_iter=100, kmax=1024, sigma_min=1e-3, kappa_max=1e5):
    """Mixture generation (Sec. 6; mixgen.c): DP-means (vmf False, lam a
    squared-distance penalty) or DP-vMF-means (vmf True, lam a cosine
    threshold), then the maximum-likelihood GMM (sigma) or vMFMM (kappa).
    Returns dict(k, mu, sigma | kappa, phi, labels, passes); k = -1 when
    more than kmax clusters would be needed."""
    x = _f64(x, (-1, 3))
    n = len(x)
    mu = np.zeros((kmax, 3))
    spread = np.zeros(kmax)
    phi = np.zeros(kmax)
    labels = np.zeros(n, dtype=np.int32)
    passes = C.c_int()
    k = lib().om_dp_cluster(int(bool(vmf)), n, _p(x), float(lam), int(max_iter), int(kmax), float(sigma_min),
                            float(kappa_max), _p(mu), _p(spread), _p(phi),
                            labels.ctypes.data_as(C.POINTER(C.c_int)), C.byref(passes))
    out = {"k": k, "labels": labels, "passes": passes.value}
    if k > 0:
        out.update(mu=mu[:k], phi=phi[:k])
        out["kappa" if vmf else "sigma"] = spread[:k]
    return out
