"""Python binding of libgosma (include/gosma.h): argument marshalling only.

Every step of the branch-and-bound path runs in the CUDA library; this
module converts numpy arrays or torch tensors to pointers and sizes and
turns error codes into exceptions.  There is no fallback: if the library
is missing or no sm_103 device is present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgosma.so")

GOSMA_OK = 0
ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ETIMEOUT", -5: "ENOTREADY"}
STATUS = {0: "optimal", 1: "node_limit", 2: "time_limit", 3: "queue_full", 4: "running"}

D = C.POINTER(C.c_double)


class Cube(C.Structure):
    _fields_ = [("r0", C.c_double * 3), ("r_hw", C.c_double), ("t0", C.c_double * 3), ("t_hw", C.c_double * 3)]


class Bound(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("lb", "ub", "self_lb", "cross_ub", "self_c", "cross_c", "psi_r", "psi_t_max")]


class Opts(C.Structure):
    _fields_ = [("eps", C.c_double), ("pop", C.c_int), ("max_nodes", C.c_longlong), ("max_seconds", C.c_double),
                ("use_sma", C.c_int), ("sma_max_iter", C.c_int), ("queue_capacity", C.c_longlong),
                ("bound_block", C.c_int), ("bound_cubes", C.c_int)]


class Result(C.Structure):
    _fields_ = [("R", C.c_double * 9), ("r", C.c_double * 3), ("t", C.c_double * 3), ("objective", C.c_double),
                ("objective_norm", C.c_double), ("lower_bound", C.c_double), ("gap_norm", C.c_double),
                ("c22", C.c_double), ("nodes", C.c_longlong), ("iterations", C.c_longlong),
                ("sma_calls", C.c_longlong), ("queue_peak", C.c_longlong), ("seconds", C.c_double),
                ("status", C.c_int), ("cross_pairs", C.c_longlong), ("self_pairs", C.c_longlong),
                ("bound_ms", C.c_double), ("iteration_ms", C.c_double), ("queue_size", C.c_longlong),
                ("launches", C.c_longlong), ("block_size", C.c_int), ("cubes_per_block", C.c_int),
                ("tunings", C.c_int), ("dstar_iteration", C.c_longlong)]


class Problem(C.Structure):
    _fields_ = [("n1", C.c_int), ("mu1", D), ("sigma1", D), ("phi1", D), ("n2", C.c_int), ("mu2", D),
                ("kappa2", D), ("phi2", D), ("t_lo", C.c_double * 3), ("t_hi", C.c_double * 3), ("zeta", C.c_double),
                ("nclass", C.c_int), ("n1c", C.POINTER(C.c_int)), ("n2c", C.POINTER(C.c_int)), ("w", D)]


# exported symbols and their signatures (restype, argtypes); the header is the authority
FP = C.POINTER(C.c_float)


class LearnOpts(C.Structure):
    _fields_ = [("use_mlp", C.c_int), ("beta", C.c_float), ("seed", C.c_int), ("trace_cap", C.c_int),
                ("active_iters", C.c_int)]


# gosma_trace_point as a numpy record
HISTORY_DTYPE = np.dtype([("iteration", "<i8"), ("seconds", "<f8"), ("dstar", "<f8"), ("lower_bound", "<f8"),
                          ("queue_size", "<i8"), ("nodes", "<i8")])

# gosma_node as a numpy record
NODE_DTYPE = np.dtype([("lb", "<f8"), ("self_lb", "<f8"), ("self_c", "<f8"), ("r", "<u4", (3,)), ("t", "<u4", (3,)),
                       ("lr", "<u2"), ("lt", "<u2"), ("psit", "<f4"), ("flags", "<u4"), ("ubf", "<f4")])
assert NODE_DTYPE.itemsize == 64

# gosma_trace_rec as a numpy record
TRACE_DTYPE = np.dtype([("feat", "<f4", (16,)), ("cube", "<f8", (10,)), ("lb", "<f8"), ("ub", "<f8"),
                        ("dstar", "<f8"), ("problem", "<i4"), ("iteration", "<i4")])
assert TRACE_DTYPE.itemsize == 176

SIGNATURES = {
    "gosma_create": (C.c_int, [C.c_int, C.c_void_p, C.POINTER(C.c_void_p)]),
    "gosma_destroy": (None, [C.c_void_p]),
    "gosma_last_error": (C.c_char_p, [C.c_void_p]),
    "gosma_set_mixtures": (C.c_int, [C.c_void_p, C.c_int, D, D, D, C.c_int, D, D, D]),
    "gosma_set_mixtures_classes": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), D, D, D, D,
                                             D, D, D]),
    "gosma_set_domain": (C.c_int, [C.c_void_p, D, D, C.c_double]),
    "gosma_set_psi_r_mode": (C.c_int, [C.c_void_p, C.c_int]),
    "gosma_eval_bounds": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int]),
    "gosma_eval_bounds_detail": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_int]),
    "gosma_eval_objective": (C.c_int, [C.c_void_p, D, D, D]),
    "gosma_eval_objective_grad": (C.c_int, [C.c_void_p, C.c_int, D, D, D]),
    "gosma_eval_objective_grad_noalloc": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "gosma_dp_means": (C.c_int, [C.c_void_p, C.c_int, D, C.c_double, C.c_int, C.c_int, C.c_double,
                                 C.POINTER(C.c_int), D, D, D, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "gosma_dp_vmf_means": (C.c_int, [C.c_void_p, C.c_int, D, C.c_double, C.c_int, C.c_int, C.c_double,
                                     C.POINTER(C.c_int), D, D, D, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "gosma_sma_batch": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.c_void_p, C.c_int]),
    "gosma_bnb_solve": (C.c_int, [C.c_void_p, C.POINTER(Opts), C.POINTER(Result)]),
    "gosma_bnb_start": (C.c_int, [C.c_void_p, C.POINTER(Opts)]),
    "gosma_bnb_solve_batch": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.POINTER(Opts), C.c_void_p]),
    "gosma_bnb_solve_batch_ex": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.POINTER(Opts), C.c_void_p, C.c_void_p,
                                           C.c_void_p, C.c_void_p]),
    "gosma_bnb_step": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(Result)]),
    "gosma_bnb_history": (C.c_int, [C.c_void_p, C.c_longlong, C.c_void_p, C.POINTER(C.c_longlong)]),
    "gosma_bnb_last_children": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.POINTER(C.c_int)]),
    "gosma_bnb_export": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.POINTER(C.c_int)]),
    "gosma_bnb_import": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "gosma_bnb_set_incumbent": (C.c_int, [C.c_void_p, C.c_double, D]),
    "gosma_bnb_save": (C.c_int, [C.c_void_p, C.c_char_p]),
    "gosma_bnb_load": (C.c_int, [C.c_void_p, C.c_char_p]),
    "gosma_selftest_approx": (C.c_int, [C.c_void_p, D, D]),
    "gosma_selftest_wait_timeout": (C.c_int, [C.c_void_p, C.c_double]),
    "gosma_selftest_pipe_rates": (C.c_int, [C.c_void_p, D, D]),
    "gosma_selftest_rodrigues": (C.c_int, [C.c_void_p, C.c_int, D, D]),
    "gosma_debug_fail_allocations": (C.c_int, [C.c_void_p, C.c_int]),
    "gosma_kernel_launches": (C.c_longlong, [C.c_void_p]),
    "gosma_mlp_set_params": (C.c_int, [C.c_void_p, FP]),
    "gosma_mlp_get_params": (C.c_int, [C.c_void_p, FP]),
    "gosma_mlp_forward": (C.c_int, [C.c_void_p, C.c_int, FP, FP]),
    "gosma_mlp_grad": (C.c_int, [C.c_void_p, C.c_int, FP, FP, FP]),
    "gosma_mlp_train": (C.c_int, [C.c_void_p, C.c_int, FP, FP, FP, C.c_int, C.c_int, C.c_float, C.c_float, FP]),
}
MLP_NPARAM = 20752

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libgosma.so and declare its signatures.  Raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError("libgosma.so is not built (run __graft_entry__.build()); there is no fallback path")
        L = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class GosmaError(RuntimeError):
    pass


class GosmaArgumentError(GosmaError, ValueError):
    """An argument refused before the library is called: array lengths that
    disagree, or a device buffer of the wrong dtype, shape, layout or device."""


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    return a.reshape(shape) if shape is not None else a


def _p(a):
    return a.ctypes.data_as(D)


def _f32(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    return a.reshape(shape) if shape is not None else a


def _pf(a):
    return a.ctypes.data_as(FP)


def _is_torch_cuda(x):
    return type(x).__module__.startswith("torch") and getattr(x, "is_cuda", False)


_MIX_NAMES = ("mu1", "sigma1", "phi1", "mu2", "kappa2", "phi2")


def _mixture_arrays(mu1, sigma1, phi1, mu2, kappa2, phi2):
    """FP64 C-contiguous copies of one problem's mixtures.  The library takes
    n1 = len(sigma1) and n2 = len(kappa2) and reads n1 rows of mu1 and phi1
    and n2 rows of mu2 and phi2, so every length is checked against those."""
    a = [_f64(mu1, (-1, 3)), _f64(sigma1, (-1,)), _f64(phi1, (-1,)), _f64(mu2, (-1, 3)), _f64(kappa2, (-1,)),
         _f64(phi2, (-1,))]
    n1, n2 = len(a[1]), len(a[4])
    for name, arr, n in zip(_MIX_NAMES, a, (n1, n1, n1, n2, n2, n2)):
        if len(arr) != n:
            raise GosmaArgumentError("%s has %d rows, expected %d" % (name, len(arr), n))
    return a


def _class_arrays(n1c, n2c, w, n1, n2):
    """Class sizes (int32) and weights of a semantic problem; the sizes must
    add up to the mixtures' lengths, which the library does not see."""
    n1c = np.ascontiguousarray(np.asarray(n1c, dtype=np.int32).reshape(-1))
    n2c = np.ascontiguousarray(np.asarray(n2c, dtype=np.int32).reshape(-1))
    w = _f64(w, (-1,))
    if not len(n1c) == len(n2c) == len(w):
        raise GosmaArgumentError("n1c, n2c and w have %d, %d and %d entries" % (len(n1c), len(n2c), len(w)))
    if int(n1c.astype(np.int64).sum()) != n1 or int(n2c.astype(np.int64).sum()) != n2:
        raise GosmaArgumentError("class sizes add up to %d x %d components, the mixtures have %d x %d"
                         % (n1c.astype(np.int64).sum(), n2c.astype(np.int64).sum(), n1, n2))
    return n1c, n2c, w


def _dev(t, name, dtype, shape, device):
    """A device buffer handed to the library: a torch tensor of `dtype` and
    exactly `shape`, C-contiguous, on CUDA device `device`.  The library sees
    only the pointer, so a smaller or differently typed buffer would let a
    kernel run past it; such tensors are refused here."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise GosmaArgumentError("%s: expected a torch tensor, got %s" % (name, type(t).__name__))
    if t.dtype != dtype:
        raise GosmaArgumentError("%s: expected %s, got %s" % (name, dtype, t.dtype))
    if tuple(t.shape) != tuple(shape):
        raise GosmaArgumentError("%s: expected shape %s, got %s" % (name, tuple(shape), tuple(t.shape)))
    if not t.is_contiguous():
        raise GosmaArgumentError("%s: must be contiguous" % name)
    if not t.is_cuda or t.device.index != device:
        raise GosmaArgumentError("%s: must be a CUDA tensor on cuda:%d, got %s" % (name, device, t.device))
    return C.c_void_p(t.data_ptr())


class Gosma:
    """One libgosma context on one CUDA device and stream."""

    node_dtype = NODE_DTYPE  # queue records of bnb_export / bnb_import

    def __init__(self, device: int = 0, stream=None):
        self.L = load_library()
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream(device).cuda_stream
            except Exception:
                stream = None
        elif hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        self._stream = stream or 0
        h = C.c_void_p()
        rc = self.L.gosma_create(int(device), C.c_void_p(self._stream), C.byref(h))
        if rc != GOSMA_OK:
            raise GosmaError("gosma_create failed (%s): no usable sm_103 device" % ERRORS.get(rc, rc))
        self.h = h
        self.device = device
        self.n1 = self.n2 = 0

    def close(self):
        if getattr(self, "h", None):
            self.L.gosma_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, what):
        if rc != GOSMA_OK:
            msg = self.L.gosma_last_error(self.h)
            raise GosmaError("%s failed (%s): %s" % (what, ERRORS.get(rc, rc), msg.decode() if msg else ""))

    # ---------------------------------------------------------------- set-up
    def set_mixtures(self, mu1, sigma1, phi1, mu2, kappa2, phi2):
        mu1, sigma1, phi1, mu2, kappa2, phi2 = _mixture_arrays(mu1, sigma1, phi1, mu2, kappa2, phi2)
        self._check(self.L.gosma_set_mixtures(self.h, len(sigma1), _p(mu1), _p(sigma1), _p(phi1), len(kappa2),
                                              _p(mu2), _p(kappa2), _p(phi2)), "set_mixtures")
        self.n1, self.n2 = len(sigma1), len(kappa2)

    def set_domain(self, t_lo, t_hi, zeta):
        lo, hi = _f64(t_lo, (3,)), _f64(t_hi, (3,))
        self._check(self.L.gosma_set_domain(self.h, _p(lo), _p(hi), float(zeta)), "set_domain")

    def set_mixtures_classes(self, n1c, n2c, w, mu1, sigma1, phi1, mu2, kappa2, phi2):
        """Semantic form: per-class sizes n1c, n2c and weights w; arrays class by class."""
        mu1, sigma1, phi1, mu2, kappa2, phi2 = _mixture_arrays(mu1, sigma1, phi1, mu2, kappa2, phi2)
        n1c, n2c, w = _class_arrays(n1c, n2c, w, len(sigma1), len(kappa2))
        ip = C.POINTER(C.c_int)
        self._check(self.L.gosma_set_mixtures_classes(self.h, len(n1c), n1c.ctypes.data_as(ip), n2c.ctypes.data_as(ip),
                                                      _p(w), _p(mu1), _p(sigma1), _p(phi1), _p(mu2), _p(kappa2),
                                                      _p(phi2)), "set_mixtures_classes")
        self.n1, self.n2 = len(sigma1), len(kappa2)

    def set_problem(self, prob):
        """Mixtures and domain of a problem dict (synth); semantic problems
        (with "n1c", "n2c", "w") go through the class entry point."""
        if "n1c" in prob:
            self.set_mixtures_classes(prob["n1c"], prob["n2c"], prob["w"], prob["mu1"], prob["sigma1"], prob["phi1"],
                                      prob["mu2"], prob["kappa2"], prob["phi2"])
        else:
            self.set_mixtures(prob["mu1"], prob["sigma1"], prob["phi1"], prob["mu2"], prob["kappa2"], prob["phi2"])
        self.set_domain(prob["t_lo"], prob["t_hi"], prob["zeta"])

    def set_psi_r_mode(self, point: bool):
        """Rotation uncertainty of the bounds computed afterwards (Lemma 2):
        point=False the point-independent sqrt(3) h, True one angle per model
        direction (gosma_set_psi_r_mode)."""
        self._check(self.L.gosma_set_psi_r_mode(self.h, 1 if point else 0), "set_psi_r_mode")

    # ---------------------------------------------------------------- bounds
    def eval_bounds(self, cubes, lb=None, ub=None):
        """Theorem 1 bounds.  cubes: (n, 10) float64 numpy array (host path) or
        a CUDA torch tensor (device path, asynchronous on the context stream)."""
        if _is_torch_cuda(cubes):
            import torch
            n = cubes.shape[0]
            pc = _dev(cubes, "cubes", torch.float64, (n, 10), self.device)
            if lb is None:
                lb = torch.empty(n, dtype=torch.float64, device=cubes.device)
            if ub is None:
                ub = torch.empty(n, dtype=torch.float64, device=cubes.device)
            pl = _dev(lb, "lb", torch.float64, (n,), self.device)
            pu = _dev(ub, "ub", torch.float64, (n,), self.device)
            self._check(self.L.gosma_eval_bounds(self.h, pc, n, pl, pu, 1), "eval_bounds")
            return lb, ub
        cubes = _f64(cubes, (-1, 10))
        n = cubes.shape[0]
        lb = np.empty(n)
        ub = np.empty(n)
        self._check(self.L.gosma_eval_bounds(self.h, cubes.ctypes.data, n, lb.ctypes.data, ub.ctypes.data, 0),
                    "eval_bounds")
        return lb, ub

    def eval_bounds_detail(self, cubes, out=None):
        """Full per-cube records, (n, 8): lb, ub, self_lb, cross_ub, self_c, cross_c, psi_r, psi_t_max."""
        if _is_torch_cuda(cubes):
            import torch
            n = cubes.shape[0]
            pc = _dev(cubes, "cubes", torch.float64, (n, 10), self.device)
            if out is None:
                out = torch.empty((n, 8), dtype=torch.float64, device=cubes.device)
            po = _dev(out, "out", torch.float64, (n, 8), self.device)
            self._check(self.L.gosma_eval_bounds_detail(self.h, pc, n, po, 1), "eval_bounds_detail")
            return out
        cubes = _f64(cubes, (-1, 10))
        n = cubes.shape[0]
        out = np.empty((n, 8))
        self._check(self.L.gosma_eval_bounds_detail(self.h, cubes.ctypes.data, n, out.ctypes.data, 0),
                    "eval_bounds_detail")
        return out

    # ---------------------------------------------------------------- objective
    def eval_objective(self, r, t):
        r, t = _f64(r, (3,)), _f64(t, (3,))
        f = C.c_double()
        self._check(self.L.gosma_eval_objective(self.h, _p(r), _p(t), C.byref(f)), "eval_objective")
        return f.value

    def eval_objective_grad(self, x):
        x = _f64(x, (-1, 6))
        n = x.shape[0]
        f = np.empty(n)
        g = np.empty((n, 6))
        self._check(self.L.gosma_eval_objective_grad(self.h, n, _p(x), _p(f), _p(g)), "eval_objective_grad")
        return f, g

    def eval_objective_grad_noalloc(self, x_dev, out_dev):
        """Allocation-free f and gradient for callers that cannot let the
        library allocate: x_dev (count, 6) and out_dev (count, 7) are CUDA
        float64 tensors owned by the caller; asynchronous on the context stream."""
        import torch
        n = x_dev.shape[0]
        px = _dev(x_dev, "x_dev", torch.float64, (n, 6), self.device)
        po = _dev(out_dev, "out_dev", torch.float64, (n, 7), self.device)
        self._check(self.L.gosma_eval_objective_grad_noalloc(self.h, n, px, po), "eval_objective_grad_noalloc")
        return out_dev

    def _dp(self, fn, name, x, lam, max_iter, kmax, param, key):
        x = _f64(x, (-1, 3))
        n = len(x)
        mu, spread, phi = np.zeros((kmax, 3)), np.zeros(kmax), np.zeros(kmax)
        labels = np.zeros(n, dtype=np.int32)
        k, passes = C.c_int(), C.c_int()
        ip = C.POINTER(C.c_int)
        self._check(fn(self.h, n, _p(x), float(lam), int(max_iter), int(kmax), float(param), C.byref(k), _p(mu),
                       _p(spread), _p(phi), labels.ctypes.data_as(ip), C.byref(passes)), name)
        K = k.value
        return {"k": K, "mu": mu[:K], key: spread[:K], "phi": phi[:K], "labels": labels, "passes": passes.value}

    def dp_means(self, x, lam, max_iter=100, kmax=1024, sigma_min=1e-3):
        """Mixture generation (Sec. 6): DP-means of the (n, 3) points and the
        fitted GMM; returns dict(k, mu, sigma, phi, labels, passes)."""
        return self._dp(self.L.gosma_dp_means, "dp_means", x, lam, max_iter, kmax, sigma_min, "sigma")

    def dp_vmf_means(self, x, lam, max_iter=100, kmax=1024, kappa_max=1e5):
        """Mixture generation (Sec. 6): DP-vMF-means of the (n, 3) unit vectors
        and the fitted vMFMM; returns dict(k, mu, kappa, phi, labels, passes)."""
        return self._dp(self.L.gosma_dp_vmf_means, "dp_vmf_means", x, lam, max_iter, kmax, kappa_max, "kappa")

    def sma_batch(self, x0, max_iter=100, precision=32, x=None, f=None, grad=None, iters=None, with_grad=True):
        """SMA (Sec. 5) from many seed poses at once on the device.

        Host call: x0 is an (n, 6) array; returns dict(x, f, grad, iters) of
        numpy arrays (grad None unless with_grad).  Device call: x0 is a CUDA
        float64 tensor (n, 6) and x (n, 6), f (n,) and optionally grad (n, 6),
        iters (n,) int32 are CUDA tensors filled asynchronously on the context
        stream; returns them."""
        if _is_torch_cuda(x0):
            import torch
            n = x0.shape[0]
            p0 = _dev(x0, "x0", torch.float64, (n, 6), self.device)
            px = _dev(x, "x", torch.float64, (n, 6), self.device)
            pf = _dev(f, "f", torch.float64, (n,), self.device)
            pg = _dev(grad, "grad", torch.float64, (n, 6), self.device) if grad is not None else None
            pi = _dev(iters, "iters", torch.int32, (n,), self.device) if iters is not None else None
            self._check(self.L.gosma_sma_batch(self.h, n, p0, int(max_iter), int(precision), px, pf, pg, pi, 1),
                        "sma_batch")
            return dict(x=x, f=f, grad=grad, iters=iters)
        x0 = _f64(x0, (-1, 6))
        n = x0.shape[0]
        xo, fo, it = np.empty((n, 6)), np.empty(n), np.empty(n, dtype=np.int32)
        go = np.empty((n, 6)) if with_grad else None
        self._check(self.L.gosma_sma_batch(self.h, n, x0.ctypes.data, int(max_iter), int(precision), xo.ctypes.data,
                                           fo.ctypes.data, go.ctypes.data if with_grad else None, it.ctypes.data, 0),
                    "sma_batch")
        return dict(x=xo, f=fo, grad=go, iters=it)

    # ---------------------------------------------------------------- branch-and-bound
    @staticmethod
    def _opts(eps, pop, max_nodes, max_seconds, use_sma, sma_max_iter, queue_capacity, shape=None):
        b, g = shape if shape is not None else (0, 0)
        return Opts(float(eps), int(pop), int(max_nodes), float(max_seconds), int(bool(use_sma)), int(sma_max_iter),
                    int(queue_capacity), int(b), int(g))

    @staticmethod
    def _result(r):
        return {
            "f": r.objective, "f_norm": r.objective_norm, "lb": r.lower_bound, "gap_norm": r.gap_norm,
            "c22": r.c22, "R": np.array(r.R[:]).reshape(3, 3), "r": np.array(r.r[:]), "t": np.array(r.t[:]),
            "nodes": r.nodes, "iterations": r.iterations, "sma_calls": r.sma_calls, "queue_peak": r.queue_peak,
            "seconds": r.seconds, "status": r.status, "status_name": STATUS.get(r.status, str(r.status)),
            "cross_pairs": r.cross_pairs, "self_pairs": r.self_pairs, "bound_ms": r.bound_ms,
            "iteration_ms": r.iteration_ms, "queue_size": r.queue_size, "launches": r.launches,
            "block_size": r.block_size, "cubes_per_block": r.cubes_per_block, "tunings": r.tunings,
            "dstar_iteration": r.dstar_iteration,
        }

    def bnb_solve(self, eps=0.1, pop=0, max_nodes=0, max_seconds=0.0, use_sma=True, sma_max_iter=100,
                  queue_capacity=0):
        """Algorithm 1 to termination; returns the certificate and the pose."""
        o = self._opts(eps, pop, max_nodes, max_seconds, use_sma, sma_max_iter, queue_capacity)
        r = Result()
        self._check(self.L.gosma_bnb_solve(self.h, C.byref(o), C.byref(r)), "bnb_solve")
        return self._result(r)

    def bnb_solve_batch(self, problems, eps=0.1, pop=0, max_nodes=0, max_seconds=0.0, use_sma=True,
                        sma_max_iter=100, queue_capacity=0, learned=None, trace_cap=0, shape=None):
        """Algorithm 1 for many independent problems at once (list of problem
        dicts as produced by synth); returns one result dict per problem.

        ``shape``: None (the autotuner picks the bound kernel's shape) or
        (threads per block, sub-cubes per block).

        ``learned``: None (plain) or a dict with ``beta``, ``seed`` and
        ``active_iters`` for the network-ordered form (parameters loaded with
        mlp_set_params).  With
        ``trace_cap > 0`` returns ``(results, traces)``, traces a list of
        TRACE_DTYPE arrays, one per problem, in pop order."""
        if not problems:
            return ([], []) if trace_cap > 0 else []
        keep = []
        arr = (Problem * len(problems))()
        for k, pr in enumerate(problems):
            a = _mixture_arrays(*(pr[k] for k in _MIX_NAMES))
            keep.append(a)
            p = arr[k]
            p.n1, p.mu1, p.sigma1, p.phi1 = len(a[1]), _p(a[0]), _p(a[1]), _p(a[2])
            p.n2, p.mu2, p.kappa2, p.phi2 = len(a[4]), _p(a[3]), _p(a[4]), _p(a[5])
            for q in range(3):
                p.t_lo[q] = float(pr["t_lo"][q])
                p.t_hi[q] = float(pr["t_hi"][q])
            p.zeta = float(pr["zeta"])
            if "n1c" in pr:  # semantic problem
                c = _class_arrays(pr["n1c"], pr["n2c"], pr["w"], len(a[1]), len(a[4]))
                keep.append(c)
                ip = C.POINTER(C.c_int)
                p.nclass, p.n1c, p.n2c, p.w = len(c[0]), c[0].ctypes.data_as(ip), c[1].ctypes.data_as(ip), _p(c[2])
        o = self._opts(eps, pop, max_nodes, max_seconds, use_sma, sma_max_iter, queue_capacity, shape)
        res = (Result * len(problems))()
        lo = LearnOpts(0, 0.0, 0, int(trace_cap), 0)
        if learned is not None:
            lo.use_mlp, lo.beta, lo.seed = 1, float(learned.get("beta", 0.0)), int(bool(learned.get("seed", True)))
            lo.active_iters = int(learned.get("active_iters", 0))
        tr = np.zeros(max(1, len(problems) * int(trace_cap)), dtype=TRACE_DTYPE)
        cnt = np.zeros(len(problems), dtype=np.int32)
        self._check(self.L.gosma_bnb_solve_batch_ex(self.h, len(problems), C.cast(arr, C.c_void_p), C.byref(o),
                                                    C.byref(lo), C.cast(res, C.c_void_p),
                                                    tr.ctypes.data_as(C.c_void_p), cnt.ctypes.data_as(C.c_void_p)),
                    "bnb_solve_batch")
        out = [self._result(r) for r in res]
        if trace_cap > 0:
            tr = tr.reshape(len(problems), trace_cap)
            return out, [tr[k, :cnt[k]].copy() for k in range(len(problems))]
        return out

    def bnb_start(self, eps=0.1, pop=0, max_nodes=0, max_seconds=0.0, use_sma=True, sma_max_iter=100,
                  queue_capacity=0):
        o = self._opts(eps, pop, max_nodes, max_seconds, use_sma, sma_max_iter, queue_capacity)
        self._check(self.L.gosma_bnb_start(self.h, C.byref(o)), "bnb_start")

    def bnb_step(self, max_iters=1):
        r = Result()
        self._check(self.L.gosma_bnb_step(self.h, int(max_iters), C.byref(r)), "bnb_step")
        return self._result(r)

    # ---- queue-ordering network
    def mlp_set_params(self, params):
        p = _f32(params, (MLP_NPARAM,))
        self._check(self.L.gosma_mlp_set_params(self.h, _pf(p)), "mlp_set_params")

    def mlp_get_params(self):
        p = np.zeros(MLP_NPARAM, dtype=np.float32)
        self._check(self.L.gosma_mlp_get_params(self.h, _pf(p)), "mlp_get_params")
        return p

    def mlp_forward(self, x):
        x = _f32(x, (-1, 16))
        y = np.zeros((len(x), 16), dtype=np.float32)
        self._check(self.L.gosma_mlp_forward(self.h, len(x), _pf(x), _pf(y)), "mlp_forward")
        return y

    def mlp_grad(self, x, dy):
        x = _f32(x, (-1, 16))
        dy = _f32(dy, (len(x), 16))
        g = np.zeros(MLP_NPARAM, dtype=np.float32)
        self._check(self.L.gosma_mlp_grad(self.h, len(x), _pf(x), _pf(dy), _pf(g)), "mlp_grad")
        return g

    def mlp_train(self, x, label, target, batch, steps, lr=1e-3, lam=1.0):
        x = _f32(x, (-1, 16))
        label = _f32(label, (len(x),))
        target = _f32(target, (len(x), 6))
        losses = np.zeros(max(steps, 1), dtype=np.float32)
        self._check(self.L.gosma_mlp_train(self.h, len(x), _pf(x), _pf(label), _pf(target), int(batch), int(steps),
                                           float(lr), float(lam), _pf(losses)), "mlp_train")
        return losses[:steps]

    def bnb_set_incumbent(self, f, x):
        """Offer (f, x) as an incumbent to the run in progress; d* becomes f if smaller."""
        x = _f64(x, (6,))
        self._check(self.L.gosma_bnb_set_incumbent(self.h, float(f), _p(x)), "bnb_set_incumbent")

    def bnb_history(self):
        """Per-iteration (iteration, seconds, dstar, lower_bound, queue_size, nodes) of the run (Fig. 5)."""
        n = C.c_longlong(0)
        self._check(self.L.gosma_bnb_history(self.h, 0, None, C.byref(n)), "bnb_history")
        out = np.zeros(n.value, dtype=HISTORY_DTYPE)
        if n.value:
            self._check(self.L.gosma_bnb_history(self.h, n.value, out.ctypes.data_as(C.c_void_p), C.byref(n)),
                        "bnb_history")
        return out

    def bnb_last_children(self):
        """The children bounded by the last iteration: (cubes (n, 10), records
        (n, 8) as in eval_bounds_detail)."""
        n = C.c_int(0)
        self._check(self.L.gosma_bnb_last_children(self.h, 0, None, None, C.byref(n)), "bnb_last_children")
        cubes = np.zeros((n.value, 10))
        rec = np.zeros((n.value, 8))
        if n.value:
            self._check(self.L.gosma_bnb_last_children(self.h, n.value, cubes.ctypes.data, rec.ctypes.data,
                                                       C.byref(n)),
                        "bnb_last_children")
        return cubes, rec

    def bnb_export(self, max_nodes):
        """Remove up to max_nodes live sub-cubes from the run; returns them as a
        NODE_DTYPE array (gosma_bnb_export)."""
        out = np.zeros(max(0, int(max_nodes)), dtype=NODE_DTYPE)
        n = C.c_int(0)
        self._check(self.L.gosma_bnb_export(self.h, int(max_nodes), out.ctypes.data, C.byref(n)), "bnb_export")
        return out[:n.value].copy()

    def bnb_import(self, nodes):
        """Append queue records (a NODE_DTYPE array) to the run (gosma_bnb_import)."""
        nodes = np.ascontiguousarray(nodes, dtype=NODE_DTYPE)
        self._check(self.L.gosma_bnb_import(self.h, len(nodes), nodes.ctypes.data), "bnb_import")

    def bnb_save(self, path):
        self._check(self.L.gosma_bnb_save(self.h, os.fsencode(path)), "bnb_save")

    def bnb_load(self, path):
        self._check(self.L.gosma_bnb_load(self.h, os.fsencode(path)), "bnb_load")

    def kernel_launches(self):
        return int(self.L.gosma_kernel_launches(self.h))

    def selftest_pipe_rates(self):
        """Measured lane operations per SM per clock: dict(ffma, ffma2, ex2, sqrt, rcp, rsqrt, lg2, clock_mhz)."""
        r = np.zeros(7)
        mhz = C.c_double()
        self._check(self.L.gosma_selftest_pipe_rates(self.h, _p(r), C.byref(mhz)), "selftest_pipe_rates")
        return dict(zip(("ffma", "ffma2", "ex2", "sqrt", "rcp", "rsqrt", "lg2"), r.tolist()), clock_mhz=mhz.value)

    def selftest_rodrigues(self, r):
        """The pre-pass's rotation matrices (double-float, summed in FP64) for rotation vectors r (n x 3)."""
        r = _f64(r, (-1, 3))
        R = np.zeros((len(r), 3, 3))
        self._check(self.L.gosma_selftest_rodrigues(self.h, len(r), _p(r), _p(R)), "selftest_rodrigues")
        return R

    def selftest_wait_timeout(self, limit_seconds=0.05):
        """Returns the library's return code (GOSMA_ETIMEOUT when the bounded wait gave up)."""
        return int(self.L.gosma_selftest_wait_timeout(self.h, float(limit_seconds)))

    def debug_fail_allocations(self, n):
        self._check(self.L.gosma_debug_fail_allocations(self.h, int(n)), "debug_fail_allocations")

    def selftest_approx(self):
        m = np.zeros(5)
        a = np.zeros(5)
        self._check(self.L.gosma_selftest_approx(self.h, _p(m), _p(a)), "selftest_approx")
        return m, a
