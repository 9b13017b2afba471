"""FP64 reference of the queue-ordering network (an extension, not in the paper).

TEST INFRASTRUCTURE ONLY: tests, ``__graft_entry__.smoke()`` and the CPU
baseline of ``bench.py`` call it; the product package never imports it.

The network scores a sub-cube and proposes a seed pose for local refinement
(SMA, Sec. 5):

    h1 = GELU(W1 x + b1)      x: 16 cube features
    h2 = GELU(W2 h1 + b2)     128 hidden units each
    y  = W3 h2 + b3           y[0]: priority logit, y[1:7]: seed offset

GELU(z) = z * Phi(z) with Phi the standard normal CDF (the exact form, not the
tanh approximation).  The device keeps weights and activations in BF16 and
accumulates in FP32; ``bf16=True`` rounds the weights, the input and both
hidden activations to BF16 (round to nearest even) exactly where the device
does, so that the two agree up to FP32 summation order.

Training loss per row (mean over rows):
    BCE(y[0], label) + lam * label * sum_k (y[1+k] - target[k])^2
with BCE the logistic loss on the logit.
"""
from __future__ import annotations

import math

import numpy as np

F_IN, HID, F_OUT = 16, 128, 16
N_SEED = 6
SQRT2 = math.sqrt(2.0)


def bf16_round(a):
    """Round float32 values to the nearest BF16 (ties to even), as float64."""
    a32 = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = a32.view(np.uint32).astype(np.uint64)
    bias = 0x7FFF + ((u >> 16) & 1)
    r = ((u + bias) & 0xFFFF0000).astype(np.uint32)
    nan = np.isnan(a32)
    out = r.view(np.float32).astype(np.float64)
    out[nan] = np.nan
    return out


_erf = np.vectorize(math.erf, otypes=[np.float64])


def gelu(z):
    return 0.5 * z * (1.0 + _erf(z / SQRT2))


def gelu_grad(z):
    """d GELU / dz = Phi(z) + z phi(z)."""
    return 0.5 * (1.0 + _erf(z / SQRT2)) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def init_params(seed: int):
    """He-style initialisation (FP32 master copy): dict of W1 b1 W2 b2 W3 b3."""
    rng = np.random.default_rng(seed)
    p = {
        "W1": rng.standard_normal((HID, F_IN)) * math.sqrt(2.0 / F_IN),
        "b1": np.zeros(HID),
        "W2": rng.standard_normal((HID, HID)) * math.sqrt(2.0 / HID),
        "b2": np.zeros(HID),
        "W3": rng.standard_normal((F_OUT, HID)) * math.sqrt(1.0 / HID),
        "b3": np.zeros(F_OUT),
    }
    p["W3"][1 + N_SEED:] = 0.0
    return {k: v.astype(np.float32).astype(np.float64) for k, v in p.items()}


def forward(p, x, bf16=False):
    """Returns (y, cache) for inputs x (n x 16)."""
    x = np.asarray(x, dtype=np.float64)
    rd = bf16_round if bf16 else (lambda a: a)
    W1, W2, W3 = rd(p["W1"]), rd(p["W2"]), rd(p["W3"])
    x0 = rd(x)
    z1 = x0 @ W1.T + p["b1"]
    h1 = rd(gelu(z1))
    z2 = h1 @ W2.T + p["b2"]
    h2 = rd(gelu(z2))
    y = h2 @ W3.T + p["b3"]
    return y, dict(x0=x0, z1=z1, h1=h1, z2=z2, h2=h2, W1=W1, W2=W2, W3=W3)


def backward(cache, dy, bf16=False):
    """Parameter gradients for an upstream gradient dy (n x 16) of the outputs.
    ``bf16=True`` rounds dy and the two pre-activation gradients to BF16
    where the device stores them as tensor-core operands."""
    rd = bf16_round if bf16 else (lambda a: a)
    dy = rd(np.asarray(dy, dtype=np.float64))
    g = {"W3": dy.T @ cache["h2"], "b3": dy.sum(0)}
    dz2 = rd((dy @ cache["W3"]) * gelu_grad(cache["z2"]))
    g["W2"] = dz2.T @ cache["h1"]
    g["b2"] = dz2.sum(0)
    dz1 = rd((dz2 @ cache["W2"]) * gelu_grad(cache["z1"]))
    g["W1"] = dz1.T @ cache["x0"]
    g["b1"] = dz1.sum(0)
    return g


def pack(p):
    """Packed FP32 parameter vector: W1, b1, W2, b2, W3, b3 (row-major)."""
    return np.concatenate([np.asarray(p[k], dtype=np.float64).ravel() for k in ("W1", "b1", "W2", "b2", "W3", "b3")])


def unpack(v):
    v = np.asarray(v, dtype=np.float64)
    shapes = (("W1", (HID, F_IN)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)), ("W3", (F_OUT, HID)),
              ("b3", (F_OUT,)))
    out, o = {}, 0
    for k, sh in shapes:
        n = int(np.prod(sh))
        out[k] = v[o:o + n].reshape(sh)
        o += n
    return out


def loss_and_dy(y, label, target, lam=1.0):
    """Mean loss over rows and its gradient with respect to y."""
    n = y.shape[0]
    s = y[:, 0]
    # logistic loss, written stably: log(1 + e^s) - label * s
    bce = np.logaddexp(0.0, s) - label * s
    r = y[:, 1:1 + N_SEED] - target
    loss = (bce + lam * label * (r * r).sum(1)).mean()
    dy = np.zeros_like(y)
    dy[:, 0] = (1.0 / (1.0 + np.exp(-s)) - label) / n
    dy[:, 1:1 + N_SEED] = 2.0 * lam * label[:, None] * r / n
    return loss, dy
