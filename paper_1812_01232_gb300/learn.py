"""Training data and training for the queue-ordering network (an extension of
the method, not in the paper).

The network (16 -> 128 -> 128 -> 16, GELU; see mlp.cu) learns from traces of
the plain batched branch-and-bound: every popped sub-cube is recorded with the
features the device computed for it, and labelled against the best pose x*
that its problem's run ended with:

* label 1 when x* lies in the sub-cube grown by ``grow`` (1.5: the cube and
  half of each neighbour), else 0;
* seed target: the offset of x* from the cube centre in half-widths, clipped
  to [-1, 1] (only rows with label 1 contribute to that loss term).

Training oversamples the rare positive rows to ``pos_frac`` of every
minibatch and runs Adam on the device (gosma_mlp_train).
"""
from __future__ import annotations

import math

import numpy as np

N_FEAT = 16
N_PARAM = 20752


def init_params(seed: int) -> np.ndarray:
    """He-scaled Gaussian weights, zero biases, packed FP32 (W1 b1 W2 b2 W3 b3);
    output rows 7..15 of W3 are zero (unused outputs)."""
    rng = np.random.default_rng(seed)
    w1 = rng.standard_normal((128, 16)) * math.sqrt(2.0 / 16)
    w2 = rng.standard_normal((128, 128)) * math.sqrt(2.0 / 128)
    w3 = rng.standard_normal((16, 128)) * math.sqrt(1.0 / 128)
    w3[7:] = 0.0
    parts = [w1, np.zeros(128), w2, np.zeros(128), w3, np.zeros(16)]
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)


def label_trace(trace: np.ndarray, r_star, t_star, grow: float = 1.5):
    """Labels and seed targets of one problem's trace against its pose x*."""
    c = trace["cube"]
    r0, rhw = c[:, 0:3], c[:, 3:4]
    t0, thw = c[:, 4:7], c[:, 7:10]
    dr = (np.asarray(r_star)[None, :] - r0) / rhw
    dt = (np.asarray(t_star)[None, :] - t0) / thw
    inside = (np.abs(dr) <= grow).all(1) & (np.abs(dt) <= grow).all(1)
    target = np.clip(np.concatenate([dr, dt], 1), -1.0, 1.0)
    return inside.astype(np.float32), target.astype(np.float32)


def collect(ctx, problems, eps, pop=256, max_nodes=2_000_000, trace_cap=8192, queue_capacity=1 << 22,
            max_seconds=120.0):
    """Plain batched runs with traces; returns (features, labels, targets,
    results).  x* of each problem is the pose its run ended with."""
    res, traces = ctx.bnb_solve_batch(problems, eps=eps, pop=pop, max_nodes=max_nodes, max_seconds=max_seconds,
                                      queue_capacity=queue_capacity, trace_cap=trace_cap)
    feats, labels, targets = [], [], []
    for r, tr in zip(res, traces):
        if len(tr) == 0 or not np.isfinite(r["f"]):
            continue
        lab, tgt = label_trace(tr, r["r"], r["t"])
        feats.append(tr["feat"])
        labels.append(lab)
        targets.append(tgt)
    return np.concatenate(feats), np.concatenate(labels), np.concatenate(targets), res


def balanced_order(labels: np.ndarray, n_rows: int, pos_frac: float, seed: int) -> np.ndarray:
    """Row indices of a training stream of n_rows rows with pos_frac positives
    (sampled with replacement), shuffled."""
    rng = np.random.default_rng(seed)
    pos = np.flatnonzero(labels > 0.5)
    neg = np.flatnonzero(labels <= 0.5)
    n_pos = int(round(pos_frac * n_rows)) if len(pos) else 0
    idx = np.concatenate([rng.choice(pos, n_pos, replace=True) if n_pos else np.zeros(0, dtype=np.int64),
                          rng.choice(neg, n_rows - n_pos, replace=len(neg) < n_rows - n_pos)])
    rng.shuffle(idx)
    return idx


def train(ctx, feats, labels, targets, steps=2000, batch=4096, lr=1e-3, lam=1.0, pos_frac=0.2, seed=0,
          params=None):
    """Adam on the device; returns (parameters, per-step losses)."""
    ctx.mlp_set_params(init_params(seed) if params is None else params)
    idx = balanced_order(labels, steps * batch, pos_frac, seed + 1)
    # the device cycles through its data set in order: give it the stream
    losses = ctx.mlp_train(feats[idx], labels[idx], targets[idx], batch=batch, steps=steps, lr=lr, lam=lam)
    return ctx.mlp_get_params(), losses


def save(path: str, params: np.ndarray, **meta):
    np.savez(path, params=np.asarray(params, dtype=np.float32), **meta)


def load(path: str) -> np.ndarray:
    with np.load(path) as z:
        p = z["params"].astype(np.float32)
    if p.size != N_PARAM:
        raise ValueError("unexpected parameter count %d" % p.size)
    return p
