"""Tensor-core (tcgen05) MLP kernels against the FP64 reference.

The reference rounds the weights, the inputs, both hidden activations and
the backward operands to BF16 exactly where the device does, so the two
differ by FP32 summation order and by the odd BF16 rounding flip that order
causes.  Tolerances: outputs within 2e-3 of the output scale; each gradient
block within 1e-2 of its norm.
"""
import numpy as np
import pytest

from oracle import mlp_oracle as M

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1812_01232_gb300 import build
    build.build()
    from paper_1812_01232_gb300.gosma import Gosma
    c = Gosma(0)
    yield c
    c.close()


def _data(seed, n):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, M.F_IN)).astype(np.float32)


@pytest.mark.parametrize("n", [1, 128, 1000, 4096])
def test_forward_parity(ctx, n):
    p = M.init_params(11)
    p["b1"] = np.random.default_rng(1).standard_normal(M.HID).astype(np.float32) * 0.1
    p["b3"][:7] = 0.25
    ctx.mlp_set_params(M.pack(p).astype(np.float32))
    x = _data(12, n)
    y = ctx.mlp_forward(x)
    ref, _ = M.forward(p, x, bf16=True)
    scale = np.abs(ref).max() + 1.0
    err = np.abs(y - ref).max() / scale
    assert err <= 2e-3, err
    # the padded outputs carry only their bias
    assert np.allclose(y[:, 7:], p["b3"][7:], atol=1e-6)


def test_gradient_parity(ctx):
    p = M.init_params(13)
    ctx.mlp_set_params(M.pack(p).astype(np.float32))
    x = _data(14, 700)
    dy = np.random.default_rng(15).standard_normal((700, M.F_OUT)).astype(np.float32) / 700
    g = M.unpack(ctx.mlp_grad(x, dy))
    _, cache = M.forward(p, x, bf16=True)
    ref = M.backward(cache, dy, bf16=True)
    for k in ref:
        e = np.linalg.norm(g[k] - ref[k]) / (np.linalg.norm(ref[k]) + 1e-30)
        assert e <= 1e-2, (k, e)


def test_training_reduces_loss(ctx):
    """A separable labelling (sign of a fixed linear form) and a linear seed
    target: the loss falls by more than half within 300 Adam steps."""
    rng = np.random.default_rng(16)
    n = 8192
    x = rng.standard_normal((n, M.F_IN)).astype(np.float32)
    w = rng.standard_normal(M.F_IN)
    label = (x @ w > 0).astype(np.float32)
    target = (x[:, :6] * 0.5).astype(np.float32)
    ctx.mlp_set_params(M.pack(M.init_params(17)).astype(np.float32))
    losses = ctx.mlp_train(x, label, target, batch=1024, steps=300, lr=2e-3, lam=1.0)
    assert np.all(np.isfinite(losses))
    assert losses[-8:].mean() < 0.5 * losses[:8].mean()
    # the trained network separates the classes on fresh data
    xt = rng.standard_normal((2048, M.F_IN)).astype(np.float32)
    yt = ctx.mlp_forward(xt)
    acc = ((yt[:, 0] > 0) == (xt @ w > 0)).mean()
    assert acc > 0.9, acc
    # the master parameters changed and remain finite
    q = ctx.mlp_get_params()
    assert np.all(np.isfinite(q)) and not np.allclose(q, M.pack(M.init_params(17)))
