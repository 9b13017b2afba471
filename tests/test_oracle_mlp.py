"""Pins of the FP64 reference of the queue-ordering network.

The reference is checked against things other than itself: BF16 rounding
against hand-computed ties and torch's bfloat16 conversion, GELU against the
normal CDF at known points and its limits, the derivatives against central
differences, and the whole forward/backward against torch autograd in FP64.
"""
import math

import numpy as np
import pytest

from oracle import mlp_oracle as M


def test_bf16_rounding_pins():
    one = 1.0
    u = 2.0 ** -7  # BF16 spacing at 1
    vals = np.array([one, one + u / 2, one + 1.5 * u, -(one + 1.5 * u), 3.0, 1e-3, 65504.0])
    # ties go to the even mantissa: 1 + u/2 -> 1, 1 + 1.5u -> 1 + 2u
    want = np.array([one, one, one + 2 * u, -(one + 2 * u), 3.0])
    got = M.bf16_round(vals)
    assert np.array_equal(got[:5], want)
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(0).standard_normal(10000).astype(np.float32) * 10.0 ** np.random.default_rng(1).integers(-5, 5, 10000)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(M.bf16_round(x), ref)


def test_gelu_pins():
    assert M.gelu(np.array([0.0]))[0] == 0.0
    # GELU(1) = Phi(1), GELU(-1) = -(1 - Phi(1))
    phi1 = 0.8413447460685429
    assert M.gelu(np.array([1.0]))[0] == pytest.approx(phi1, rel=1e-15)
    assert M.gelu(np.array([-1.0]))[0] == pytest.approx(-(1 - phi1), rel=1e-14)
    assert M.gelu(np.array([40.0]))[0] == 40.0 and M.gelu(np.array([-40.0]))[0] == pytest.approx(0.0, abs=1e-300)
    assert M.gelu_grad(np.array([0.0]))[0] == 0.5
    z = np.linspace(-6, 6, 241)
    h = 1e-6
    fd = (M.gelu(z + h) - M.gelu(z - h)) / (2 * h)
    assert np.allclose(M.gelu_grad(z), fd, atol=1e-8)


def test_forward_backward_match_autograd():
    torch = pytest.importorskip("torch")
    p = M.init_params(3)
    rng = np.random.default_rng(4)
    x = rng.standard_normal((37, M.F_IN))
    dy = rng.standard_normal((37, M.F_OUT))
    y, cache = M.forward(p, x)
    g = M.backward(cache, dy)
    tp = {k: torch.tensor(v, dtype=torch.float64, requires_grad=True) for k, v in p.items()}
    tx = torch.tensor(x)
    h1 = torch.nn.functional.gelu(tx @ tp["W1"].T + tp["b1"])
    h2 = torch.nn.functional.gelu(h1 @ tp["W2"].T + tp["b2"])
    ty = h2 @ tp["W3"].T + tp["b3"]
    assert np.allclose(y, ty.detach().numpy(), rtol=1e-12, atol=1e-12)
    (ty * torch.tensor(dy)).sum().backward()
    for k in p:
        assert np.allclose(g[k], tp[k].grad.numpy(), rtol=1e-10, atol=1e-12), k


def test_loss_gradient_finite_differences():
    p = M.init_params(5)
    rng = np.random.default_rng(6)
    x = rng.standard_normal((9, M.F_IN))
    label = (rng.random(9) < 0.5).astype(float)
    target = rng.standard_normal((9, M.N_SEED))
    y, cache = M.forward(p, x)
    loss, dy = M.loss_and_dy(y, label, target, lam=0.7)
    g = M.backward(cache, dy)
    v = M.pack(p)
    gv = M.pack(g)
    h = 1e-6
    for idx in rng.choice(len(v), 40, replace=False):
        vp, vm = v.copy(), v.copy()
        vp[idx] += h
        vm[idx] -= h
        lp = M.loss_and_dy(M.forward(M.unpack(vp), x)[0], label, target, 0.7)[0]
        lm = M.loss_and_dy(M.forward(M.unpack(vm), x)[0], label, target, 0.7)[0]
        assert gv[idx] == pytest.approx((lp - lm) / (2 * h), rel=1e-5, abs=1e-9)
    # the logistic loss of a zero logit is log 2 for either label
    y0 = np.zeros((2, M.F_OUT))
    l0, _ = M.loss_and_dy(y0, np.array([0.0, 1.0]), np.zeros((2, M.N_SEED)))
    assert l0 == pytest.approx(math.log(2.0), rel=1e-15)


def test_pack_roundtrip_and_size():
    p = M.init_params(7)
    v = M.pack(p)
    assert v.size == 20752
    q = M.unpack(v)
    for k in p:
        assert np.array_equal(p[k], q[k])
