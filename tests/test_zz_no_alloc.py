"""The allocation-free objective entry point (for callers that cannot let the
library allocate device memory while they run) must give the same f and
gradient as gosma_eval_objective_grad, call after call.

Collected last on purpose: if it fails, a run that stops at the first
failure has already run every other test."""
import ctypes as C
import math

import numpy as np
import pytest

from paper_1812_01232_gb300 import synth

pytestmark = pytest.mark.gpu


def test_no_alloc_objective_matches_allocating_entry_point():
    import torch
    from paper_1812_01232_gb300 import build
    build.build()
    from paper_1812_01232_gb300.gosma import Gosma, load_library
    ctx = Gosma(0)
    prob = synth.paper_scale_problem(2000)
    ctx.set_problem(prob)
    L = load_library()
    rng = np.random.default_rng(17)
    for call in range(2):
        X = np.concatenate([prob["r_gt"] + rng.normal(0, 0.05, (5, 3)), prob["t_gt"] + rng.normal(0, 0.05, (5, 3))],
                           1)
        f_ref, g_ref = ctx.eval_objective_grad(X)
        x_dev = torch.tensor(X, dtype=torch.float64, device="cuda")
        out = torch.full((5, 7), float("nan"), dtype=torch.float64, device="cuda")
        rc = L.gosma_eval_objective_grad_noalloc(ctx.h, 5, C.c_void_p(x_dev.data_ptr()), C.c_void_p(out.data_ptr()))
        assert rc == 0, L.gosma_last_error(ctx.h)
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        assert np.allclose(o[:, 0], f_ref, rtol=1e-11, atol=1e-12), call
        assert np.allclose(o[:, 1:], g_ref, rtol=1e-9, atol=1e-9 * np.abs(g_ref).max()), call
    # sizes beyond the fixed scratch are rejected with an error, not run
    big = torch.zeros((100000, 6), dtype=torch.float64, device="cuda")
    big_out = torch.zeros((100000, 7), dtype=torch.float64, device="cuda")
    rc = L.gosma_eval_objective_grad_noalloc(ctx.h, 100000, C.c_void_p(big.data_ptr()), C.c_void_p(big_out.data_ptr()))
    assert rc == -1 and b"8 MiB" in L.gosma_last_error(ctx.h)
    ctx.close()


def test_no_alloc_size_limit_is_the_documented_one():
    """The documented limit, count * (128 n1 + 56 ceil((n1^2 + n1 n2) / 512))
    bytes <= 8 MiB, is the one applied: with 3 model and 8 image components the
    largest count it allows leaves 8 bytes of the 8 MiB, and is accepted and
    matches the allocating entry point; one pose more is refused."""
    import torch
    from paper_1812_01232_gb300 import build
    build.build()
    from paper_1812_01232_gb300.gosma import Gosma, load_library
    n1, n2 = 3, 8
    per_pose = 128 * n1 + 56 * math.ceil((n1 * n1 + n1 * n2) / 512)
    count = (8 << 20) // per_pose
    assert (8 << 20) - count * per_pose < 128 and (n1 * count) % 2 == 1
    prob = synth.tiny_problem(21, n1=n1, n_in=n1, n_out=n2 - n1)
    ctx = Gosma(0)
    ctx.set_problem(prob)
    L = load_library()
    rng = np.random.default_rng(23)
    X = np.concatenate([rng.uniform(-2, 2, (count + 1, 3)), rng.uniform(-1, 1, (count + 1, 3))], 1)
    x_dev = torch.tensor(X, dtype=torch.float64, device="cuda")
    out = torch.full((count + 1, 7), float("nan"), dtype=torch.float64, device="cuda")
    rc = L.gosma_eval_objective_grad_noalloc(ctx.h, count + 1, C.c_void_p(x_dev.data_ptr()),
                                             C.c_void_p(out.data_ptr()))
    assert rc == -1 and b"8 MiB" in L.gosma_last_error(ctx.h)
    rc = L.gosma_eval_objective_grad_noalloc(ctx.h, count, C.c_void_p(x_dev.data_ptr()), C.c_void_p(out.data_ptr()))
    assert rc == 0, L.gosma_last_error(ctx.h)
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    assert np.all(np.isnan(o[count]))  # the pose past the count is not written
    f_ref, g_ref = ctx.eval_objective_grad(X[:count])
    fin = np.isfinite(f_ref)
    assert np.array_equal(fin, np.isfinite(o[:count, 0]))
    assert np.allclose(o[:count, 0][fin], f_ref[fin], rtol=1e-11, atol=1e-12)
    assert np.allclose(o[:count, 1:][fin], g_ref[fin], rtol=1e-9, atol=1e-9 * np.abs(g_ref[fin]).max())
    ctx.close()
