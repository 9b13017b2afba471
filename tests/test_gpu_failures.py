"""Failure detection without a GPU fault.

* A bounded device wait is made to run out (an mbarrier that nothing arrives
  on): the call reports GOSMA_ETIMEOUT and the context keeps working.
* Device allocations are made to fail from the host: every entry point
  returns an error instead of crashing, and the same call succeeds when
  retried on the same context.
"""
import numpy as np
import pytest

from paper_1812_01232_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture()
def fresh():
    from paper_1812_01232_gb300 import build
    build.build()
    from paper_1812_01232_gb300.gosma import Gosma
    c = Gosma(0)
    yield c
    c.close()


def test_bounded_wait_times_out_and_context_survives(fresh, oracle_mod):
    assert fresh.selftest_wait_timeout(0.05) == -4  # GOSMA_ETIMEOUT
    p = synth.tiny_problem(1000)
    fresh.set_problem(p)
    cubes = synth.tree_cubes(3, 64, p["t_lo"], p["t_hi"], 0, 10)
    lb, ub = fresh.eval_bounds(cubes)
    ref = oracle_mod.bounds(oracle_mod.Mixtures.from_problem(p), cubes, p["zeta"])
    fin = np.isfinite(ref[:, 0])
    assert np.all(lb[fin] <= ref[fin, 0] + 1e-12 * np.abs(ref[fin, 0]))
    assert fresh.selftest_wait_timeout(0.01) == -4


def _fails_then_works(ctx, fn):
    from paper_1812_01232_gb300.gosma import GosmaError
    ctx.debug_fail_allocations(1)
    with pytest.raises(GosmaError):
        fn()
    ctx.debug_fail_allocations(0)
    return fn()


def test_allocation_failures_are_reported_and_recoverable(fresh):
    from paper_1812_01232_gb300 import learn
    p = synth.tiny_problem(1000)
    _fails_then_works(fresh, lambda: fresh.set_problem(p))
    cubes = synth.tree_cubes(4, 128, p["t_lo"], p["t_hi"], 0, 10)
    lb, ub = _fails_then_works(fresh, lambda: fresh.eval_bounds(cubes))
    lb2, ub2 = fresh.eval_bounds(cubes)
    assert np.array_equal(lb, lb2) and np.array_equal(ub, ub2)
    f = _fails_then_works(fresh, lambda: fresh.eval_objective(p["r_gt"], p["t_gt"]))
    assert np.isfinite(f)
    r = _fails_then_works(fresh, lambda: fresh.bnb_solve(eps=1e-2, pop=256, max_seconds=60, queue_capacity=1 << 22))
    assert r["status_name"] == "optimal"
    rb = _fails_then_works(fresh, lambda: fresh.bnb_solve_batch([p], eps=1e-2, pop=256, max_seconds=60,
                                                                queue_capacity=1 << 22))
    assert rb[0]["status_name"] == "optimal" and abs(rb[0]["f"] - r["f"]) <= 1e-2 * r["c22"]
    _fails_then_works(fresh, lambda: fresh.mlp_set_params(learn.init_params(0)))
    y = fresh.mlp_forward(np.zeros((3, 16), dtype=np.float32))
    assert np.all(np.isfinite(y))
