"""Checkpoint / resume of a branch-and-bound run: a run saved between two
steps and resumed on a fresh context ends with exactly the certificate,
pose and counters of the uninterrupted run."""
import numpy as np
import pytest

from paper_1812_01232_gb300 import synth

pytestmark = pytest.mark.gpu


def _ctx():
    from paper_1812_01232_gb300 import build
    build.build()
    from paper_1812_01232_gb300.gosma import Gosma
    return Gosma(0)


@pytest.mark.parametrize("seed,steps", [(1000, 40), (3001, 300)])
def test_resume_replays_the_run(tmp_path, seed, steps):
    p = synth.tiny_problem(seed)
    a = _ctx()
    a.set_problem(p)
    a.bnb_start(eps=1e-3, pop=1024, queue_capacity=1 << 25)
    mid = a.bnb_step(steps)
    assert mid["status_name"] == "running"
    path = str(tmp_path / "run.gosma")
    a.bnb_save(path)
    full = a.bnb_step(0)
    a.close()
    b = _ctx()
    b.set_problem(p)
    b.bnb_load(path)
    res = b.bnb_step(0)
    b.close()
    assert full["status_name"] == res["status_name"] == "optimal"
    for k in ("f", "lb", "nodes", "iterations", "sma_calls", "queue_peak", "cross_pairs", "self_pairs",
              "dstar_iteration"):
        assert res[k] == full[k], k
    assert np.array_equal(res["r"], full["r"]) and np.array_equal(res["t"], full["t"])


def test_load_checks_the_problem(tmp_path):
    from paper_1812_01232_gb300.gosma import GosmaError
    p = synth.tiny_problem(1000)
    a = _ctx()
    a.set_problem(p)
    with pytest.raises(GosmaError):
        a.bnb_save(str(tmp_path / "none.gosma"))  # no run yet
    a.bnb_start(eps=1e-3, pop=256, queue_capacity=1 << 22)
    a.bnb_step(5)
    path = str(tmp_path / "run.gosma")
    a.bnb_save(path)
    a.set_problem(synth.tiny_problem(1001))
    with pytest.raises(GosmaError):
        a.bnb_load(path)  # other mixtures
    # the same image mixture (so the same C22) and sizes, the model means moved
    # by 1 mm: only the mixture fingerprint tells the problems apart
    q = dict(p)
    q["mu1"] = p["mu1"] + 1e-3
    a.set_problem(q)
    with pytest.raises(GosmaError, match="other mixtures"):
        a.bnb_load(path)
    # one model scale changed
    q = dict(p)
    q["sigma1"] = p["sigma1"].copy()
    q["sigma1"][3] *= 1.5
    a.set_problem(q)
    with pytest.raises(GosmaError, match="other mixtures"):
        a.bnb_load(path)
    (tmp_path / "junk.gosma").write_bytes(b"not a checkpoint")
    a.set_problem(p)
    with pytest.raises(GosmaError):
        a.bnb_load(str(tmp_path / "junk.gosma"))
    a.bnb_load(path)
    assert a.bnb_step(1)["iterations"] == 6
    a.close()
