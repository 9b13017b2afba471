"""Argument checks of the Python binding, run on CPU: the C ABI sees only
pointers and the sizes it is given, so the binding refuses arrays whose
lengths disagree and device buffers of the wrong dtype, shape, layout or
device before any call reaches the library."""
import numpy as np
import pytest
import torch

from paper_1812_01232_gb300 import gosma, synth
from paper_1812_01232_gb300.gosma import GosmaArgumentError, GosmaError

MIX = gosma._MIX_NAMES


def test_argument_error_is_both_kinds():
    e = GosmaArgumentError("x")
    assert isinstance(e, GosmaError) and isinstance(e, ValueError)


def test_mixture_lengths():
    p = synth.paper_scale_problem(3)
    a = gosma._mixture_arrays(*(p[k] for k in MIX))
    assert [x.shape for x in a] == [(128, 3), (128,), (128,), (64, 3), (64,), (64,)]
    assert all(x.dtype == np.float64 and x.flags.c_contiguous for x in a)
    for k, cut in (("mu1", 1), ("phi1", 1), ("mu2", 2), ("phi2", 5)):
        bad = dict(p)
        bad[k] = p[k][:-cut]
        with pytest.raises(GosmaArgumentError, match=k):
            gosma._mixture_arrays(*(bad[q] for q in MIX))
    bad = dict(p, mu1=p["mu1"][:, :2])  # not n x 3: the reshape to rows of 3 gives the wrong count or fails
    with pytest.raises((GosmaArgumentError, ValueError)):
        gosma._mixture_arrays(*(bad[q] for q in MIX))


def test_class_sizes():
    p = synth.semantic_problem(5, nclass=3)
    n1, n2 = len(p["sigma1"]), len(p["kappa2"])
    n1c, n2c, w = gosma._class_arrays(p["n1c"], p["n2c"], p["w"], n1, n2)
    assert n1c.dtype == np.int32 and n2c.dtype == np.int32 and len(w) == 3
    with pytest.raises(GosmaArgumentError, match="entries"):
        gosma._class_arrays(p["n1c"], p["n2c"], p["w"][:2], n1, n2)
    with pytest.raises(GosmaArgumentError, match="add up"):
        gosma._class_arrays(np.asarray(p["n1c"]) + [1, 0, 0], p["n2c"], p["w"], n1, n2)
    with pytest.raises(GosmaArgumentError, match="add up"):
        gosma._class_arrays(p["n1c"], np.asarray(p["n2c"]) - [0, 0, 1], p["w"], n1, n2)


def test_device_buffers():
    t = torch.zeros(5, 10, dtype=torch.float64)
    with pytest.raises(GosmaArgumentError, match="torch tensor"):
        gosma._dev(np.zeros((5, 10)), "cubes", torch.float64, (5, 10), 0)
    with pytest.raises(GosmaArgumentError, match="expected torch.float64"):
        gosma._dev(t.float(), "cubes", torch.float64, (5, 10), 0)
    with pytest.raises(GosmaArgumentError, match="shape"):
        gosma._dev(t[:4], "cubes", torch.float64, (5, 10), 0)
    with pytest.raises(GosmaArgumentError, match="shape"):
        gosma._dev(t.reshape(10, 5), "cubes", torch.float64, (5, 10), 0)
    with pytest.raises(GosmaArgumentError, match="contiguous"):
        gosma._dev(torch.zeros(10, 5, dtype=torch.float64).t(), "cubes", torch.float64, (5, 10), 0)
    with pytest.raises(GosmaArgumentError, match="CUDA tensor on cuda:0"):
        gosma._dev(t, "cubes", torch.float64, (5, 10), 0)  # the right tensor, but in host memory
    with pytest.raises(GosmaArgumentError, match="expected torch.int32"):
        gosma._dev(torch.zeros(5, dtype=torch.int64), "iters", torch.int32, (5,), 0)
