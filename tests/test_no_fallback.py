"""The product path has no CPU fallback: without the CUDA library the
binding refuses to load, and without a usable GPU creating a context fails
with the library's error (checked here, on a machine without a GPU)."""
import os

import pytest

from paper_1812_01232_gb300 import gosma


def test_missing_library_raises(monkeypatch, tmp_path):
    monkeypatch.setattr(gosma, "_lib", None)
    with pytest.raises(RuntimeError, match="no fallback"):
        gosma.load_library(str(tmp_path / "libgosma.so"))


def test_context_needs_a_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1812_01232_gb300 import build
    build.build()
    assert os.path.exists(gosma.LIB_PATH)
    with pytest.raises(gosma.GosmaError, match="gosma_create failed"):
        gosma.Gosma(0)
