"""The C-ABI library loads and exports every function include/gosma.h declares
(no GPU needed: nothing is called)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gosma.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gosma_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("gosma_create", "gosma_destroy", "gosma_set_mixtures", "gosma_set_domain", "gosma_eval_bounds",
              "gosma_eval_objective", "gosma_bnb_solve", "gosma_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_1812_01232_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for n in _declared():
        assert hasattr(lib, n), n


def test_binding_signatures_cover_header():
    from paper_1812_01232_gb300 import gosma
    assert set(gosma.SIGNATURES) == set(_declared())


def test_product_package_does_not_touch_the_oracle():
    pkg = os.path.join(ROOT, "paper_1812_01232_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"import\s+oracle|from\s+oracle|liboracle|gosma_oracle", text), f
