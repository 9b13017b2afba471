"""The Python binding and the C header describe the same ABI (CPU only).

ctypes sees neither the header nor the library's types: a structure field
out of place or an argument list one entry short corrupts memory without an
error.  So (1) a small C program compiled against include/gosma.h prints the
size and every field offset of each structure, which must equal the ctypes
structures and numpy record types of the binding, and (2) every prototype in
the header is parsed and compared, parameter by parameter, with the
binding's argtypes and restype."""
import ctypes as C
import os
import re
import shutil
import subprocess

import pytest

from paper_1812_01232_gb300 import gosma as G

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gosma.h")

# C structure -> (binding type, its field names as the C structure names them)
STRUCTS = {
    "gosma_cube": G.Cube,
    "gosma_bound": G.Bound,
    "gosma_opts": G.Opts,
    "gosma_result": G.Result,
    "gosma_problem": G.Problem,
    "gosma_learn_opts": G.LearnOpts,
    "gosma_trace_point": G.HISTORY_DTYPE,
    "gosma_trace_rec": G.TRACE_DTYPE,
    "gosma_node": G.NODE_DTYPE,
}


def _fields(t):
    if isinstance(t, type) and issubclass(t, C.Structure):
        return C.sizeof(t), {f[0]: getattr(t, f[0]).offset for f in t._fields_}
    return t.itemsize, {n: t.fields[n][1] for n in t.names}


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_structure_layouts_match_the_header(tmp_path):
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "gosma.h"', "int main(void) {"]
    for cname, t in STRUCTS.items():
        _, offs = _fields(t)
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for f in offs:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for ln in filter(None, out):
        s, f, v = ln.split(" ")
        got[(s, f)] = int(v)
    for cname, t in STRUCTS.items():
        size, offs = _fields(t)
        assert got[(cname, "size")] == size, cname
        for f, o in offs.items():
            assert got[(cname, f)] == o, (cname, f)


# ---------------------------------------------------------------- prototypes
_STRUCT_PTR = {"gosma_cube": G.Cube, "gosma_bound": G.Bound, "gosma_opts": G.Opts, "gosma_result": G.Result,
               "gosma_problem": G.Problem, "gosma_learn_opts": G.LearnOpts}
_SCALAR = {"int": C.c_int, "double": C.c_double, "float": C.c_float, "long long": C.c_longlong}


def _prototypes():
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    src = re.sub(r"#[^\n]*", "", src)
    out = {}
    for ret, name, args in re.findall(r"([A-Za-z_][A-Za-z_ ]*?\**)\s*\b(gosma_[a-z_]+)\s*\(([^)]*)\)\s*;", src):
        params = [a.strip() for a in args.split(",")] if args.strip() != "void" else []
        out[name] = (" ".join(ret.split()), params)
    return out


def _accepts(ctype, decl):
    """Whether the ctypes type passes the C parameter `decl` correctly."""
    d = " ".join(decl.replace("const ", "").split())
    m = re.match(r"^([A-Za-z_ ]+?)\s*(\**)\s*([A-Za-z_0-9]+)?\s*(\[\d*\])?$", d)
    assert m, decl
    base, stars = m.group(1).strip(), len(m.group(2)) + (1 if m.group(4) else 0)
    if stars == 0:
        return ctype is _SCALAR[base]
    if base == "gosma_ctx":
        return ctype is C.c_void_p if stars == 1 else ctype == C.POINTER(C.c_void_p)
    if stars != 1:
        return False
    if ctype is C.c_void_p:  # any data pointer may go as an address
        return base != "char"
    if base == "char":
        return ctype is C.c_char_p
    if base in _STRUCT_PTR:
        return ctype == C.POINTER(_STRUCT_PTR[base])
    return base in _SCALAR and ctype == C.POINTER(_SCALAR[base])


def test_prototypes_match_the_binding():
    protos = _prototypes()
    assert set(protos) == set(G.SIGNATURES)
    rets = {"int": C.c_int, "void": None, "const char *": C.c_char_p, "long long": C.c_longlong}
    for name, (ret, params) in protos.items():
        restype, argtypes = G.SIGNATURES[name]
        assert rets[ret.replace("char*", "char *")] is restype, name
        assert len(argtypes) == len(params), (name, params)
        for k, (a, p) in enumerate(zip(argtypes, params)):
            assert _accepts(a, p), (name, k, p, a)
