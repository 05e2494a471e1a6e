"""The CUDA path and the CPU oracle share no code, and the product path has no
CPU fallback.

The package (binding, build script, CUDA sources, input generators) must not
import, include or link anything under oracle/, and the oracle must not use
the package's code, headers or library.  Only the seeded input generators
(synth.py) serve both sides, and they hold none of the method's arithmetic:
they import neither side's solver.  Loading a missing library raises instead
of falling back.
"""
import ast
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2411_03040_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def _files(top, exts):
    out = []
    for d, dirs, names in os.walk(top):
        dirs[:] = [x for x in dirs if x not in ("__pycache__", "_build")]
        out += [os.path.join(d, n) for n in names if n.endswith(exts)]
    return sorted(out)


def _py_imports(path):
    tree = ast.parse(open(path).read(), path)
    mods = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            mods |= {a.name.split(".")[0] for a in node.names}
        elif isinstance(node, ast.ImportFrom) and node.module and node.level == 0:
            mods.add(node.module.split(".")[0])
    return mods


def _includes(path):
    return re.findall(r'^\s*#\s*include\s*[<"]([^>"]+)[>"]', open(path).read(), re.M)


def test_package_does_not_use_the_oracle():
    py = _files(PKG, (".py",))
    assert py
    for f in py:
        assert "oracle" not in _py_imports(f), f
    native = _files(PKG, (".cu", ".cuh", ".h", ".cpp", ".c"))
    assert native
    for f in native:
        for inc in _includes(f):
            assert "oracle" not in inc, (f, inc)
        assert "liboracle" not in open(f).read(), f
    for f in _files(os.path.join(ROOT, "include"), (".h",)):
        assert not any("oracle" in inc for inc in _includes(f)), f


def test_oracle_does_not_use_the_package():
    py = _files(ORACLE, (".py",))
    assert py
    for f in py:
        mods = _py_imports(f)
        assert "paper_2411_03040_gb300" not in mods and "torch" not in mods, (f, mods)
        text = open(f).read()
        assert "libmgt" not in text and "magritte_gpu.h" not in text, f
    for f in _files(ORACLE, (".c", ".h", ".cu", ".cuh")):
        incs = _includes(f)
        assert not any(("mgt" in i or "magritte" in i or "cuda" in i) for i in incs), (f, incs)


def test_input_generators_import_no_solver():
    mods = _py_imports(os.path.join(PKG, "synth.py"))
    assert "oracle" not in mods
    text = open(os.path.join(PKG, "synth.py")).read()
    assert not re.search(r"^\s*(from\s+\.|import\s+\.|from\s+paper_2411_03040_gb300)", text, re.M)
    assert "libmgt" not in text and "ctypes" not in mods


def test_library_is_built_from_package_sources_only():
    from paper_2411_03040_gb300 import build
    for src in build.SOURCES:
        assert os.path.exists(os.path.join(build.CSRC, src)), src
        assert "oracle" not in src


def test_missing_library_raises(tmp_path):
    from paper_2411_03040_gb300 import mgt
    saved = mgt._lib
    mgt._lib = None
    try:
        with pytest.raises(RuntimeError, match="no CPU fallback"):
            mgt.load(str(tmp_path / "libmgt.so"))
    finally:
        mgt._lib = saved
