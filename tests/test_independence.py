"""Structural checks of the product/oracle split: the package neither imports
nor reads anything under oracle/ (and the oracle nothing from the package), the
CUDA sources include nothing from the oracle, and the binding refuses to run
without its compiled library instead of falling back to any CPU path."""
import ast
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2506_05558_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def _py_files(d):
    for dirpath, _, files in os.walk(d):
        if "__pycache__" in dirpath or "_build" in dirpath or "_lib" in dirpath:
            continue
        for f in files:
            if f.endswith(".py"):
                yield os.path.join(dirpath, f)


def _imported_modules(path):
    tree = ast.parse(open(path).read(), path)
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            for a in node.names:
                yield a.name
        elif isinstance(node, ast.ImportFrom):
            yield node.module or ""


def test_package_never_imports_the_oracle():
    for path in _py_files(PKG):
        for mod in _imported_modules(path):
            assert not (mod == "oracle" or mod.startswith("oracle.")), (path, mod)
        assert "oracle/" not in open(path).read().replace("\\", "/"), path


def test_oracle_never_imports_the_package():
    for path in _py_files(ORACLE):
        for mod in _imported_modules(path):
            assert not mod.startswith("paper_2506_05558_gb300"), (path, mod)
    for name in os.listdir(ORACLE):
        if name.endswith((".c", ".h")):
            text = open(os.path.join(ORACLE, name)).read()
            assert "csrc" not in text and "gs.h" not in text, name


def test_cuda_sources_include_nothing_from_the_oracle():
    csrc = os.path.join(PKG, "csrc")
    for name in os.listdir(csrc):
        if name.endswith((".cu", ".cuh", ".h", ".cpp")):
            for inc in re.findall(r'#include\s+"([^"]+)"', open(os.path.join(csrc, name)).read()):
                assert "oracle" not in inc, (name, inc)


def test_binding_fails_loudly_without_its_library(monkeypatch):
    from paper_2506_05558_gb300 import gs
    monkeypatch.setattr(gs, "_lib", None)
    monkeypatch.setattr(gs, "LIB_PATH", os.path.join(ROOT, "no_such_dir", "libgs.so"))
    with pytest.raises(RuntimeError, match="not built"):
        gs.lib()
    with pytest.raises(RuntimeError, match="not built"):
        gs.config(sh_degree=3)
