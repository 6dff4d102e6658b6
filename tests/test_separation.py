"""The product path and the oracle stay apart: nothing in the package imports,
includes or names the oracle; the oracle imports nothing of the package; the
seeded input generators import neither; and the binding raises when the CUDA
library is missing instead of falling back to anything."""
import ast
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1509_06865_gb300")


def _files(top, exts):
    for d, _, names in os.walk(top):
        if "__pycache__" in d or "_build" in d:
            continue
        for n in names:
            if n.endswith(exts):
                yield os.path.join(d, n)


def _imports(path):
    tree = ast.parse(open(path).read(), path)
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            yield from (a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom) and node.module and node.level == 0:
            yield node.module.split(".")[0]


def test_package_never_uses_the_oracle():
    for f in _files(PKG, (".py",)):
        assert "oracle" not in set(_imports(f)), f
    for f in _files(PKG, (".cu", ".cuh", ".h", ".cpp")):
        text = open(f).read()
        assert "oracle/" not in text and "#include \"../../oracle" not in text, f
    for f in _files(os.path.join(ROOT, "include"), (".h",)):
        assert "oracle/" not in open(f).read(), f


def test_oracle_and_generators_never_use_the_package():
    for top in ("oracle", "synth"):
        for f in _files(os.path.join(ROOT, top), (".py",)):
            mods = set(_imports(f))
            assert "paper_1509_06865_gb300" not in mods, f
            if top == "synth":
                assert "oracle" not in mods, f
    for f in _files(os.path.join(ROOT, "oracle"), (".c", ".h", ".py")):
        assert "csrc" not in open(f).read(), f


def test_binding_raises_without_the_library(monkeypatch, tmp_path):
    from paper_1509_06865_gb300 import _lib
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "libmgeig.so"))
    with pytest.raises(ImportError):
        _lib.load()
