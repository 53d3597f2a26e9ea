"""CPU guards of the product / test-infrastructure boundary.

The product package never imports the oracle (the oracle is test
infrastructure; only tests/, the smoke check and bench.py's CPU-baseline and
reference legs use it), and the binding has no fallback: without the compiled
CUDA library every operator call fails loudly.
"""
import ast
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1906_03489_gb300")


def _imports(path):
    tree = ast.parse(open(path).read())
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            for a in node.names:
                yield a.name, node
        elif isinstance(node, ast.ImportFrom):
            yield (node.module or ""), node


def test_product_package_never_imports_the_oracle():
    for name in sorted(os.listdir(PKG)):
        if name.endswith(".py"):
            for mod, _ in _imports(os.path.join(PKG, name)):
                assert not mod.split(".")[0] == "oracle", (name, mod)


def test_bench_imports_the_oracle_only_inside_its_cpu_legs():
    """bench.py may use the oracle only in the functions that time it on the host."""
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    allowed = {"oracle_sample_rate"}
    for fn in tree.body:
        if isinstance(fn, ast.FunctionDef):
            for node in ast.walk(fn):
                if isinstance(node, ast.ImportFrom) and (node.module or "").split(".")[0] == "oracle":
                    assert fn.name in allowed, fn.name
        elif isinstance(fn, (ast.Import, ast.ImportFrom)):
            mods = [a.name for a in fn.names] if isinstance(fn, ast.Import) else [fn.module or ""]
            assert not any(m.split(".")[0] == "oracle" for m in mods)


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    from paper_1906_03489_gb300 import _lib
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "libspx.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        _lib.lib()
