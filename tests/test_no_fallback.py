"""The product path has no CPU fallback and never touches the oracle (CPU checks).

* Without the compiled library the binding raises on first use, before any
  computation, instead of computing anything another way.
* No module of the package imports the oracle, and no CUDA or C++ source of it
  includes or names the oracle's library: the FP64 oracle is test
  infrastructure only.
"""
import ast
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2212_09807_gb300")


def test_binding_raises_without_the_library(monkeypatch):
    from paper_2212_09807_gb300 import sim
    from synth import params
    missing = os.path.join(ROOT, "_build", "no_such_folder", "libsim.so")
    assert not os.path.exists(missing)
    monkeypatch.setattr(sim, "LIB_PATH", missing)
    monkeypatch.setattr(sim, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        sim.lib()
    cfg = sim.make_config(params.module_config())
    with pytest.raises(RuntimeError, match="not built"):
        sim.workspace_size(cfg, 100, 1000, 100)


def _py_files():
    for d, _, files in os.walk(PKG):
        for f in files:
            if f.endswith(".py"):
                yield os.path.join(d, f)


def test_package_never_imports_the_oracle():
    for path in _py_files():
        tree = ast.parse(open(path).read(), path)
        for node in ast.walk(tree):
            if isinstance(node, ast.Import):
                names = [a.name for a in node.names]
            elif isinstance(node, ast.ImportFrom):
                names = [node.module or ""]
            else:
                continue
            assert not any(n == "oracle" or n.startswith("oracle.") for n in names), (path, names)


def test_native_sources_never_name_the_oracle():
    for d, _, files in os.walk(os.path.join(PKG, "csrc")):
        for f in files:
            src = open(os.path.join(d, f), errors="replace").read()
            assert "larsim_oracle" not in src and "ora_" not in src, f
    for f in os.listdir(os.path.join(ROOT, "include")):
        assert "larsim_oracle" not in open(os.path.join(ROOT, "include", f)).read(), f
