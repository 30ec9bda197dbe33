"""The product path has no CPU fallback and no route through the oracle (CPU):
a missing library raises, host tensors are refused without computing
anything, and neither the package nor the oracle imports or includes the
other (only the seeded input generators are shared)."""
import ast
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1908_09606_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def _py_files(top):
    for dirpath, dirnames, files in os.walk(top):
        dirnames[:] = [d for d in dirnames if not d.startswith(("_build", "__pycache__"))]
        for f in files:
            if f.endswith(".py"):
                yield os.path.join(dirpath, f)


def _imported_modules(path):
    tree = ast.parse(open(path).read(), filename=path)
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            for a in node.names:
                yield a.name
        elif isinstance(node, ast.ImportFrom) and node.level == 0 and node.module:
            yield node.module


def test_missing_library_raises(tmp_path):
    from paper_1908_09606_gb300 import cosma
    with pytest.raises(RuntimeError, match="not built"):
        cosma.load(str(tmp_path / "libcosma_gb300.so"))


def test_host_tensors_are_refused_without_computing():
    import torch
    from paper_1908_09606_gb300 import build as b
    b.build()
    from paper_1908_09606_gb300 import cosma
    A = torch.ones((8, 8), dtype=torch.float64)
    B = torch.ones((8, 8), dtype=torch.float64)
    C = torch.full((8, 8), float("nan"), dtype=torch.float64)
    with pytest.raises((AssertionError, cosma.CosmaError)):
        cosma.gemm(A, B, C, "f64")
    assert torch.isnan(C).all()
    # the C entry point itself refuses host memory for the device entry
    rc = cosma.cosma_gemm(8, 8, 8, A.data_ptr(), 8, B.data_ptr(), 8, C.data_ptr(), 8,
                          cosma.COSMA_F64)
    assert rc == cosma.COSMA_ERR_INVALID_ARG and torch.isnan(C).all()


def test_package_never_imports_the_oracle():
    for path in _py_files(PKG):
        for mod in _imported_modules(path):
            assert mod.split(".")[0] != "oracle", (path, mod)
    for dirpath, _, files in os.walk(os.path.join(PKG, "csrc")):
        for f in files:
            text = open(os.path.join(dirpath, f), errors="replace").read()
            for inc in re.findall(r'#\s*include\s*[<"]([^>"]+)[>"]', text):
                assert "oracle" not in inc, (f, inc)


def test_oracle_never_imports_the_package():
    for path in _py_files(ORACLE):
        for mod in _imported_modules(path):
            assert mod.split(".")[0] != "paper_1908_09606_gb300", (path, mod)
    for f in os.listdir(ORACLE):
        if f.endswith((".c", ".h")):
            text = open(os.path.join(ORACLE, f)).read()
            for inc in re.findall(r'#\s*include\s*[<"]([^>"]+)[>"]', text):
                assert "cosma.h" not in inc and "csrc" not in inc, (f, inc)


def test_shared_input_generators_import_neither_side():
    top = os.path.join(ROOT, "cosma_inputs")
    for path in _py_files(top):
        for mod in _imported_modules(path):
            assert mod.split(".")[0] not in ("oracle", "paper_1908_09606_gb300"), (path, mod)
    for dirpath, dirnames, files in os.walk(top):
        dirnames[:] = [d for d in dirnames if d != "_build"]
        for f in files:
            if f.endswith((".c", ".h", ".cu", ".cuh", ".cpp")):
                text = open(os.path.join(dirpath, f), errors="replace").read()
                for inc in re.findall(r'#\s*include\s*[<"]([^>"]+)[>"]', text):
                    assert "oracle" not in inc and "cosma.h" not in inc, (f, inc)


def test_bench_reaches_the_oracle_only_in_its_cpu_legs():
    """bench.py imports the oracle only inside the CPU-timing helpers, the
    reference arm, or a branch guarded by the --no-cpu switch (the CPU-baseline
    leg), never on the timed GPU path."""
    path = os.path.join(ROOT, "bench.py")
    src = open(path).read()
    tree = ast.parse(src)
    parents = {}
    for node in ast.walk(tree):
        for child in ast.iter_child_nodes(node):
            parents[child] = node
    helpers = {"oracle_sample", "tiled_sample", "grouped_oracle_sample", "run_reference"}
    found = 0
    for node in ast.walk(tree):
        names = []
        if isinstance(node, ast.ImportFrom) and node.module:
            names = [node.module]
        elif isinstance(node, ast.Import):
            names = [a.name for a in node.names]
        if not any(nm.split(".")[0] == "oracle" for nm in names):
            continue
        found += 1
        p, ok = parents.get(node), False
        while p is not None and not ok:
            if isinstance(p, ast.FunctionDef) and p.name in helpers:
                ok = True
            if isinstance(p, ast.If) and "no_cpu" in ast.get_source_segment(src, p.test):
                ok = True
            p = parents.get(p)
        assert ok, f"oracle import at bench.py:{node.lineno} outside the CPU legs"
    assert found >= 3
    # and the CPU-timing helpers are called only from those places too
    for node in ast.walk(tree):
        if not (isinstance(node, ast.Call) and isinstance(node.func, ast.Name)
                and node.func.id in ("oracle_sample", "tiled_sample",
                                     "grouped_oracle_sample")):
            continue
        p, ok = parents.get(node), False
        while p is not None and not ok:
            if isinstance(p, ast.FunctionDef) and p.name == "run_reference":
                ok = True
            if isinstance(p, ast.If) and "no_cpu" in ast.get_source_segment(src, p.test):
                ok = True
            p = parents.get(p)
        assert ok, f"{node.func.id} called at bench.py:{node.lineno} outside the CPU legs"
