"""The product path never reaches the oracle.

The CUDA library, its Python binding and the benchmark's timed legs must not
import, link, load or name anything under oracle/: the oracle is test
infrastructure, and a product path that routed through it would make every
parity result meaningless.  Only bench.py's CPU legs (the CPU baseline and
the reference arm) may call it.  Everything here reads source text or the
built library's dynamic section; no GPU is needed.
"""
import ast
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1810_08218_gb300")
# bench.py functions allowed to use the oracle: the CPU baseline leg and the
# reference arm, both timed on the host
BENCH_ORACLE_LEGS = {"cpu_oracle_full_map", "run_reference", "_oracle_worker", "reference_accuracy"}


def _docstring_nodes(tree):
    out = set()
    for node in ast.walk(tree):
        if isinstance(node, (ast.Module, ast.FunctionDef, ast.AsyncFunctionDef, ast.ClassDef)):
            body = getattr(node, "body", [])
            if body and isinstance(body[0], ast.Expr) and isinstance(body[0].value, ast.Constant) \
                    and isinstance(body[0].value.value, str):
                out.add(id(body[0].value))
    return out


def _oracle_uses(tree, skip_functions=()):
    """Imports of `oracle`, dynamic imports naming it, and non-docstring
    string constants naming it, outside the functions in skip_functions."""
    docs = _docstring_nodes(tree)
    skipped = set()
    for node in ast.walk(tree):
        if isinstance(node, (ast.FunctionDef, ast.AsyncFunctionDef)) and node.name in skip_functions:
            for sub in ast.walk(node):
                skipped.add(id(sub))
    hits = []
    for node in ast.walk(tree):
        if id(node) in skipped:
            continue
        if isinstance(node, ast.Import):
            hits += [a.name for a in node.names if a.name.split(".")[0] == "oracle"]
        elif isinstance(node, ast.ImportFrom):
            mod = node.module or ""
            if mod.split(".")[0] == "oracle" or (node.level == 0 and any(a.name == "oracle" for a in node.names)):
                hits.append(f"from {mod} import ...")
        elif isinstance(node, ast.Constant) and isinstance(node.value, str) and id(node) not in docs:
            # a module or path naming the oracle ("oracle", "oracle/...",
            # "../oracle", "oracle.ptp"); prose that mentions it is not a use
            v = node.value.strip()
            if v == "oracle" or re.search(r"(^|[/\\])oracle([/\\.]|$)", v):
                hits.append(repr(v[:60]))
    return hits


def _package_modules():
    out = []
    for dirpath, _, files in os.walk(PKG):
        if "_build" in dirpath or "__pycache__" in dirpath:
            continue
        out += [os.path.join(dirpath, f) for f in files if f.endswith(".py")]
    return sorted(out)


@pytest.mark.parametrize("path", _package_modules(), ids=lambda p: os.path.relpath(p, ROOT))
def test_package_module_never_names_the_oracle(path):
    tree = ast.parse(open(path).read(), path)
    assert _oracle_uses(tree) == [], path


def test_native_sources_never_include_the_oracle():
    for d in (os.path.join(PKG, "csrc"), os.path.join(ROOT, "include")):
        for f in os.listdir(d):
            text = open(os.path.join(d, f)).read()
            code = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            code = re.sub(r"//[^\n]*", "", code)
            assert "oracle" not in code, f


def test_build_compiles_only_the_package_sources():
    from paper_1810_08218_gb300 import build

    for src in build.sources():
        assert os.path.dirname(src) == os.path.join(PKG, "csrc"), src
    assert "oracle" not in " ".join(build.NVCC_FLAGS)


def test_library_links_no_oracle():
    from paper_1810_08218_gb300 import build

    lib = build.build()
    try:
        dyn = subprocess.run(["readelf", "-d", lib], capture_output=True, text=True, check=True).stdout
    except (OSError, subprocess.CalledProcessError):
        pytest.skip("readelf unavailable")
    needed = re.findall(r"\(NEEDED\).*\[(.*?)\]", dyn)
    assert needed, dyn
    assert not [n for n in needed if "oracle" in n], needed


def test_bench_timed_legs_never_use_the_oracle():
    path = os.path.join(ROOT, "bench.py")
    tree = ast.parse(open(path).read(), path)
    hits = _oracle_uses(tree, skip_functions=BENCH_ORACLE_LEGS)
    assert hits == [], hits
    # and the allowed legs exist, so the exemption names real functions
    names = {n.name for n in ast.walk(tree) if isinstance(n, ast.FunctionDef)}
    assert {"cpu_oracle_full_map", "run_reference"} <= names


def test_guard_catches_a_planted_import():
    planted = ast.parse("import numpy\n\ndef f():\n    from oracle import mlp\n    return mlp\n")
    assert _oracle_uses(planted) != []
    planted = ast.parse("import os\np = os.path.join('x', 'oracle', 'lib.so')\n")
    assert _oracle_uses(planted) != []
    planted = ast.parse("import ctypes\nlib = ctypes.CDLL('repo/oracle/_build/liboracle.so')\n")
    assert _oracle_uses(planted) != []
    planted = ast.parse("import importlib\nm = importlib.import_module('oracle.mlp')\n")
    assert _oracle_uses(planted) != []
    clean = ast.parse('"""Checked against the oracle in the tests."""\nimport numpy\n')
    assert _oracle_uses(clean) == []
