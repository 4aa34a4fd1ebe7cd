"""The oracle and the CUDA path share no code and call each other nowhere.

Static checks over the sources: nothing in the package (Python, CUDA, the
C header) imports, includes or loads anything under ``oracle/``; nothing under
``oracle/`` imports the package, except the seeded input generators of
``workloads`` (which hold none of the method's arithmetic); and the only
places outside ``tests/`` that reach the oracle are ``__graft_entry__``'s
``build``/``smoke`` and ``bench.py``'s ``run_reference``/``cpu_baseline``.
"""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2111_10140_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def _files(top, exts):
    for d, _, names in os.walk(top):
        if "_build" in d or "__pycache__" in d:
            continue
        for n in names:
            if n.endswith(exts):
                yield os.path.join(d, n)


def _imports(path):
    tree = ast.parse(open(path).read(), path)
    out = []
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            out += [a.name for a in node.names]
        elif isinstance(node, ast.ImportFrom) and node.module:
            out.append(node.module)
    return out


def test_package_never_reaches_the_oracle():
    for path in _files(PKG, (".py",)):
        for mod in _imports(path):
            assert not mod.split(".")[0] == "oracle", f"{path} imports {mod}"
        text = open(path).read()
        assert "anova_oracle" not in text and "liboracle" not in text, path
    for path in list(_files(PKG, (".cu", ".cuh", ".h", ".cpp"))) + list(_files(os.path.join(ROOT, "include"), (".h",))):
        text = open(path).read()
        assert not re.search(r'#\s*include\s*[<"][^>"]*oracle', text), path
        assert "orc_" not in text, f"{path} names an oracle symbol"


def test_oracle_imports_only_the_input_generators():
    for path in _files(ORACLE, (".py",)):
        for mod in _imports(path):
            if mod.startswith("paper_2111_10140_gb300"):
                assert mod == "paper_2111_10140_gb300.workloads", f"{path} imports {mod}"
    for path in _files(ORACLE, (".c", ".h")):
        text = open(path).read()
        assert "anova_gb300" not in text and "#include \"" not in text, path


def _functions_importing_oracle(path):
    tree = ast.parse(open(path).read(), path)
    hits = set()
    for fn in ast.walk(tree):
        if isinstance(fn, (ast.FunctionDef, ast.AsyncFunctionDef)):
            for node in ast.walk(fn):
                if isinstance(node, ast.Import) and any(a.name.split(".")[0] == "oracle" for a in node.names):
                    hits.add(fn.name)
                elif isinstance(node, ast.ImportFrom) and (node.module or "").split(".")[0] == "oracle":
                    hits.add(fn.name)
    top = [n for n in tree.body if isinstance(n, (ast.Import, ast.ImportFrom))]
    for node in top:
        names = [a.name for a in node.names] if isinstance(node, ast.Import) else [node.module or ""]
        assert not any(n.split(".")[0] == "oracle" for n in names), f"{path} imports the oracle at module level"
    return hits


def test_only_the_baseline_legs_reach_the_oracle():
    assert _functions_importing_oracle(os.path.join(ROOT, "bench.py")) <= {"run_reference", "cpu_baseline"}
    assert _functions_importing_oracle(os.path.join(ROOT, "__graft_entry__.py")) <= {"build", "smoke"}


def test_workloads_hold_no_method_arithmetic():
    """The shared generators draw and map inputs; they name none of the
    method's steps (no window, kernel coefficients, FFT, spreading)."""
    text = open(os.path.join(PKG, "workloads.py")).read()
    code = "\n".join(l for l in text.splitlines() if not l.lstrip().startswith("#"))
    code = re.sub(r'"""(.|\n)*?"""', "", code)
    for word in ("fft", "bessel", "sinh", "kaiser", "spread", "gather", "kreg", "kernel_coeffs"):
        assert word not in code.lower(), f"workloads.py mentions {word}"
