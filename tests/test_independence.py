"""CPU: the CUDA library and the oracle stay apart.  Neither side imports or includes the other,
the library build compiles only the library's own sources, and the benchmark and the entry module
reach the oracle only inside functions (the CPU legs, the accuracy checks and the smoke check),
never at import time."""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2403_04578_gb300")
ORC = os.path.join(ROOT, "oracle")


def _py_files(d):
    return [os.path.join(d, f) for f in sorted(os.listdir(d)) if f.endswith(".py")]


def _imports(path, top_level_only=False):
    tree = ast.parse(open(path).read(), path)
    nodes = tree.body if top_level_only else ast.walk(tree)
    out = set()
    for n in nodes:
        if isinstance(n, ast.Import):
            out.update(a.name.split(".")[0] for a in n.names)
        elif isinstance(n, ast.ImportFrom) and n.module and n.level == 0:
            out.add(n.module.split(".")[0])
    return out


def _includes(path):
    return re.findall(r'^\s*#\s*include\s*[<"]([^>"]+)[>"]', open(path).read(), re.M)


def test_library_python_never_imports_the_oracle():
    files = _py_files(PKG)
    assert files
    for f in files:
        assert "oracle" not in _imports(f), f


def test_oracle_never_imports_the_library():
    files = _py_files(ORC)
    assert files
    for f in files:
        assert "paper_2403_04578_gb300" not in _imports(f), f


def test_c_sources_include_nothing_from_the_other_side():
    csrc = os.path.join(PKG, "csrc")
    lib_sources = [os.path.join(csrc, f) for f in os.listdir(csrc)]
    assert lib_sources
    for f in lib_sources:
        for inc in _includes(f):
            assert "oracle" not in inc and "fpi" not in inc, (f, inc)
    for f in [os.path.join(ORC, x) for x in os.listdir(ORC) if x.endswith((".c", ".h"))]:
        for inc in _includes(f):
            assert "/" not in inc and not inc.startswith("tpf"), (f, inc)  # system headers only


def test_library_build_compiles_only_its_own_sources():
    import importlib.util

    spec = importlib.util.spec_from_file_location("_tpf_build_probe", os.path.join(PKG, "build.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    assert os.path.samefile(b.CSRC, os.path.join(PKG, "csrc"))
    for src in b.SOURCES:
        assert os.path.isfile(os.path.join(b.CSRC, src)), src
        assert "oracle" not in src and "fpi" not in src


def test_inputs_module_holds_no_solver():
    """The shared input generators draw random numbers only: no linear algebra, no oracle."""
    path = os.path.join(PKG, "inputs.py")
    assert _imports(path) <= {"__future__", "dataclasses", "math", "concurrent", "numpy", "torch"}
    text = open(path).read()
    for word in ("linalg", "solve(", "inv(", "scipy"):
        assert word not in text, word


def test_bench_and_entry_reach_the_oracle_only_inside_functions():
    for name in ("bench.py", "__graft_entry__.py"):
        path = os.path.join(ROOT, name)
        assert "oracle" not in _imports(path, top_level_only=True), name
        assert "oracle" in _imports(path), name  # the CPU legs / smoke check do use it
