"""The oracle and the CUDA path share no code (host test, no GPU).

The product package (the ctypes binding, the build script and csrc/) never imports or names the
oracle; the oracle imports neither the package nor the input generators; the input generators
(synthetic/) import neither; __graft_entry__ reaches the oracle only from smoke(), where the
smoke run checks the library against it."""
import ast
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = "paper_2110_14514_gb300"


def _py_files(folder):
    for dirpath, _, files in os.walk(os.path.join(ROOT, folder)):
        if "__pycache__" in dirpath or "_build" in dirpath:
            continue
        for f in files:
            if f.endswith(".py"):
                yield os.path.join(dirpath, f)


def _imported_roots(path):
    """(top-level module, enclosing function or None, line) of every import in a file; relative
    imports count as the file's own package."""
    tree = ast.parse(open(path).read())
    parents = {c: p for p in ast.walk(tree) for c in ast.iter_child_nodes(p)}
    out = []
    for n in ast.walk(tree):
        if isinstance(n, ast.Import):
            mods = [a.name for a in n.names]
        elif isinstance(n, ast.ImportFrom):
            mods = ["." if n.level else (n.module or "")]
        else:
            continue
        fn, c = None, n
        while c in parents:
            c = parents[c]
            if isinstance(c, ast.FunctionDef):
                fn = c.name
        out += [(m.split(".")[0], fn, n.lineno) for m in mods]
    return out


def test_package_never_imports_the_oracle():
    files = list(_py_files(PKG))
    assert any(f.endswith("__init__.py") for f in files)
    for f in files:
        for mod, _, line in _imported_roots(f):
            assert mod != "oracle", f"{f}:{line} imports the oracle"
            assert mod != "synthetic", f"{f}:{line} imports the input generators"


def test_product_sources_do_not_name_the_oracle():
    csrc = os.path.join(ROOT, PKG, "csrc")
    files = [os.path.join(csrc, f) for f in sorted(os.listdir(csrc))]
    files += [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))]
    files += list(_py_files(PKG))
    assert len(files) > 10
    for f in files:
        assert "oracle" not in open(f).read().lower(), f


def test_oracle_imports_neither_the_package_nor_the_generators():
    files = list(_py_files("oracle"))
    assert len(files) >= 3
    for f in files:
        for mod, _, line in _imported_roots(f):
            assert mod not in (PKG, "synthetic", "bench", "torch"), f"{f}:{line} imports {mod}"


def test_generators_import_neither_side():
    for f in _py_files("synthetic"):
        for mod, _, line in _imported_roots(f):
            assert mod not in (PKG, "oracle"), f"{f}:{line} imports {mod}"


def test_entry_module_reaches_the_oracle_only_from_smoke():
    uses = [(fn, line) for mod, fn, line in _imported_roots(os.path.join(ROOT, "__graft_entry__.py"))
            if mod == "oracle"]
    assert uses, "smoke() checks the library against the oracle"
    assert all(fn == "smoke" for fn, _ in uses), uses
