"""The oracle and the CUDA path share no code: the oracle imports nothing from
the package, the package never imports the oracle, and the seeded input
generators (imported by both sides' tests) hold no arithmetic of the method
(they import nothing but NumPy)."""
import ast
import glob
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def imported_modules(path):
    tree = ast.parse(open(path).read(), path)
    mods = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            mods.update(a.name for a in node.names)
        elif isinstance(node, ast.ImportFrom):
            mods.add(("." * node.level) + (node.module or ""))
    return mods


def test_oracle_imports_nothing_from_the_package():
    for path in glob.glob(os.path.join(ROOT, "oracle", "*.py")):
        for m in imported_modules(path):
            assert not m.startswith("paper_1810_02719_gb300"), (path, m)


def test_package_never_imports_the_oracle():
    for path in glob.glob(os.path.join(ROOT, "paper_1810_02719_gb300", "**", "*.py"),
                          recursive=True):
        for m in imported_modules(path):
            assert not m.startswith("oracle"), (path, m)


def test_input_generators_import_only_numpy():
    mods = imported_modules(os.path.join(ROOT, "paper_1810_02719_gb300", "synth.py"))
    assert mods <= {"__future__", "numpy"}, mods


def test_cuda_sources_include_nothing_from_the_oracle():
    for path in glob.glob(os.path.join(ROOT, "paper_1810_02719_gb300", "csrc", "*")):
        for line in open(path, errors="ignore"):
            if line.lstrip().startswith("#include"):
                assert "oracle" not in line, (path, line)
