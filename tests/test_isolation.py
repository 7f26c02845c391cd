"""The product path and the oracle share no code: nothing in the package (Python binding, CUDA
sources, header) loads the oracle, and the oracle loads nothing of the package; the only
shared module is the seeded input generator, which holds none of the method's arithmetic."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _sources(folder, exts):
    for d, _, files in os.walk(os.path.join(ROOT, folder)):
        if "_build" in d or "__pycache__" in d:
            continue
        for f in files:
            if f.endswith(exts):
                yield os.path.join(d, f)


def test_package_does_not_load_the_oracle():
    pat = re.compile(r"^\s*(import\s+oracle|from\s+oracle\b)|bltc_oracle|liboracle", re.M)
    for path in list(_sources("paper_2003_01836_gb300", (".py", ".cu", ".cuh", ".cpp", ".h"))) + \
            [os.path.join(ROOT, "include", "bltc.h")]:
        with open(path) as f:
            assert not pat.search(f.read()), path


def test_oracle_does_not_load_the_package():
    pat = re.compile(r"^\s*(import\s+paper_2003_01836_gb300|from\s+paper_2003_01836_gb300)|libbltc|#\s*include\s*\"bltc\.h\"",
                     re.M)
    for path in _sources("oracle", (".py", ".c", ".h")):
        with open(path) as f:
            assert not pat.search(f.read()), path


def test_input_module_holds_no_treecode_arithmetic():
    with open(os.path.join(ROOT, "paper_2003_01836_gb300", "inputs.py")) as f:
        text = f.read()
    for word in ("cheb", "lagrange", "rsqrt", "theta", "modified charge", "import oracle"):
        assert word not in text.lower(), word
