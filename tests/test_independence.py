"""The oracle and the CUDA path share no code: the package never imports the
oracle, the oracle imports nothing of the package (its inputs come from the
caller), and neither side's C/CUDA sources include the other's.  CPU only."""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1510_02148_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def _py_files(d):
    for dp, _, fs in os.walk(d):
        if "__pycache__" in dp or "_build" in dp:
            continue
        for f in fs:
            if f.endswith(".py"):
                yield os.path.join(dp, f)


def _imports(path):
    tree = ast.parse(open(path).read(), path)
    out = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            out.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom) and node.level == 0 and node.module:
            out.add(node.module.split(".")[0])
    return out


def test_package_never_imports_the_oracle():
    for f in _py_files(PKG):
        assert "oracle" not in _imports(f), f


def test_oracle_imports_nothing_of_the_package():
    for f in _py_files(ORACLE):
        assert "paper_1510_02148_gb300" not in _imports(f), f


def test_c_sources_do_not_cross():
    inc = re.compile(r'#\s*include\s*[<"]([^>"]+)[>"]')
    csrc = os.path.join(PKG, "csrc")
    cuda_names = set(os.listdir(csrc))
    oracle_c = [f for f in os.listdir(ORACLE) if f.endswith((".c", ".h"))]
    for f in os.listdir(csrc):
        for h in inc.findall(open(os.path.join(csrc, f), errors="replace").read()):
            assert "oracle" not in h and os.path.basename(h) not in oracle_c, (f, h)
    for f in oracle_c:
        for h in inc.findall(open(os.path.join(ORACLE, f)).read()):
            assert os.path.basename(h) not in cuda_names and "sld.h" not in h, (f, h)
