"""The C-ABI library builds, loads and exports every entry point declared in include/*.h, and the
Python binding declares a signature for each (no compute calls: runs without a GPU)."""
import glob
import os
import re

from paper_2310_08408_gb300 import build, xl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = []
    for h in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(xl_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = xl.load(path)
    names = declared()
    assert "xl_rs_propagate" in names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"
        assert n in xl.SIGNATURES, f"{n} has no ctypes signature in the binding"
    assert set(xl.SIGNATURES) <= set(names)
    assert xl.version().startswith("xl ")


def test_oracle_and_library_share_no_source():
    """The oracle neither includes nor links the CUDA sources (and vice versa)."""
    orc = open(os.path.join(ROOT, "oracle", "xl_oracle.cpp")).read()
    assert "csrc" not in orc and "xl.h" not in orc
    for f in glob.glob(os.path.join(ROOT, "paper_2310_08408_gb300", "csrc", "*")):
        src = open(f).read()
        assert not re.search(r"#\s*include\s*[<\"][^>\"]*oracle", src), f
    for f in glob.glob(os.path.join(ROOT, "paper_2310_08408_gb300", "*.py")):
        src = open(f).read()
        assert not re.search(r"^\s*(import|from)\s+oracle", src, flags=re.M), f


def test_binding_calls_match_signatures():
    """Every call the binding makes to an entry point passes as many arguments as its ctypes
    signature declares (checked on the source, no GPU needed)."""
    import ast
    src = open(os.path.join(ROOT, "paper_2310_08408_gb300", "xl.py")).read()
    bad = []
    for node in ast.walk(ast.parse(src)):
        if (isinstance(node, ast.Call) and isinstance(node.func, ast.Attribute)
                and node.func.attr in xl.SIGNATURES
                and not any(isinstance(a, ast.Starred) for a in node.args)):
            if len(node.args) != len(xl.SIGNATURES[node.func.attr][0]):
                bad.append((node.func.attr, node.lineno))
    assert not bad, bad
