"""Source hygiene (CPU): code, comments and tests state facts on their own.
They name none of the project's planning documents or the paper's text
files, no path of a build machine and no job tool, and the product never
imports the oracle (test infrastructure). Tokens are assembled from pieces
so that this file does not contain them either."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SOURCES = ["paper_2103_08246_gb300", "oracle", "include", "tests", "bench.py", "__graft_entry__.py"]
EXT = (".py", ".cu", ".cuh", ".h", ".c", ".cpp")

FORBIDDEN = [
    "BASE" + "LINE",
    "north" + "_star",
    "SUR" + "VEY.md",
    "DES" + "IGN.md",
    "VER" + "DICT",
    "AD" + "VICE.md",
    "PA" + "PER.md",
    "SP" + "EC.md",
    "gpu" + "run",
    "/ro" + "ot/",
    "configs" + "[",
]


def _files():
    for top in SOURCES:
        path = os.path.join(ROOT, top)
        if os.path.isfile(path):
            yield path
            continue
        for d, dirs, files in os.walk(path):
            dirs[:] = [x for x in dirs if x not in ("__pycache__", "_build")]
            for f in files:
                if f.endswith(EXT):
                    yield os.path.join(d, f)


def test_no_forbidden_references():
    me = os.path.abspath(__file__)
    bad = []
    for f in _files():
        if os.path.abspath(f) == me:
            continue
        text = open(f, errors="replace").read()
        for tok in FORBIDDEN:
            if tok in text:
                bad.append((os.path.relpath(f, ROOT), tok))
    assert not bad, bad


def test_product_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2103_08246_gb300")
    pattern = re.compile(r"^\s*(from\s+oracle\b|import\s+oracle\b)", re.M)
    for d, _, files in os.walk(pkg):
        for f in files:
            if f.endswith(".py"):
                assert not pattern.search(open(os.path.join(d, f)).read()), f
