"""The oracle and the CUDA path share no code and neither uses the other: checked
on the sources.  Only the seeded input generators (paper_1111_3297_gb300/
workloads.py, no sieve arithmetic) may serve both, and the oracle does not need them."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1111_3297_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def sources(top, exts):
    for d, dirs, files in os.walk(top):
        dirs[:] = [x for x in dirs if not x.startswith(("_", "."))]
        for f in files:
            if f.endswith(exts):
                yield os.path.join(d, f)


def test_product_never_uses_the_oracle():
    pat = re.compile(r"^\s*(import\s+oracle|from\s+oracle\b)|#\s*include\s*[<\"].*oracle", re.M)
    bad = [p for p in sources(PKG, (".py", ".cu", ".cuh", ".h", ".c", ".cpp")) if pat.search(open(p).read())]
    assert not bad, bad
    # the library build compiles only its own sources
    from paper_1111_3297_gb300 import build
    text = open(build.__file__).read()
    assert "oracle" not in text


def test_oracle_never_uses_the_product():
    pat = re.compile(r"paper_1111_3297_gb300|gbsieve|csrc|sieve_internal", re.M)
    bad = [p for p in sources(ORACLE, (".py", ".c", ".h")) if pat.search(open(p).read())]
    assert not bad, bad


def test_shared_input_module_holds_no_sieve_arithmetic():
    text = open(os.path.join(PKG, "workloads.py")).read()
    code = re.sub(r'""".*?"""', "", text, flags=re.S)
    code = "\n".join(ln.split("#")[0] for ln in code.splitlines()).lower()
    for word in ("prime", "isqrt", "barrett", "lemma", "first_hit", "atomic", "sieve"):
        assert word not in code, word
