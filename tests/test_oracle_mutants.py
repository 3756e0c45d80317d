"""The oracle pins must reject plausible mistakes planted in the oracle.

Each mutant is a copy of oracle/oracle.c with one textual change (a dropped
strictness test, a ceiling instead of a floor, a transposed operand, a reversed
scan, a wrong partition weight), compiled on the CPU and loaded through
GRES_ORACLE_LIB; the pin suite must fail against every one of them.
"""
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTANTS = {
    "no_strictness": ("return strictly_better_somewhere;", "return 1;"),
    "ceil_projection": ("for (int i = 0; i < d; i++) q[i] = t[i] / delta;",
                        "for (int i = 0; i < d; i++) q[i] = (uint32_t)(((uint64_t)t[i] + delta - 1) / delta);"),
    "transposed": ("if (oracle_dominates(qs, qt, d, dir)) { result = k; break; }",
                   "if (oracle_dominates(qt, qs, d, dir)) { result = k; break; }"),
    "descending_scan": ("for (int32_t k = 0; k < K && result == K; k++) {\n            project(t, d, steps[k], qt);",
                        "for (int32_t kk = K - 1, k = kk; kk >= 0 && result == K; kk--, k = kk) {\n            project(t, d, steps[k], qt);"),
    "last_not_first": ("for (int32_t k = 0; k < K && result == K; k++) {\n            project(t, d, steps[k], qt);",
                       "for (int32_t k = 0; k < K; k++) {\n            project(t, d, steps[k], qt);"),
    "grid_weight": ("p += (int64_t)c * w;\n            w *= m;", "p += (int64_t)c * w;\n            w *= m + 1;"),
    "bnl_keeps_dominated": ("if (oracle_dominates(data + win[j] * d, tx, d, dir)) { dominated = 1; break; }",
                            "if (0) { dominated = 1; break; }"),
}


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_reject_mutant(name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor for {name} not found"
    src = src.replace(old, new)
    with tempfile.TemporaryDirectory() as tmp:
        c = os.path.join(tmp, "mut.c")
        so = os.path.join(tmp, "libmut.so")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", c, "-o", so, "-lm"],
                       check=True, capture_output=True)
        env = dict(os.environ, GRES_ORACLE_LIB=so)
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                            os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
        assert r.returncode != 0, f"pins accepted mutant {name}:\n{r.stdout[-2000:]}"
