"""Each planted mistake in a copy of the oracle must make a pin fail.

The mistakes are the plausible ones: a dropped conjugation, a transposed
index map, a wrong matrix stride, a sign error in the complex product or in
complex alpha, C read when beta = 0, and a dropped double-double term.  Each
mutant is built on the CPU from the oracle's source with one textual edit
and the oracle pins are re-run against it in a subprocess."""
from __future__ import annotations

import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "sbgemm_oracle.c")

MUTANTS = {
    "no_conj_a": ("if (opa == 2) ai = -ai;", ";"),
    "transposed_index": ("return op == 0 ? r + ld * c + ld2 * p", "return op != 0 ? r + ld * c + ld2 * p"),
    "wrong_batch_stride": ("r + ld * c + ld2 * p    /*", "r + ld * c + ld * p    /*"),
    "complex_sign": ("re = dd_add(re, dd_neg(two_prod(ai, bi)));", "re = dd_add(re, two_prod(ai, bi));"),
    "alpha_imag_sign": ("dd_neg(dd_mul_d(im, alpha[1]))", "dd_mul_d(im, alpha[1])"),
    "reads_c_when_beta_zero": ("const int read_c = !(", "const int read_c = 1 || !("),
    "dropped_dd_term": ("s.lo += t.hi;", ";"),
    # variable-size arenas addressed with a wrong element size per type
    "vbatch_es_z": ("(type == OR_Z) ? 16 : 2;", "(type == OR_Z) ? 8 : 2;"),
    "vbatch_es_16bit": ("(type == OR_Z) ? 16 : 2;", "(type == OR_Z) ? 16 : 4;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name):
    src = open(SRC).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    with tempfile.TemporaryDirectory() as td:
        c = os.path.join(td, "mut.c")
        so = os.path.join(td, "libmut.so")
        open(c, "w").write(src.replace(old, new))
        subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                        "-ffp-contract=off", c, "-o", so, "-lm"], check=True)
        env = dict(os.environ, SBGEMM_ORACLE_LIB=so)
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                            os.path.join(ROOT, "tests", "test_oracle.py")],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
        assert r.returncode != 0, f"mutant {name} passed every pin:\n{r.stdout[-2000:]}"
