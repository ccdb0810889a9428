"""The pins must catch plausible mistakes in the oracle.  Each case plants one
mistake in a copy of the oracle's C source (a dropped term, a wrong
comparison, a swapped constant, a wrong sign, a transposed operand, a skipped
rounding step, the literal reading of Algorithm 7, misplaced outputs of the
quotient algorithms), builds it, and runs the pin suites against it in a
subprocess: they have to fail.  CPU only."""
import os
import shutil
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
ORACLE = os.path.join(ROOT, "oracle")

# (name, file, text in the oracle, replacement)
MUTANTS = [
    ("Algorithm 6 drops the third square", "oracle_impl.h",
     "REAL rt = SQRT(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);", "REAL rt = SQRT(t[0] * t[0] + t[1] * t[1]);"),
    ("Scale2D compares m > tau_min", "oracle_impl.h",
     "    if (m >= TAU_MIN) {\n        if (m <= TAU_MAX) { *sigma = 1; t[0] = x1; t[1] = x2; return OR_CODE_ONE; }",
     "    if (m > TAU_MIN) {\n        if (m <= TAU_MAX) { *sigma = 1; t[0] = x1; t[1] = x2; return OR_CODE_ONE; }"),
    ("Scale3D scales large vectors by sigma_min", "oracle_impl.h",
     "t[0] = SIGMA_MAX * x1; t[1] = SIGMA_MAX * x2; t[2] = SIGMA_MAX * x3;",
     "t[0] = SIGMA_MIN * x1; t[1] = SIGMA_MIN * x2; t[2] = SIGMA_MIN * x3;"),
    ("Algorithm 7 read literally (m <- |x4| without the Else)", "oracle_impl.h",
     "            } else {\n                m = FABS(x4);\n            }",
     "            }\n            m = FABS(x4);"),
    ("Normalize2D divides instead of multiplying by h", "oracle_impl.h",
     "    y[0] = h * t[0];\n    y[1] = h * t[1];\n    *hout = h;",
     "    y[0] = t[0] / rt;\n    y[1] = t[1] / rt;\n    *hout = h;"),
    ("Normalize3D returns the scaled norm", "oracle_impl.h",
     "    *r = sigma * rt;\n    y[0] = h * t[0];\n    y[1] = h * t[1];\n    y[2] = h * t[2];",
     "    *r = rt;\n    y[0] = h * t[0];\n    y[1] = h * t[1];\n    y[2] = h * t[2];"),
    ("CR(n) drops the second term of each slot", "oracle_impl.h",
     "for (int64_t k = j + OR_CR_SLOTS; k < n; k += OR_CR_SLOTS)",
     "for (int64_t k = j + 2 * OR_CR_SLOTS; k < n; k += OR_CR_SLOTS)"),
    ("CR(n) tree stops one level early", "oracle_impl.h",
     "for (int64_t s = OR_CR_SLOTS / 2; s >= 1; s /= 2)", "for (int64_t s = OR_CR_SLOTS / 2; s >= 2; s /= 2)"),
    ("backward adds y_k dot instead of subtracting", "oracle_impl.h",
     "REAL tk = g[k] - y[k] * dot;", "REAL tk = g[k] + y[k] * dot;"),
    ("rotation matrix with a transposed operand", "oracle_impl.h",
     "R[1] = 2 * (q1 * q2 - q3 * q4);", "R[1] = 2 * (q1 * q3 - q2 * q4);"),
    ("Algorithm 2 with pivot x1 writes its outputs to the wrong places", "oracle_impl.h",
     "else SFX(quotient2_pivot)(x1, x3, x2, r, &y[0], &y[2], &y[1]);",
     "else SFX(quotient2_pivot)(x1, x3, x2, r, &y[2], &y[0], &y[1]);"),
    ("Algorithm 2 drops the sign of the pivot", "oracle_impl.h",
     "REAL s = COPYSIGN((REAL)1, xp) / h;", "REAL s = 1 / h;"),
    ("Algorithm 1 divides the scaled components by r", "oracle_impl.h",
     "    y[0] = x[0] / rr;\n    y[1] = x[1] / rr;\n    y[2] = x[2] / rr;",
     "    y[0] = t1 / rr;\n    y[1] = t2 / rr;\n    y[2] = t3 / rr;"),
]


@pytest.fixture(scope="module")
def cc():
    c = shutil.which("gcc")
    if c is None:
        pytest.skip("no C compiler")
    import oracle
    return c, oracle.CFLAGS


@pytest.mark.parametrize("name,fname,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(cc, tmp_path, name, fname, old, new):
    compiler, cflags = cc
    for f in ("normalize_oracle.c", "oracle_impl.h"):
        shutil.copy(os.path.join(ORACLE, f), tmp_path / f)
    path = tmp_path / fname
    text = path.read_text()
    assert text.count(old) == 1, f"mutation site not unique or missing: {name}"
    path.write_text(text.replace(old, new))
    lib = str(tmp_path / "liboracle_mutant.so")
    subprocess.run([compiler, *cflags, str(tmp_path / "normalize_oracle.c"), "-o", lib, "-lm"], check=True)
    env = dict(os.environ, NGB_ORACLE_LIB=lib)
    out = subprocess.run([sys.executable, "-m", "pytest", os.path.join(HERE, "test_oracle_pins.py"),
                          os.path.join(HERE, "test_oracle_quotient_pins.py"), "-x", "-q", "-p", "no:cacheprovider",
                          "-k", "not full_exponent_grid and not whole_config0"],  # the long bound sweeps: ~15 s each
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode != 0, f"the pins did not catch: {name}\n{out.stdout[-2000:]}"
