"""The values arXiv 1606.06508 prints (tests/golden/, each file citing the
table, section or lemma it transcribes) against the constants the oracle pins
and the exact checks use (CPU only)."""
import math
import os
from fractions import Fraction as Fr

from oracle import exact
import test_oracle_pins as pins

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [line.split() for line in f if line.strip() and not line.lstrip().startswith("#")]


def table2():
    out = {}
    for row in _rows("table2_ieee_parameters.txt"):
        if row[0] == "u":
            out.setdefault("u_printed", {})[row[1]] = float(row[2])
        else:
            alg = [int(v) for v in row[1:5]]
            hw = [int(v) for v in row[6:10]]
            out[row[0]] = (alg, hw)
    return out


def test_table2_constants_are_the_pinned_ones():
    t = table2()
    for fmt_name, key in (("single", "f32"), ("double", "f64")):
        alg, _ = t[fmt_name]
        assert tuple(Fr(2) ** e for e in alg) == pins.TABLE2[key], fmt_name


def test_table2_hardware_columns_match_the_formats():
    """Table 2 prints u, alpha, nu and omega as powers of ten; each is within a
    factor of ten of the exact binary32/binary64 value the checks use."""
    t = table2()
    for fmt_name, fmt in (("single", exact.F32), ("double", exact.F64)):
        _, hw = t[fmt_name]
        for k, v in zip(hw, (fmt.u, fmt.alpha, fmt.nu, fmt.omega)):
            lg = (math.log2(v.numerator) - math.log2(v.denominator)) * math.log10(2)
            assert abs(lg - k) < 1, (fmt_name, k, lg)


def test_unit_roundoff_printed_in_section_2():
    t = table2()["u_printed"]
    for fmt_name, fmt in (("single", exact.F32), ("double", exact.F64)):
        assert float(f"{float(fmt.u):.1e}") == t[fmt_name], fmt_name


def test_lemma_bounds_are_the_checked_ones():
    rows = _rows("error_bounds.txt")
    assert rows
    for key, n, value in rows:
        n, v = int(n), Fr(value)
        if key == "direction":
            assert exact.direction_bound(n, exact.F64.u) == v
        elif key == "norm":
            assert exact.norm_bound(n, exact.F64.u) == v
        elif key == "sin_phi":
            assert exact.SIN_BOUND_U == v
        elif key == "pair_const":
            assert exact.PAIR_BOUND_U[0] == v
        elif key == "pair_slope":
            assert exact.PAIR_BOUND_U[1] == v
        else:
            raise AssertionError(f"unknown key {key}")
