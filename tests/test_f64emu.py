"""The integer-pipe binary64 square, product, sum, square root, reciprocal and
power-of-two scaling (csrc/ngb_f64emu.cuh) against the host's IEEE 754 multiply,
add, divide and square root, on random and structured operands (ties, carries,
exponent limits, subnormal results, zeros, exact squares, perturbed Newton
starting points).  The header is plain C++ on the
host; the device build uses the same source."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1606_06508_gb300", "csrc")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("f64emu") / "f64emu_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC,
                    os.path.join(HERE, "f64emu_check.cpp"), "-o", exe], check=True)
    return exe


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_square_and_sum_match_ieee(checker, seed):
    out = subprocess.run([checker, "3000000", str(seed)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    rows = {line.split()[0]: [int(v) for v in line.split()[1:]] for line in out.stdout.splitlines()}
    cases, taken, bad = rows["square"]
    assert bad == 0 and taken > cases // 3
    cases, taken, bad = rows["mul"]
    assert bad == 0 and taken > cases // 2
    cases, taken, bad = rows["mul_signed"]
    assert bad == 0 and taken > cases // 2
    cases, taken, bad = rows["add"]
    assert bad == 0 and taken > cases // 2
    cases, taken, bad = rows["add_signed"]
    assert bad == 0 and taken == cases
    cases, taken, bad = rows["sqrt"]
    assert bad == 0 and taken == cases
    cases, taken, bad = rows["rcp"]
    assert bad == 0 and taken > cases * 9 // 10
    cases, taken, bad = rows["ldexp"]
    assert bad == 0 and taken == cases
