"""The decimal fast path of the device strtod (Clinger's exact case), built
for the host and compared with the C library's strtod: same value bits and
same end pointer wherever the fast path answers; hex floats, inf/nan, long
mantissas and large exponents must be left to the library."""
import os
import re
import subprocess

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

FIXED = ["0", "-0", "+0", "1.5", "-2.25e3", "  42", "\t7", "3.14159265358979", "1e22", "1e23", "0.1", "-.5",
         "123456789012345678", "1.7976931348623157e308", "4.9e-324", "inf", "-inf", "nan", "NaN", "infinity",
         "0x1p-2", "0X10", "-0x1.8p1", "0x", "abc", "12abc", ".e1", "1e", "1e+", "1e-", "0.000123",
         "999999999999999", "1000000000000000", "9007199254740993", "5e-1", "00012.5000", "1.", "7e-22",
         "7e-23", "0e99999", "0.0e-400", "-0.0", "123456789012345e-22", "1.23456789012345e7", "12e", "1.5E+3x",
         "  -  1", "+-1", ".", "-", "", "000000000000000000000000001.5", "1.000000000000000"]
NOT_FAST = ["0x1p-2", "0X10", "-0x1.8p1", "inf", "-inf", "nan", "NaN", "infinity", "123456789012345678", "1e23",
            "7e-23", "abc", ".e1", "", "-"]


def cases():
    rng = np.random.default_rng(11)
    out = list(FIXED)
    for _ in range(20000):
        nd = int(rng.integers(1, 21))
        digits = "".join(str(int(d)) for d in rng.integers(0, 10, nd))
        dot = int(rng.integers(0, nd + 1))
        s = digits[:dot] + "." + digits[dot:] if rng.random() < 0.7 else digits
        if rng.random() < 0.6:
            s += rng.choice(["e", "E"]) + str(int(rng.integers(-30, 31)))
        if rng.random() < 0.1:
            s += rng.choice(["x", " 1", "e", ".5", "abc"])
        out.append(rng.choice(["", "-", "+", " "]) + s)
    return out


def _run(tmp_path, lines):
    exe = str(tmp_path / "strtod_check")
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2306_11686_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "host", "strtod_check.cpp"), "-o", exe], check=True,
                   capture_output=True)
    (tmp_path / "in.txt").write_text("\n".join(lines) + "\n")
    out = subprocess.run([exe, str(tmp_path / "in.txt")], capture_output=True, text=True, timeout=120).stdout
    m = re.search(r"handled (\d+) of (\d+), mismatches (\d+)", out)
    assert m, out
    return int(m.group(1)), int(m.group(2)), int(m.group(3)), out


def test_fast_path_matches_libc(tmp_path):
    lines = cases()
    handled, n, bad, out = _run(tmp_path, lines)
    assert n == len(lines) and bad == 0, out
    assert handled > n // 3, out                     # the fast path is taken for most short decimals


def test_fast_path_declines_what_it_cannot_do_exactly(tmp_path):
    for s in NOT_FAST:
        handled, n, bad, out = _run(tmp_path, [s])
        assert handled == 0, s
