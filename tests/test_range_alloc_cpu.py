"""The admission bookkeeping of the heap and ring pools (first-fit unit
ranges, host/range_alloc.h) against a brute-force bitmap model on the CPU."""
import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2306_11686_gb300", "csrc")


def test_range_alloc_matches_first_fit_model(tmp_path):
    out = str(tmp_path / "range_alloc_check")
    subprocess.run(["g++", "-std=c++17", "-O2", "-I", CSRC, os.path.join(ROOT, "tests", "host", "range_alloc_check.cpp"),
                    "-o", out], check=True)
    p = subprocess.run([out], capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stdout + p.stderr
    assert p.stdout.startswith("OK")
