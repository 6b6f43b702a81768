"""Integer-pipe FP64 helpers (correctly rounded add, fabs, division by an
invariant integer) built for the host and compared with IEEE arithmetic."""
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_intpipe_helpers_match_ieee(tmp_path):
    exe = str(tmp_path / "intpipe_check")
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-I",
                    os.path.join(ROOT, "paper_2306_11686_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "host", "intpipe_check.cpp"), "-o", exe],
                   check=True, capture_output=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300).stdout
    for name, floor in (("dadd", 4_000_000), ("fabs", 100_000), ("udiv", 4_000_000_000)):
        m = re.search(name + r" checked (\d+) mismatches (\d+)", out)
        assert m, out
        assert int(m.group(1)) >= floor and int(m.group(2)) == 0, out
