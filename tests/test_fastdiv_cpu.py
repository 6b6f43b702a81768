"""gf_div6_int (division by 6 on the integer pipe) equals IEEE x / 6.0 bit
for bit, checked on the CPU (the header compiles for host and device)."""
import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_div6_int_matches_ieee_on_cpu(tmp_path):
    exe = str(tmp_path / "div6_check")
    subprocess.run(["nvcc", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2306_11686_gb300", "csrc"),
                    "-x", "cu", os.path.join(ROOT, "tests", "host", "div6_check.cu"), "-o", exe],
                   check=True, capture_output=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300).stdout
    assert out.strip().endswith("mismatches 0"), out
