"""The host printf landing pad's to_chars fast path produces the same
characters as snprintf for every conversion it accepts."""
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_fmt_fast_matches_snprintf(tmp_path):
    exe = str(tmp_path / "fmt_check")
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2306_11686_gb300", "csrc", "host"),
                    os.path.join(ROOT, "tests", "host", "fmt_check.cpp"), "-o", exe], check=True, capture_output=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120).stdout
    m = re.search(r"fmt checked (\d+) fast (\d+) mismatches (\d+)", out)
    assert m, out
    n, fast, bad = map(int, m.groups())
    assert bad == 0 and fast > n // 2, out


def test_printf_plan_matches_snprintf(tmp_path):
    """Whole formats through the host landing pad (format cut once into
    literal runs and conversions) against one snprintf call each: flags,
    widths, '*', every length modifier, %%, %n, strings, formats that run
    out of arguments or end inside a conversion."""
    exe = str(tmp_path / "plan_check")
    csrc = os.path.join(ROOT, "paper_2306_11686_gb300", "csrc")
    subprocess.run(["g++", "-O2", "-std=c++17", "-pthread", "-w", "-I", os.path.join(ROOT, "include"), "-I", csrc,
                    os.path.join(ROOT, "tests", "host", "printf_plan_check.cpp"),
                    os.path.join(csrc, "host", "server.cpp"), "-o", exe], check=True, capture_output=True)
    p = subprocess.run([exe, str(tmp_path / "out.txt")], capture_output=True, text=True, timeout=300)
    m = re.search(r"plan checked (\d+) mismatches (\d+)", p.stdout)
    assert m, p.stdout + p.stderr
    n, bad = map(int, m.groups())
    assert p.returncode == 0 and bad == 0 and n > 20000, p.stdout
