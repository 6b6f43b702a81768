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


def test_jacobi_arithmetic_matches_the_serial_program(tmp_path, oracle_bin):
    """The device sweep's arithmetic (index split, boundary test, integer-pipe
    adds, /6 and |.|), built for the host, gives the serial program's output
    byte for byte at every split of the adds, on the grids the GPU parity test
    uses: unit, signed, subnormal, 2^200-scaled, constant and smooth."""
    import numpy as np
    from paper_2306_11686_gb300 import inputs
    exe = str(tmp_path / "jacobi_intpipe_check")
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-I",
                    os.path.join(ROOT, "paper_2306_11686_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "host", "jacobi_intpipe_check.cpp"), "-o", exe],
                   check=True, capture_output=True)
    n, sweeps = 37, 4
    base = inputs.jacobi_input(n, seed=9)
    x = np.sin(np.pi * np.arange(n) / (n - 1))
    kinds = {
        "unit": base,
        "signed": np.where(base != 0.0, 2.0 * base - 1.0, 0.0),
        "tiny": base * 2.0 ** -1060,
        "huge": base * 2.0 ** 200,
        "ties": np.where(base != 0.0, 0.5, 0.0),
        "smooth": np.where(base != 0.0, (x[:, None, None] * x[None, :, None] * x[None, None, :]).reshape(-1), 0.0),
    }
    for kind, g in kinds.items():
        inputs.write_f64(tmp_path / "in.bin", g)
        want = subprocess.run([oracle_bin("jacobi"), str(n), str(sweeps), str(tmp_path / "in.bin"),
                               str(tmp_path / "ref.bin")], capture_output=True, text=True, check=True).stdout
        ref = (tmp_path / "ref.bin").read_bytes()
        for k in range(6):
            got = subprocess.run([exe, str(n), str(sweeps), str(k), str(tmp_path / "in.bin"), str(tmp_path / "got.bin")],
                                 capture_output=True, text=True, check=True).stdout
            assert got == want, (kind, k)
            assert (tmp_path / "got.bin").read_bytes() == ref, (kind, k)
