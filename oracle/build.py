"""Builds the C oracles (test infrastructure only: tests/, __graft_entry__ and
bench.py's cpu_baseline leg are the only callers).

Each oracle is plain C11 compiled with ``-O2 -ffp-contract=off`` so that a
product and a following sum round separately, as in the C abstract machine.
Binaries land in ``oracle/_build/``.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "_build")
SOURCES = ["axpy_sum", "jacobi", "exact_sum", "stress", "spmv_serve", "loops", "loops_rpc", "synth"]
CFLAGS = ["-O2", "-std=gnu11", "-ffp-contract=off", "-Wall", "-Wno-unknown-pragmas"]


def binary(name: str) -> str:
    return os.path.join(OUT, name)


def build(force: bool = False) -> None:
    os.makedirs(OUT, exist_ok=True)
    procs = []
    for name in SOURCES:
        src = os.path.join(HERE, name + ".c")
        if not os.path.exists(src):
            continue
        out = binary(name)
        if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
            continue
        procs.append((name, subprocess.Popen(["gcc", *CFLAGS, "-o", out, src, "-lm"],
                                             stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    # the same Jacobi source built with OpenMP: a timed all-core CPU baseline
    # (bench.py), never a parity reference
    src = os.path.join(HERE, "jacobi.c")
    out = binary("jacobi_omp")
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        procs.append(("jacobi_omp", subprocess.Popen(["gcc", *CFLAGS, "-fopenmp", "-o", out, src, "-lm"],
                                                     stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    for name, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            raise RuntimeError(f"oracle {name} failed to build:\n{out.decode()}")


if __name__ == "__main__":
    build(force="--force" in sys.argv)
