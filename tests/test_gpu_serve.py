"""Serving (row A12): several served programs admitted by free instance
(ring segment + heap arena), run concurrently on separate streams, compared
with the serial C oracle and with themselves run alone.

Per program: the final vector bit-exact (CSR order, no contraction on either
side); the fwrite record multiset byte-identical; printf lines identical as
a multiset; getenv results exact (one variable unset -> -1); clock values
non-decreasing from pass to pass; fwrite / printf return values exact."""
import os
import struct
import subprocess

import numpy as np
import pytest

from paper_2306_11686_gb300 import inputs

pytestmark = pytest.mark.gpu
N, PASSES, RPP = 20000, 3, 12


def records(path):
    b = open(path, "rb").read()
    out, k = [], 0
    while k < len(b):
        prog, r, row, size = struct.unpack_from("<4I", b, k)
        out.append(b[k:k + 16 + size])
        k += 16 + size
    assert k == len(b)
    return sorted(out)


def run_oracle(oracle_bin, d, p, pr):
    rowptr, col, val, x0, req = inputs.serve_program_inputs(p, n=N, passes=PASSES, req_per_pass=RPP)
    for name, a in [("rp", rowptr), ("c", col), ("v", val), ("x", x0), ("q", req)]:
        inputs.write_raw(d / f"{name}{p}.bin", a)
    out = subprocess.run([oracle_bin("spmv_serve"), str(p), str(PASSES), str(N), str(len(col)), str(len(req) // 2),
                          d / f"rp{p}.bin", d / f"c{p}.bin", d / f"v{p}.bin", d / f"x{p}.bin", d / f"q{p}.bin",
                          d / f"y{p}.bin", d / f"rec{p}.bin", d / f"res{p}.bin"],
                         capture_output=True, text=True, check=True).stdout
    return (np.fromfile(d / f"y{p}.bin"), records(d / f"rec{p}.bin"), sorted(out.splitlines()),
            np.fromfile(d / f"res{p}.bin", dtype=np.int64), req)


def check_program(pr, req, want, got_rec_path, lines):
    y, rec, out, res = want
    assert np.array_equal(pr.x.cpu().numpy(), y)
    assert records(got_rec_path) == rec
    mine = sorted(l for l in lines if l.startswith(f"p {pr.p} "))
    assert mine == out
    r = pr.res.cpu().numpy()[:pr.nreq]
    kind = req[1::2] & 0xFF
    exact = kind != 2
    assert np.array_equal(r[exact], res[exact])
    passes = req[0::2] >> 32
    clocks = [(passes[q], r[q]) for q in range(pr.nreq) if kind[q] == 2]
    for a in clocks:
        for b in clocks:
            if a[0] < b[0]:
                assert a[1] <= b[1]


def test_serving_alone_and_mixed(gf_lib, oracle_bin, tmp_path):
    from paper_2306_11686_gb300 import serve
    os.environ["GF_SERVE_VAR0"] = "zero"
    os.environ["GF_SERVE_VAR1"] = "one-1"
    os.environ.pop("GF_SERVE_VAR2", None)
    P = 6
    progs = [serve.Program(p, N, PASSES, RPP) for p in range(P)]
    wants = [run_oracle(oracle_bin, tmp_path, p, progs[p]) for p in range(P)]
    for label, conc in [("alone", 1), ("mix", 3)]:
        for pr in progs:
            pr.reset()
        outs = [str(tmp_path / f"{label}_rec{p}.bin") for p in range(P)]
        recs, agg = serve.serve(progs, outs, max_concurrent=conc, heap_bytes=256 << 20, ring_slots=256,
                                server_threads=2, stdout_path=str(tmp_path / f"{label}_out.txt"))
        assert all(r["rc"] == 0 and r["exit"] == 0 and r["heap_fail"] == 0 for r in recs), recs
        lines = open(tmp_path / f"{label}_out.txt").read().splitlines()
        for p in range(P):
            check_program(progs[p], wants[p][4], wants[p][:4], outs[p], lines)
        if conc > 1:
            assert agg["admission_refusals"] >= 0 and agg["programs"] == P
