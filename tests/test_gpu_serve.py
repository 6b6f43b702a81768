"""Serving (row A12): served programs admitted by ring and heap memory, run
concurrently on separate streams, compared with the serial C oracle and with
themselves run alone.

Per program: the final vector bit-exact (CSR order, no contraction on either
side); the fwrite record multiset byte-identical; printf lines identical as
a multiset; getenv results exact (one variable unset -> -1); clock values
non-decreasing from pass to pass; fwrite / printf return values exact.

Scale: the small case runs 6 programs; the serving-scale cases run 64
programs with 16 instances and 4 host server threads (n = 2^17 rows, 10
passes, about 64 requests per pass), a quota-limited pool that must refuse
admissions (GF_EBUSY) with 8 server threads, so that every DMA lane carries
in-region fwrites, and 8 programs at the full 2^20 rows x 10 passes."""
import os
import struct
import subprocess
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

from paper_2306_11686_gb300 import inputs

pytestmark = pytest.mark.gpu
PASSES, RPP = 10, 64


def records(path):
    b = open(path, "rb").read()
    out, k = [], 0
    while k < len(b):
        prog, r, row, size = struct.unpack_from("<4I", b, k)
        out.append(b[k:k + 16 + size])
        k += 16 + size
    assert k == len(b)
    return sorted(out)


def run_oracle(oracle_bin, d, pr):
    """The serial C program on program pr's inputs: (y, records, lines, results)."""
    p, n = pr.p, pr.n
    rowptr, col, val, x0, req = inputs.serve_program_inputs(p, n=n, passes=pr.passes, req_per_pass=pr.rpp)
    tag = f"{p}_{n}"
    for name, a in [("rp", rowptr), ("c", col), ("v", val), ("x", x0), ("q", req)]:
        inputs.write_raw(d / f"{name}{tag}.bin", a)
    out = subprocess.run([oracle_bin("spmv_serve"), str(p), str(pr.passes), str(n), str(len(col)), str(len(req) // 2),
                          d / f"rp{tag}.bin", d / f"c{tag}.bin", d / f"v{tag}.bin", d / f"x{tag}.bin",
                          d / f"q{tag}.bin", d / f"y{tag}.bin", d / f"rec{tag}.bin", d / f"res{tag}.bin"],
                         capture_output=True, text=True, check=True).stdout
    want = (np.fromfile(d / f"y{tag}.bin"), records(d / f"rec{tag}.bin"), sorted(out.splitlines()),
            np.fromfile(d / f"res{tag}.bin", dtype=np.int64), req)
    for name in ("rp", "c", "v", "x", "q", "y", "rec", "res"):
        os.remove(d / f"{name}{tag}.bin")
    return want


def oracles(oracle_bin, d, progs):
    with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4)) as ex:
        return list(ex.map(lambda pr: run_oracle(oracle_bin, d, pr), progs))


def check_program(pr, want, got_rec_path, lines):
    y, rec, out, res, req = want
    assert np.array_equal(pr.x.cpu().numpy(), y), f"program {pr.p}: final vector"
    assert records(got_rec_path) == rec, f"program {pr.p}: fwrite records"
    mine = sorted(l for l in lines if l.startswith(f"p {pr.p} "))
    assert mine == out, f"program {pr.p}: printf lines"
    r = pr.res.cpu().numpy()[:pr.nreq]
    kind = req[1::2] & 0xFF
    exact = kind != 2
    assert np.array_equal(r[exact], res[exact]), f"program {pr.p}: request results"
    passes = req[0::2] >> 32
    clocks = [(passes[q], r[q]) for q in range(pr.nreq) if kind[q] == 2]
    for a in clocks:
        for b in clocks:
            if a[0] < b[0]:
                assert a[1] <= b[1]


def set_env():
    os.environ["GF_SERVE_VAR0"] = "zero"
    os.environ["GF_SERVE_VAR1"] = "one-1"
    os.environ.pop("GF_SERVE_VAR2", None)


def run_and_check(serve, progs, wants, tmp_path, label, **kw):
    for pr in progs:
        pr.reset()
    outs = [str(tmp_path / f"{label}_rec{k}.bin") for k in range(len(progs))]
    recs, agg = serve.serve(progs, outs, stdout_path=str(tmp_path / f"{label}_out.txt"), **kw)
    assert all(r["rc"] == 0 and r["exit"] == 0 and r["heap_fail"] == 0 and r["error"] == 0 for r in recs), recs
    lines = open(tmp_path / f"{label}_out.txt").read().splitlines()
    for k, pr in enumerate(progs):
        check_program(pr, wants[k], outs[k], lines)
        os.remove(outs[k])
    return recs, agg


def test_serving_alone_and_mixed(gf_lib, oracle_bin, tmp_path):
    from paper_2306_11686_gb300 import serve
    set_env()
    progs = [serve.Program(p, 20000, 3, 12) for p in range(6)]
    wants = oracles(oracle_bin, tmp_path, progs)
    recs, agg = run_and_check(serve, progs, wants, tmp_path, "alone", max_concurrent=1, heap_bytes=256 << 20,
                              ring_slots=256, server_threads=2)
    assert agg["max_overlap"] == 1
    recs, agg = run_and_check(serve, progs, wants, tmp_path, "mix", max_concurrent=3, heap_bytes=256 << 20,
                              ring_slots=256, server_threads=2)
    assert agg["programs"] == 6


def test_serving_64_programs_16_instances(gf_lib, oracle_bin, tmp_path):
    """64 programs through 16 instances and 4 server threads: every result
    equals the oracle's, and programs' device intervals overlap."""
    from paper_2306_11686_gb300 import serve
    set_env()
    progs = [serve.Program(p, 1 << 17, PASSES, RPP) for p in range(64)]
    wants = oracles(oracle_bin, tmp_path, progs)
    recs, agg = run_and_check(serve, progs, wants, tmp_path, "s64", max_concurrent=16, heap_bytes=128 << 20,
                              ring_slots=1024, server_threads=4)
    assert agg["programs"] == 64
    assert agg["max_overlap"] >= 2, agg            # continuous batching: work overlaps on the device


def test_serving_admission_by_heap_and_ring_quota(gf_lib, oracle_bin, tmp_path):
    """Programs ask for different heap and ring quotas from pools that cannot
    hold them all at once: the runtime must refuse some launches (GF_EBUSY)
    although instances are free, and every refused program must run later
    with results equal to the oracle's and to its run alone."""
    from paper_2306_11686_gb300 import serve
    set_env()
    P = 24
    progs = [serve.Program(p, 1 << 17, PASSES, RPP) for p in range(P)]
    wants = oracles(oracle_bin, tmp_path, progs)
    quotas = [((128 if k % 3 else 384) << 20, 256 if k % 2 else 1024) for k in range(P)]
    recs, agg = run_and_check(serve, progs, wants, tmp_path, "quota", max_concurrent=16, heap_bytes=128 << 20,
                              ring_slots=256, server_threads=8, quotas=quotas, heap_pool_bytes=1 << 30,
                              ring_pool_slots=4096)
    assert agg["admission_refusals"] >= 1, agg
    refused = [r for r in recs if r["refused"] > 0]
    assert refused                                   # those were checked against the oracle above
    for r in recs:
        hq, rq = quotas[r["program"]]
        assert r["heap_quota"] == hq and r["ring_quota"] == rq
    # never more admitted at once than the pools hold
    ev = sorted([(r["t_start_ns"], 1, r["program"]) for r in recs] + [(r["t_end_ns"], -1, r["program"]) for r in recs])
    heap = ring = 0
    for _, d, k in ev:
        heap += d * quotas[k][0]
        ring += d * quotas[k][1]
        assert heap <= 1 << 30 and ring <= 4096
    # alone: the same results as in the mix
    alone = [progs[r["program"]] for r in refused[:2]]
    run_and_check(serve, alone, [wants[pr.p] for pr in alone], tmp_path, "quota_alone", max_concurrent=1,
                  heap_bytes=384 << 20, ring_slots=1024, server_threads=8)


def test_serving_full_size_subset(gf_lib, oracle_bin, tmp_path):
    """8 programs at the full 2^20 rows x 16 nnz x 10 passes, 8 at once."""
    from paper_2306_11686_gb300 import serve
    set_env()
    progs = [serve.Program(p, 1 << 20, PASSES, RPP) for p in range(8)]
    wants = oracles(oracle_bin, tmp_path, progs)
    recs, agg = run_and_check(serve, progs, wants, tmp_path, "full", max_concurrent=8, heap_bytes=256 << 20,
                              ring_slots=1024, server_threads=4)
    assert agg["max_overlap"] >= 2, agg
