"""Batching of many independent loops (row A10): the plain runtime (one region
per loop), ONE batched region (warps pull (loop, chunk) items; static and
dynamic item schedules), and the CUDA-graph form (one kernel node per loop).
All must give z bit-exact equal to the serial C oracle (two roundings, no
contraction on either side).  The loops_rpc cases add libc to the bodies
(a heap block and a printf every 4096 iterations, all loops sharing one
ring), with launch shapes picked by the project's autotuner."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from paper_2306_11686_gb300 import inputs

pytestmark = pytest.mark.gpu


def oracle_z(oracle_bin, tmp_path, trips, a, off, x, y, z_in):
    total = len(x)
    for name, arr in [("t", trips), ("a", a), ("o", off), ("x", x), ("y", y), ("z", z_in)]:
        inputs.write_raw(tmp_path / f"{name}.bin", arr)
    subprocess.run([oracle_bin("loops"), str(len(trips)), tmp_path / "t.bin", tmp_path / "a.bin", tmp_path / "o.bin",
                    tmp_path / "x.bin", tmp_path / "y.bin", tmp_path / "z.bin", tmp_path / "zo.bin", str(total)],
                   check=True)
    return np.fromfile(tmp_path / "zo.bin", dtype=np.float64)


@pytest.fixture(scope="module")
def small_case():
    trips, a, off, x, y = inputs.loops_inputs(n=37, seed=5, lo=1, hi=1 << 14)
    trips[3] = 0                                       # an empty loop
    off[1:] = np.cumsum(trips)[:-1]
    total = int(trips.sum())
    return trips, a, off, x[:total].copy(), y[:total].copy()


@pytest.mark.parametrize("mode,chunk,sched", [(0, 1, 0), (1, 64, 1), (1, 2048, 1), (1, 100, 0), (1, 1, 1)])
def test_loops_program_parity(gf_lib, oracle_bin, tmp_path, small_case, mode, chunk, sched):
    import torch
    gf = gf_lib
    trips, a, off, x, y = small_case
    z_in = np.full(len(x), -7.0)
    want = oracle_z(oracle_bin, tmp_path, trips, a, off, x, y, z_in)
    dv = lambda v: torch.from_numpy(np.ascontiguousarray(v)).cuda()
    z = dv(z_in)
    prefix = torch.zeros(len(trips) + 1, dtype=torch.int64, device="cuda")
    with gf.Context(timeout_ns=10_000_000_000, heap_bytes=64 << 20) as c:
        rc, ec = c.run("loops", [mode, len(trips), chunk, sched],
                       [(dv(trips), 1), (dv(a), 1), (dv(off), 1), (dv(x), 1), (dv(y), 1), (z, 1), (prefix, 1)])
        st = c.stats()
    assert ec == 0
    assert np.array_equal(z.cpu().numpy(), want)
    assert st.regions == (int((trips > 0).sum()) if mode == 0 else 1)


def test_loops_graph_parity(gf_lib, oracle_bin, tmp_path, small_case):
    import torch
    gf = gf_lib
    trips, a, off, x, y = small_case
    z_in = np.zeros(len(x))
    want = oracle_z(oracle_bin, tmp_path, trips, a, off, x, y, z_in)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    z = torch.from_numpy(z_in).cuda()
    grid = np.array([1 + (k % 5) for k in range(len(trips))], dtype=np.uint32)   # odd shapes on purpose
    block = np.array([32 * (1 + k % 8) for k in range(len(trips))], dtype=np.uint32)
    ms = ctypes.c_float()
    P = lambda arr: ctypes.c_void_p(arr.ctypes.data)
    rc = gf.gf_axpy_batch_graph(len(trips), P(trips), P(a), P(off), ctypes.c_void_p(xd.data_ptr()),
                                ctypes.c_void_p(yd.data_ptr()), ctypes.c_void_p(z.data_ptr()), P(grid), P(block),
                                3, None, ctypes.byref(ms))
    assert rc == 0 and ms.value > 0
    torch.cuda.synchronize()
    assert np.array_equal(z.cpu().numpy(), want)


def test_loops_256_full_size(gf_lib, oracle_bin, tmp_path):
    """The 256-loop batch at its full size (trip counts 2^10..2^22), batched region."""
    import torch
    gf = gf_lib
    trips, a, off, x, y = inputs.loops_inputs()
    z_in = np.zeros(len(x))
    want = oracle_z(oracle_bin, tmp_path, trips, a, off, x, y, z_in)
    dv = lambda v: torch.from_numpy(np.ascontiguousarray(v)).cuda()
    z = dv(z_in)
    prefix = torch.zeros(len(trips) + 1, dtype=torch.int64, device="cuda")
    with gf.Context(timeout_ns=20_000_000_000, heap_bytes=64 << 20) as c:
        rc, ec = c.run("loops", [1, 256, 4096, 1],
                       [(dv(trips), 1), (dv(a), 1), (dv(off), 1), (dv(x), 1), (dv(y), 1), (z, 1), (prefix, 1)])
    assert ec == 0
    assert np.array_equal(z.cpu().numpy(), want)


# ------------------------------------------------------------------ loops that call libc
def oracle_rpc(oracle_bin, tmp_path, trips, a, off, x, y, z_in):
    """z and the printed lines of the serial program (oracle/loops_rpc.c)."""
    total = len(x)
    for name, arr in [("t", trips), ("a", a), ("o", off), ("x", x), ("y", y), ("z", z_in)]:
        inputs.write_raw(tmp_path / f"{name}.bin", arr)
    out = subprocess.run([oracle_bin("loops_rpc"), str(len(trips)), tmp_path / "t.bin", tmp_path / "a.bin",
                          tmp_path / "o.bin", tmp_path / "x.bin", tmp_path / "y.bin", tmp_path / "z.bin",
                          tmp_path / "zo.bin", str(total)], check=True, capture_output=True, text=True).stdout
    return np.fromfile(tmp_path / "zo.bin", dtype=np.float64), sorted(out.splitlines())


def run_loops_rpc(gf, tmp_path, trips, a, off, x, y, z_in, argv, label, server_threads=4):
    import torch
    dv = lambda v: torch.from_numpy(np.ascontiguousarray(v)).cuda()
    z = dv(z_in)
    fails = torch.zeros(1, dtype=torch.int64, device="cuda")
    prefix = torch.zeros(len(trips) + 1, dtype=torch.int64, device="cuda")
    out = tmp_path / f"{label}.txt"
    with gf.Context(timeout_ns=20_000_000_000, heap_bytes=1 << 30, server_threads=server_threads,
                    stdout_path=out) as c:
        rc, ec = c.run("loops_rpc", argv, [(dv(trips), 1), (dv(a), 1), (dv(off), 1), (dv(x), 1), (dv(y), 1), (z, 1),
                                           (prefix, 1), (fails, 1)])
        st = c.stats()
    assert ec == 0
    return z.cpu().numpy(), sorted(open(out).read().splitlines()), int(fails.item()), st


@pytest.mark.parametrize("mode,chunk,sched", [(0, 1, 0), (1, 4096, 1), (1, 1000, 0), (1, 64, 1)])
def test_loops_rpc_program_parity(gf_lib, oracle_bin, tmp_path, small_case, mode, chunk, sched):
    """Loops whose bodies print and use heap blocks: z bit-exact, the printed
    lines equal to the serial program's as a multiset (iterations of one loop
    run concurrently, so their order is not defined), no heap failure."""
    trips, a, off, x, y = small_case
    z_in = np.full(len(x), -7.0)
    want_z, want_lines = oracle_rpc(oracle_bin, tmp_path, trips, a, off, x, y, z_in)
    z, lines, fails, st = run_loops_rpc(gf_lib, tmp_path, trips, a, off, x, y, z_in,
                                        [mode, len(trips), chunk, sched], f"m{mode}")
    assert np.array_equal(z, want_z)
    assert lines == want_lines
    assert fails == 0 and st.heap_fail == 0 and st.heap_alloc == len(want_lines) == st.heap_free


def test_loops_rpc_256_full_size_tuned(gf_lib, oracle_bin, tmp_path):
    """The 256-loop batch at full size (trip 2^10..2^22) with its RPC and heap
    traffic: the autotuner picks the batched region's chunk and schedule, and
    per-loop grid and block for the graph form; every form gives the serial
    program's z and lines."""
    import torch
    from paper_2306_11686_gb300 import tune
    gf = gf_lib
    trips, a, off, x, y = inputs.loops_inputs()
    z_in = np.zeros(len(x))
    want_z, want_lines = oracle_rpc(oracle_bin, tmp_path, trips, a, off, x, y, z_in)
    dv = lambda v: torch.from_numpy(np.ascontiguousarray(v)).cuda()
    td, ad, od, xd, yd = dv(trips), dv(a), dv(off), dv(x), dv(y)
    zd = dv(z_in)
    fails = torch.zeros(1, dtype=torch.int64, device="cuda")
    prefix = torch.zeros(len(trips) + 1, dtype=torch.int64, device="cuda")
    bufs = [(td, 1), (ad, 1), (od, 1), (xd, 1), (yd, 1), (zd, 1), (prefix, 1), (fails, 1)]
    with gf.Context(timeout_ns=30_000_000_000, heap_bytes=1 << 30, server_threads=4, stdout_path=os.devnull) as c:
        (chunk, sched), table = tune.tune_batch(c, bufs, len(trips), reps=1)
        sms = c.grid_info("loops_rpc")[0]
        grid, block, _, _ = tune.tune_graph(c, trips, a, off, xd, yd, zd, fails, sms, reps=1)
    assert f"{chunk}/{sched}" in table and grid.min() >= 1 and block.max() <= 256
    z, lines, nf, st = run_loops_rpc(gf, tmp_path, trips, a, off, x, y, z_in, [1, len(trips), chunk, sched], "tuned")
    assert np.array_equal(z, want_z)
    assert lines == want_lines
    assert nf == 0 and st.heap_fail == 0
    # graph form with the tuned shapes, once
    zd.copy_(torch.from_numpy(z_in))
    fails.zero_()
    P = lambda arr: ctypes.c_void_p(arr.ctypes.data)
    out = tmp_path / "graph.txt"
    with gf.Context(timeout_ns=30_000_000_000, heap_bytes=1 << 30, server_threads=4, stdout_path=out) as c:
        rc = gf.gf_loops_rpc_graph(c.h, len(trips), P(trips), P(a), P(off), ctypes.c_void_p(xd.data_ptr()),
                                   ctypes.c_void_p(yd.data_ptr()), ctypes.c_void_p(zd.data_ptr()),
                                   ctypes.c_void_p(fails.data_ptr()), P(grid), P(block), 1, 0, None, None)
    assert rc == gf.GF_OK
    assert np.array_equal(zd.cpu().numpy(), want_z)
    assert sorted(open(out).read().splitlines()) == want_lines
    assert fails.item() == 0
