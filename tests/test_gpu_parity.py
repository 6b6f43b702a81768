"""Parity of the GPU path against the serial C oracle, through the C ABI.

Bar (written here, per kind of result):
- printf text, written files, integer/index results: bit-exact;
- elementwise FP64 (axpy y, Jacobi grid, residuals): bit-exact, since both
  sides evaluate the same expression with no contraction (oracle built with
  -ffp-contract=off, device code with --fmad=false) and IEEE division;
- FP64 sums: |gpu - oracle| <= 1e-12 |oracle|, and |gpu - exact| <= 2 eps sum|y|
  against the exactly rounded sum.
stdout is compared as a multiset of lines (OpenMP leaves the interleaving of
output from different threads unspecified).
"""
import os
import subprocess

import numpy as np
import pytest

from paper_2306_11686_gb300 import inputs

pytestmark = pytest.mark.gpu
EPS = 2.0 ** -52


def oracle(oracle_bin, name, *args):
    p = subprocess.run([oracle_bin(name), *map(str, args)], capture_output=True, text=True)
    assert p.returncode == 0, p.stderr
    return p.stdout


def split_sum(lines):
    body = sorted(l for l in lines if not l.startswith("sum "))
    s = [float(l.split()[1]) for l in lines if l.startswith("sum ")]
    return body, s


@pytest.mark.parametrize("n", [0, 1, 1023, 1025, 5000 + 17, 1 << 20])
def test_axpy_sum_parity(gf_lib, oracle_bin, tmp_path, n):
    import torch
    gf = gf_lib
    x, y = inputs.axpy_inputs(n, seed=1)
    inputs.write_f64(tmp_path / "x.bin", x)
    inputs.write_f64(tmp_path / "y.bin", y)
    want = oracle(oracle_bin, "axpy_sum", n, tmp_path / "x.bin", tmp_path / "y.bin", tmp_path / "ref.bin")
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    with gf.Context(timeout_ns=10_000_000_000, stdout_path=tmp_path / "out.txt", heap_bytes=64 << 20) as ctx:
        rc, ec = ctx.run("axpy_sum", [n, tmp_path / "gpu.bin"], [(xd, gf.GF_BUF_IN), (yd, gf.GF_BUF_IN)])
        st = ctx.stats()
    assert ec == 0
    got = open(tmp_path / "out.txt").read().splitlines()
    gb, gs = split_sum(got)
    wb, ws = split_sum(want.splitlines())
    assert gb == wb
    assert len(gs) == 1 and len(ws) == 1
    assert abs(gs[0] - ws[0]) <= 1e-12 * abs(ws[0])
    ex = dict(l.split() for l in oracle(oracle_bin, "exact_sum", tmp_path / "ref.bin").splitlines())
    assert abs(gs[0] - float(ex["exact"])) <= 2 * EPS * float(ex["absum"])
    assert (tmp_path / "gpu.bin").read_bytes() == (tmp_path / "ref.bin").read_bytes()
    assert st.rpc_calls[gf.OP_PRINTF] == (n + 1023) // 1024 + 1
    # axpy and sum regions, plus one grid copy per bulk-arena chunk of the final fwrite (32 MiB halves)
    chunks = 0 if 8 * n <= 2048 else -(-8 * n // (32 << 20))
    assert st.regions == (2 + chunks if n else 0)


def test_axpy_closed_form_sum_is_exact(gf_lib, tmp_path):
    import torch
    gf = gf_lib
    n = 1 << 20
    x, y = inputs.axpy_closed_form_inputs(n)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    with gf.Context(timeout_ns=10_000_000_000, stdout_path=tmp_path / "out.txt", heap_bytes=64 << 20) as ctx:
        ctx.run("axpy_sum", [n, tmp_path / "gpu.bin"], [(xd, gf.GF_BUF_IN), (yd, gf.GF_BUF_IN)])
    s = [l for l in open(tmp_path / "out.txt").read().splitlines() if l.startswith("sum ")]
    assert s == ["sum %.17g" % (2.5 * n * (n - 1) / 2 + n)]


def test_axpy_host_buffers_e2e(gf_lib, oracle_bin, tmp_path):
    """Host (numpy) buffers: the loader stages them in and out."""
    gf = gf_lib
    n = 70000
    x, y = inputs.axpy_inputs(n, seed=3)
    inputs.write_f64(tmp_path / "x.bin", x)
    inputs.write_f64(tmp_path / "y.bin", y)
    oracle(oracle_bin, "axpy_sum", n, tmp_path / "x.bin", tmp_path / "y.bin", tmp_path / "ref.bin")
    yh = y.copy()
    with gf.Context(timeout_ns=10_000_000_000, stdout_path=tmp_path / "out.txt", heap_bytes=64 << 20) as ctx:
        rc, ec = ctx.run("axpy_sum", [n, tmp_path / "gpu.bin"], [(x, gf.GF_BUF_IN), (yh, gf.GF_BUF_IN | gf.GF_BUF_OUT)])
    assert ec == 0
    assert np.array_equal(yh, np.fromfile(tmp_path / "ref.bin"))


@pytest.mark.parametrize("n,sweeps", [(1, 2), (2, 2), (3, 2), (8, 3), (12, 60), (18, 4), (20, 40), (67, 5),
                                     (256, 100)])
def test_jacobi_parity(gf_lib, oracle_bin, tmp_path, n, sweeps):
    """Bit-exact against the serial program.  The small grids with many
    sweeps reuse the same few heap blocks while they fit in an SM's L1, so a
    read of a grid through the read-only path that saw data from two sweeps
    earlier would change the result."""
    import torch
    gf = gf_lib
    g = inputs.jacobi_input(n, seed=2)
    inputs.write_f64(tmp_path / "in.bin", g)
    want = oracle(oracle_bin, "jacobi", n, sweeps, tmp_path / "in.bin", tmp_path / "ref.bin")
    gd = torch.from_numpy(g).cuda()
    heap = max(64 << 20, 4 * n ** 3 * 8 + (64 << 20))
    with gf.Context(timeout_ns=10_000_000_000, stdout_path=tmp_path / "out.txt", heap_bytes=heap, heap_small_pct=5) as ctx:
        rc, ec = ctx.run("jacobi", [n, sweeps, tmp_path / "gpu.bin"], [(gd, gf.GF_BUF_IN)])
        st = ctx.stats()
    assert ec == 0
    got = open(tmp_path / "out.txt").read().splitlines()
    assert sorted(got) == sorted(want.splitlines())          # residual text bit-exact
    assert (tmp_path / "gpu.bin").read_bytes() == (tmp_path / "ref.bin").read_bytes()
    assert st.heap_alloc == sweeps and st.heap_free == sweeps and st.heap_bad_free == 0
    assert st.heap_live_bytes == 0


@pytest.mark.parametrize("n,sweeps,kseg", [(1, 2, 1), (2, 2, 1), (3, 2, 2), (8, 3, 3), (18, 4, 18), (67, 5, 7),
                                            (256, 100, 8)])
def test_jacobi_column_parity(gf_lib, oracle_bin, tmp_path, n, sweeps, kseg):
    """The sweep as columns of kseg planes: the serial program's residual
    lines and grid bits, including ragged last segments and the full-size
    benchmark grid."""
    import torch
    gf = gf_lib
    g = inputs.jacobi_input(n, seed=2)
    inputs.write_f64(tmp_path / "in.bin", g)
    want = oracle(oracle_bin, "jacobi", n, sweeps, tmp_path / "in.bin", tmp_path / "ref.bin")
    heap = max(64 << 20, 4 * n ** 3 * 8 + (64 << 20))
    with gf.Context(timeout_ns=10_000_000_000, stdout_path=tmp_path / "out.txt", heap_bytes=heap, heap_small_pct=5) as ctx:
        rc, ec = ctx.run("jacobi", [n, sweeps, tmp_path / "gpu.bin", 1, kseg],
                         [(torch.from_numpy(g).cuda(), gf.GF_BUF_IN)])
    assert ec == 0
    assert sorted(open(tmp_path / "out.txt").read().splitlines()) == sorted(want.splitlines())
    assert (tmp_path / "gpu.bin").read_bytes() == (tmp_path / "ref.bin").read_bytes()


@pytest.mark.parametrize("kseg", [0, 3, 16])
@pytest.mark.parametrize("int_adds", [0, 1, 2, 3, 4, 5])
@pytest.mark.parametrize("kind", ["unit", "signed", "tiny", "huge", "ties", "smooth"])
def test_jacobi_parity_every_pipe_split(gf_lib, oracle_bin, tmp_path, int_adds, kind, kseg):
    """Every split of the neighbour adds between the integer and FP64 pipes
    gives the serial program's bits, one iteration per point (kseg 0) and as
    columns of 3 or 16 planes: on the standard grid, on a grid of mixed
    signs (opposite-sign adds take the FP64 path), on grids scaled into the
    subnormal range and up by 2^200, on a constant interior (residuals tie)
    and on a smooth grid whose residual grows along the iteration order."""
    import torch
    gf = gf_lib
    n, sweeps = 67, 5
    g = inputs.jacobi_input(n, seed=9)
    if kind == "signed":
        g = np.where(g != 0.0, 2.0 * g - 1.0, 0.0)
    elif kind == "tiny":
        g = g * 2.0 ** -1060
    elif kind == "huge":
        g = g * 2.0 ** 200
    elif kind == "ties":
        g = np.where(g != 0.0, 0.5, 0.0)
    elif kind == "smooth":
        x = np.sin(np.pi * np.arange(n) / (n - 1))
        g = np.where(g != 0.0, (x[:, None, None] * x[None, :, None] * x[None, None, :]).reshape(-1), 0.0)
    inputs.write_f64(tmp_path / "in.bin", g)
    want = oracle(oracle_bin, "jacobi", n, sweeps, tmp_path / "in.bin", tmp_path / "ref.bin")
    with gf.Context(timeout_ns=10_000_000_000, stdout_path=tmp_path / "out.txt", heap_bytes=64 << 20,
                    heap_small_pct=5) as ctx:
        rc, ec = ctx.run("jacobi", [n, sweeps, tmp_path / "gpu.bin", int_adds, kseg],
                         [(torch.from_numpy(g).cuda(), gf.GF_BUF_IN)])
    assert ec == 0
    assert sorted(open(tmp_path / "out.txt").read().splitlines()) == sorted(want.splitlines())
    assert (tmp_path / "gpu.bin").read_bytes() == (tmp_path / "ref.bin").read_bytes()


@pytest.mark.parametrize("T,aggregate", [(4096 + 7, 1), (4096 + 7, 0), (1 << 20, 1)])
def test_stress_parity(gf_lib, oracle_bin, tmp_path, T, aggregate):
    """Heap + RPC stress: line multiset and per-thread line order, per-thread
    heap checksums bit-exact, no allocation failure, heap empty at the end."""
    import torch
    gf = gf_lib
    sizes = inputs.loguniform_int(3, 8 * T, 16, 65536).astype(np.uint32)
    inputs.write_raw(tmp_path / "s.bin", sizes)
    want = oracle(oracle_bin, "stress", T, tmp_path / "s.bin", tmp_path / "cs.bin").splitlines()
    cs = torch.zeros(T, dtype=torch.int64, device="cuda")
    fails = torch.zeros(1, dtype=torch.int64, device="cuda")
    with gf.Context(timeout_ns=20_000_000_000, stdout_path=tmp_path / "out.txt", heap_bytes=8 << 30,
                    heap_small_pct=95, aggregate=aggregate) as ctx:
        rc, ec = ctx.run("stress", [T], [(torch.from_numpy(sizes.view(np.int32)).cuda(), 1), (cs, 1), (fails, 1)])
        st = ctx.stats()
    assert ec == 0 and fails.item() == 0
    got = open(tmp_path / "out.txt").read().splitlines()
    assert sorted(got) == sorted(want)
    pos = {l: k for k, l in enumerate(got)}
    body = want[:-1]
    for t in range(0, T, max(1, T // 4096)):                  # each thread's 4 lines in program order
        idx = [pos[body[4 * t + j]] for j in range(4)]
        assert idx == sorted(idx)
    assert np.array_equal(cs.cpu().numpy().view(np.uint64), np.fromfile(tmp_path / "cs.bin", dtype=np.uint64))
    assert st.heap_alloc == 8 * T and st.heap_free == 8 * T and st.heap_fail == 0 and st.heap_live_bytes == 0
    assert st.rpc_calls[gf.OP_PRINTF] == 4 * T + 1
    if aggregate:
        # lanes reach printf out of step after divergent malloc/free paths, so
        # slots carry fewer records than in a printf-only loop
        assert st.rpc_slots[gf.OP_PRINTF] * 2 < st.rpc_calls[gf.OP_PRINTF]
    else:
        assert st.rpc_slots[gf.OP_PRINTF] == st.rpc_calls[gf.OP_PRINTF]
