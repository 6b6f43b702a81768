"""The paper's kernel split (Sec. 3.3, Fig. 3) as a comparator: with
split_regions the program kernel is one block and every parallel region is
an RPC on which the host launches the region as its own kernel.  The same
programs must give the same results as on the persistent grid and as the
serial C oracle."""
import math
import subprocess

import numpy as np
import pytest

from paper_2306_11686_gb300 import inputs

pytestmark = pytest.mark.gpu


def _oracle(oracle_bin, name, *args):
    p = subprocess.run([oracle_bin(name), *map(str, args)], capture_output=True, text=True)
    assert p.returncode == 0, p.stderr
    return p.stdout


def test_split_axpy_sum_matches_oracle(gf_lib, oracle_bin, tmp_path):
    import torch
    gf = gf_lib
    n = 50000 + 17
    x, y = inputs.axpy_inputs(n, seed=1)
    inputs.write_f64(tmp_path / "x.bin", x)
    inputs.write_f64(tmp_path / "y.bin", y)
    want = _oracle(oracle_bin, "axpy_sum", n, tmp_path / "x.bin", tmp_path / "y.bin", tmp_path / "ref.bin").splitlines()
    with gf.Context(split_regions=1, timeout_ns=10_000_000_000, heap_bytes=64 << 20,
                    stdout_path=tmp_path / "out.txt") as ctx:
        rc, ec = ctx.run("axpy_sum", [n, tmp_path / "gpu.bin"],
                         [(torch.from_numpy(x).cuda(), gf.GF_BUF_IN), (torch.from_numpy(y).cuda(), gf.GF_BUF_IN)])
        st = ctx.stats()
    assert ec == 0
    got = open(tmp_path / "out.txt").read().splitlines()
    body = lambda ls: sorted(l for l in ls if not l.startswith("sum "))
    assert body(got) == body(want)
    s_got = float([l for l in got if l.startswith("sum ")][0].split()[1])
    s_want = float([l for l in want if l.startswith("sum ")][0].split()[1])
    assert abs(s_got - s_want) <= 1e-12 * abs(s_want)
    assert (tmp_path / "gpu.bin").read_bytes() == (tmp_path / "ref.bin").read_bytes()
    assert st.regions >= 2 and st.rpc_calls[gf.OP_REGION] == st.regions     # one launch RPC per region


def test_split_jacobi_bit_exact(gf_lib, oracle_bin, tmp_path):
    import torch
    gf = gf_lib
    n, sweeps = 67, 5
    g = inputs.jacobi_input(n, seed=9)
    inputs.write_f64(tmp_path / "in.bin", g)
    want = _oracle(oracle_bin, "jacobi", n, sweeps, tmp_path / "in.bin", tmp_path / "ref.bin")
    with gf.Context(split_regions=1, timeout_ns=10_000_000_000, heap_bytes=64 << 20, heap_small_pct=5,
                    stdout_path=tmp_path / "out.txt") as ctx:
        rc, ec = ctx.run("jacobi", [n, sweeps, tmp_path / "gpu.bin"], [(torch.from_numpy(g).cuda(), gf.GF_BUF_IN)])
    assert ec == 0
    assert sorted(open(tmp_path / "out.txt").read().splitlines()) == sorted(want.splitlines())
    assert (tmp_path / "gpu.bin").read_bytes() == (tmp_path / "ref.bin").read_bytes()


@pytest.mark.parametrize("n,sched,chunk", [(1, 0, 1), (123457, 0, 1), (123457, 1, 5), (99, 0, 0)])
def test_split_reductions(gf_lib, n, sched, chunk):
    import torch
    gf = gf_lib
    rng = np.random.default_rng(n + 1)
    x = rng.standard_normal(n) * 10.0 ** rng.integers(-8, 8, n)
    v = rng.integers(-2 ** 40, 2 ** 40, n)
    out = torch.zeros(6, dtype=torch.int64, device="cuda")
    with gf.Context(split_regions=1, timeout_ns=10_000_000_000, heap_bytes=64 << 20) as ctx:
        rc, ec = ctx.run("reduce_probe", [n, sched, chunk],
                         [(torch.from_numpy(x).cuda(), 1), (torch.from_numpy(v).cuda(), 1), (out, 1)])
    assert ec == 0
    o = out.cpu().numpy()
    d = o[:3].view(np.float64)
    assert abs(d[0] - math.fsum(x)) <= 2 * 2.0 ** -52 * np.abs(x).sum()
    assert d[1] == x.min() and d[2] == x.max()
    assert o[3] == int(v.sum()) and o[4] == v.min() and o[5] == v.max()


@pytest.mark.parametrize("e,sched,chunk", [(300017, 0, 1), (300017, 1, 13), (1000, 0, 0)])
def test_split_schedules(gf_lib, e, sched, chunk):
    """Every iteration exactly once; in a region kernel every thread is a
    worker, so ids run 0 .. grid x 256 - 1 with no offset."""
    import torch
    gf = gf_lib
    hits = torch.zeros(e, dtype=torch.int32, device="cuda")
    owner = torch.full((e,), -1, dtype=torch.int64, device="cuda")
    info = torch.zeros(2, dtype=torch.int64, device="cuda")
    with gf.Context(split_regions=1, timeout_ns=10_000_000_000, heap_bytes=64 << 20) as ctx:
        sms, per = ctx.grid_info("sched_probe")
        rc, ec = ctx.run("sched_probe", [0, e, sched, chunk], [(hits, 1), (owner, 1), (info, 1)])
    assert ec == 0
    T = info[0].item()
    assert T == (sms * per - 1) * 256                       # the region kernel's grid: all blocks but the program's
    assert info[1].item() == 1
    assert torch.all(hits == 1)
    o = owner.cpu().numpy()
    i = np.arange(e)
    if sched == 0 and chunk == 1:
        assert np.array_equal(o, i % T)
    elif sched == 0 and chunk == 0:
        assert np.array_equal(o, i // -(-e // T))
    else:
        assert o.min() >= 0 and o.max() < T
