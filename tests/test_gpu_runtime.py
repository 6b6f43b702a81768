"""GPU tests of the runtime mechanisms, each against brute force or a closed
form: schedules (every iteration exactly once, OpenMP static assignment),
reductions, the cross-block barrier, RPC landing pads, warp aggregation, the
heap audit (pairwise non-overlap, alignment, bounds) and bounded waits."""
import math
import os

import numpy as np
import pytest

from paper_2306_11686_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(gf_lib, tmp_path_factory):
    d = tmp_path_factory.mktemp("rt")
    c = gf_lib.Context(timeout_ns=10_000_000_000, stdout_path=d / "out.txt", heap_bytes=1 << 30)
    yield c
    c.close()


@pytest.mark.parametrize("b,e,sched,chunk", [
    (0, 1, 0, 1), (0, 1000, 0, 1), (5, 300017, 0, 1), (0, 300017, 0, 0), (3, 100000, 0, 7),
    (0, 777777, 1, 1), (11, 500000, 1, 13), (0, 31, 1, 64), (0, 0, 0, 1)])
def test_schedules(gf_lib, ctx, b, e, sched, chunk):
    import torch
    gf = gf_lib
    n = e - b
    hits = torch.zeros(max(n, 1), dtype=torch.int32, device="cuda")
    owner = torch.full((max(n, 1),), -1, dtype=torch.int64, device="cuda")
    info = torch.zeros(2, dtype=torch.int64, device="cuda")
    rc, ec = ctx.run("sched_probe", [b, e, sched, chunk], [(hits, 1), (owner, 1), (info, 1)])
    assert ec == 0
    if n == 0:
        assert info[0].item() == 0
        return
    T = info[0].item()
    sms, per = ctx.grid_info("sched_probe")
    assert T == sms * per * 256 - 32                       # every SM, continuous ids
    assert info[1].item() == 1                              # serial part: a team of one
    assert torch.all(hits[:n] == 1)                         # each iteration exactly once
    o = owner[:n].cpu().numpy()
    i = np.arange(n)
    if sched == 0 and chunk == 1:
        assert np.array_equal(o, i % T)
    elif sched == 0 and chunk > 1:
        assert np.array_equal(o, (i // chunk) % T)
    elif sched == 0:
        per_t = -(-n // T)
        assert np.array_equal(o, i // per_t)
    else:
        assert o.min() >= 0 and o.max() < T


@pytest.mark.parametrize("b,n", [(1 << 40, 1000), (1 << 40, (1 << 31) - 2), (-(1 << 35), (1 << 31) + 7)])
def test_static1_ranges(gf_lib, ctx, b, n):
    """Static chunk-1 loops with a large (or negative) base, on both sides of
    2^31 iterations: below it they run in the 32-bit trampoline, above it in
    the generic 64-bit loop.  Every index is visited once: the count, the
    sum of i - b, min and max of i."""
    import torch
    out = torch.zeros(4, dtype=torch.int64, device="cuda")
    rc, ec = ctx.run("range_probe", [b, b + n], [(out, 1)])
    assert ec == 0
    o = out.cpu().tolist()
    assert o == [n, n * (n - 1) // 2, b, b + n - 1]


@pytest.mark.parametrize("n,sched,chunk", [(1, 0, 1), (1000, 0, 1), (1 << 20, 0, 1), (123457, 1, 5), (99, 0, 0)])
def test_reductions(gf_lib, ctx, n, sched, chunk):
    import torch
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) * 10.0 ** rng.integers(-8, 8, n)
    v = rng.integers(-2 ** 40, 2 ** 40, n)
    out = torch.zeros(6, dtype=torch.int64, device="cuda")
    ctx.run("reduce_probe", [n, sched, chunk],
            [(torch.from_numpy(x).cuda(), 1), (torch.from_numpy(v).cuda(), 1), (out, 1)])
    o = out.cpu().numpy()
    d = o[:3].view(np.float64)
    exact = math.fsum(x)
    assert abs(d[0] - exact) <= 2 * 2.0 ** -52 * np.abs(x).sum()
    assert d[1] == x.min() and d[2] == x.max()
    assert o[3] == int(v.sum()) and o[4] == v.min() and o[5] == v.max()


def test_reduction_deterministic(gf_lib, ctx):
    import torch
    n = 1 << 19
    x = inputs.uniform_pm1(9, n) * 1e6
    xd = torch.from_numpy(x).cuda()
    vd = torch.zeros(n, dtype=torch.int64, device="cuda")
    res = set()
    for _ in range(3):
        out = torch.zeros(6, dtype=torch.int64, device="cuda")
        ctx.run("reduce_probe", [n, 1, 3], [(xd, 1), (vd, 1), (out, 1)])
        res.add(out[0].item())
    assert len(res) == 1


def test_grid_barrier(gf_lib, ctx):
    import torch
    sms, per = ctx.grid_info("barrier_probe")
    T = sms * per * 256 - 32
    a = torch.zeros(T, dtype=torch.int64, device="cuda")
    err = torch.zeros(1, dtype=torch.int64, device="cuda")
    rc, ec = ctx.run("barrier_probe", [20], [(a, 1), (err, 1)])
    assert ec == 0 and err.item() == 0


@pytest.mark.parametrize("bulk", [64 << 20, 1 << 20, 0])   # arena (1 and several chunks), copy-engine DMA
def test_rpc_landing_pads(gf_lib, tmp_path, bulk):
    import torch
    gf = gf_lib
    os.environ["GF_PROBE_VAR"] = "value-42"
    os.environ.pop("GF_PROBE_UNSET_VAR", None)
    nbig = (3 << 20) + 123
    big = torch.from_numpy(np.frombuffer(np.random.default_rng(1).bytes(nbig), dtype=np.uint8).copy()).cuda()
    ref = big.clone()
    res = torch.zeros(32, dtype=torch.int64, device="cuda")
    with gf.Context(timeout_ns=10_000_000_000, stdout_path=tmp_path / "out.txt", heap_bytes=64 << 20,
                    bulk_bytes=bulk) as c:
        rc, ec = c.run("rpc_probe", [tmp_path / "small.txt", tmp_path / "big.bin", nbig], [(res, 1), (big, 1)])
    assert ec == 0
    lines = open(tmp_path / "out.txt").read().splitlines()
    want = [
        "int %d %i %u %x %X %o|" % (-42, 7, 4000000000, 255, 3054, 8),
        "long %d %d %d %x" % (-5000000000, 123456789012345, 18446744073709551615, 0xdeadbeefcafe),
        "dbl %f %e %g %.17g %10.3f|%-8.2e|%+.0f" % (3.14159, -1.5e-300, 1e100, 0.1, 2.5, 12345.678, 2.5),
        "str [%s] [%10s] [%-6s] [%.3s] %c%c %%" % ("hello", "right", "left", "truncate", "o", "k"),
        "star [%*d] [%-*d] [%.*f]" % (6, 42, 5, 7, 3, 1.0 / 3.0),
        "no args",
    ]
    assert lines == want
    r = res.cpu().tolist()
    assert r[:6] == [len(w) + 1 for w in want]
    assert r[6] == 1 and r[7] == len("to file 99 ok\n") and r[8] == 16 and r[9] == 0
    assert open(tmp_path / "small.txt").read() == "to file 99 ok\n0123456789abcdef"
    assert r[10] == nbig and r[11] == 0
    assert (tmp_path / "big.bin").read_bytes() == ref.cpu().numpy().tobytes()
    assert r[12] == 20
    h = 0
    for ch in b"to file 99 ok\n012345":
        h = (h * 31 + ch) & ((1 << 64) - 1)
    assert r[13] == (h if h < 1 << 63 else h - (1 << 64))
    assert r[14] == nbig and torch.equal(big, ref)           # fread by DMA restored the bytes
    assert r[15] == len("value-42") and r[16] == ord("v") and r[17] == 0
    assert r[18] == 1 and r[19] == 1


@pytest.mark.parametrize("aggregate", [1, 0])
def test_rpc_storm_order_and_multiset(gf_lib, tmp_path, aggregate):
    import torch
    gf = gf_lib
    n, calls = 20000, 4
    bad = torch.zeros(1, dtype=torch.int64, device="cuda")
    with gf.Context(timeout_ns=10_000_000_000, stdout_path=tmp_path / "out.txt", heap_bytes=64 << 20, aggregate=aggregate) as c:
        rc, ec = c.run("rpc_storm", [n, calls], [(bad, 1)])
        st = c.stats()
    assert ec == 0 and bad.item() == 0
    lines = open(tmp_path / "out.txt").read().splitlines()
    want = ["t %d k %d v %.6e" % (i, k, i * 0.5 + k) for i in range(n) for k in range(calls)]
    assert sorted(lines) == sorted(want)
    last = {}
    for l in lines:                                          # per-thread program order
        p = l.split()
        i, k = int(p[1]), int(p[3])
        assert last.get(i, -1) == k - 1
        last[i] = k
    assert st.rpc_calls[gf.OP_PRINTF] == n * calls
    if aggregate:
        assert st.rpc_slots[gf.OP_PRINTF] < st.rpc_calls[gf.OP_PRINTF] / 8
    else:
        assert st.rpc_slots[gf.OP_PRINTF] == st.rpc_calls[gf.OP_PRINTF]


@pytest.mark.parametrize("aggregate", [1, 0])
def test_rpc_divergent_groups_share_slots(gf_lib, tmp_path, aggregate):
    """Odd and even lanes print from two call sites with one format: every
    line and return value as printf gives them, and with aggregation a slot
    holds at least a half warp's records (the two call sites' groups either
    share a slot or the compiler merged the sites)."""
    import torch
    gf = gf_lib
    n = 20000 + 13
    ret = torch.zeros(n, dtype=torch.int32, device="cuda")
    with gf.Context(timeout_ns=10_000_000_000, stdout_path=tmp_path / "out.txt", heap_bytes=64 << 20,
                    aggregate=aggregate, server_threads=2) as c:
        rc, ec = c.run("rpc_diverge", [n], [(ret, 1)])
        st = c.stats()
    assert ec == 0
    want = ["d %d %d" % (i, i & 1) for i in range(n)]
    assert sorted(open(tmp_path / "out.txt").read().splitlines()) == sorted(want)
    assert ret.cpu().tolist() == [len(w) + 1 for w in want]
    calls, slots = int(st.rpc_calls[gf.OP_PRINTF]), int(st.rpc_slots[gf.OP_PRINTF])
    assert calls == n
    if aggregate:
        assert calls >= 16 * slots, (calls, slots)
    else:
        assert slots == calls


def test_heap_audit(gf_lib, tmp_path):
    import torch
    gf = gf_lib
    n, per = 4096, 8
    sizes = inputs.loguniform_int(11, n * per, 16, 65536).astype(np.uint32)
    ptrs = torch.zeros(n * per, dtype=torch.int64, device="cuda")
    info = torch.zeros(4, dtype=torch.int64, device="cuda")
    with gf.Context(timeout_ns=10_000_000_000, heap_bytes=2 << 30, heap_small_pct=90) as c:
        rc, ec = c.run("heap_audit", [n, per], [(torch.from_numpy(sizes.view(np.int32)).cuda(), 1), (ptrs, 1), (info, 1)])
        st = c.stats()
        hb = c.cfg.heap_bytes
    assert ec == 0
    p = ptrs.cpu().numpy().view(np.uint64)
    assert (p != 0).all()
    cls = np.maximum(16, 1 << np.ceil(np.log2(sizes)).astype(np.int64))
    order = np.argsort(p)
    ps, cs = p[order].astype(np.int64), cls[order]
    assert (ps % 16 == 0).all()
    assert (ps[1:] >= ps[:-1] + cs[:-1]).all()               # pairwise non-overlap
    assert ps[-1] + cs[-1] - ps[0] <= hb                     # inside the arena
    inf = info.cpu().tolist()
    assert inf[0] == 0                                       # every block kept its tags
    assert inf[1] == int(cls.sum()) and inf[2] == 0          # live bytes, then all freed
    assert inf[3] == n * per                                 # reuse succeeds
    assert st.heap_fail == 0 and st.heap_bad_free == 0


def test_heap_large_path(gf_lib):
    import torch
    gf = gf_lib
    out = torch.zeros(16, dtype=torch.int64, device="cuda")
    with gf.Context(timeout_ns=10_000_000_000, heap_bytes=1 << 30, heap_small_pct=0) as c:
        rc, ec = c.run("heap_big", [100 << 20, 4], [(out, 1)])
        st = c.stats()
    o = out.cpu().numpy().view(np.uint64)
    assert ec == 0
    assert len(set(o[:4].tolist())) == 4 and (o[:4] != 0).all()
    assert o[4] == o[1]                                      # first fit reuses the hole
    assert o[5] == o[0]                                      # all extents merged back
    assert st.heap_bad_free == 1 and st.heap_live_bytes == 0


def test_heap_out_of_memory_returns_null(gf_lib):
    import torch
    gf = gf_lib
    out = torch.zeros(16, dtype=torch.int64, device="cuda")
    with gf.Context(timeout_ns=10_000_000_000, heap_bytes=256 << 20, heap_small_pct=0) as c:
        rc, ec = c.run("heap_big", [100 << 20, 4], [(out, 1)])
        st = c.stats()
    o = out.cpu().numpy()
    assert o[0] != 0 and o[1] != 0 and o[2] == 0 and o[3] == 0   # only two 100 MiB blocks fit
    assert st.heap_fail >= 2


def test_heap_small_class_exhaustion_and_reuse(gf_lib):
    """Small-class exhaustion: the first pass gets every block the small heap
    holds (then NULL, counted as failures); after all are freed the second
    pass gets exactly the same set of blocks back, which it can only find on
    the per-lane free stacks of other lanes and other SMs."""
    import torch
    gf = gf_lib
    T, per, bytes_ = 4096, 2, 4096
    ptrs = torch.zeros(2 * T * per, dtype=torch.int64, device="cuda")
    with gf.Context(timeout_ns=10_000_000_000, heap_bytes=8 << 20, heap_small_pct=100) as c:
        rc, ec = c.run("heap_exhaust", [T, per, bytes_], [(ptrs, 1)])
        st = c.stats()
    assert ec == 0
    p = ptrs.cpu().numpy().view(np.uint64).reshape(2, T * per)
    assert not (p & np.uint64(15)).any()                     # 16-byte aligned, no block flagged as shared
    got = [set(p[k][p[k] != 0].tolist()) for k in range(2)]
    n1 = int((p[0] != 0).sum())
    assert len(got[0]) == n1                                  # pairwise distinct
    slabs = (8 << 20) >> 18
    assert (slabs - 2) * ((1 << 18) // bytes_) <= n1 <= slabs * ((1 << 18) // bytes_)
    assert got[1] == got[0] and int((p[1] != 0).sum()) == n1  # the same blocks again, each once
    a = np.array(sorted(got[0]), dtype=np.uint64)
    assert (np.diff(a) >= bytes_).all()                        # no overlap
    assert st.heap_fail == 2 * (T * per - n1)
    assert st.heap_live_bytes == 0 and st.heap_bad_free == 0


def test_rpc_timeout_without_server(gf_lib):
    gf = gf_lib
    with gf.Context(server_threads=0, timeout_ns=200_000_000, heap_bytes=64 << 20) as c:
        rc, h = c.launch("rpc_timeout", [])
        assert rc == 0
        import time
        t0 = time.time()
        while not gf.gf_done(h):
            assert time.time() - t0 < 30
            time.sleep(0.01)
        rc, ec = c.wait(h)
    assert ec == 1 and rc == gf.GF_ETIMEDOUT


def test_div6_matches_ieee_division(gf_lib, ctx):
    """gf_div6_rn (Markstein's correction) and gf_div6_int (integer pipe)
    equal x / 6.0 bit for bit on the GPU."""
    import torch
    rng = np.random.default_rng(6)
    n = 1 << 22
    e = rng.integers(-1074, 1024, n).astype(np.float64)
    m = rng.random(n) + 1.0
    x = np.ldexp(m, e.astype(np.int64))
    x[: n // 4] = rng.random(n // 4) * 6.0                       # the Jacobi range
    x[n // 4: n // 4 + 1000] = np.arange(1000, dtype=np.float64)  # integers and 0
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 5e-324, 2.0 ** -1000, 2.0 ** -1000 * (1 - 2 ** -53),
                        2.0 ** 1001, np.nextafter(2.0 ** 1001, 0), 1.7976931348623157e308, 6.0, 3.0, 12.0])
    x[-len(special):] = special
    x[n // 2: n // 2 + 10000] *= -1.0
    x[n // 2 + 10000: n // 2 + 20000] = np.ldexp(3.0 * 2.0 ** 51 + np.arange(-5000, 5000), -52)  # k switch
    out = torch.zeros(3 * n, dtype=torch.float64, device="cuda")
    rc, ec = ctx.run("div6_probe", [n], [(torch.from_numpy(x).cuda(), 1), (out, 1)])
    assert ec == 0
    o = out.cpu().numpy().view(np.uint64).reshape(n, 3)
    assert np.array_equal(o[:, 0], o[:, 1])
    assert np.array_equal(o[:, 0], o[:, 2])
    ref = (x / 6.0).view(np.uint64)                              # numpy's IEEE division agrees too
    finite = np.isfinite(x)
    assert np.array_equal(o[finite, 0], ref[finite])


def test_dadd_int_matches_fp64_add(gf_lib, ctx):
    """gf_dadd_int (same-sign add on the integer pipe) equals the FP64 add bit
    for bit on the GPU: every exponent gap, ties (of both paths), carries, the Jacobi range,
    zeros, subnormals, overflow, NaN/inf and random bit patterns."""
    import torch
    rng = np.random.default_rng(8)
    n = 1 << 22
    q = n // 8
    ea = rng.integers(1, 2047, q).astype(np.uint64)
    eb = np.maximum(ea.astype(np.int64) - rng.integers(0, 71, q), 1).astype(np.uint64)
    frac = lambda k: rng.integers(0, 1 << 52, k, dtype=np.uint64)
    sgn = (rng.integers(0, 2, q).astype(np.uint64) << np.uint64(63))
    xa = sgn | (ea << np.uint64(52)) | frac(q)
    xb = sgn | (eb << np.uint64(52)) | frac(q)
    ties_e = rng.integers(60, 1960, q).astype(np.uint64)
    tx = (ties_e << np.uint64(52)) | frac(q)
    th = ((ties_e - np.uint64(53)) << np.uint64(52)) + rng.integers(-1, 2, q).astype(np.uint64)
    ones = (ea << np.uint64(52)) | np.uint64((1 << 52) - 1)
    # exponent gaps 1..10 with the dropped bits exactly one half (ties of the short path)
    dg = rng.integers(1, 11, q).astype(np.uint64)
    se = rng.integers(20, 2040, q).astype(np.uint64)
    low = (np.uint64(1) << dg) - np.uint64(1)
    sfrac = (frac(q) & ~low) | (np.uint64(1) << (dg - np.uint64(1)))
    sx_ = (se << np.uint64(52)) | frac(q)
    sy_ = ((se - dg) << np.uint64(52)) | sfrac
    xa = np.concatenate([xa, sx_])
    xb = np.concatenate([xb, sy_])
    x = np.concatenate([xa.view(np.float64), tx.view(np.float64), ones.view(np.float64),
                        rng.random(q) * 6.0, rng.integers(0, 2 ** 63, q, dtype=np.uint64).view(np.float64) *
                        np.where(rng.random(q) < 0.5, -1.0, 1.0)])
    y = np.concatenate([xb.view(np.float64), th.view(np.float64), xb[:q].view(np.float64) * np.sign(ones.view(np.float64)),
                        rng.random(q) * 6.0, rng.integers(0, 2 ** 64, q, dtype=np.uint64).view(np.float64)])
    special = np.array([0.0, -0.0, 1.0, -1.0, np.inf, -np.inf, np.nan, 5e-324, -5e-324, 2.2250738585072014e-308,
                        1.7976931348623157e308, float.fromhex("0x1.fffffffffffffp1022"), 2.0 ** 1023, 3.0])
    sx, sy = np.meshgrid(special, special)
    x = np.concatenate([x, sx.ravel()])
    y = np.concatenate([y, sy.ravel()])
    m = len(x)
    out = torch.zeros(2 * m, dtype=torch.float64, device="cuda")
    rc, ec = ctx.run("dadd_probe", [m], [(torch.from_numpy(x).cuda(), 1), (torch.from_numpy(y).cuda(), 1), (out, 1)])
    assert ec == 0
    o = out.cpu().numpy().reshape(m, 2)
    nan = np.isnan(o[:, 0])
    assert np.array_equal(np.isnan(o[:, 1]), nan)
    assert np.array_equal(o[~nan, 0].view(np.uint64), o[~nan, 1].view(np.uint64))
    with np.errstate(all="ignore"):
        ref = x + y                                              # numpy's IEEE add agrees too
    assert np.array_equal(ref[~nan].view(np.uint64), o[~nan, 0].view(np.uint64))


@pytest.mark.parametrize("bulk", [64 << 20, 0])
def test_fwrite_append_mode_in_order(gf_lib, tmp_path, bulk):
    import torch
    gf = gf_lib
    n = (40 << 20) + 17                                          # several arena halves / DMA chunks
    data = np.frombuffer(np.random.default_rng(2).bytes(n), dtype=np.uint8).copy()
    (tmp_path / "a.bin").write_bytes(b"head")
    with gf.Context(timeout_ns=10_000_000_000, heap_bytes=64 << 20, bulk_bytes=bulk) as c:
        rc, ec = c.run("fwrite_modes", [tmp_path / "a.bin", n], [(torch.from_numpy(data).cuda(), 1)])
    assert ec == 0
    assert (tmp_path / "a.bin").read_bytes() == b"head" + data.tobytes() * 2


def test_link_probe_round_trip_and_rpc_latency(gf_lib, tmp_path):
    """The host-link probe moves the bytes it times: device -> mapped host
    arena -> device restores a pattern exactly (sizes off the 16-byte path
    too); the single-thread RPC timer reports one positive time per call."""
    import torch
    gf = gf_lib
    pat = torch.from_numpy(np.frombuffer(np.random.default_rng(4).bytes(1 << 20), dtype=np.uint8).copy()).cuda()
    ns = torch.zeros(64, dtype=torch.int64, device="cuda")
    with gf.Context(timeout_ns=10_000_000_000, heap_bytes=64 << 20, bulk_bytes=1 << 20,
                    stdout_path=tmp_path / "out.txt") as c:
        for n in (64, 1000, 4096, (1 << 20) - 3, 1 << 20):
            dev = pat.clone()
            rc, ec = c.run("link_probe", [n, 2, 0], [(dev, 1), (ns, 1)])       # device -> host arena
            assert ec == 0 and (ns[:2] > 0).all()
            dev[:n] = 0
            rc, ec = c.run("link_probe", [n, 2, 1], [(dev, 1), (ns, 1)])       # host arena -> device
            assert ec == 0
            assert torch.equal(dev, pat), n
        rc, ec = c.run("link_probe", [(1 << 20) + 16, 1, 0], [(pat, 1), (ns, 1)])
        assert ec == 2                                                       # larger than the arena: refused
        for mode in (0, 1):
            ns.zero_()
            rc, ec = c.run("rpc_latency", [50, mode], [(ns, 1)])
            assert ec == 0
            v = ns[:50].cpu().numpy()
            assert (v > 0).all() and (v < 10_000_000_000).all()
            assert (ns[50:].cpu().numpy() == 0).all()


@pytest.mark.parametrize("prog", ["axpy_width", "axpy_width4", "axpy_width8"])
@pytest.mark.parametrize("n", [0, 1, 2, 1001, 1 << 16])
def test_axpy_access_width(gf_lib, prog, n):
    """The axpy loop with 8-byte and 16-byte accesses (even index, scalar
    tail) gives torch's own results, at every compiled occupancy; 16-byte
    accesses refuse a misaligned buffer."""
    import torch
    gf = gf_lib
    x = torch.empty(n + 1, dtype=torch.float64, device="cuda").uniform_(-1, 1)
    y = torch.empty(n + 1, dtype=torch.float64, device="cuda").uniform_(-1, 1)
    nb = torch.tensor([n], dtype=torch.int64, device="cuda")
    with gf.Context(timeout_ns=10_000_000_000, heap_bytes=64 << 20) as ctx:
        for w in (1, 2):
            z = torch.zeros(n + 1, dtype=torch.float64, device="cuda")
            rc, ec = ctx.run(prog, [w], [(nb, 1), (x[:n], 1), (y[:n], 1), (z[:n], 1)])
            assert ec == 0
            assert torch.equal(z[:n], 2.5 * x[:n] + y[:n]) and z[n] == 0
        if n >= 2:
            z = torch.zeros(n + 1, dtype=torch.float64, device="cuda")
            rc, ec = ctx.run(prog, [2], [(nb, 1), (x[1:], 1), (y[1:], 1), (z[1:], 1)])
            assert ec == 2 and not z.any()


def test_main_printf_buffered(gf_lib, tmp_path):
    """The initial thread's printf records share ring slots: every line once
    and in program order across full and partial batches, format changes,
    a string argument, a record larger than the buffer, other calls in
    between and records still buffered when main returns; a result read in
    its own statement is the character count; fewer slots than calls."""
    import torch
    gf = gf_lib
    res = torch.zeros(8, dtype=torch.int64, device="cuda")
    with gf.Context(timeout_ns=10_000_000_000, stdout_path=tmp_path / "out.txt", heap_bytes=64 << 20) as c:
        rc, ec = c.run("main_printf_batch", [tmp_path / "f.txt"], [(res, 1)])
        st = c.stats()
    assert ec == 0
    assert open(tmp_path / "f.txt").read().splitlines() == [f"f {k} x" for k in range(50)] and res[5].item() == 0
    big = "".join(chr(ord("a") + k % 26) for k in range(1399))
    want = [f"a {k}" for k in range(100)] + ["b str -1", "c 7", "big " + big]
    want += ["d %d %.17g" % (k, 0.5 if k == 0 else k * 0.25) for k in range(40)] + ["e 1", "e 2"]
    assert open(tmp_path / "out.txt").read().splitlines() == want
    r = res.cpu().tolist()
    assert r[0] == 4 and r[1] == 1 and r[2] == len("big ") + 1399 + 1 and r[3] == 1 and r[4] == -1
    assert st.rpc_calls[gf.OP_PRINTF] == len(want) + 50
    assert st.rpc_slots[gf.OP_PRINTF] <= 17                # 195 calls in at most 17 slots
