"""Native device libc (rand, realloc, strtod) against the host's real libc,
and the interleaved-layout pair (array of structs vs struct of arrays).

- rand: the device sequence after srand(seed) equals the host libc's
  rand() sequence (glibc's generator) for several seeds;
- strtod: value bits and consumed length equal the host strtod's for every
  string (native fast path or RPC fallback alike);
- realloc: in place within a block, moved with its bytes, NULL / 0 cases;
- interleave: both layouts give the same bits as the elementwise
  definition (each product and sum rounded once)."""
import ctypes
import ctypes.util

import numpy as np
import pytest

from paper_2306_11686_gb300 import inputs

pytestmark = pytest.mark.gpu
LIBC = ctypes.CDLL(ctypes.util.find_library("c"))
LIBC.strtod.restype = ctypes.c_double
LIBC.strtod.argtypes = [ctypes.c_char_p, ctypes.POINTER(ctypes.c_char_p)]


def host_rand(seed, n):
    LIBC.srand(ctypes.c_uint(seed))
    return [LIBC.rand() for _ in range(n)]


def strtod_cases():
    fixed = ["0", "-0", "1.5", "-2.25e3", "  42", "3.14159265358979", "1e22", "1e23", "0.1", "-.5",
             "123456789012345678", "1.7976931348623157e308", "4.9e-324", "2.2250738585072014e-308", "inf", "-inf",
             "nan", "0x1p-2", "abc", "12abc", ".e1", "1e", "1e+", "0.000123", "999999999999999", "1000000000000000",
             "9007199254740993", "5e-1", "00012.5000", "1.", "7e-22", "7e-23"]
    rng = np.random.default_rng(3)
    rand = []
    for _ in range(400):
        nd = int(rng.integers(1, 21))
        digits = "".join(str(int(d)) for d in rng.integers(0, 10, nd))
        dot = int(rng.integers(0, nd + 1))
        s = digits[:dot] + "." + digits[dot:] if rng.random() < 0.7 else digits
        if rng.random() < 0.6:
            s += "e" + str(int(rng.integers(-30, 31)))
        rand.append(("-" if rng.random() < 0.3 else "") + s)
    return fixed + rand


def test_rand_realloc_strtod(gf_lib):
    import torch
    gf = gf_lib
    strs = strtod_cases()
    blob = b"".join(s.encode() + b"\0" for s in strs)
    off = np.cumsum([0] + [len(s) + 1 for s in strs[:-1]]).astype(np.int64)
    for seed in (1, 12345, 4000000000):
        rnd = torch.zeros(200, dtype=torch.int32, device="cuda")
        val = torch.zeros(len(strs), dtype=torch.float64, device="cuda")
        used = torch.zeros(len(strs), dtype=torch.int64, device="cuda")
        rea = torch.zeros(8, dtype=torch.int64, device="cuda")
        sb = torch.from_numpy(np.frombuffer(blob, dtype=np.uint8).copy()).cuda()
        with gf.Context(timeout_ns=10_000_000_000, heap_bytes=64 << 20) as c:
            rc, ec = c.run("libc_probe", [seed, 200, len(strs)],
                           [(rnd, 1), (sb, 1), (torch.from_numpy(off).cuda(), 1), (val, 1), (used, 1), (rea, 1)])
        assert ec == 0
        assert rnd.cpu().tolist() == host_rand(seed, 200), seed
    assert rea.cpu().tolist()[:6] == [1, 1, 1, 1, 1, 1]
    v = val.cpu().numpy()
    u = used.cpu().numpy()
    for k, s in enumerate(strs):
        end = ctypes.c_char_p()
        buf = ctypes.create_string_buffer(s.encode())
        want = LIBC.strtod(buf, ctypes.byref(end))
        want_used = ctypes.cast(end, ctypes.c_void_p).value - ctypes.addressof(buf)
        got = v[k]
        assert (np.isnan(got) and np.isnan(want)) or np.float64(got).tobytes() == np.float64(want).tobytes(), s
        assert u[k] == want_used, s


@pytest.mark.parametrize("n", [1, 1000, 1 << 20])
def test_interleave_layouts(gf_lib, n):
    import torch
    gf = gf_lib
    a, b, c, d = (inputs.uniform_pm1(40 + k, n) for k in range(4))
    aos = np.stack([a, b, c, d], axis=1).reshape(-1).copy()
    want = (a + (b * c)) - d
    dv = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    outs = []
    with gf.Context(timeout_ns=10_000_000_000, heap_bytes=64 << 20) as ctx:
        for layout in (0, 1):
            out = torch.zeros(n, dtype=torch.float64, device="cuda")
            rc, ec = ctx.run("interleave", [layout, n], [(dv(aos), 1), (dv(a), 1), (dv(b), 1), (dv(c), 1),
                                                        (dv(d), 1), (out, 1)])
            assert ec == 0
            outs.append(out.cpu().numpy())
    assert np.array_equal(outs[0], want) and np.array_equal(outs[1], want)
