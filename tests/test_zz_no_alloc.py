"""The allocation-free reduction entry point (for callers that may not
allocate device memory) against the existing worksharing reduction reached
through gf_run_main, on two calls in a row.

Tolerance as in the other reduction tests: min and max exactly equal; sums
each within 2 eps sum|x| of the exactly rounded sum, so within 4 eps sum|x| of
each other.  This file is collected last on purpose."""
import ctypes
import math

import numpy as np
import pytest

from paper_2306_11686_gb300 import inputs

pytestmark = pytest.mark.gpu
EPS = 2.0 ** -52


def existing(gf, ctx, xd, n):
    import torch
    out = torch.zeros(6, dtype=torch.int64, device="cuda")
    vd = torch.zeros(max(n, 1), dtype=torch.int64, device="cuda")
    rc, ec = ctx.run("reduce_probe", [n, 0, 1], [(xd, 1), (vd, 1), (out, 1)])
    assert ec == 0
    return out[:3].cpu().numpy().view(np.float64)


def noalloc(gf, xd, n, op, blocks=0):
    import torch
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    rc = gf.gf_reduce_f64_noalloc(ctypes.c_void_p(xd.data_ptr()), n, op, ctypes.c_void_p(out.data_ptr()),
                                  blocks, ctypes.c_void_p(stream.cuda_stream))
    assert rc == gf.GF_OK
    torch.cuda.synchronize()
    return out.item()


@pytest.mark.parametrize("n", [0, 1, 1000, 777777, 1 << 22])
def test_noalloc_matches_existing_twice(gf_lib, n):
    import torch
    gf = gf_lib
    x = inputs.uniform_pm1(17 + n, n) * 1e3
    xd = torch.from_numpy(x).cuda() if n else torch.zeros(1, dtype=torch.float64, device="cuda")
    absum = math.fsum(np.abs(x))
    with gf.Context(timeout_ns=10_000_000_000, heap_bytes=64 << 20) as ctx:
        ref = existing(gf, ctx, xd, n)
    for _ in range(2):
        got = [noalloc(gf, xd, n, op) for op in (gf.GF_REDUCE_SUM, gf.GF_REDUCE_MIN, gf.GF_REDUCE_MAX)]
        assert abs(got[0] - ref[0]) <= 4 * EPS * absum
        assert got[1] == ref[1] and got[2] == ref[2]
        if n:
            assert abs(got[0] - math.fsum(x)) <= 2 * EPS * absum


def test_noalloc_rejects_too_many_blocks(gf_lib):
    import torch
    gf = gf_lib
    xd = torch.ones(10, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc = gf.gf_reduce_f64_noalloc(ctypes.c_void_p(xd.data_ptr()), 10, gf.GF_REDUCE_SUM,
                                  ctypes.c_void_p(out.data_ptr()), 4096, None)
    assert rc == gf.GF_EINVAL
    assert noalloc(gf, xd, 10, gf.GF_REDUCE_SUM, blocks=2048) == 10.0
    assert noalloc(gf, xd, 10, gf.GF_REDUCE_SUM, blocks=1) == 10.0
