"""Launch-shape tuning (row A11): the C++ MLP forward pass and feature
function on the CPU; the synthetic loop against its serial C oracle and a
small end-to-end autotune / train / evaluate run on the GPU."""
import ctypes
import subprocess

import numpy as np
import pytest

from paper_2306_11686_gb300 import inputs


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as ge
    ge.build()
    from paper_2306_11686_gb300 import gf
    return gf


def np_forward(P, nin, width, depth, x):
    mean, sd = P[:nin], P[nin:2 * nin]
    a = (x - mean) / sd
    off, d = 2 * nin, nin
    for _ in range(depth):
        W = P[off:off + width * d].reshape(width, d)
        off += width * d
        b = P[off:off + width]
        off += width
        a = np.maximum(a @ W.T + b, 0.0)
        d = width
    w = P[off:off + width]
    return a @ w + P[off + width]


def test_mlp_forward_matches_numpy(lib):
    gf = lib
    rng = np.random.default_rng(0)
    nin, width, depth, n = 9, 64, 3, 50
    size = 2 * nin + (nin * width + width) + 2 * (width * width + width) + width + 1
    P = rng.standard_normal(size).astype(np.float32) * 0.3
    P[nin:2 * nin] = np.abs(P[nin:2 * nin]) + 0.5
    x = rng.standard_normal((n, nin)).astype(np.float32)
    y = np.zeros(n, dtype=np.float32)
    rc = gf.gf_mlp_forward(P.ctypes.data, nin, width, depth, x.ctypes.data, n, y.ctypes.data)
    assert rc == 0
    want = np_forward(P.astype(np.float64), nin, width, depth, x.astype(np.float64))
    assert np.allclose(y, want, rtol=1e-4, atol=1e-4)


def test_features_and_choose(lib):
    gf = lib
    from paper_2306_11686_gb300 import tune
    loop = dict(trip=1 << 20, bytes=64, flops=16, div_thresh=2 ** 30, rpc_thresh=2 ** 22, seed=7)
    shs = tune.shapes(152)
    f = tune.features(loop, shs, 152)
    assert f.shape == (len(shs), 9)
    assert f[0, 0] == 20.0 and f[0, 1] == 6.0 and f[0, 2] == 4.0
    assert abs(f[0, 3] - 0.25) < 1e-6 and abs(f[0, 4] - 1000 * 2 ** 22 / 2 ** 32) < 1e-4
    assert set(f[:, 5]) == {0.0, 1.0, 2.0, 3.0} and set(f[:, 8]) == {0.0, 1.0}
    # a "model" whose prediction is the block-size feature picks a 128-thread shape
    nin, width, depth = 9, 64, 3
    P = np.zeros(2 * nin + (nin * width + width) + 2 * (width * width + width) + width + 1, dtype=np.float32)
    P[nin:2 * nin] = 1.0
    off = 2 * nin
    P[off + 6] = 1.0                                   # unit 0 of layer 1 copies feature 6 (log2 block)
    off += nin * width + width
    P[off] = 1.0                                       # layer 2 passes unit 0 through
    off += width * width + width
    P[off] = 1.0                                       # layer 3 passes unit 0 through
    off += width * width + width
    P[off] = 1.0                                       # output = unit 0
    best = tune.choose(P, loop, shs, 152)
    assert shs[best][1] == 128


@pytest.mark.gpu
def test_synth_loop_parity(lib, oracle_bin, tmp_path):
    import torch
    gf = lib
    from paper_2306_11686_gb300 import tune
    cases = [dict(trip=1, bytes=8, flops=1, div_thresh=0, rpc_thresh=0, seed=1),
             dict(trip=5000, bytes=24, flops=7, div_thresh=2 ** 31, rpc_thresh=2 ** 24, seed=2),
             dict(trip=33333, bytes=256, flops=64, div_thresh=2 ** 32 - 1, rpc_thresh=0, seed=3),
             dict(trip=70001, bytes=8, flops=3, div_thresh=12345678, rpc_thresh=2 ** 22, seed=4)]
    with gf.Context(timeout_ns=10_000_000_000, heap_bytes=64 << 20, server_threads=2) as ctx:
        sms = ctx.grid_info("jacobi")[0]
        for d in cases:
            nx = d["trip"] * d["bytes"] // 8
            x = inputs.uniform_pm1(d["seed"] + 50, nx) * 4.0
            inputs.write_f64(tmp_path / "x.bin", x)
            subprocess.run([oracle_bin("synth"), str(d["trip"]), str(d["bytes"]), str(d["flops"]),
                            str(d["div_thresh"]), str(d["rpc_thresh"]), str(d["seed"]), tmp_path / "x.bin",
                            tmp_path / "z.bin"], check=True, capture_output=True)
            want = np.fromfile(tmp_path / "z.bin")
            xd = torch.from_numpy(x).cuda()
            for shape in [(sms, 256, 64, 0), (3, 96, 7, 1), (2 * sms, 1024, 4096, 1)]:
                zd = torch.full((d["trip"],), np.nan, dtype=torch.float64, device="cuda")
                rc = gf.gf_synth_run(ctx.h, ctypes.byref(tune.c_loop(d)), ctypes.c_void_p(xd.data_ptr()), nx,
                                     ctypes.c_void_p(zd.data_ptr()), tune.c_shapes([shape]), None)
                assert rc == 0
                assert np.array_equal(zd.cpu().numpy(), want), (d, shape)


@pytest.mark.gpu
def test_tune_pipeline_small(lib):
    """Autotune 60 small loops over all shapes, train on 48, evaluate on 12."""
    from paper_2306_11686_gb300 import tune
    import paper_2306_11686_gb300.tune as T
    orig = T.config4_loops
    T.config4_loops = lambda n, seed=4: [dict(d, trip=min(d["trip"], 1 << 18)) for d in orig(n, seed)]
    try:
        res = tune.run(n_loops=60, n_train=48, reps=1, epochs=40, log=None)
    finally:
        T.config4_loops = orig
    assert res["n"] == 12
    t = res["table"]
    assert 0.0 <= t["refined"]["mean"] <= t["top1"]["mean"] and t["plain"]["mean"] >= 0.0
    assert all(np.isfinite(v["mean"]) for v in res["retimed"].values())
    # the model has learned something: its top-1 shape beats a shape drawn at
    # random from the same candidates, on the held-out loops
    assert t["top1"]["mean"] < t["random"]["mean"], t
