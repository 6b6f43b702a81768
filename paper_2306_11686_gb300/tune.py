"""Autotuner and learned launch-shape model for synthetic legacy loops.

Pipeline (the learned-model pattern on top of the runtime):
  1. `measure`: the autotuner times every candidate shape of every loop
     natively (gf_synth_time: CUDA events, fastest of `reps` runs after a
     warm-up); its per-loop optimum is the reference regret is measured
     against.
  2. `train`: an FP32 MLP (3 hidden layers of 64 ReLU units) learns, from
     gf_tune_features(loop, shape) on the training loops (torch), the log of
     a shape's time relative to that loop's fastest shape: only the ranking
     of a loop's shapes matters for the choice, and removing each loop's own
     scale leaves the network the shape effects to fit.
  3. `evaluate`: on held-out loops the model's choice (gf_mlp_choose, the C++
     forward pass) is compared with the autotuner's optimum:
     regret = t(model's shape) / t(best measured shape) - 1; also against the
     plain runtime's fixed shape (the heuristic fallback).

Feature extraction and inference are the library's own (C ABI); Python only
orchestrates and trains.
"""
from __future__ import annotations

import ctypes
import json
import math
import os
import time

import numpy as np

from . import gf, inputs

WIDTH, DEPTH = 64, 3
GRID_MULT = (1, 2, 4, 8)          # blocks per SM
BLOCKS = (128, 256, 512, 1024)
CHUNKS = (64, 512, 4096)
SCHEDS = (0, 1)


def shapes(sms: int):
    out = []
    for gm in GRID_MULT:
        for b in BLOCKS:
            for c in CHUNKS:
                for s in SCHEDS:
                    out.append((gm * sms, b, c, s))
    return out


# ---------------------------------------------------------------- batched loops
BATCH_CHUNKS = (1024, 4096, 16384, 65536)
GRAPH_BLOCKS = (128, 256)
GRAPH_GRID_MULT = (1, 2, 4, 8)


def tune_batch(ctx, bufs, n, reps=3, stream=None, chunks=BATCH_CHUNKS, scheds=SCHEDS):
    """The autotuner for a batched region of `n` loops (program loops_rpc,
    mode 1): every (chunk, schedule) candidate is timed `reps` times after a
    warm-up (CUDA events around the whole program); returns the fastest
    (chunk, sched) and the table {"chunk/sched": best seconds}."""
    import torch
    s = stream or torch.cuda.current_stream()
    table = {}
    for c in chunks:
        for sc in scheds:
            argv = [1, n, c, sc]
            ts = []
            for r in range(reps + 1):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(s)
                rc, ec = ctx.run("loops_rpc", argv, bufs)
                e1.record(s)
                torch.cuda.synchronize()
                if ec != 0:
                    raise RuntimeError(f"loops_rpc exit code {ec}")
                if r:
                    ts.append(e0.elapsed_time(e1) / 1e3)
            table[f"{c}/{sc}"] = min(ts)
    best = min(table, key=table.get)
    c, sc = best.split("/")
    return (int(c), int(sc)), table


def graph_candidates(trip, sms):
    """Launch shapes tried for one loop of the graph form: 128 or 256 threads,
    1 to 8 blocks per SM, never more blocks than the loop has iterations
    for, plus the one-pass cover of the loop."""
    out = set()
    for b in GRAPH_BLOCKS:
        cover = max(1, -(-trip // b))
        out.add((min(cover, 8 * sms), b))
        for m in GRAPH_GRID_MULT:
            out.add((max(1, min(m * sms, cover)), b))
    return sorted(out)


def tune_graph(ctx, trips, a, off, x, y, z, fails, sms, reps=2, stream=None):
    """The autotuner for the graph form: each loop alone (a one-node graph) is
    timed under each of its candidate shapes; returns per-loop grid and block
    arrays (uint32) and the summed per-loop best and default times."""
    grid = np.zeros(len(trips), dtype=np.uint32)
    block = np.zeros(len(trips), dtype=np.uint32)
    best_sum = default_sum = 0.0
    P = lambda arr: ctypes.c_void_p(arr.ctypes.data)
    for k in range(len(trips)):
        t1, a1, o1 = trips[k:k + 1].copy(), a[k:k + 1].copy(), off[k:k + 1].copy()
        best = None
        for g, b in graph_candidates(int(trips[k]), sms):
            g1, b1 = np.array([g], dtype=np.uint32), np.array([b], dtype=np.uint32)
            ms = ctypes.c_float()
            rc = gf.gf_loops_rpc_graph(ctx.h, 1, P(t1), P(a1), P(o1), ctypes.c_void_p(x.data_ptr()),
                                       ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(z.data_ptr()),
                                       ctypes.c_void_p(fails.data_ptr()), P(g1), P(b1), 1, reps, stream,
                                       ctypes.byref(ms))
            if rc != gf.GF_OK:
                raise gf.GFError(rc, f"gf_loops_rpc_graph(loop {k})")
            if best is None or ms.value < best[0]:
                best = (ms.value, g, b)
            if b == 256 and g == min(-(-int(trips[k]) // 256), 8 * sms):
                default_sum += ms.value
        best_sum += best[0]
        grid[k], block[k] = best[1], best[2]
    return grid, block, best_sum, default_sum


def heuristic_shape(sms: int):
    """The plain runtime's fixed choice: 4 blocks of 256 per SM, small static items."""
    return (4 * sms, 256, 64, 0)


def config4_loops(n: int = 2000, seed: int = 4):
    """trip log-uniform 2^10..2^26, bytes/iter in {8..256}, flops 1..64,
    divergent fraction U[0, 0.5], RPC rate U[0, 1e-3] (as thresholds of 2^32)."""
    trip = inputs.loguniform_int(seed, n, 1 << 10, 1 << 26).astype(np.int64)
    bytes_ = np.array([8, 16, 32, 64, 128, 256], dtype=np.int64)[inputs.uniform_int(seed + 1, n, 0, 5)]
    flops = inputs.uniform_int(seed + 2, n, 1, 64)
    div = inputs.uniform01(seed + 3, n) * 0.5
    rpc = inputs.uniform01(seed + 4, n) * 1e-3
    loops = []
    for k in range(n):
        loops.append(dict(trip=int(trip[k]), bytes=int(bytes_[k]), flops=int(flops[k]),
                          div_thresh=int(div[k] * 2 ** 32), rpc_thresh=int(rpc[k] * 2 ** 32), seed=1000 + k))
    return loops


def c_loop(d):
    L = gf.gf_synth_loop()
    L.trip, L.bytes, L.flops = d["trip"], d["bytes"], d["flops"]
    L.div_thresh, L.rpc_thresh, L.seed = d["div_thresh"], d["rpc_thresh"], d["seed"]
    return L


def c_shapes(shs):
    arr = (gf.gf_shape * len(shs))()
    for k, (g, b, c, s) in enumerate(shs):
        arr[k].grid, arr[k].block, arr[k].chunk, arr[k].sched = g, b, c, s
    return arr


def features(loop, shs, sms):
    L = c_loop(loop)
    out = np.zeros((len(shs), gf.GF_TUNE_NFEAT), dtype=np.float32)
    sa = c_shapes(shs)
    for k in range(len(shs)):
        gf.gf_tune_features(ctypes.byref(L), ctypes.byref(sa[k]), sms, out[k].ctypes.data_as(ctypes.c_void_p))
    return out


def measure(ctx, loops, shs, x, z, reps=2, stream=None, log=None):
    """ms[loop, shape] from the native timer."""
    ms = np.zeros((len(loops), len(shs)), dtype=np.float32)
    sa = c_shapes(shs)
    xlen = x.numel()
    t0 = time.time()
    for k, d in enumerate(loops):
        L = c_loop(d)
        row = (ctypes.c_float * len(shs))()
        rc = gf.gf_synth_time(ctx.h, ctypes.byref(L), ctypes.c_void_p(x.data_ptr()), xlen,
                              ctypes.c_void_p(z.data_ptr()), sa, len(shs), reps, stream, row)
        if rc != gf.GF_OK:
            raise gf.GFError(rc, f"gf_synth_time(loop {k})")
        ms[k] = np.frombuffer(row, dtype=np.float32)
        if log and (k + 1) % 100 == 0:
            log(f"measured {k + 1}/{len(loops)} loops in {time.time() - t0:.1f} s")
    return ms


def train(X, y, epochs=300, seed=0, device=None, log=None):
    """FP32 MLP (3 x 64 ReLU) regression of log(ms); returns the flat parameter
    vector in gf_mlp_forward's layout."""
    import torch
    torch.manual_seed(seed)
    dev = device or ("cuda" if torch.cuda.is_available() else "cpu")
    mean = X.mean(0)
    sd = X.std(0) + 1e-6
    Xt = torch.from_numpy((X - mean) / sd).float().to(dev)
    yt = torch.from_numpy(y).float().to(dev)
    layers, d = [], X.shape[1]
    for _ in range(DEPTH):
        layers += [torch.nn.Linear(d, WIDTH), torch.nn.ReLU()]
        d = WIDTH
    layers.append(torch.nn.Linear(d, 1))
    net = torch.nn.Sequential(*layers).to(dev)
    opt = torch.optim.Adam(net.parameters(), lr=2e-3)
    sched = torch.optim.lr_scheduler.CosineAnnealingLR(opt, epochs)
    n = Xt.shape[0]
    bs = 4096
    for ep in range(epochs):
        perm = torch.randperm(n, device=dev)
        tot = 0.0
        for i in range(0, n, bs):
            idx = perm[i:i + bs]
            loss = torch.mean((net(Xt[idx]).squeeze(1) - yt[idx]) ** 2)
            opt.zero_grad()
            loss.backward()
            opt.step()
            tot += loss.item() * len(idx)
        sched.step()
        if log and (ep + 1) % 50 == 0:
            log(f"epoch {ep + 1}: mse {tot / n:.4f}")
    parts = [mean.astype(np.float32), sd.astype(np.float32)]
    for m in net:
        if isinstance(m, torch.nn.Linear):
            parts += [m.weight.detach().cpu().numpy().astype(np.float32).reshape(-1),
                      m.bias.detach().cpu().numpy().astype(np.float32).reshape(-1)]
    return np.concatenate(parts).astype(np.float32)


def choose(params, loop, shs, sms):
    best = ctypes.c_int(-1)
    rc = gf.gf_mlp_choose(params.ctypes.data_as(ctypes.c_void_p), WIDTH, DEPTH, ctypes.byref(c_loop(loop)),
                          c_shapes(shs), len(shs), sms, ctypes.byref(best))
    if rc != gf.GF_OK:
        raise gf.GFError(rc, "gf_mlp_choose")
    return best.value


def topk(params, loop, shs, sms, k):
    idx = (ctypes.c_int * k)()
    rc = gf.gf_mlp_topk(params.ctypes.data_as(ctypes.c_void_p), WIDTH, DEPTH, ctypes.byref(c_loop(loop)),
                        c_shapes(shs), len(shs), sms, k, idx)
    if rc != gf.GF_OK:
        raise gf.GFError(rc, "gf_mlp_topk")
    return list(idx)


def _stats(r):
    r = np.asarray(r)
    return {"mean": float(r.mean()), "p90": float(np.percentile(r, 90)), "max": float(r.max())}


def evaluate(params, loops, shs, ms, sms, refine_k=3, ctx=None, x=None, z=None, reps=5):
    """Regret of the model's choice on held-out loops.

    top1:    the model's single choice;
    refined: the fastest (by the table's measurement) of the model's top
             `refine_k` predictions -- the model prunes 96 shapes to k timed runs;
    table:   regret against the minimum of the autotuner's table (biased
             upwards: that minimum is the luckiest of 96 noisy timings);
    retimed: the model's choices, the autotuner's choice and the plain shape
             re-timed side by side (`reps` runs each), regret against the
             autotuner's choice -- the fair comparison.  Needs ctx, x, z."""
    h = shs.index(heuristic_shape(sms))
    res = {"n": len(loops), "refine_k": refine_k}
    t1, tr, th, trand = [], [], [], []
    retimed = {"top1": [], "refined": [], "plain": []}
    for k, d in enumerate(loops):
        cand = topk(params, d, shs, sms, refine_k)
        c1 = cand[0]
        cr = min(cand, key=lambda s: ms[k, s])
        auto = int(np.argmin(ms[k]))
        best = float(ms[k, auto])
        t1.append(float(ms[k, c1]) / best - 1.0)
        tr.append(float(ms[k, cr]) / best - 1.0)
        th.append(float(ms[k, h]) / best - 1.0)
        trand.append(float(np.mean(ms[k])) / best - 1.0)     # a shape drawn uniformly at random
        if ctx is not None:
            picks = [c1, cr, auto, h]
            sa = c_shapes([shs[s] for s in picks])
            row = (ctypes.c_float * 4)()
            rc = gf.gf_synth_time(ctx.h, ctypes.byref(c_loop(d)), ctypes.c_void_p(x.data_ptr()), x.numel(),
                                  ctypes.c_void_p(z.data_ptr()), sa, 4, reps, None, row)
            if rc != gf.GF_OK:
                raise gf.GFError(rc, "gf_synth_time (re-timing)")
            ta = row[2]
            retimed["top1"].append(row[0] / ta - 1.0)
            retimed["refined"].append(row[1] / ta - 1.0)
            retimed["plain"].append(row[3] / ta - 1.0)
    res["table"] = {"top1": _stats(t1), "refined": _stats(tr), "plain": _stats(th), "random": _stats(trand)}
    if ctx is not None:
        res["retimed"] = {k: _stats(v) for k, v in retimed.items()}
        res["learned_vs_plain_speedup_geomean"] = float(np.exp(np.mean(
            np.log1p(np.array(retimed["plain"])) - np.log1p(np.array(retimed["refined"])))))
    return res


def run(n_loops=2000, n_train=1600, reps=2, epochs=300, out=None, log=print):
    """Full pipeline on cuda:0; returns the evaluation dict."""
    import torch
    ctx = gf.Context(server_threads=4, heap_bytes=64 << 20, timeout_ns=60_000_000_000)
    sms = ctx.grid_info("jacobi")[0]
    shs = shapes(sms)
    loops = config4_loops(n_loops)
    xlen = max(d["trip"] * d["bytes"] // 8 for d in loops)
    x = torch.empty(xlen, dtype=torch.float64, device="cuda").uniform_(-1, 1)
    z = torch.empty(max(d["trip"] for d in loops), dtype=torch.float64, device="cuda")
    t0 = time.time()
    ms = measure(ctx, loops, shs, x, z, reps=reps, log=log)
    t_meas = time.time() - t0
    X = np.concatenate([features(d, shs, sms) for d in loops[:n_train]])
    lm = np.log(np.maximum(ms[:n_train], 1e-4))
    y = (lm - lm.min(axis=1, keepdims=True)).reshape(-1)     # log time relative to the loop's fastest shape
    params = train(X, y, epochs=epochs, log=log)
    res = evaluate(params, loops[n_train:], shs, ms[n_train:], sms, ctx=ctx, x=x, z=z)
    res.update({"loops": n_loops, "train": n_train, "shapes": len(shs), "reps": reps,
                "measure_s": round(t_meas, 1)})
    if out:
        np.savez(out, ms=ms, params=params, sms=sms)
        with open(os.path.splitext(out)[0] + ".json", "w") as f:
            json.dump(res, f, indent=1)
    ctx.close()
    return res
