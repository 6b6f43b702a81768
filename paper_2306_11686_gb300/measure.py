"""Measurements of the non-benchmark configurations (used by bench.py --workload).

Each function prints one JSON line with its own metric:
  stress   printf calls/s with warp aggregation on vs off (printf-only loop,
           2^20 iterations x 4 calls), device RPC p50/p99, heap alloc/free
           pairs/s (2^20 x 8 pairs, log-uniform 16 B..64 KiB), the full
           stress program's time;
  batch    256 axpy loops (trip 2^10..2^22): one region per loop vs one
           batched region vs one CUDA graph; loop GB/s (24 B per iteration);
  learned  autotuner + MLP over 2000 synthetic loops (1600 train / 400
           held out): regret vs the autotuner's optimum, speedup vs the plain
           runtime's fixed shape;
  serve    64 served programs (CSR SpMV, 1M rows, 16 nnz/row, 10 passes,
           ~64 libc requests per pass) under continuous batching: calls/s,
           RPC p50/p99, admission -> done latency, SpMV GB/s;
  split    the persistent grid against the paper's kernel split (one RPC and
           one host-launched kernel per region): a 64-byte region, config 1's
           axpy program, the 256 per-loop regions, Jacobi 256^3 x 100;
  link     the host link's measured peaks, the denominators of the RPC and
           bulk-I/O figures: pinned cudaMemcpy H2D/D2H and grid-wide device
           stores/loads of mapped host memory for 64 B .. 64 MiB, and the
           single-thread RPC round trip (empty call; the paper's 128-byte
           fprintf experiment).
"""
from __future__ import annotations

import json
import os
import shutil
import tempfile
import time

import numpy as np

from . import gf, inputs


def _out_dir(args):
    """Where programs' output files go: --out-dir, else /dev/shm when it is a
    writable tmpfs (as for the benchmark), else the system temp directory."""
    if getattr(args, "out_dir", None):
        return args.out_dir
    return "/dev/shm" if os.path.isdir("/dev/shm") and os.access("/dev/shm", os.W_OK) else None


def _timed_run(ctx, stream, name, argv, bufs):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    rc, ec = ctx.run(name, argv, bufs)
    e1.record(stream)
    torch.cuda.synchronize()
    if ec != 0:
        raise RuntimeError(f"{name} exit code {ec}")
    return e0.elapsed_time(e1) / 1e3


def printf_rate(T=1 << 20, out_dir=None, server_threads=4):
    """The printf-only half of the stress program (T iterations x 4 printf,
    mixed int/double formats) with warp aggregation on and off: calls/s, the
    device round-trip p50/p99 and the lane records per ring slot."""
    import torch
    tmp = tempfile.mkdtemp(prefix="gfprintf", dir=out_dir)
    stream = torch.cuda.Stream()
    out = {}
    for agg in (1, 0):
        with gf.Context(aggregate=agg, stream=stream, heap_bytes=64 << 20, server_threads=server_threads,
                        stdout_path=os.path.join(tmp, "out.txt"), timeout_ns=int(120e9)) as ctx:
            _timed_run(ctx, stream, "printf_only", [1 << 14], [])          # warm-up
            t = _timed_run(ctx, stream, "printf_only", [T], [])
            st = ctx.stats()
            calls = int(st.rpc_calls[gf.OP_PRINTF])
            if calls != 4 * T:
                raise RuntimeError(f"printf_only: {calls} calls served, {4 * T} issued")
            out["aggregated" if agg else "per_thread"] = {
                "calls_per_s": round(4 * T / t), "seconds": round(t, 4), "rpc_p50_ns": st.rpc_p50_ns,
                "rpc_p99_ns": st.rpc_p99_ns, "records_per_slot": round(calls / max(1, int(st.rpc_slots[gf.OP_PRINTF])), 2)}
    shutil.rmtree(tmp, ignore_errors=True)
    out["aggregation_speedup"] = round(out["aggregated"]["calls_per_s"] / out["per_thread"]["calls_per_s"], 2)
    out["workload"] = f"{T} iterations x 4 printf, host server {server_threads} threads"
    return out


def stress(args):
    import torch
    T = 1 << 20
    nthr = getattr(args, "server_threads", None) or 4
    tmp = tempfile.mkdtemp(prefix="gfstress", dir=_out_dir(args))
    sizes = torch.from_numpy(inputs.loguniform_int(3, 8 * T, 16, 65536).astype(np.int32)).cuda()
    cs = torch.zeros(T, dtype=torch.int64, device="cuda")
    fails = torch.zeros(1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.Stream()
    out = {}
    for agg in (1, 0):
        with gf.Context(aggregate=agg, stream=stream, heap_bytes=8 << 30, heap_small_pct=95, server_threads=nthr,
                        stdout_path=os.path.join(tmp, "out.txt"), timeout_ns=int(120e9)) as ctx:
            _timed_run(ctx, stream, "printf_only", [1 << 14], [])          # warm-up
            b0 = ctx.stats().host_ring_bytes
            t = _timed_run(ctx, stream, "printf_only", [T], [])
            st = ctx.stats()
            out[agg] = dict(calls_per_s=4 * T / t, seconds=t, p50_ns=st.rpc_p50_ns, p99_ns=st.rpc_p99_ns,
                            slots=int(st.rpc_slots[gf.OP_PRINTF]), calls=int(st.rpc_calls[gf.OP_PRINTF]),
                            ring_GBps=(st.host_ring_bytes - b0) / t / 1e9,
                            ring_bytes_per_call=(st.host_ring_bytes - b0) / (4 * T))
            if agg:
                hb = [(sizes, 1), (cs, 1), (fails, 1)]
                _timed_run(ctx, stream, "heap_only", [T], hb)                # warm-up: slabs carved
                th = min(_timed_run(ctx, stream, "heap_only", [T], hb) for _ in range(3))
                hst = ctx.stats()
                ts = min(_timed_run(ctx, stream, "stress", [T], hb) for _ in range(3))
                sst = ctx.stats()
    line = {"metric": "RPC calls/s + p99 latency", "value": round(out[1]["calls_per_s"]), "unit": "calls/s",
            "n_gpus": 1, "higher_is_better": True, "dtype": "int/bytes", "data": "synthetic",
            "config": {"workload": f"2^20 iterations x 4 printf (int/double formats), host server {nthr} threads",
                       "output": os.path.dirname(tmp)},
            "detail": {"aggregated": out[1], "per_thread": out[0],
                       "aggregation_speedup": out[1]["calls_per_s"] / out[0]["calls_per_s"],
                       "heap_pairs_per_s": 8 * T / th, "heap_fail": int(hst.heap_fail),
                       "stress_program_s": ts, "stress_slots": int(sst.rpc_slots[gf.OP_PRINTF]),
                       "stress_calls": int(sst.rpc_calls[gf.OP_PRINTF])}}
    print(json.dumps(line))
    shutil.rmtree(tmp, ignore_errors=True)


def batch(args):
    import ctypes
    import torch
    trips, a, off, x, y = inputs.loops_inputs()
    n, total = len(trips), int(trips.sum())
    dv = lambda v: torch.from_numpy(np.ascontiguousarray(v)).cuda()
    td, ad, od, xd, yd = dv(trips), dv(a), dv(off), dv(x), dv(y)
    z = torch.zeros(total, dtype=torch.float64, device="cuda")
    prefix = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.Stream()
    res = {}
    with gf.Context(stream=stream, heap_bytes=64 << 20, timeout_ns=int(60e9)) as ctx:
        for label, argv in [("regions", [0, n, 1, 0]), ("batched_dynamic", [1, n, 4096, 1]),
                            ("batched_static", [1, n, 4096, 0])]:
            bufs = [(td, 1), (ad, 1), (od, 1), (xd, 1), (yd, 1), (z, 1), (prefix, 1)]
            _timed_run(ctx, stream, "loops", argv, bufs)
            ts = [_timed_run(ctx, stream, "loops", argv, bufs) for _ in range(3)]
            st = ctx.stats()
            res[label] = {"program_s": min(ts), "region_s": st.region_ns / 1e9, "regions": int(st.regions),
                          "GBps_regions": 24 * total / (st.region_ns / 1e9) / 1e9}
    ms = ctypes.c_float()
    P = lambda arr: ctypes.c_void_p(arr.ctypes.data)
    rc = gf.gf_axpy_batch_graph(n, P(trips), P(a), P(off), ctypes.c_void_p(xd.data_ptr()),
                                ctypes.c_void_p(yd.data_ptr()), ctypes.c_void_p(z.data_ptr()), None, None, 5,
                                ctypes.c_void_p(stream.cuda_stream), ctypes.byref(ms))
    res["graph"] = {"replay_s": ms.value / 1e3, "GBps": 24 * total / (ms.value / 1e3) / 1e9, "rc": rc}
    res["with_rpc_and_heap"] = batch_rpc(trips, a, off, td, ad, od, xd, yd, total, stream, _out_dir(args))
    best = res["batched_dynamic"]["GBps_regions"]
    line = {"metric": "loop GB/s (% HBM peak)", "value": round(best, 1), "unit": "GB/s", "n_gpus": 1,
            "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{n} axpy loops, trip log-uniform 2^10..2^22, {total} iterations, 24 B/iter"},
            "detail": res}
    print(json.dumps(line))


def batch_rpc(trips, a, off, td, ad, od, xd, yd, total, stream, out_dir):
    """The 256 loops with a heap block and a printf every 4096 iterations
    (loops_rpc): one region per loop, one batched region at the fixed chunk
    4096 / dynamic and at the autotuner's (chunk, schedule), and the graph
    form at its default shapes and at the autotuner's per-loop shapes.  Loop
    GB/s counts the 24 B per iteration of the loop bodies."""
    import ctypes
    import torch
    from . import tune
    n = len(trips)
    z = torch.zeros(total, dtype=torch.float64, device="cuda")
    fails = torch.zeros(1, dtype=torch.int64, device="cuda")
    prefix = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    bufs = [(td, 1), (ad, 1), (od, 1), (xd, 1), (yd, 1), (z, 1), (prefix, 1), (fails, 1)]
    out = {}
    with gf.Context(stream=stream, heap_bytes=1 << 30, server_threads=4, timeout_ns=int(60e9),
                    stdout_path=os.devnull) as ctx:
        t0 = time.time()
        (chunk, sched), table = tune.tune_batch(ctx, bufs, n, reps=3, stream=stream)
        out["batch_tuning"] = {"choice": {"chunk": chunk, "sched": sched}, "table_s": table,
                               "tuning_s": round(time.time() - t0, 2)}
        for label, argv in [("regions", [0, n, 1, 0]), ("batched_fixed_4096_dynamic", [1, n, 4096, 1]),
                            ("batched_tuned", [1, n, chunk, sched])]:
            _timed_run(ctx, stream, "loops_rpc", argv, bufs)
            ts = [_timed_run(ctx, stream, "loops_rpc", argv, bufs) for _ in range(3)]
            st = ctx.stats()
            out[label] = {"program_s": min(ts), "GBps": 24 * total / min(ts) / 1e9, "regions": int(st.regions),
                          "printf_calls": int(st.rpc_calls[gf.OP_PRINTF]),
                          "records_per_slot": round(int(st.rpc_calls[gf.OP_PRINTF]) /
                                                    max(1, int(st.rpc_slots[gf.OP_PRINTF])), 2)}
        sms = ctx.grid_info("loops_rpc")[0]
        t0 = time.time()
        grid, block, tuned_sum, default_sum = tune.tune_graph(ctx, trips, a, off, xd, yd, z, fails, sms, reps=2,
                                                              stream=ctypes.c_void_p(stream.cuda_stream))
        out["graph_tuning"] = {"per_loop_best_sum_s": tuned_sum / 1e3, "per_loop_default_sum_s": default_sum / 1e3,
                               "tuning_s": round(time.time() - t0, 2)}
        P = lambda arr: ctypes.c_void_p(arr.ctypes.data)
        for label, g, b in [("graph_default", None, None), ("graph_tuned", P(grid), P(block))]:
            ms = ctypes.c_float()
            rc = gf.gf_loops_rpc_graph(ctx.h, n, P(trips), P(a), P(off), ctypes.c_void_p(xd.data_ptr()),
                                       ctypes.c_void_p(yd.data_ptr()), ctypes.c_void_p(z.data_ptr()),
                                       ctypes.c_void_p(fails.data_ptr()), g, b, 1, 3,
                                       ctypes.c_void_p(stream.cuda_stream), ctypes.byref(ms))
            if rc != gf.GF_OK:
                raise gf.GFError(rc, "gf_loops_rpc_graph")
            out[label] = {"replay_s": ms.value / 1e3, "GBps": 24 * total / (ms.value / 1e3) / 1e9}
    out["heap_fails"] = int(fails.item())
    return out


def learned(args):
    from . import tune
    res = tune.run(n_loops=2000, n_train=1600, reps=2, epochs=300, log=lambda m: print("#", m, flush=True),
                   out=os.path.join(args.out_dir or ".", "learned_ds.npz") if args.out_dir else None)
    line = {"metric": "learned vs plain config", "value": round(res["retimed"]["top1"]["mean"], 4),
            "unit": "mean regret of the model's top-1 shape, re-timed beside the autotuner's (top-3 in detail)",
            "n_gpus": 1, "higher_is_better": False, "dtype": "fp32 model", "data": "synthetic",
            "config": {"workload": "2000 synthetic loops (1600 train / 400 held out), 96 launch shapes"},
            "detail": res}
    print(json.dumps(line))


SERVE_THREADS = 4


def _serve_threads(args):
    return getattr(args, "server_threads", None) or SERVE_THREADS


def _spmv_alone(serve, n, P, tmp, fp64_peak=None):
    """The served SpMV without its libc requests: P programs at once (16
    instances), device time of the whole set (first start to last end)."""
    progs = [serve.Program(p, n, 10, 64, requests=False) for p in range(P)]
    outs = [os.path.join(tmp, f"norq{p}.bin") for p in range(P)]
    serve.serve(progs, outs, max_concurrent=min(16, P), heap_bytes=256 << 20, ring_slots=1024,
                server_threads=SERVE_THREADS, stdout_path=os.devnull)             # warm-up
    for pr in progs:
        pr.reset()
    recs, agg = serve.serve(progs, outs, max_concurrent=min(16, P), heap_bytes=256 << 20, ring_slots=1024,
                            server_threads=SERVE_THREADS, stdout_path=os.devnull)
    t = agg["device_s"]
    nbytes = sum(pr.bytes_moved() for pr in progs)
    ops = sum(pr.fp64_ops() for pr in progs)
    out = {"programs": P, "device_s": t, "GBps": nbytes / t / 1e9, "hbm_frac": None,
           "fp64_Gops": ops / t / 1e9, "fp64_frac": None if not fp64_peak else ops / t / fp64_peak,
           "errors": sum(1 for r in recs if r["rc"] or r["exit"])}
    peak = _hbm_peak()
    if peak:
        out["hbm_frac"] = out["GBps"] / peak
    return out


def spmv(args):
    """The served SpMV alone: one request-free program (10 passes of a 1 M-row
    CSR SpMV, 16 nonzeros per row) after a warm-up, against the HBM and FP64
    peaks."""
    import ctypes
    from . import serve
    tmp = tempfile.mkdtemp(prefix="gfspmv", dir=_out_dir(args))
    ms, adds = ctypes.c_float(), ctypes.c_double()
    gf.gf_fp64_add_rate(0, 512, None, ctypes.byref(ms), ctypes.byref(adds))
    peak = adds.value / (ms.value / 1e3)
    one = _spmv_alone(serve, 1 << 20, 1, tmp, peak)
    line = {"metric": "loop GB/s (% HBM peak)", "value": round(one["GBps"], 1), "unit": "GB/s", "n_gpus": 1,
            "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "CSR SpMV 1M rows x 16 nnz, 10 passes, one program, no requests"},
            "roofline": {"bound": "fp64", "achieved": round(one["fp64_Gops"], 1), "peak": round(peak / 1e9, 1),
                         "unit": "G FP64 op/s", "frac": round(one["fp64_frac"], 4)},
            "detail": one}
    print(json.dumps(line))
    shutil.rmtree(tmp, ignore_errors=True)


def serve_run(args):
    import ctypes
    from . import serve
    P, n = 64, 1 << 20
    os.environ.setdefault("GF_SERVE_VAR0", "zero")
    os.environ.setdefault("GF_SERVE_VAR1", "one-1")
    os.environ.pop("GF_SERVE_VAR2", None)
    tmp = tempfile.mkdtemp(prefix="gfserve", dir=_out_dir(args))
    t0 = time.time()
    progs = [serve.Program(p, n, 10, 64) for p in range(P)]
    t_gen = time.time() - t0
    outs = [os.path.join(tmp, f"rec{p}.bin") for p in range(P)]
    runs = []
    for _ in range(3):                  # the median of three runs (a run varies by about 10%)
        recs, agg = serve.serve(progs, outs, max_concurrent=16, rate_hz=400.0, heap_bytes=1 << 30, ring_slots=1024,
                                server_threads=_serve_threads(args), stdout_path=os.path.join(tmp, "out.txt"))
        agg["errors"] = sum(1 for r in recs if r["rc"] or r["exit"])
        runs.append(agg)
    runs.sort(key=lambda a: a["calls_per_s"])
    agg = dict(runs[1])
    agg["calls_per_s_runs"] = [round(a["calls_per_s"]) for a in runs]
    agg["errors"] = sum(a["errors"] for a in runs)
    agg["server_threads"] = _serve_threads(args)
    agg["input_gen_s"] = t_gen
    # the plain single-program runtime on the same GPU: the same programs one at a time
    for pr in progs:
        pr.reset()
    recs1, one = serve.serve(progs, outs, max_concurrent=1, heap_bytes=1 << 30, ring_slots=1024,
                             server_threads=_serve_threads(args), stdout_path=os.path.join(tmp, "out1.txt"))
    agg["single_program_runtime"] = {k: one[k] for k in ("wall_s", "calls_per_s", "rpc_p50_ns_median",
                                                          "rpc_p99_ns_max", "latency_p50_s", "latency_p99_s")}
    agg["single_program_runtime"]["errors"] = sum(1 for r in recs1 if r["rc"] or r["exit"])
    del progs
    # the SpMV alone (no libc requests): one program, then 16 at once
    ms, adds = ctypes.c_float(), ctypes.c_double()
    gf.gf_fp64_add_rate(0, 8192, None, ctypes.byref(ms), ctypes.byref(adds))
    peak = adds.value / (ms.value / 1e3)
    agg["spmv_only"] = {"one": _spmv_alone(serve, n, 1, tmp, peak), "sixteen": _spmv_alone(serve, n, 16, tmp, peak),
                        "fp64_add_peak_Gops": peak / 1e9,
                        "bytes_per_spmv": 16 * n * 12 + (n + 1) * 8 + 2 * n * 8}
    line = {"metric": "RPC calls/s + p99 latency", "value": round(agg["calls_per_s"]), "unit": "calls/s",
            "n_gpus": 1, "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "64 programs, CSR SpMV 1M rows x 16 nnz, 10 passes, Poisson libc requests, "
                                   "16 concurrent instances, arrivals 400/s",
                       "output": os.path.dirname(tmp)},
            "detail": agg}
    print(json.dumps(line))
    shutil.rmtree(tmp, ignore_errors=True)


def e1(args):
    """The paper's allocator grid (Sec. 5.1, Fig. 6): teams x threads/team in
    {1, 32, 64, 128, 256}^2, one 64 B allocate/use/free per thread, for the
    slab heap, the paper's balanced and generic allocators, and CUDA malloc."""
    import ctypes
    kinds = {0: "slab", 1: "balanced", 2: "generic", 3: "cuda_malloc"}
    sizes = (1, 32, 64, 128, 256)
    table = {}
    with gf.Context(heap_bytes=1 << 30, timeout_ns=int(60e9)) as ctx:
        for k, name in kinds.items():
            for teams in sizes:
                for threads in sizes:
                    ms, fails = ctypes.c_float(), ctypes.c_uint64()
                    rc = gf.gf_alloc_e1(ctx.h, k, teams, threads, 64, 5, None, ctypes.byref(ms),
                                        ctypes.byref(fails))
                    if rc:
                        raise gf.GFError(rc, f"gf_alloc_e1({name}, {teams}, {threads})")
                    table[f"{name}/{teams}x{threads}"] = {"s": ms.value / 1e3, "fails": int(fails.value)}
    big = lambda n: table[f"{n}/256x256"]["s"]
    line = {"metric": "allocator alloc/free pairs/s", "value": round(65536 / big("slab")), "unit": "pairs/s",
            "n_gpus": 1, "higher_is_better": True, "dtype": "bytes", "data": "synthetic",
            "config": {"workload": "paper Fig. 6 grid: teams x threads in {1,32,64,128,256}^2, 64 B per thread"},
            "detail": {"seconds": table,
                       "speedup_vs_cuda_malloc_256x256": big("cuda_malloc") / big("slab"),
                       "speedup_vs_balanced_256x256": big("balanced") / big("slab"),
                       "balanced_vs_cuda_malloc_256x256": big("cuda_malloc") / big("balanced"),
                       "balanced_vs_cuda_malloc_1x1": table["cuda_malloc/1x1"]["s"] / table["balanced/1x1"]["s"],
                       "balanced_vs_cuda_malloc_256x32": table["cuda_malloc/256x32"]["s"]
                       / table["balanced/256x32"]["s"]}}
    print(json.dumps(line))


def link(args):
    import torch
    sizes = [64 << (2 * k) for k in range(11)]                  # 64 B .. 64 MiB
    big = sizes[-1]
    dev = torch.zeros(big, dtype=torch.uint8, device="cuda")
    host = torch.zeros(big, dtype=torch.uint8).pin_memory()
    stream = torch.cuda.Stream()
    table = {}
    for n in sizes:
        reps = 200 if n <= (1 << 20) else 20
        for name, dst, src in (("memcpy_h2d", dev[:n], host[:n]), ("memcpy_d2h", host[:n], dev[:n])):
            with torch.cuda.stream(stream):
                for _ in range(3):
                    dst.copy_(src, non_blocking=True)
                e0, e1_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(reps):
                    dst.copy_(src, non_blocking=True)
                e1_.record(stream)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1_) / 1e3 / reps
            table[f"{name}/{n}"] = {"us": round(t * 1e6, 3), "GBps": round(n / t / 1e9, 3)}
    reps = 20
    ns = torch.zeros(max(reps, 1000), dtype=torch.int64, device="cuda")
    with gf.Context(bulk_bytes=big, heap_bytes=64 << 20, timeout_ns=int(60e9), stdout_path=os.devnull) as ctx:
        for n in sizes:
            for d, name in ((0, "device_store_mapped"), (1, "device_load_mapped")):
                rc, ec = ctx.run("link_probe", [n, reps, d], [(dev, 1), (ns, 1)])
                if ec != 0:
                    raise RuntimeError(f"link_probe exit {ec}")
                t = float(np.median(ns[1:reps].cpu().numpy())) / 1e9
                table[f"{name}/{n}"] = {"us": round(t * 1e6, 3), "GBps": round(n / t / 1e9, 3)}
        rtt = {}
        for mode, name in ((0, "clock"), (1, "fprintf_128B")):
            rc, ec = ctx.run("rpc_latency", [1000, mode], [(ns, 1)])
            if ec != 0:
                raise RuntimeError(f"rpc_latency exit {ec}")
            v = ns[:1000].cpu().numpy().astype(np.float64) / 1e3
            rtt[name] = {"mean_us": round(float(v.mean()), 3), "p50_us": round(float(np.median(v)), 3),
                         "p99_us": round(float(np.percentile(v, 99)), 3), "calls_per_s": round(1e6 / v.mean())}
    peak = {k: max(v["GBps"] for kk, v in table.items() if kk.startswith(k + "/"))
            for k in ("memcpy_h2d", "memcpy_d2h", "device_store_mapped", "device_load_mapped")}
    line = {"metric": "host link GB/s and RPC round trip", "value": peak["device_store_mapped"], "unit": "GB/s",
            "n_gpus": 1, "higher_is_better": True, "dtype": "bytes", "data": "synthetic",
            "config": {"workload": "message sizes 64 B .. 64 MiB; 1000 single-thread RPCs per kind"},
            "detail": {"peak_GBps": peak, "single_thread_rpc": rtt, "table": table}}
    print(json.dumps(line))


def _hbm_peak():
    try:
        with open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except Exception:
        return None


def axpy_regions(logs, reps=5):
    """One axpy loop z = 2.5 x + y through the plain runtime (one static
    chunk-1 parallel region, 24 B per iteration) at N = 2^k for k in logs;
    the best of `reps` region times.  Checked against torch's own axpy."""
    import torch
    res = {}
    stream = torch.cuda.Stream()
    for lg in logs:
        n = 1 << lg
        x = torch.empty(n, dtype=torch.float64, device="cuda").uniform_(-1, 1)
        y = torch.empty(n, dtype=torch.float64, device="cuda").uniform_(-1, 1)
        z = torch.zeros(n, dtype=torch.float64, device="cuda")
        i64 = lambda v: torch.tensor(v, dtype=torch.int64, device="cuda")
        bufs = [(i64([n]), 1), (torch.tensor([2.5], dtype=torch.float64, device="cuda"), 1), (i64([0]), 1),
                (x, 1), (y, 1), (z, 1),
                (torch.zeros(2, dtype=torch.int64, device="cuda"), 1)]
        with gf.Context(stream=stream, heap_bytes=64 << 20, timeout_ns=int(60e9)) as ctx:
            _timed_run(ctx, stream, "loops", [0, 1, 1, 0], bufs)
            ts = []
            for _ in range(reps):
                _timed_run(ctx, stream, "loops", [0, 1, 1, 0], bufs)
                st = ctx.stats()
                ts.append(st.region_ns / max(1, st.regions) / 1e9)
        ok = bool(torch.equal(z, 2.5 * x + y))
        t = min(ts)
        res[f"2^{lg}"] = {"region_s": t, "GBps": 24 * n / t / 1e9, "bytes": 24 * n, "correct": ok}
        del x, y, z
    return res


def axpy_width_table(lg=28, reps=6):
    """The same axpy loop (one static chunk-1 region, N = 2^lg) with 8-byte and
    16-byte accesses (program axpy_width, argument 1 or 2) at 3, 4 and 8
    resident blocks per SM: GB/s of the best region after the first."""
    import torch
    n = 1 << lg
    x = torch.empty(n, dtype=torch.float64, device="cuda").uniform_(-1, 1)
    y = torch.empty(n, dtype=torch.float64, device="cuda").uniform_(-1, 1)
    z = torch.zeros(n, dtype=torch.float64, device="cuda")
    nb = torch.tensor([n], dtype=torch.int64, device="cuda")
    stream = torch.cuda.Stream()
    out = {}
    with gf.Context(stream=stream, heap_bytes=64 << 20, timeout_ns=int(60e9)) as ctx:
        for prog in ("axpy_width", "axpy_width4", "axpy_width8"):
            row = {"blocks_per_sm": ctx.grid_info(prog)[1]}
            for w in (1, 2):
                ts = []
                for _ in range(reps):
                    z.zero_()
                    rc, ec = ctx.run(prog, [w], [(nb, 1), (x, 1), (y, 1), (z, 1)])
                    if ec != 0:
                        raise RuntimeError(f"{prog} exit code {ec}")
                    st = ctx.stats()
                    ts.append(st.region_ns / max(1, st.regions) / 1e9)
                t = min(ts[1:])
                row[f"{8 * w}B"] = {"GBps": round(24 * n / t / 1e9, 1), "correct": bool(torch.equal(z, 2.5 * x + y))}
            out[prog] = row
    return out


def hbm(args):
    """One large legacy loop through the plain runtime at N = 2^26 and 2^28:
    inputs far larger than L2, so the region's GB/s is HBM bandwidth."""
    peak = _hbm_peak()
    res = axpy_regions((args.hbm_log2,) if getattr(args, "hbm_log2", None) else (26, 28))
    best = max(v["GBps"] for v in res.values())
    res["access_width"] = axpy_width_table()
    line = {"metric": "loop GB/s (% HBM peak)", "value": round(best, 1), "unit": "GB/s", "n_gpus": 1,
            "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "one axpy loop z = 2.5 x + y, N = " + " and ".join(res) + ", static chunk 1, "
                                   "inputs larger than L2"},
            "roofline": {"bound": "hbm", "achieved": round(best, 1), "peak": peak, "unit": "GB/s",
                         "frac": None if not peak else round(best / peak, 4), "peak_kind": "measured"},
            "detail": res}
    print(json.dumps(line))


def split(args):
    import torch
    tmp = tempfile.mkdtemp(prefix="gfsplit", dir=_out_dir(args))
    stream = torch.cuda.Stream()
    res = {"persistent": {}, "split": {}}
    dev = torch.zeros(1 << 20, dtype=torch.uint8, device="cuda")
    ns = torch.zeros(400, dtype=torch.int64, device="cuda")
    n1 = 1 << 20
    x1, y1 = inputs.axpy_inputs(n1, seed=1)
    x1d, y1d = torch.from_numpy(x1).cuda(), torch.from_numpy(y1).cuda()
    trips, a, off, x, y = inputs.loops_inputs()
    nl, total = len(trips), int(trips.sum())
    dv = lambda v: torch.from_numpy(np.ascontiguousarray(v)).cuda()
    lb = [dv(trips), dv(a), dv(off), dv(x), dv(y), torch.zeros(total, dtype=torch.float64, device="cuda"),
          torch.zeros(nl + 1, dtype=torch.int64, device="cuda")]
    g = torch.from_numpy(inputs.jacobi_input(256, seed=2)).cuda()
    for mode in ("persistent", "split"):
        r = res[mode]
        kw = dict(split_regions=1 if mode == "split" else 0, stream=stream, timeout_ns=int(60e9),
                  stdout_path=os.path.join(tmp, f"out_{mode}.txt"))
        with gf.Context(bulk_bytes=1 << 20, heap_bytes=64 << 20, **kw) as ctx:
            rc, ec = ctx.run("link_probe", [64, 400, 0], [(dev, 1), (ns, 1)])
            v = ns[10:].cpu().numpy().astype(np.float64) / 1e3
            r["region_64B_us"] = {"p50": round(float(np.median(v)), 2), "min": round(float(v.min()), 2)}
            y1c = y1d.clone()
            _timed_run(ctx, stream, "axpy_sum", [n1, os.path.join(tmp, "axpy.bin")], [(x1d, 1), (y1c, 1)])
            y1c = y1d.clone()
            t = _timed_run(ctx, stream, "axpy_sum", [n1, os.path.join(tmp, "axpy.bin")], [(x1d, 1), (y1c, 1)])
            r["axpy_sum_2^20_ms"] = round(t * 1e3, 3)
            bufs = [(b, 1) for b in lb]
            _timed_run(ctx, stream, "loops", [0, nl, 1, 0], bufs)
            t = _timed_run(ctx, stream, "loops", [0, nl, 1, 0], bufs)
            st = ctx.stats()
            r["loops_256_regions"] = {"program_ms": round(t * 1e3, 3), "GBps": round(24 * total / t / 1e9, 1)}
        with gf.Context(heap_bytes=3 * 256 ** 3 * 8 + (256 << 20), heap_small_pct=5, **kw) as ctx:
            _timed_run(ctx, stream, "jacobi", [256, 100, "-"], [(g, gf.GF_BUF_IN)])
            t = _timed_run(ctx, stream, "jacobi", [256, 100, "-"], [(g, gf.GF_BUF_IN)])
            st = ctx.stats()
            r["jacobi_256x100_ms"] = round(t * 1e3, 3)
            r["jacobi_sweep_us"] = round(st.region_ns / max(1, st.regions) / 1e3, 2)
            r["jacobi_region_rpcs"] = int(st.rpc_calls[gf.OP_REGION])
    p, q = res["persistent"], res["split"]
    line = {"metric": "region cost: persistent grid vs kernel split", "value": q["region_64B_us"]["p50"],
            "unit": "us per 64-byte region (kernel split)", "n_gpus": 1, "higher_is_better": False,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": "64-byte region x 400; axpy_sum N = 2^20; 256 loops one region each; "
                                   "Jacobi 256^3 x 100 sweeps (no final write)"},
            "detail": {**res,
                       "split_over_persistent": {"region_64B": round(q["region_64B_us"]["p50"] /
                                                                     p["region_64B_us"]["p50"], 2),
                                                 "axpy_sum": round(q["axpy_sum_2^20_ms"] / p["axpy_sum_2^20_ms"], 2),
                                                 "loops_256": round(q["loops_256_regions"]["program_ms"] /
                                                                    p["loops_256_regions"]["program_ms"], 2),
                                                 "jacobi": round(q["jacobi_256x100_ms"] / p["jacobi_256x100_ms"], 3)}}}
    print(json.dumps(line))
    shutil.rmtree(tmp, ignore_errors=True)


def run(args):
    {"stress": stress, "batch": batch, "learned": learned, "serve": serve_run, "spmv": spmv, "e1": e1,
     "link": link, "hbm": hbm, "split": split}[args.workload](args)
