"""Serving loop over the C ABI: many device programs at once, continuous batching.

Programs arrive at the host as a seeded Poisson process and queue in
arrival order.  The head of the queue is launched with gf_launch_q on a free
stream with an equal share of the SMs and its own heap and ring-slot quota;
the runtime admits it only when a program instance, that much of the
context's heap pool and that many of its ring slots are free, and answers
GF_EBUSY otherwise.  A refused program stays at the head of the queue until a
running program has been collected (gf_wait as soon as gf_done reports it),
which gives its quotas back: requests that arrive while others are on the GPU
are admitted as slots and memory free up.

The host RPC server threads of the context serve every running program's
ring segment.  Reported: per-program admission -> done latency, device RPC
round-trip percentiles, calls/s and aggregate SpMV bandwidth.
"""
from __future__ import annotations

import collections
import time

import numpy as np

from . import gf, inputs


class Program:
    """Device buffers of one served program (CSR SpMV with libc requests)."""

    def __init__(self, p, n, passes, req_per_pass, device="cuda", requests=True):
        """requests=False drops the program's libc requests: the SpMV passes alone."""
        import torch
        rowptr, col, val, x0, req = inputs.serve_program_inputs(p, n=n, passes=passes, req_per_pass=req_per_pass)
        if not requests:
            req = req[:0]
        self.p, self.n, self.passes, self.rpp = p, n, passes, req_per_pass
        self.nnz = len(col)
        self.nreq = len(req) // 2
        self.req = req
        self.x0 = x0
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
        self.rowptr, self.col, self.val = t(rowptr), t(col), t(val)
        self.x = t(x0)
        self.y = torch.zeros(n, dtype=torch.float64, device=device)
        self.reqd = t(req) if len(req) else torch.zeros(2, dtype=torch.int64, device=device)
        self.res = torch.zeros(max(1, self.nreq), dtype=torch.int64, device=device)

    def reset(self):
        import torch
        self.x.copy_(torch.from_numpy(self.x0))
        self.res.zero_()

    def bufs(self):
        return [(self.rowptr, 1), (self.col, 1), (self.val, 1), (self.x, 1), (self.y, 1),
                (self.reqd if self.nreq else self.reqd[:0], 1), (self.res, 1)]

    def bytes_moved(self):
        """Algorithmic SpMV bytes: values, columns, row pointers, x gather, y write."""
        return self.passes * (self.nnz * 12 + (self.n + 1) * 8 + self.n * 8 * 2)

    def fp64_ops(self):
        """FP64 operations of the SpMV passes: a multiply and an add per nonzero."""
        return self.passes * self.nnz * 2


def max_overlap(recs):
    """Most programs whose device intervals [t_start_ns, t_end_ns] (one
    %globaltimer clock for the device) contain a common instant."""
    ev = sorted([(r["t_start_ns"], 1) for r in recs] + [(r["t_end_ns"], -1) for r in recs])
    best = cur = 0
    for _, d in ev:
        cur += d
        best = max(best, cur)
    return best


def serve(programs, out_paths, max_concurrent=16, rate_hz=None, seed=7, heap_bytes=1 << 30, ring_slots=1024,
          server_threads=4, stdout_path=None, timeout_s=600.0, quotas=None, heap_pool_bytes=0, ring_pool_slots=0,
          heap_small_pct=50):
    """Run every program once through the serving loop; returns per-program
    records and aggregate statistics.  quotas[k] = (heap bytes, ring slots)
    of program k (None: the context's defaults heap_bytes, ring_slots); the
    pools default to max_concurrent times the defaults."""
    import torch
    ctx = gf.Context(max_programs=max_concurrent, heap_bytes=heap_bytes, heap_small_pct=heap_small_pct,
                     ring_slots=ring_slots, server_threads=server_threads, stdout_path=stdout_path,
                     timeout_ns=int(60e9), bulk_bytes=0, heap_pool_bytes=heap_pool_bytes,
                     ring_pool_slots=ring_pool_slots)
    streams = [torch.cuda.Stream() for _ in range(max_concurrent)]
    rng = np.random.default_rng(seed)
    n = len(programs)
    if rate_hz:
        arrivals = np.cumsum(rng.exponential(1.0 / rate_hz, n))
        arrivals -= arrivals[0]
    else:
        arrivals = np.zeros(n)
    queue = collections.deque()
    running = {}
    free_streams = list(range(max_concurrent))
    recs = [None] * n
    nxt = 0
    refused = 0
    refused_by = collections.Counter()
    blocked = False          # the head was refused; admission can change only when a program ends
    t0 = time.perf_counter()
    while nxt < n or queue or running:
        now = time.perf_counter() - t0
        while nxt < n and arrivals[nxt] <= now:
            queue.append((nxt, time.perf_counter()))
            nxt += 1
        while queue and free_streams and not blocked:
            k, t_arr = queue[0]
            s = free_streams[-1]
            pr = programs[k]
            hq, rq = quotas[k] if quotas else (0, 0)
            rc, h = ctx.launch("spmv_serve", [pr.p, pr.passes, pr.n, out_paths[k]], pr.bufs(), stream=streams[s],
                               heap_bytes=hq, ring_slots=rq)
            if rc == gf.GF_EBUSY:
                refused += 1
                refused_by[k] += 1
                blocked = True
                break
            if rc != gf.GF_OK:
                raise gf.GFError(rc, f"gf_launch_q(program {k})")
            queue.popleft()
            free_streams.pop()
            running[k] = (h, s, t_arr, time.perf_counter())
        for k in list(running):
            h, s, t_arr, t_adm = running[k]
            if gf.gf_done(h):
                rc, ec = ctx.wait(h)
                st = ctx.stats()
                t_done = time.perf_counter()
                recs[k] = dict(program=k, rc=rc, exit=ec, queue_s=t_adm - t_arr, run_s=t_done - t_adm,
                               latency_s=t_done - t_arr, calls=int(sum(st.rpc_calls)), slots=int(sum(st.rpc_slots)),
                               p50_ns=st.rpc_p50_ns, p99_ns=st.rpc_p99_ns, main_ns=st.main_ns, error=st.error,
                               heap_fail=st.heap_fail, t_start_ns=st.t_start_ns, t_end_ns=st.t_end_ns,
                               heap_quota=st.heap_quota, ring_quota=st.ring_quota, refused=refused_by[k])
                del running[k]
                free_streams.append(s)
                blocked = False
        if time.perf_counter() - t0 > timeout_s:
            raise TimeoutError("serving loop timed out")
        if running and (not queue or blocked or not free_streams):
            time.sleep(20e-6)
    wall = time.perf_counter() - t0
    ctx.close()
    calls = sum(r["calls"] for r in recs)
    lat = np.array([r["latency_s"] for r in recs])
    return recs, {"programs": n, "wall_s": wall, "calls": calls, "calls_per_s": calls / wall,
                  "latency_p50_s": float(np.percentile(lat, 50)), "latency_p99_s": float(np.percentile(lat, 99)),
                  "rpc_p50_ns_median": float(np.median([r["p50_ns"] for r in recs])),
                  "rpc_p99_ns_max": float(max(r["p99_ns"] for r in recs)),
                  "admission_refusals": refused,
                  "max_overlap": max_overlap(recs),
                  "spmv_GBps": sum(p.bytes_moved() for p in programs) / wall / 1e9,
                  "device_s": (max(r["t_end_ns"] for r in recs) - min(r["t_start_ns"] for r in recs)) / 1e9}
