"""Benchmark: the legacy 3-D Jacobi program run whole on the GPU.

Workload (one step = one complete program run through the C ABI):
  256^3 FP64 grid, interior ~ U[0,1) (seed 2), zero Dirichlet boundary,
  100 sweeps; each sweep takes a fresh grid from the device heap and frees
  the old one, fuses the max-residual reduction into the stencil region and
  prints one line over RPC; the final grid is fwrite'd (copy-engine DMA).

metric  loop GB/s: algorithmic loop bytes of the whole program (per sweep:
        read the grid once, write the new grid once = 2 * 8 * 256^3 B)
        divided by the device time of the whole program (CUDA events on the
        launch stream around gf_run_main).
e2e     same metric through the same call with a HOST input buffer (the
        loader's H2D copy inside the timed region) and the program's fwrite
        of the result to a file (D2H) inside it.

--impl reference times the serial C oracle of the same program on the host
cores (a bounded sample of sweeps per step) under the same metric.
"""
import argparse
import json
import os
import shutil
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N, SWEEPS = 256, 100
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP64 operations of the serial program per interior point: 5 neighbour adds,
# the division by 6, the residual's subtract.
FP64_OPS_PER_POINT = 7
# DRAM bytes (read + write) of one full launch (100 sweeps and the final
# fwrite), from an ncu capture of the current program kernel on this
# workload: dram__bytes_read.sum 16.047640 GB + dram__bytes_write.sum
# 15.610922 GB.
TRAFFIC_PER_LAUNCH = 16_047_640_000 + 15_610_922_000


def fp64_pipe_ops_per_point(int_adds):
    """Operations per interior point that issue on the FP64 pipe: the
    neighbour adds left to it, plus the residual's subtract.  The division by 6,
    the absolute value and `int_adds` of the five adds run on the integer pipe."""
    return (5 - int_adds) + 1


def fp64_add_peak(gf, stream, tries=3, iters=512):
    """The measured FP64 add rate of this GPU (gf_fp64_add_rate: eight
    independent add chains per thread, CUDA events), best of `tries`, with the
    SM clock sampled while it runs."""
    import ctypes
    best = 0.0
    with Clocks() as clk:
        for _ in range(tries):
            ms, adds = ctypes.c_float(), ctypes.c_double()
            rc = gf.gf_fp64_add_rate(0, iters, ctypes.c_void_p(stream.cuda_stream), ctypes.byref(ms),
                                     ctypes.byref(adds))
            if rc != gf.GF_OK:
                raise gf.GFError(rc, "gf_fp64_add_rate")
            best = max(best, adds.value / (ms.value / 1e3))
    return best, clk.summary()


def max_over_ranks(seconds, world, device):
    """Replicas: the job takes as long as its slowest rank."""
    if world <= 1:
        return seconds
    import torch
    import torch.distributed as dist
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def job_rate(units_per_rank, world, seconds):
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    return units_per_rank * world / seconds


def loop_bytes(n, sweeps):
    return 2 * 8 * n ** 3 * sweeps


def hbm_peak():
    try:
        with open(PEAKS) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def default_out_dir():
    """/dev/shm when it is a writable directory, else the system temp dir."""
    d = "/dev/shm"
    return d if os.path.isdir(d) and os.access(d, os.W_OK) else None


def fs_type(path):
    """File system type of the mount holding path (from /proc/mounts), or None."""
    try:
        best, kind = "", None
        real = os.path.realpath(path)
        with open("/proc/mounts") as f:
            for line in f:
                parts = line.split()
                if len(parts) >= 3 and (real == parts[1] or real.startswith(parts[1].rstrip("/") + "/")) \
                        and len(parts[1]) > len(best):
                    best, kind = parts[1], parts[2]
        return kind
    except OSError:
        return None


class Clocks:
    """Samples SM clock and throttle reasons with nvidia-smi during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.rows, self.proc = [], None

    def __enter__(self):
        if shutil.which("nvidia-smi"):
            dev = os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0] or "0"
            self.proc = subprocess.Popen(["nvidia-smi", "-i", dev, f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()
            self.t.join(timeout=2)

    def summary(self):
        sm = [float(r[0]) for r in self.rows if r and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) > 1 and r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4)
                          if len(r) > 3 + k and r[3 + k].lower().startswith("active")})
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm)}


def host_cores():
    """Cores this process may run on (the GPU machine's host share)."""
    try:
        return sorted(os.sched_getaffinity(0))
    except AttributeError:
        return list(range(os.cpu_count() or 1))


def cpu_oracle_sample(n, sweeps, tmp, omp=False, reps=3):
    """Times the serial C oracle on `sweeps` sweeps of the same grid: pinned to
    one core, best of `reps`.  omp=True times the same C built with OpenMP on
    every available core instead (a CPU baseline like the paper's; timing
    only).  Returns (GB/s, seconds, cores)."""
    from oracle import build as ob
    from paper_2306_11686_gb300 import inputs
    ob.build()
    path = os.path.join(tmp, "in.bin")
    if not os.path.exists(path):
        inputs.write_f64(path, inputs.jacobi_input(n, seed=2))
    cores = host_cores()
    env = dict(os.environ)
    if omp:
        env["OMP_NUM_THREADS"] = str(len(cores))
        env["OMP_PROC_BIND"] = "close"
    # pinning by a taskset prefix, not preexec_fn: this process has live threads
    pin = ["taskset", "-c", str(cores[0])] if not omp and shutil.which("taskset") else []
    best = None
    for _ in range(reps):
        t0 = time.perf_counter()
        subprocess.run(pin + [ob.binary("jacobi_omp" if omp else "jacobi"), str(n), str(sweeps), path,
                              os.path.join(tmp, "ref.bin")], check=True, stdout=subprocess.DEVNULL, env=env)
        dt = time.perf_counter() - t0
        best = dt if best is None else min(best, dt)
    return loop_bytes(n, sweeps) / best / 1e9, best, (len(cores) if omp else 1), bool(pin) or omp


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    tmp = tempfile.mkdtemp(prefix="gfbench", dir=args.out_dir or default_out_dir())
    sample = max(1, args.ref_sweeps)
    for _ in range(args.warmup):
        cpu_oracle_sample(N, sample, tmp, reps=1)
    vals, times = [], []
    for _ in range(args.steps):
        v, dt, _, _ = cpu_oracle_sample(N, sample, tmp, reps=1)
        vals.append(v)
        times.append(dt)
    v = sum(loop_bytes(N, sample) for _ in times) / sum(times) / 1e9
    line = {"impl": "reference", "metric": "loop GB/s (% HBM peak)", "value": round(v, 3), "unit": "GB/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * sum(times) / len(times), 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"jacobi-7pt {N}^3 fp64, {sample} sweeps per step (bounded sample of 100)",
                       "l2": "grid larger than L2"},
            "cpu_baseline": {"value": round(v, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
                             "sample": f"{sample} sweeps of {N}^3 per step"},
            "e2e": {"value": round(v, 3), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    shutil.rmtree(tmp, ignore_errors=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20,
                    help="timed programs (20 x 22 ms: long enough for several clock samples)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gf", choices=["gf", "reference"])
    ap.add_argument("--ref-sweeps", type=int, default=4)
    ap.add_argument("--cpu-sweeps", type=int, default=8)
    ap.add_argument("--out-dir", default=None,
                    help="where the program writes its final grid (default: /dev/shm when it is a writable "
                         "tmpfs, so the number measures the runtime and the page cache, not the disk)")
    ap.add_argument("--sweeps", type=int, default=SWEEPS, help="sweeps per program (100 = the benchmark workload)")
    ap.add_argument("--hbm-log2", type=int, default=None,
                    help="--workload hbm: one loop of 2^k iterations only (default: 2^26 and 2^28)")
    ap.add_argument("--bulk-mib", type=int, default=None,
                    help="bulk arena of the context in MiB (the final fwrite's staging; library default 64)")
    ap.add_argument("--int-adds", type=int, default=None,
                    help="how many of the five neighbour adds run on the integer pipe (0..5; the program's "
                         "default when omitted)")
    ap.add_argument("--kseg", type=int, default=None,
                    help="run each sweep as columns of K planes per parallel iteration (0 = one iteration per "
                         "point; the program's default when omitted)")
    ap.add_argument("--server-threads", type=int, default=None,
                    help="host server threads for --workload serve and stress (a power of two; the "
                         "workload's default when omitted)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer leg (profiling runs)")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the same-process extra measurements (printf calls/s with and without warp "
                         "aggregation, one axpy loop at 2^28 against HBM, the measured FP64 add peak)")
    ap.add_argument("--no-write", action="store_true",
                    help="the program skips its final fwrite (profiling runs that isolate the sweeps)")
    ap.add_argument("--workload", default="jacobi", choices=["jacobi", "stress", "batch", "learned", "serve", "spmv", "e1", "link", "hbm", "split"],
                    help="jacobi = the benchmark; the others measure the RPC/heap stress, 256-loop batching, "
                         "learned launch shapes, serving, host-link peaks, single large loops and the "
                         "persistent grid against the paper's kernel split")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "jacobi":
        from paper_2306_11686_gb300 import measure
        return measure.run(args)
    sweeps = args.sweeps

    import numpy as np
    import torch
    from paper_2306_11686_gb300 import gf, inputs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    out_dir = args.out_dir or default_out_dir()
    tmp = tempfile.mkdtemp(prefix="gfbench", dir=out_dir)
    out_path = os.path.join(tmp, f"grid_r{rank}.bin")

    g = inputs.jacobi_input(N, seed=2)
    gd = torch.from_numpy(g).to(dev)
    gh = torch.from_numpy(g).pin_memory()
    stream = torch.cuda.Stream(device=dev)
    heap = 3 * N ** 3 * 8 + (256 << 20)
    ckw = {} if args.bulk_mib is None else {"bulk_bytes": args.bulk_mib << 20}
    ctx = gf.Context(stream=stream, heap_bytes=heap, heap_small_pct=5,
                     stdout_path=os.path.join(tmp, f"stdout_r{rank}.txt"), **ckw)
    argv = [N, sweeps, "-" if args.no_write else out_path]
    if args.int_adds is not None or args.kseg is not None:
        argv.append(1 if args.int_adds is None else args.int_adds)
    if args.kseg is not None:
        argv.append(args.kseg)

    def step(buf):
        rc, ec = ctx.run("jacobi", argv, [(buf, gf.GF_BUF_IN)])
        if ec != 0:
            raise RuntimeError(f"jacobi exit code {ec}")

    for _ in range(args.warmup):
        step(gd)
    torch.cuda.synchronize(dev)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    # ---- value: inputs resident in HBM
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    with Clocks() as clk:
        for k in range(args.steps):
            ev[k][0].record(stream)
            step(gd)
            ev[k][1].record(stream)
        torch.cuda.synchronize(dev)
    barrier()
    per = [a.elapsed_time(b) / 1e3 for a, b in ev]
    total = max_over_ranks(sum(per), world, dev)
    st = ctx.stats()
    value = job_rate(loop_bytes(N, sweeps) * args.steps, world, total) / 1e9

    # ---- e2e: host input staged in by the loader, result written by the program's fwrite
    e2e = None
    if not args.no_e2e:
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e2e_steps = args.steps
        step(gh)            # warm-up: the first host-buffer run maps its staging allocation
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(e2e_steps):
            step(gh)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        e2e_t = e0.elapsed_time(e1) / 1e3
        e2e = loop_bytes(N, sweeps) * e2e_steps * world / e2e_t / 1e9

    peak, peak_kind = hbm_peak()
    # Algorithmic bytes of one launch: every sweep reads the grid once and
    # writes the new one (2 x 8 B per point), and the final fwrite reads the
    # last grid once more.
    launch_bytes = loop_bytes(N, sweeps) + (0 if args.no_write else 8 * N ** 3)
    achieved = launch_bytes / (total / args.steps) / 1e9
    # the program's own regions (the sweeps), without the final fwrite's copies
    sweep_s = max(st.region_ns - st.copy_ns, 1) / max(1, st.regions - st.copy_regions) / 1e9
    # The sweep's binding roofline is the FP64 pipe, not HBM: GB300 retires
    # FP64 adds at a small fraction of its other rates, and the serial
    # program's 7 FP64 operations per interior point need several times longer
    # on that pipe than the point's 16 bytes need on HBM.  The program runs
    # the division by 6, the absolute value and one of the five adds on the
    # integer pipe (bit-identical results), so the roofline counts what
    # issues on the FP64 pipe -- the other four adds and the residual's
    # subtract -- against the FP64 add rate measured on this GPU in this run.
    # HBM is reported beside it.
    sms = ctx.grid_info("jacobi")[0]
    int_adds = 1 if args.int_adds is None else args.int_adds
    pipe_per_point = fp64_pipe_ops_per_point(int_adds)
    fp64_peak, peak_clocks = fp64_add_peak(gf, stream)                     # FP64 adds / s
    fp64_ops = pipe_per_point * (N - 2) ** 3 * sweeps
    extra = None
    if rank == 0 and not args.no_extra:
        from paper_2306_11686_gb300 import measure
        ax = measure.axpy_regions((28,))["2^28"]
        extra = {"fp64_peak": {"adds_per_s": round(fp64_peak), "per_sm_per_clock":
                               round(fp64_peak / (sms * peak_clocks["sm_mhz"] * 1e6), 3)
                               if peak_clocks.get("sm_mhz") else None,
                               "clocks": peak_clocks,
                               "how": "gf_fp64_add_rate: SMs x resident blocks of 256 threads, 8 independent "
                                      "add.rn.f64 chains x 512 per thread (2.4 ms per launch), CUDA events, "
                                      "best of 3"},
                 "hbm": {"workload": "one axpy loop z = 2.5 x + y, N = 2^28, one static chunk-1 region "
                                     "through the plain runtime (24 B per iteration, 6.4 GB)",
                         "GBps": round(ax["GBps"], 1), "frac": round(ax["GBps"] / peak, 4),
                         "peak": peak, "peak_kind": peak_kind, "correct": ax["correct"]},
                 "stress": measure.printf_rate(1 << 20, out_dir=out_dir, server_threads=16)}
    cpu = cpu_omp = None
    if rank == 0 and args.cpu_sweeps > 0:
        cv, cdt, cc, pinned = cpu_oracle_sample(N, args.cpu_sweeps, tmp)
        cpu = {"value": round(cv, 3), "unit": "GB/s", "cores": cc, "kind": "oracle",
               "sample": f"{args.cpu_sweeps} sweeps of the {N}^3 grid, "
                         f"{'pinned to one core' if pinned else 'one thread (not pinned)'}, best of 3 "
                         f"({cdt:.2f} s); host cores available: {len(host_cores())}"}
        ov, odt, oc, _ = cpu_oracle_sample(N, args.cpu_sweeps, tmp, omp=True)
        cpu_omp = {"value": round(ov, 3), "unit": "GB/s", "cores": oc, "kind": "oracle source built with OpenMP",
                   "sample": f"{args.cpu_sweeps} sweeps of the {N}^3 grid on {oc} threads, best of 3 ({odt:.3f} s)"}
    if rank == 0:
        line = {
            "metric": "loop GB/s (% HBM peak)", "value": round(value, 2), "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * total / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"jacobi-7pt {N}^3 fp64, {sweeps} sweeps, per-sweep device malloc/free, "
                                   "fused max-residual, printf per sweep, final fwrite",
                       "grid": st.grid, "block": st.block, "l2": "inputs larger than L2 (2 x 134 MB grids)",
                       "output": None if args.no_write else {"dir": os.path.dirname(tmp), "fs": fs_type(tmp)},
                       "parallelism": "replicas" if world > 1 else "single"},
            "roofline": {"bound": "alu", "achieved": round(fp64_ops / (total / args.steps) / 1e9, 1),
                         "peak": round(fp64_peak / 1e9, 1), "unit": "G FP64 add/s",
                         "frac": round(fp64_ops / (total / args.steps) / fp64_peak, 4),
                         "traffic": TRAFFIC_PER_LAUNCH,
                         "peak_kind": "measured: gf_fp64_add_rate in this run (extra.fp64_peak), "
                                      f"sampled SM clock {peak_clocks.get('sm_mhz')} MHz",
                         "kernel": "program_kernel<jacobi>",
                         "algorithmic": f"{pipe_per_point} FP64-pipe operations per interior point ({5 - int_adds} "
                                        f"neighbour adds + the residual's subtract) x {N - 2}^3 x {sweeps} sweeps; "
                                        f"the /6, |.| and {int_adds} add(s) run on the integer pipe",
                         "all_fp64_ops": {"per_point": FP64_OPS_PER_POINT,
                                          "on_integer_pipe": int_adds + 1,
                                          "achieved": round(FP64_OPS_PER_POINT * (N - 2) ** 3 * sweeps /
                                                            (total / args.steps) / 1e9, 1)},
                         "sweeps_only": {"achieved": round(fp64_ops / sweeps / sweep_s / 1e9, 1),
                                         "frac": round(fp64_ops / sweeps / sweep_s / fp64_peak, 4),
                                         "sweep_us": round(sweep_s * 1e6, 2)},
                         "hbm": {"achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                                 "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
                                 "algorithmic_bytes_per_launch": launch_bytes,
                                 "sweeps_only": round(loop_bytes(N, 1) / sweep_s / 1e9, 1)}},
            "e2e": None if e2e is None else {"value": round(e2e, 2), "unit": "GB/s", "h2d_bytes_per_step": N ** 3 * 8,
                    "d2h_bytes_per_step": N ** 3 * 8 + 100 * 24, "steps": e2e_steps, "warmup": 1},
            "gpu_launches": args.steps,
            "cpu_baseline": cpu,
            "cpu_openmp": cpu_omp,
            "clocks": clk.summary(),
            "extra": extra,
            "detail": {"main_ns": st.main_ns, "regions": st.regions, "region_ns": st.region_ns,
                       "sweep_us": round(sweep_s * 1e6, 2),
                       "sweep_GBps": round(loop_bytes(N, 1) / sweep_s / 1e9, 1),
                       "program_ms": {"sweeps": round((st.region_ns - st.copy_ns) / 1e6, 3),
                                      "fwrite_copy_regions": round(st.copy_ns / 1e6, 3),
                                      "rpc_waits": round(st.rpc_wait_ns / 1e6, 3),
                                      "rpc_waits_by_call": {
                                          "printf": round(st.rpc_wait_op_ns[gf.OP_PRINTF] / 1e6, 3),
                                          "fwrite": round(st.rpc_wait_op_ns[gf.OP_FWRITE] / 1e6, 3),
                                          "fopen_fclose": round((st.rpc_wait_op_ns[gf.OP_FOPEN] +
                                                                 st.rpc_wait_op_ns[gf.OP_FCLOSE]) / 1e6, 3),
                                          "fopen": round(st.rpc_wait_op_ns[gf.OP_FOPEN] / 1e6, 3),
                                          "fclose": round(st.rpc_wait_op_ns[gf.OP_FCLOSE] / 1e6, 3)},
                                      "rpc_client": round(st.rpc_client_ns / 1e6, 3),
                                      "serial_heap": round(st.heap_ns / 1e6, 3),
                                      "rest": round((st.main_ns - st.region_ns - st.rpc_wait_ns - st.heap_ns -
                                                     st.rpc_client_ns) / 1e6, 3)},
                       "rpc_p50_ns": st.rpc_p50_ns, "rpc_p99_ns": st.rpc_p99_ns, "rpc_wait_ns": st.rpc_wait_ns,
                       "step_s": [round(p, 6) for p in per]},
        }
        print(json.dumps(line))
    ctx.close()
    shutil.rmtree(tmp, ignore_errors=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
