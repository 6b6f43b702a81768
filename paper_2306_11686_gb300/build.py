"""Builds libgf.so (runtime + programs) for sm_103a, in-tree.

Every .cu is compiled by nvcc for `-gencode arch=compute_103a,code=sm_103a`
with `--fmad=false` (C semantics without floating-point contraction, so loop
bodies round like the serial program), the host server with g++, and
everything is linked into paper_2306_11686_gb300/libgf.so.  Translation units
compile in parallel; unchanged objects are reused.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libgf.so")
NVCC = os.environ.get("NVCC", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
INC = ["-I", os.path.join(ROOT, "include"), "-I", CSRC]
NVFLAGS = ARCH + INC + ["-O3", "-lineinfo", "-std=c++17", "--fmad=false", "-Xcompiler", "-fPIC,-fvisibility=hidden",
                        "-Xptxas", "-v", "-diag-suppress", "177"]
CXXFLAGS = INC + ["-O2", "-std=c++17", "-fPIC", "-fvisibility=hidden", "-Wall"]

CU = ["runtime.cu", "noalloc.cu", "peak.cu", "programs/legacy.cu", "programs/probes_sched.cu", "programs/probes_rpc.cu",
      "programs/probes_heap.cu", "programs/probes_misc.cu", "programs/stress.cu", "programs/batch.cu",
      "programs/synth.cu", "programs/serve.cu",
      "programs/alloc_e1.cu", "programs/libc.cu"]
CPP = ["host/server.cpp", "host/mlp.cpp"]
HEADERS = ["gf_layout.h", "gf_device.cuh", "gf_device_rpc.cuh", "gf_device_heap.cuh", "gf_program.h",
           "host/server.h", "host/range_alloc.h", "gf_errors.h", "gf_internal.h", "gf_fastdiv.cuh", "gf_paper_alloc.cuh", "gf_device_libc.cuh",
           "gf_intpipe.cuh", "gf_strtod_fast.h", "host/fmt_fast.h", "host/dtoa_fixed.h"]


def _newer(obj, deps):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def _run(cmd, log):
    p = subprocess.run(cmd, capture_output=True, text=True)
    with open(log, "w") as f:
        f.write(" ".join(cmd) + "\n" + p.stdout + p.stderr)
    if p.returncode != 0:
        raise RuntimeError(f"build failed: {' '.join(cmd)}\n{p.stdout}\n{p.stderr}")
    return p.stderr


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(ROOT, "include", "gf.h")]
    jobs, objs = [], []
    for src in CU + CPP:
        path = os.path.join(CSRC, src)
        if not os.path.exists(path):
            continue
        obj = os.path.join(OUT, src.replace("/", "_") + ".o")
        objs.append(obj)
        if force or _newer(obj, [path] + hdrs):
            if src.endswith(".cu"):
                cmd = [NVCC, *NVFLAGS, "-c", path, "-o", obj]
            else:
                cmd = ["g++", *CXXFLAGS, "-c", path, "-o", obj]
            jobs.append((cmd, obj + ".log"))
    with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        outs = list(ex.map(lambda j: _run(*j), jobs))
    if verbose:
        for o in outs:
            sys.stderr.write(o)
    if force or jobs or not os.path.exists(LIB) or _newer(LIB, objs):
        _run([NVCC, *ARCH, "-shared", "-o", LIB, *objs, "-lpthread"], os.path.join(OUT, "link.log"))
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
