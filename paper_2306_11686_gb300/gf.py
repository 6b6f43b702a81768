"""ctypes binding of the C ABI in include/gf.h (argument marshalling only).

Every function of the header is exposed under its own name; `Context` is a
thin convenience wrapper.  Importing this module loads libgf.so and raises
ImportError when it has not been built: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgf.so")
if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is not built; run __graft_entry__.build() (nvcc, sm_103a)")
_lib = ctypes.CDLL(LIB_PATH, mode=ctypes.RTLD_GLOBAL)

GF_OK, GF_EINVAL, GF_ENOMEM, GF_ERING, GF_ETIMEDOUT, GF_EHOST, GF_ECUDA, GF_ENOENT, GF_EBUSY = (
    0, -1, -2, -3, -4, -5, -6, -7, -8)
GF_BUF_IN, GF_BUF_OUT = 1, 2
SCHED_STATIC, SCHED_DYNAMIC = 0, 1
OP_PRINTF, OP_FOPEN, OP_FWRITE, OP_FCLOSE, OP_CLOCK, OP_GETENV, OP_FREAD, OP_FFLUSH = 1, 2, 3, 4, 5, 6, 7, 8
OP_STRTOD, OP_REGION = 9, 10
NOPS = 16


class gf_config(ctypes.Structure):
    _fields_ = [
        ("heap_bytes", ctypes.c_uint64),
        ("heap_small_pct", ctypes.c_uint32),
        ("ring_slots", ctypes.c_uint32),
        ("slot_bytes", ctypes.c_uint32),
        ("aggregate", ctypes.c_uint32),
        ("server_threads", ctypes.c_uint32),
        ("max_programs", ctypes.c_uint32),
        ("grid", ctypes.c_uint32),
        ("timeout_ns", ctypes.c_int64),
        ("stream", ctypes.c_void_p),
        ("stdout_path", ctypes.c_char_p),
        ("fmt_cache", ctypes.c_uint32),
        ("device", ctypes.c_int32),
        ("bulk_bytes", ctypes.c_uint64),
        ("split_regions", ctypes.c_uint32),
        ("pad0", ctypes.c_uint32),
        ("heap_pool_bytes", ctypes.c_uint64),
        ("ring_pool_slots", ctypes.c_uint32),
        ("pad1", ctypes.c_uint32),
    ]


class gf_quota(ctypes.Structure):
    _fields_ = [("heap_bytes", ctypes.c_uint64), ("ring_slots", ctypes.c_uint32), ("pad", ctypes.c_uint32)]


class gf_buf(ctypes.Structure):
    _fields_ = [("ptr", ctypes.c_void_p), ("bytes", ctypes.c_uint64), ("dir", ctypes.c_uint32),
                ("pad", ctypes.c_uint32)]


class gf_stats(ctypes.Structure):
    _fields_ = [
        ("rpc_calls", ctypes.c_uint64 * NOPS),
        ("rpc_slots", ctypes.c_uint64 * NOPS),
        ("rpc_wait_ns", ctypes.c_uint64),
        ("rpc_p50_ns", ctypes.c_double),
        ("rpc_p99_ns", ctypes.c_double),
        ("regions", ctypes.c_uint64),
        ("region_ns", ctypes.c_uint64),
        ("heap_alloc", ctypes.c_uint64),
        ("heap_free", ctypes.c_uint64),
        ("heap_fail", ctypes.c_uint64),
        ("heap_bad_free", ctypes.c_uint64),
        ("heap_live_bytes", ctypes.c_uint64),
        ("heap_high_water", ctypes.c_uint64),
        ("main_ns", ctypes.c_uint64),
        ("host_slots", ctypes.c_uint64),
        ("host_records", ctypes.c_uint64),
        ("host_ns", ctypes.c_uint64),
        ("host_dma_bytes", ctypes.c_uint64),
        ("grid", ctypes.c_int32),
        ("block", ctypes.c_int32),
        ("error", ctypes.c_int32),
        ("exit_code", ctypes.c_int32),
        ("heap_ns", ctypes.c_uint64),
        ("copy_regions", ctypes.c_uint64),
        ("copy_ns", ctypes.c_uint64),
        ("host_ring_bytes", ctypes.c_uint64),
        ("t_start_ns", ctypes.c_uint64),
        ("t_end_ns", ctypes.c_uint64),
        ("heap_quota", ctypes.c_uint64),
        ("ring_quota", ctypes.c_uint64),
        ("rpc_wait_op_ns", ctypes.c_uint64 * NOPS),
        ("rpc_client_ns", ctypes.c_uint64),
    ]

    def as_dict(self):
        d = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            d[name] = list(v) if hasattr(v, "__len__") else v
        return d


class gf_serve_opts(ctypes.Structure):
    _fields_ = [("timeout_ns", ctypes.c_int64), ("stop", ctypes.POINTER(ctypes.c_int32))]


class gf_synth_loop(ctypes.Structure):
    _fields_ = [("trip", ctypes.c_int64), ("bytes", ctypes.c_uint32), ("flops", ctypes.c_uint32),
                ("div_thresh", ctypes.c_uint32), ("rpc_thresh", ctypes.c_uint32), ("seed", ctypes.c_uint64)]


class gf_shape(ctypes.Structure):
    _fields_ = [("grid", ctypes.c_uint32), ("block", ctypes.c_uint32), ("chunk", ctypes.c_uint32),
                ("sched", ctypes.c_uint32)]


GF_TUNE_NFEAT = 9

gf_host_fn = ctypes.CFUNCTYPE(ctypes.c_int64, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p)

_P = ctypes.c_void_p
_sig = {
    "gf_config_default": (None, [ctypes.POINTER(gf_config)]),
    "gf_init": (ctypes.c_int, [ctypes.POINTER(gf_config), ctypes.POINTER(_P)]),
    "gf_finalize": (ctypes.c_int, [_P]),
    "gf_program_lookup": (ctypes.c_int, [_P, ctypes.c_char_p, ctypes.POINTER(ctypes.c_int32)]),
    "gf_run_main": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int, ctypes.POINTER(ctypes.c_char_p),
                                   ctypes.POINTER(gf_buf), ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "gf_launch": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int, ctypes.POINTER(ctypes.c_char_p),
                                 ctypes.POINTER(gf_buf), ctypes.c_int, _P, ctypes.c_uint32, ctypes.POINTER(_P)]),
    "gf_launch_q": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int, ctypes.POINTER(ctypes.c_char_p),
                                   ctypes.POINTER(gf_buf), ctypes.c_int, _P, ctypes.c_uint32, ctypes.POINTER(gf_quota),
                                   ctypes.POINTER(_P)]),
    "gf_done": (ctypes.c_int, [_P]),
    "gf_wait": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.c_int64]),
    "gf_rpc_serve": (ctypes.c_int, [_P, ctypes.POINTER(gf_serve_opts)]),
    "gf_rpc_register": (ctypes.c_int, [_P, ctypes.c_uint32, gf_host_fn, _P]),
    "gf_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(gf_stats)]),
    "gf_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "gf_grid_info": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_uint32),
                                    ctypes.POINTER(ctypes.c_uint32)]),
    "gf_reduce_f64_noalloc": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int, _P, ctypes.c_uint32, _P]),
    "gf_synth_run": (ctypes.c_int, [_P, ctypes.POINTER(gf_synth_loop), _P, ctypes.c_uint64, _P,
                                    ctypes.POINTER(gf_shape), _P]),
    "gf_synth_time": (ctypes.c_int, [_P, ctypes.POINTER(gf_synth_loop), _P, ctypes.c_uint64, _P,
                                     ctypes.POINTER(gf_shape), ctypes.c_int, ctypes.c_int, _P, ctypes.c_void_p]),
    "gf_tune_features": (None, [ctypes.POINTER(gf_synth_loop), ctypes.POINTER(gf_shape), ctypes.c_uint32, _P]),
    "gf_mlp_forward": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, ctypes.c_int, _P]),
    "gf_mlp_choose": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(gf_synth_loop),
                                     ctypes.POINTER(gf_shape), ctypes.c_int, ctypes.c_uint32,
                                     ctypes.POINTER(ctypes.c_int)]),
    "gf_rec_arg": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_uint8), ctypes.POINTER(ctypes.c_uint64),
                                  ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_uint32),
                                  ctypes.POINTER(ctypes.c_uint32)]),
    "gf_alloc_e1": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int,
                                   _P, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_uint64)]),
    "gf_mlp_topk": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(gf_synth_loop),
                                   ctypes.POINTER(gf_shape), ctypes.c_int, ctypes.c_uint32, ctypes.c_int,
                                   ctypes.POINTER(ctypes.c_int)]),
    "gf_fp64_add_rate": (ctypes.c_int, [ctypes.c_uint32, ctypes.c_int64, _P, ctypes.POINTER(ctypes.c_float),
                                        ctypes.POINTER(ctypes.c_double)]),
    "gf_loops_rpc_graph": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, _P, _P, _P, _P, _P, _P, ctypes.c_int,
                                          ctypes.c_int, _P, ctypes.POINTER(ctypes.c_float)]),
    "gf_axpy_batch_graph": (ctypes.c_int, [ctypes.c_int, _P, _P, _P, _P, _P, _P, _P, _P, ctypes.c_int, _P,
                                           ctypes.POINTER(ctypes.c_float)]),
}
GF_REDUCE_SUM, GF_REDUCE_MIN, GF_REDUCE_MAX = 1, 2, 3
for _name, (_res, _args) in _sig.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args
    globals()[_name] = _f


class GFError(RuntimeError):
    def __init__(self, rc, what):
        super().__init__(f"{what}: {gf_strerror(rc).decode()} ({rc})")
        self.rc = rc


def _check(rc, what):
    if rc != GF_OK:
        raise GFError(rc, what)


def _ptr_bytes(obj):
    """(pointer, bytes) of a torch tensor (device or host) or a numpy array."""
    if hasattr(obj, "data_ptr"):
        return obj.data_ptr(), obj.numel() * obj.element_size()
    if hasattr(obj, "ctypes"):
        return obj.ctypes.data, obj.nbytes
    raise TypeError(f"unsupported buffer {type(obj)}")


def make_bufs(bufs):
    """bufs: sequence of (array_or_tensor, dir) -> ctypes array of gf_buf."""
    arr = (gf_buf * max(1, len(bufs)))()
    for k, (obj, d) in enumerate(bufs):
        p, n = _ptr_bytes(obj)
        arr[k].ptr = p
        arr[k].bytes = n
        arr[k].dir = d
    return arr


def make_argv(argv):
    enc = [a.encode() if isinstance(a, str) else bytes(a) for a in argv]
    arr = (ctypes.c_char_p * (len(enc) + 1))(*enc, None)
    return arr, enc


class Context:
    """One gf_ctx.  Keyword arguments override gf_config fields."""

    def __init__(self, **kw):
        self.cfg = gf_config()
        gf_config_default(ctypes.byref(self.cfg))
        self._keep = []
        for k, v in kw.items():
            if k == "stdout_path" and v is not None:
                v = str(v).encode()
                self._keep.append(v)
            if k == "stream" and v is not None and not isinstance(v, int):
                v = v.cuda_stream
            setattr(self.cfg, k, v)
        self.h = _P()
        _check(gf_init(ctypes.byref(self.cfg), ctypes.byref(self.h)), "gf_init")

    def program(self, name):
        pid = ctypes.c_int32()
        _check(gf_program_lookup(self.h, name.encode(), ctypes.byref(pid)), f"gf_program_lookup({name})")
        return pid.value

    def run(self, name, argv, bufs=(), check=True):
        """gf_run_main; returns (rc, exit_code)."""
        pid = self.program(name)
        av, keep = make_argv([name] + [str(a) for a in argv])
        b = make_bufs(bufs)
        ec = ctypes.c_int(-1)
        rc = gf_run_main(self.h, pid, len(keep), av, b, len(bufs), ctypes.byref(ec))
        if check:
            _check(rc, f"gf_run_main({name})")
        return rc, ec.value

    def launch(self, name, argv, bufs=(), stream=None, grid=0, heap_bytes=0, ring_slots=0):
        """gf_launch_q with the given quotas (0 = the context's defaults);
        returns (rc, handle)."""
        pid = self.program(name)
        av, keep = make_argv([name] + [str(a) for a in argv])
        b = make_bufs(bufs)
        h = _P()
        s = stream.cuda_stream if stream is not None and not isinstance(stream, int) else stream
        q = gf_quota(heap_bytes, ring_slots, 0)
        rc = gf_launch_q(self.h, pid, len(keep), av, b, len(bufs), s, grid, ctypes.byref(q), ctypes.byref(h))
        return rc, h

    def wait(self, h, timeout_ns=0):
        ec = ctypes.c_int(-1)
        rc = gf_wait(h, ctypes.byref(ec), timeout_ns)
        return rc, ec.value

    def stats(self):
        s = gf_stats()
        _check(gf_get_stats(self.h, ctypes.byref(s)), "gf_get_stats")
        return s

    def grid_info(self, name):
        sms, per = ctypes.c_uint32(), ctypes.c_uint32()
        _check(gf_grid_info(self.h, self.program(name), ctypes.byref(sms), ctypes.byref(per)), "gf_grid_info")
        return sms.value, per.value

    def close(self):
        if self.h:
            gf_finalize(self.h)
            self.h = _P()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
