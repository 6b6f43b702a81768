"""The paper's worked example (Fig. 4) through a user landing pad.

The landing pad records, for every argument, the kind, tag, object size and
pointer offset it received (gf_rec_arg) and compares them with the golden
table transcribed from Fig. 4c (tests/golden/fig4_rpc_args.txt).  It then
writes through the write / readwrite pointers as fscanf would; the device
must see exactly those writes after the call, and nothing else of the
objects may change."""
import ctypes
import os
import struct

import pytest

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fig4_rpc_args.txt")


def golden_rows():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        k, kind, tag, nbytes, off = line.split()[:5]
        rows.append((int(k), kind, tag, int(nbytes), int(off)))
    return rows


@pytest.mark.parametrize("form", ["variadic", "array"])
def test_fig4_argument_kinds_and_copy_back(gf_lib, form):
    """Both call forms of gf_rpc: the parameter pack and the gf_arg array."""
    import torch
    gf = gf_lib
    seen = []

    def pad(user, opcode, rec):
        got = []
        for k in range(5):
            tag, word, ptr = ctypes.c_uint8(), ctypes.c_uint64(), ctypes.c_void_p()
            nbytes, off = ctypes.c_uint32(), ctypes.c_uint32()
            assert gf.gf_rec_arg(ctypes.c_void_p(rec), k, ctypes.byref(tag), ctypes.byref(word), ctypes.byref(ptr),
                                 ctypes.byref(nbytes), ctypes.byref(off)) == 0
            got.append((chr(tag.value), word.value, ptr.value, nbytes.value, off.value))
        seen.append(got)
        fmt = ctypes.string_at(got[1][2], 8)
        seen.append(fmt)
        ctypes.memmove(got[2][2], struct.pack("<f", 3.25), 4)      # %f  -> s.f
        ctypes.memmove(got[3][2], struct.pack("<i", 42), 4)        # %i  -> i
        ctypes.memmove(got[4][2], struct.pack("<i", 77), 4)        # %i  -> *p
        return 3

    cb = gf.gf_host_fn(pad)
    out = torch.zeros(8, dtype=torch.int64, device="cuda")
    with gf.Context(timeout_ns=10_000_000_000, heap_bytes=64 << 20) as c:
        assert gf.gf_rpc_register(c.h, 300, cb, None) == 0
        rc, ec = c.run("fig4_probe", [300] + (["array"] if form == "array" else []), [(out, 1)])
    assert ec == 0
    got, fmt = seen[0], seen[1]
    for k, kind, tag, nbytes, off in golden_rows():
        t, word, ptr, b, o = got[k]
        assert t == tag, (k, t, tag)
        if kind == "value":
            assert word == 0xF11E0
        else:
            assert (b, o) == (nbytes, off), (k, b, o)
    assert fmt == b"%f %i %i"
    o = out.cpu().tolist()
    assert o[0] == 3 and o[1] == 0
    assert struct.unpack("<f", struct.pack("<i", o[2]))[0] == 3.25
    assert (o[3], o[4]) == (1, 2)                   # the rest of s came back unchanged
    assert o[5] == 42 and o[6] == 77
    assert o[7] == 10 + 100 * 12 + 10000 * 13      # the rest of p's block unchanged
