"""The paper's own allocators (comparators for the slab heap) and its
allocator experiment.

balanced_probe walks one chunk of the balanced allocator through the life
cycle of the paper's Fig. 5 (16-byte in-band headers, sizes rounded to 16):
  a = 100 B at 0, b = 200 B at 128, c = 50 B at 352, watermark 432;
  free(b): the watermark stays (Fig. 5 middle row);
  free(c): c is the top entry, so the watermark drops to 352 and, chained,
  over the already-free b to 128 (Fig. 5 bottom row);
  the next 100 B entry lands at 128, where b was.
A full chunk reuses a freed entry by walking the entries; a request larger
than the chunk fails; the first chunk of a team slot is `ratio` times larger.
E1 itself: every allocator serves every thread of every team without a
NULL or a corrupted block."""
import ctypes

import pytest

pytestmark = pytest.mark.gpu


def test_balanced_allocator_fig5_cycle(gf_lib):
    import torch
    gf = gf_lib
    out = torch.zeros(16, dtype=torch.int64, device="cuda")
    with gf.Context(timeout_ns=10_000_000_000, heap_bytes=64 << 20, heap_small_pct=10) as c:
        rc, ec = c.run("balanced_probe", [], [(out, 1)])
    assert ec == 0
    o = out.cpu().tolist()
    assert o[0:4] == [16, 128 + 16, 352 + 16, 432]
    assert o[4] == 432
    assert o[5] == 128
    assert o[6] == 128 + 16
    # d takes 128..256 (16 B header + 112 B); the 1024 B chunk holds (1024 - 256) / 64 = 12 more 48 B entries
    assert o[7] == (1024 - 256) // 64
    assert o[8] == o[9]                         # the walk found the freed entry
    assert o[10] == 0 and o[12] == 0
    assert o[11] == 16                          # 1500 B fits the 2048 B first chunk


@pytest.mark.parametrize("kind", [0, 1, 2, 3])
@pytest.mark.parametrize("teams,threads", [(1, 1), (32, 32), (256, 256)])
def test_e1_no_failures(gf_lib, kind, teams, threads):
    gf = gf_lib
    ms, fails = ctypes.c_float(), ctypes.c_uint64(123)
    with gf.Context(timeout_ns=10_000_000_000, heap_bytes=1 << 30) as c:
        rc = gf.gf_alloc_e1(c.h, kind, teams, threads, 64, 2, None, ctypes.byref(ms), ctypes.byref(fails))
    assert rc == 0 and fails.value == 0 and ms.value > 0
