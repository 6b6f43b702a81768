"""The RPC ring protocol and host server with CPU threads as the fake device
(no GPU): wrap-around and credit exhaustion, warp-aggregated slots,
out-of-order publication, a claimant that dies mid-slot, a stalled server,
several server threads, and format-string caching.  Faults are injected on
the host only."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2306_11686_gb300", "csrc")


@pytest.fixture(scope="module")
def ring_bin(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("ring") / "ring_test")
    subprocess.run(["g++", "-std=c++17", "-O2", "-pthread", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
                    os.path.join(ROOT, "tests", "host", "ring_fake_device.cpp"),
                    os.path.join(CSRC, "host", "server.cpp"), "-o", out], check=True)
    return out


@pytest.mark.parametrize("scenario", ["basic", "aggregate", "ooo", "dead", "stall", "threads", "fmtcache",
                                      "bulkfile", "bulkchunks", "closerace", "retire"])
def test_ring_scenario(ring_bin, tmp_path, scenario):
    p = subprocess.run([ring_bin, scenario, str(tmp_path / "out.txt")], capture_output=True, text=True, timeout=120)
    assert p.returncode == 0, p.stdout + p.stderr
    assert p.stdout.strip().endswith("OK " + scenario)


def test_async_output_file(tmp_path):
    """The stdout file written by its own thread: lines from four threads
    (some of 65 KB, in several writes) are whole and in per-thread order
    after every drain and after close; a drain returns promptly while
    another thread keeps printing (it waits only for what was queued
    before it)."""
    exe = str(tmp_path / "async_check")
    subprocess.run(["g++", "-std=c++17", "-O2", "-pthread", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
                    os.path.join(ROOT, "tests", "host", "async_file_check.cpp"),
                    os.path.join(CSRC, "host", "server.cpp"), "-o", exe], check=True)
    p = subprocess.run([exe, str(tmp_path / "out.txt")], capture_output=True, text=True, timeout=120)
    assert p.returncode == 0 and "OK" in p.stdout, p.stdout + p.stderr
