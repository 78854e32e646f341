"""The checked build (libmctp_checked.so, kernels compiled with MCTP_CHECKED):
every main index of the histogram, filter, slicemap and render kernels is
tested against the extent of the buffer it addresses, and an index outside
sets a bit in a device status word instead of being accessed.  Here the
self-test sets and clears its bit, and the parity, batched, texture and
batched-preparation tests run again against the checked library in a child
process, each ending with a check that no bit is set (tests/conftest.py)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return dict(os.environ, MCTP_LIBRARY="checked")


def test_checked_selftest():
    env = _env()
    code = """
import ctypes, sys
sys.path.insert(0, %r)
import torch
from paper_2311_15038_gb300 import _lib
L = _lib.load()
assert L.mctp_checked_build() == 1
bits = ctypes.c_uint32()
assert L.mctp_checked_status(ctypes.byref(bits), 1) == 0
assert L.mctp_checked_selftest(None) == 0
assert L.mctp_checked_status(ctypes.byref(bits), 1) == 0 and bits.value == 1 << 31, hex(bits.value)
assert L.mctp_checked_status(ctypes.byref(bits), 0) == 0 and bits.value == 0, hex(bits.value)
print("selftest ok")
""" % ROOT
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr


def test_parity_cases_under_the_checked_build():
    env = _env()
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider",
           os.path.join(ROOT, "tests", "test_gpu_parity.py"), os.path.join(ROOT, "tests", "test_gpu_batch.py"),
           os.path.join(ROOT, "tests", "test_gpu_texture.py"), os.path.join(ROOT, "tests", "test_gpu_prepare_batch.py"),
           "-k", "not fullsize"]
    r = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=3000, cwd=ROOT)
    print(r.stdout[-2000:])
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
