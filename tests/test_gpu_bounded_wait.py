"""The bounded mbarrier wait that the tile renderer's TMA staging and the
radix downsweep's bulk copies use: a phase that never completes makes the
wait give up after its poll limit (the kernel returns, the context stays
usable), and a completed phase is seen at once.  The failure is a barrier
that nothing arrives on, not a fault."""
import ctypes
import os
import subprocess
import time

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _build(tmp_path):
    from paper_1004_1302_gb300 import splotch as S
    so = str(tmp_path / "bounded_wait.so")
    cmd = [S._nvcc(), *S.ARCH, "-O3", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
           "-I", os.path.join(ROOT, "paper_1004_1302_gb300", "csrc"),
           os.path.join(ROOT, "tests", "cuda", "bounded_wait.cu"), "-o", so]
    subprocess.run(cmd, check=True, capture_output=True, timeout=300)
    lib = ctypes.CDLL(so)
    lib.run_bounded_wait.argtypes = [ctypes.c_int, ctypes.c_uint, ctypes.POINTER(ctypes.c_int)]
    lib.run_bounded_wait.restype = ctypes.c_int
    return lib


def test_wait_gives_up_on_a_phase_that_never_completes_and_sees_one_that_does(tmp_path):
    lib = _build(tmp_path)
    out = ctypes.c_int(-1)
    t0 = time.perf_counter()
    assert lib.run_bounded_wait(0, 2000, ctypes.byref(out)) == 0
    waited = time.perf_counter() - t0
    assert out.value == 0            # gave up: nothing arrived
    assert waited < 30.0
    out.value = -1
    assert lib.run_bounded_wait(1, 2000, ctypes.byref(out)) == 0
    assert out.value == 1            # the arrival completed the phase
    # the context is still usable after the wait that gave up
    out.value = -1
    assert lib.run_bounded_wait(0, 10, ctypes.byref(out)) == 0 and out.value == 0
