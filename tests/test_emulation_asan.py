"""AddressSanitizer sweep of the stage bodies, compiled for the CPU (PME_HOST_EMULATION).

compute-sanitizer is not available for these kernels, so memory safety of their index arithmetic is checked
here: the same source, built with -fsanitize=address, runs in a child process over meshes, orders, tile edges,
bucket capacities and positions that exercise every ragged edge (tests/emu/asan_sweep.py).
"""
import os
import shutil
import subprocess
import sys

import pytest

from helpers import EMU_SRC, ROOT

ASAN_LIB = os.path.join(ROOT, "tests", "emu", "_build", "libpme_emu_asan.so")


def _libasan():
    if shutil.which("g++") is None:
        return None
    path = subprocess.run(["g++", "-print-file-name=libasan.so"], capture_output=True, text=True).stdout.strip()
    return path if os.path.isabs(path) and os.path.exists(path) else None


@pytest.mark.slow
def test_stage_bodies_under_address_sanitizer():
    libasan = _libasan()
    if libasan is None:
        pytest.skip("libasan not available")
    os.makedirs(os.path.dirname(ASAN_LIB), exist_ok=True)
    tmp = ASAN_LIB + f".{os.getpid()}.tmp"
    subprocess.check_call(["g++", "-O1", "-g", "-std=c++17", "-fPIC", "-shared", "-DPME_HOST_EMULATION",
                           "-ffp-contract=off", "-fsanitize=address", "-fno-omit-frame-pointer",
                           "-I/usr/local/cuda/include", "-x", "c++", EMU_SRC, "-o", tmp])
    os.replace(tmp, ASAN_LIB)
    env = dict(os.environ, LD_PRELOAD=libasan, ASAN_OPTIONS="detect_leaks=0:abort_on_error=0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "emu", "asan_sweep.py"), ASAN_LIB],
                       env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "asan sweep ok" in r.stdout
