"""The C-ABI library builds, loads and exports every symbol include/pme.h declares; argument validation
that needs no GPU (no compute calls here)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2009_12617_gb300 import build, pme

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build_library()
    return pme.load_library()


def _declared():
    src = open(os.path.join(ROOT, "include", "pme.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pme_[a-z0-9_]+)\s*\(", src)))


def test_header_declarations_match_binding():
    assert sorted(pme.EXPORTS) == _declared()


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name
    out = os.popen(f"nm -D --defined-only {build.library_path()}").read()
    for name in _declared():
        assert re.search(rf"\bT {name}\b", out), name


def test_strerror(lib):
    for s in range(9):
        assert pme.pme_strerror(s)
    assert pme.pme_strerror(0) == "ok"


@pytest.mark.parametrize("K,p,beta,expect", [
    ((14, 16, 16), 4, 0.3, pme.PME_EINVAL),    # 7 is not an allowed prime factor
    ((15, 16, 16), 4, 0.3, pme.PME_EINVAL),    # odd edge
    ((6, 16, 16), 4, 0.3, pme.PME_EINVAL),     # below 8
    ((256, 16, 16), 4, 0.3, pme.PME_EINVAL),   # above 128
    ((16, 16, 16), 7, 0.3, pme.PME_EUNSUPPORTED),  # an order this build does not implement
    ((16, 16, 16), 2, 0.3, pme.PME_EUNSUPPORTED),
    ((16, 16, 16), 10, 0.3, pme.PME_EUNSUPPORTED),
    ((16, 16, 16), 4, 0.0, pme.PME_EINVAL),
    ((16, 16, 16), 4, float("nan"), pme.PME_EINVAL),
])
def test_create_validation(lib, K, p, beta, expect):
    with pytest.raises(pme.PMEError) as ei:
        pme.pme_create(K, p, beta, np.eye(3) * 20.0)
    assert ei.value.status == expect
    assert ei.value.detail


def test_create_singular_box(lib):
    box = np.array([[10.0, 0, 0], [20.0, 0, 0], [0, 0, 10.0]])
    with pytest.raises(pme.PMEError) as ei:
        pme.pme_create((16, 16, 16), 4, 0.3, box)
    assert ei.value.status == pme.PME_EINVAL


def test_null_arguments(lib):
    out = ctypes.c_void_p()
    assert lib.pme_create(None, 4, 0.3, None, None, ctypes.byref(out)) == pme.PME_EINVAL
    assert lib.pme_compute(None, None, None, 0, None, None, None) == pme.PME_EINVAL
    assert lib.pme_sync(None) == pme.PME_EINVAL
    lib.pme_destroy(None)


def test_binding_address_cache():
    """The host-array binding's address cache returns each array's own data address, evicts the oldest
    entries beyond its size, and never answers for a different object that happens to get a cached id."""
    cache = pme._AddressCache(size=4)
    keep = [np.zeros((16, 3), np.float32) for _ in range(6)]
    for a in keep:
        assert cache(a) == a.ctypes.data
    assert len(cache._items) == 4
    for a in keep:  # evicted ones are recomputed, cached ones come back unchanged
        assert cache(a) == a.ctypes.data
    view = keep[0][2:]  # a new object over the same buffer: its own address
    assert cache(view) == view.ctypes.data != keep[0].ctypes.data
    import gc
    import weakref

    b = np.zeros(8, np.float32)
    cache(b)
    wb = weakref.ref(b)
    del b
    gc.collect()
    assert wb() is None  # the cache does not keep a caller's array alive
    for _ in range(50):  # fresh objects may reuse a freed id; the identity check keeps them apart
        c = np.ones(8, np.float32)
        assert cache(c) == c.ctypes.data


def test_binding_result_buffer_per_thread():
    """Energy and virial land in a 7-double buffer owned by the calling thread."""
    import threading

    ev, at = pme._result_buffer()
    assert ev.shape == (7,) and ev.dtype == np.float64 and at == ev.ctypes.data
    assert pme._result_buffer()[1] == at
    other = []
    t = threading.Thread(target=lambda: other.append(pme._result_buffer()[1]))
    t.start()
    t.join()
    assert other[0] != at


def test_product_never_reaches_the_oracle(tmp_path):
    """The package imports nothing from oracle/ (a fresh interpreter that imports it loads no oracle module),
    no product source names it in an import, and a missing CUDA library raises instead of falling back."""
    import subprocess
    import sys

    code = ("import sys; import paper_2009_12617_gb300, paper_2009_12617_gb300.pme, paper_2009_12617_gb300.build, "
            "paper_2009_12617_gb300.workloads; "
            "print(sorted(m for m in sys.modules if m == 'oracle' or m.startswith('oracle.')))")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, check=True).stdout
    assert out.strip() == "[]"
    pkg = os.path.join(ROOT, "paper_2009_12617_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", src, re.M), f
                assert "oracle/" not in src and "liboracle" not in src, f
    code = ("from paper_2009_12617_gb300 import pme\n"
            "try:\n    pme.load_library(%r)\nexcept RuntimeError as e:\n    print('raised', e)\n" % str(tmp_path / "missing.so"))
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, check=True).stdout
    assert out.startswith("raised")


def test_injected_host_allocation_failure(lib):
    """The first allocation of each constructor is its host object, made before any CUDA call: with the
    first allocation made to fail, every constructor returns PME_ENOMEM (no GPU needed), and disarming
    restores normal argument checking."""
    box = np.eye(3) * 20.0
    try:
        for make in (lambda: pme.pme_create((16, 16, 16), 4, 0.3, box), lambda: pme.pme_real_create(box, 0.3, 9.0),
                     lambda: pme.pme_server_create(1 << 20, 4)):
            pme.pme_debug_fail_alloc(1)
            with pytest.raises(pme.PMEError) as ei:
                make()
            assert ei.value.status == pme.PME_ENOMEM and "allocation" in ei.value.detail
    finally:
        pme.pme_debug_fail_alloc(0)
    with pytest.raises(pme.PMEError) as ei:
        pme.pme_debug_fail_alloc(-1)
    assert ei.value.status == pme.PME_EINVAL
