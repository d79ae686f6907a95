"""Thin Python binding of the C ABI in include/pme.h (ctypes; argument marshalling only).

Every function here has the name of the C entry point it calls, and every step of the SPME evaluation runs
in the CUDA library ``libpme_gb300.so``. Array arguments are torch CUDA tensors (float32, contiguous; the
library reads their device pointers) except in ``pme_compute_host``, which takes host numpy arrays.
There is no CPU fallback: if the library is missing, loading it raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
import weakref

import numpy as np

from . import build as _build

PME_OK = 0
PME_EINVAL = 1
PME_EUNSUPPORTED = 2
PME_ENOMEM = 3
PME_ECUDA = 4
PME_EOVERFLOW = 5
PME_EAGAIN = 6
PME_ETIMEOUT = 7
PME_PENDING = 8

PME_BATCH_AUTO = 0
PME_BATCH_GROUPED = 1
PME_BATCH_PERSISTENT = 2

STATUS_NAMES = {0: "PME_OK", 1: "PME_EINVAL", 2: "PME_EUNSUPPORTED", 3: "PME_ENOMEM", 4: "PME_ECUDA",
                5: "PME_EOVERFLOW", 6: "PME_EAGAIN", 7: "PME_ETIMEOUT", 8: "PME_PENDING"}

# every symbol include/pme.h declares
EXPORTS = ("pme_create", "pme_set_box", "pme_compute", "pme_compute_debug", "pme_enqueue", "pme_reserve", "pme_sync", "pme_compute_host",
           "pme_profile_stages", "pme_set_launch_mode", "pme_set_slab_split", "pme_plan_device_bytes", "pme_destroy", "pme_batch_create", "pme_batch_enqueue", "pme_batch_sync",
           "pme_batch_destroy", "pme_server_create", "pme_submit", "pme_poll", "pme_server_stats",
           "pme_server_destroy", "pme_strerror", "pme_last_error_detail", "pme_batch_debug_stall",
           "pme_compute_noalloc", "pme_batch_set_strategy", "pme_batch_get_strategy",
           "pme_probe_launch", "pme_real_create", "pme_real_set_box", "pme_real_reserve", "pme_real_enqueue",
           "pme_real_compute", "pme_real_destroy", "pme_autotune", "pme_tune_cache", "pme_plan_set_tiling",
           "pme_plan_get_tiling", "pme_batch_autotune", "pme_run_steps", "pme_debug_fail_alloc",
           "pme_set_influence_path", "pme_get_influence_path", "pme_slab_create", "pme_slab_layout",
           "pme_slab_stage1", "pme_slab_stage2", "pme_slab_stage3", "pme_slab_sync", "pme_slab_destroy",
           "pme_enqueue_host", "pme_host_wait")


PME_TUNE_FORCE = 1
PME_INFLUENCE_FP32 = 0
PME_INFLUENCE_TENSOR = 1


class TuneResult(ctypes.Structure):
    """pme_tune_result of include/pme.h."""
    _fields_ = [("tile_edge", ctypes.c_int), ("tile_threads", ctypes.c_int), ("us_per_eval", ctypes.c_double),
                ("default_us", ctypes.c_double), ("candidates", ctypes.c_int), ("rejected", ctypes.c_int),
                ("from_cache", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class PMEError(RuntimeError):
    def __init__(self, status: int, detail: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {detail}")
        self.status = status
        self.detail = detail


_lib = None
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_st = ctypes.c_int


class _AddressCache:
    """Data addresses of the last few numpy arrays the binding was given. Reading ``a.ctypes.data`` costs about a
    microsecond; a loop that passes the same buffers every step finds them here. Entries hold weak references
    (no caller's buffer is kept alive), and a hit needs the very same live object, so an id reused by a new
    array is never mistaken for a cached one."""

    def __init__(self, size: int = 8):
        self._items: dict = {}  # id -> (weak reference, address), oldest first
        self._size = size

    def __call__(self, a: np.ndarray) -> int:
        # no lock: each dict operation is atomic under the interpreter lock, and a race costs at most a
        # recomputed address
        items = self._items
        hit = items.get(id(a))
        if hit is not None and hit[0]() is a:
            return hit[1]
        p = a.ctypes.data
        items[id(a)] = (weakref.ref(a), p)
        while len(items) > self._size:
            try:
                del items[next(iter(items))]
            except (KeyError, RuntimeError, StopIteration):  # another thread changed it meanwhile
                break
        return p


_addr = _AddressCache()
_tls = threading.local()


def _result_buffer():
    """This thread's 7 doubles receiving energy and virial, and their address."""
    b = getattr(_tls, "ev", None)
    if b is None:
        arr = np.zeros(7)
        b = _tls.ev = (arr, arr.ctypes.data)
    return b


def load_library(path: str | None = None):
    """Load libpme_gb300.so (built by __graft_entry__.build() / paper_2009_12617_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    sig = {
        "pme_create": (_st, [ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_double), _vp, ctypes.POINTER(_vp)]),
        "pme_set_box": (_st, [_vp, ctypes.POINTER(ctypes.c_double)]),
        "pme_compute": (_st, [_vp, _vp, _vp, _i64, _vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
        "pme_compute_debug": (_st, [_vp, _vp, _vp, _i64, _vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), _vp, _vp]),
        "pme_enqueue": (_st, [_vp, _vp, _vp, _i64, _vp, _vp]),
        "pme_reserve": (_st, [_vp, _i64]),
        "pme_sync": (_st, [_vp]),
        "pme_compute_host": (_st, [_vp, _vp, _vp, _i64, _vp, _vp, _vp]),
        "pme_enqueue_host": (_st, [_vp, _vp, _vp, _i64, _vp, _vp, ctypes.POINTER(_i64)]),
        "pme_host_wait": (_st, [_vp, _i64]),
        "pme_profile_stages": (_st, [_vp, _vp, _vp, _i64, _vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
        "pme_set_launch_mode": (_st, [ctypes.c_int]),
        "pme_set_slab_split": (_st, [ctypes.c_int, ctypes.c_int]),
        "pme_plan_device_bytes": (ctypes.c_size_t, [_vp]),
        "pme_destroy": (None, [_vp]),
        "pme_batch_create": (_st, [ctypes.c_int, ctypes.POINTER(_vp), ctypes.POINTER(_i64), _vp, ctypes.POINTER(_vp)]),
        "pme_batch_enqueue": (_st, [_vp, _vp, _vp, _vp, _vp]),
        "pme_batch_sync": (_st, [_vp]),
        "pme_batch_destroy": (None, [_vp]),
        "pme_batch_debug_stall": (_st, [_vp, ctypes.c_int, _i64]),
        "pme_batch_set_strategy": (_st, [_vp, ctypes.c_int]),
        "pme_batch_get_strategy": (ctypes.c_int, [_vp]),
        "pme_autotune": (_st, [_vp, _vp, _vp, _i64, _vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(TuneResult)]),
        "pme_tune_cache": (_st, [ctypes.c_char_p]),
        "pme_plan_set_tiling": (_st, [_vp, ctypes.c_int, ctypes.c_int]),
        "pme_plan_get_tiling": (_st, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
        "pme_batch_autotune": (_st, [_vp, _vp, _vp, _vp, _vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]),
        "pme_debug_fail_alloc": (_st, [ctypes.c_int]),
        "pme_set_influence_path": (_st, [_vp, ctypes.c_int]),
        "pme_slab_create": (_st, [ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_int, _vp, ctypes.POINTER(_vp)]),
        "pme_slab_layout": (_st, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_i64)]),
        "pme_slab_stage1": (_st, [_vp, _vp, _vp, _i64, _vp]),
        "pme_slab_stage2": (_st, [_vp, _vp, _vp, _vp]),
        "pme_slab_stage3": (_st, [_vp, _vp, _vp, _vp, _i64, _vp]),
        "pme_slab_sync": (_st, [_vp]),
        "pme_slab_destroy": (None, [_vp]),
        "pme_get_influence_path": (ctypes.c_int, [_vp]),
        "pme_run_steps": (_st, [_vp, _vp, _vp, _vp, _vp, _vp, _i64, _vp, ctypes.c_double, ctypes.c_int, _vp]),
        "pme_real_create": (_st, [ctypes.POINTER(ctypes.c_double), ctypes.c_double, ctypes.c_double, _vp, ctypes.POINTER(_vp)]),
        "pme_real_set_box": (_st, [_vp, ctypes.POINTER(ctypes.c_double)]),
        "pme_real_reserve": (_st, [_vp, _i64]),
        "pme_real_enqueue": (_st, [_vp, _vp, _vp, _i64, _vp, ctypes.c_int, _vp]),
        "pme_real_compute": (_st, [_vp, _vp, _vp, _i64, _vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
        "pme_real_destroy": (None, [_vp]),
        "pme_probe_launch": (_st, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_size_t, _vp, ctypes.POINTER(ctypes.c_double)]),
        "pme_server_create": (_st, [ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(_vp)]),
        "pme_submit": (_st, [_vp, _vp, _vp, _vp, _i64, _vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_i64)]),
        "pme_poll": (_st, [_vp, _i64, ctypes.c_int]),
        "pme_server_stats": (_st, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_i64)]),
        "pme_server_destroy": (None, [_vp]),
        "pme_strerror": (ctypes.c_char_p, [_st]),
        "pme_last_error_detail": (_st, [ctypes.c_char_p, ctypes.c_size_t]),
        "pme_compute_noalloc": (_st, [ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_double), _vp, _vp, _i64, _vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), _vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def last_error_detail() -> str:
    buf = ctypes.create_string_buffer(512)
    load_library().pme_last_error_detail(buf, 512)
    return buf.value.decode(errors="replace")


def check(status: int) -> int:
    if status != PME_OK and status != PME_PENDING:
        raise PMEError(status, last_error_detail())
    return status


def _ptr(t) -> int:
    """Device pointer of a CUDA tensor (float32, contiguous), or 0 for None."""
    if t is None:
        return 0
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def _f32(t, shape_tail, name):
    import torch

    if t.dtype != torch.float32:
        raise TypeError(f"{name} must be float32")
    if tuple(t.shape[1:]) != shape_tail:
        raise ValueError(f"{name} has shape {tuple(t.shape)}")
    return _ptr(t)


def _stream_handle(stream) -> int:
    if stream is None:
        return 0
    return int(getattr(stream, "cuda_stream", stream))


# ---------------------------------------------------------------------------------------------------------
# C entry points (same names as include/pme.h)


def pme_create(K, p: int, beta: float, box, stream=None) -> int:
    K = (ctypes.c_int * 3)(*[int(k) for k in K])
    bx = np.ascontiguousarray(box, dtype=np.float64).reshape(9)
    out = _vp()
    check(load_library().pme_create(K, int(p), float(beta), bx.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                    _vp(_stream_handle(stream)), ctypes.byref(out)))
    return out.value


def pme_set_box(plan: int, box) -> None:
    bx = np.ascontiguousarray(box, dtype=np.float64).reshape(9)
    check(load_library().pme_set_box(_vp(plan), bx.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))


def pme_compute(plan: int, pos, q, forces) -> tuple[float, np.ndarray]:
    """Synchronous evaluation on torch CUDA tensors pos (n,3), q (n,), forces (n,3); returns (E, virial[6])."""
    n = int(q.shape[0])
    e = ctypes.c_double()
    vir = (ctypes.c_double * 6)()
    check(load_library().pme_compute(_vp(plan), _vp(_f32(pos, (3,), "pos")), _vp(_f32(q, (), "q")), n,
                                     _vp(_f32(forces, (3,), "forces")), ctypes.byref(e), vir))
    return e.value, np.array(vir[:])


def pme_compute_debug(plan: int, pos, q, forces, mesh=None, phi=None) -> tuple[float, np.ndarray]:
    """pme_compute that also copies the fixed-point charge mesh (int64 CUDA tensor of shape K) and the
    potential mesh (float32 CUDA tensor of shape K) into mesh / phi when given."""
    n = int(q.shape[0])
    e = ctypes.c_double()
    vir = (ctypes.c_double * 6)()
    check(load_library().pme_compute_debug(_vp(plan), _vp(_f32(pos, (3,), "pos")), _vp(_f32(q, (), "q")), n,
                                           _vp(_f32(forces, (3,), "forces")), ctypes.byref(e), vir,
                                           _vp(_ptr(mesh)), _vp(_ptr(phi))))
    return e.value, np.array(vir[:])


def pme_enqueue(plan: int, pos, q, forces, ev_dev=None) -> None:
    """Asynchronous evaluation; ev_dev is a float64 CUDA tensor of 7 (or None for the plan's own slot)."""
    n = int(q.shape[0])
    check(load_library().pme_enqueue(_vp(plan), _vp(_f32(pos, (3,), "pos")), _vp(_f32(q, (), "q")), n,
                                     _vp(_f32(forces, (3,), "forces")), _vp(_ptr(ev_dev))))


def pme_reserve(plan: int, n: int) -> None:
    check(load_library().pme_reserve(_vp(plan), int(n)))


def pme_sync(plan: int) -> None:
    check(load_library().pme_sync(_vp(plan)))


def pme_enqueue_host(plan: int, pos: np.ndarray, q: np.ndarray, forces: np.ndarray, result: np.ndarray) -> int:
    """Asynchronous evaluation on page-locked numpy arrays (pos (n,3), q (n,), forces (n,3) float32; result (8,)
    float64 receives energy, virial[6] and the status bits); returns the ticket to pass to pme_host_wait."""
    for name, a, dt in (("pos", pos, np.float32), ("q", q, np.float32), ("forces", forces, np.float32),
                        ("result", result, np.float64)):
        if a.dtype != dt or not a.flags["C_CONTIGUOUS"]:
            raise ValueError(f"{name} must be a contiguous {np.dtype(dt).name} array")
    n = int(q.shape[0])
    t = ctypes.c_int64()
    check(load_library().pme_enqueue_host(_vp(plan), _vp(_addr(pos)), _vp(_addr(q)), n, _vp(_addr(forces)),
                                          _vp(_addr(result)), ctypes.byref(t)))
    return t.value


def pme_host_wait(plan: int, ticket: int) -> None:
    """Block until pme_enqueue_host's ticket has its forces and result in host memory."""
    check(load_library().pme_host_wait(_vp(plan), int(ticket)))


def pme_compute_host(plan: int, pos: np.ndarray, q: np.ndarray, forces: np.ndarray | None = None):
    """Evaluation on HOST numpy arrays (float32); returns (forces, E, virial[6])."""
    if pos.dtype != np.float32 or not pos.flags.c_contiguous:
        pos = np.ascontiguousarray(pos, dtype=np.float32)
    if q.dtype != np.float32 or not q.flags.c_contiguous:
        q = np.ascontiguousarray(q, dtype=np.float32)
    n = int(q.shape[0])
    if pos.shape != (n, 3):
        raise ValueError("pos must be (n, 3)")
    if forces is None:
        forces = np.empty((n, 3), dtype=np.float32)
    if forces.dtype != np.float32 or forces.shape != (n, 3) or not forces.flags.c_contiguous:
        raise ValueError("forces must be a contiguous float32 (n, 3) array")
    ev, at = _result_buffer()
    check(load_library().pme_compute_host(plan, _addr(pos), _addr(q), n, _addr(forces), at, at + 8))
    return forces, float(ev[0]), ev[1:].copy()


STAGE_NAMES = ("bin", "spread", "fft_fwd", "influence", "fft_inv", "gather")


def pme_profile_stages(plan: int, pos, q, forces, reps: int = 10) -> dict:
    """Mean microseconds per stage kernel (CUDA events on the plan stream) over reps evaluations."""
    out = (ctypes.c_double * 6)()
    check(load_library().pme_profile_stages(_vp(plan), _vp(_f32(pos, (3,), "pos")), _vp(_f32(q, (), "q")),
                                            int(q.shape[0]), _vp(_f32(forces, (3,), "forces")), int(reps), out))
    return dict(zip(STAGE_NAMES, out[:]))


def pme_set_launch_mode(mode: int) -> None:
    """0 plain; programmatic dependent launch triggered 1 at kernel entry, 2 (default) at CTA exit (the influence
    stage: right after its own wait), 3 right after each kernel's own wait."""
    check(load_library().pme_set_launch_mode(int(mode)))


def pme_set_slab_split(fwd_ctas: int, inv_ctas: int | None = None) -> None:
    """CTAs (a thread-block cluster) per slab of the forward and the inverse slab stage: 1, 2 or 4 each
    (inv_ctas defaults to fwd_ctas)."""
    check(load_library().pme_set_slab_split(int(fwd_ctas), int(fwd_ctas if inv_ctas is None else inv_ctas)))


def pme_plan_device_bytes(plan: int) -> int:
    return int(load_library().pme_plan_device_bytes(_vp(plan)))


def pme_destroy(plan: int) -> None:
    if plan:
        load_library().pme_destroy(_vp(plan))


def pme_batch_create(plans, n, stream=None) -> int:
    arr = (_vp * len(plans))(*[_vp(p) for p in plans])
    ns = (_i64 * len(n))(*[int(x) for x in n])
    out = _vp()
    check(load_library().pme_batch_create(len(plans), arr, ns, _vp(_stream_handle(stream)), ctypes.byref(out)))
    return out.value


def pme_batch_enqueue(batch: int, pos, q, forces, ev_dev) -> None:
    check(load_library().pme_batch_enqueue(_vp(batch), _vp(_f32(pos, (3,), "pos")), _vp(_f32(q, (), "q")),
                                           _vp(_f32(forces, (3,), "forces")), _vp(_ptr(ev_dev))))


def pme_batch_sync(batch: int) -> int:
    return check(load_library().pme_batch_sync(_vp(batch)))


def pme_batch_destroy(batch: int) -> None:
    if batch:
        load_library().pme_batch_destroy(_vp(batch))


def pme_batch_set_strategy(batch: int, strategy: int) -> None:
    check(load_library().pme_batch_set_strategy(_vp(batch), int(strategy)))


def pme_batch_get_strategy(batch: int) -> int:
    return int(load_library().pme_batch_get_strategy(_vp(batch)))


def pme_batch_debug_stall(batch: int, enable: bool, wait_limit_ns: int = 200_000_000) -> None:
    check(load_library().pme_batch_debug_stall(_vp(batch), int(bool(enable)), int(wait_limit_ns)))


def pme_server_create(mem_budget_bytes: int, max_slots: int) -> int:
    out = _vp()
    check(load_library().pme_server_create(int(mem_budget_bytes), int(max_slots), ctypes.byref(out)))
    return out.value


class Ticket:
    """A submitted request: keeps the host result slots alive until the request completes."""

    def __init__(self):
        self.id = _i64()
        self.energy = ctypes.c_double()
        self.virial = (ctypes.c_double * 6)()


def pme_submit(srv: int, plan: int, pos, q, forces) -> Ticket:
    t = Ticket()
    st = load_library().pme_submit(_vp(srv), _vp(plan), _vp(_f32(pos, (3,), "pos")), _vp(_f32(q, (), "q")),
                                   int(q.shape[0]), _vp(_f32(forces, (3,), "forces")), ctypes.byref(t.energy),
                                   t.virial, ctypes.byref(t.id))
    if st == PME_EAGAIN:
        return None
    check(st)
    return t


def pme_poll(srv: int, ticket: Ticket, block: bool = False) -> int:
    return check(load_library().pme_poll(_vp(srv), ticket.id.value, int(bool(block))))


def pme_server_stats(srv: int) -> dict:
    c, w = _i64(), _i64()
    p50, p99 = ctypes.c_double(), ctypes.c_double()
    check(load_library().pme_server_stats(_vp(srv), ctypes.byref(c), ctypes.byref(p50), ctypes.byref(p99),
                                          ctypes.byref(w)))
    return {"completed": c.value, "p50_us": p50.value, "p99_us": p99.value, "waves": w.value}


def pme_server_destroy(srv: int) -> None:
    if srv:
        load_library().pme_server_destroy(_vp(srv))


def pme_compute_noalloc(K, p: int, beta: float, box, pos, q, forces, stream=None) -> tuple[float, np.ndarray]:
    """Allocation-free evaluation of one small system (see include/pme.h): the library allocates no device
    memory for it, using a fixed static device array instead. Returns (E, virial[6]); forces filled."""
    import torch

    n = int(q.shape[0])
    if int(pos.shape[0]) != n or int(forces.shape[0]) != n:
        raise ValueError(f"pos {tuple(pos.shape)}, q {tuple(q.shape)} and forces {tuple(forces.shape)} need the same n")
    cur = torch.cuda.current_device()
    for name, t in (("pos", pos), ("q", q), ("forces", forces)):
        if t.is_cuda and t.device.index != cur:
            raise ValueError(f"{name} is on cuda:{t.device.index}, but the call runs on the current device cuda:{cur}")
    if stream is None:  # the caller's current torch stream, so the call orders after the work that made pos / q
        stream = torch.cuda.current_stream(cur)
    Kc = (ctypes.c_int * 3)(*[int(k) for k in K])
    bx = np.ascontiguousarray(box, dtype=np.float64).reshape(9)
    e = ctypes.c_double()
    vir = (ctypes.c_double * 6)()
    check(load_library().pme_compute_noalloc(Kc, int(p), float(beta), bx.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                             _vp(_f32(pos, (3,), "pos")), _vp(_f32(q, (), "q")), n,
                                             _vp(_f32(forces, (3,), "forces")), ctypes.byref(e), vir,
                                             _vp(_stream_handle(stream))))
    return e.value, np.array(vir[:])


def pme_probe_launch(kind: int, ctas: int, rounds: int, buf, stream=None) -> float:
    """Enqueue one atomic-throughput probe kernel (kind 0: shared-memory int32 atomics, 1: global int64
    reductions) on buf (a CUDA tensor); returns the operations it performs."""
    ops = ctypes.c_double()
    check(load_library().pme_probe_launch(int(kind), int(ctas), int(rounds), _vp(_ptr(buf)),
                                          buf.numel() * buf.element_size(), _vp(_stream_handle(stream)), ctypes.byref(ops)))
    return ops.value


def pme_autotune(plan: int, pos, q, forces, reps: int = 20, force: bool = False) -> dict:
    """Tune the plan's tile edge and CTA size on these atoms (see include/pme.h); returns pme_tune_result."""
    res = TuneResult()
    check(load_library().pme_autotune(_vp(plan), _vp(_f32(pos, (3,), "pos")), _vp(_f32(q, (), "q")), int(q.shape[0]),
                                      _vp(_f32(forces, (3,), "forces")), int(reps), PME_TUNE_FORCE if force else 0,
                                      ctypes.byref(res)))
    return res.as_dict()


def pme_tune_cache(path) -> None:
    check(load_library().pme_tune_cache(None if path is None else os.fsencode(path)))


def pme_plan_set_tiling(plan: int, tile_edge: int = 0, tile_threads: int = 0) -> None:
    check(load_library().pme_plan_set_tiling(_vp(plan), int(tile_edge), int(tile_threads)))


def pme_plan_get_tiling(plan: int) -> tuple[int, int]:
    e, t = ctypes.c_int(), ctypes.c_int()
    check(load_library().pme_plan_get_tiling(_vp(plan), ctypes.byref(e), ctypes.byref(t)))
    return e.value, t.value


def pme_batch_autotune(batch: int, pos, q, forces, ev_dev, reps: int = 10) -> tuple[int, float]:
    """Tune a batch's strategy and tile CTA size; returns (strategy, us per batch)."""
    st, us = ctypes.c_int(), ctypes.c_double()
    check(load_library().pme_batch_autotune(_vp(batch), _vp(_f32(pos, (3,), "pos")), _vp(_f32(q, (), "q")),
                                            _vp(_f32(forces, (3,), "forces")), _vp(_ptr(ev_dev)), int(reps),
                                            ctypes.byref(st), ctypes.byref(us)))
    return st.value, us.value


def pme_run_steps(plan: int, pos, vel, q, forces, dt: float, steps: int, rs: int = 0, inv_mass=None,
                  ev_steps=None) -> None:
    """Enqueue `steps` leapfrog time steps on the device (see include/pme.h); pme_sync(plan) waits."""
    n = int(q.shape[0])
    if inv_mass is not None:
        _f32(inv_mass, (), "inv_mass")
    check(load_library().pme_run_steps(_vp(plan), _vp(rs or 0), _vp(_f32(pos, (3,), "pos")), _vp(_f32(vel, (3,), "vel")),
                                       _vp(_f32(q, (), "q")), _vp(_ptr(inv_mass)), n, _vp(_f32(forces, (3,), "forces")),
                                       float(dt), int(steps), _vp(_ptr(ev_steps))))


def pme_real_create(box, beta: float, rcut: float, stream=None) -> int:
    bx = np.ascontiguousarray(box, dtype=np.float64).reshape(9)
    out = _vp()
    check(load_library().pme_real_create(bx.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), float(beta), float(rcut),
                                         _vp(_stream_handle(stream)), ctypes.byref(out)))
    return out.value


def pme_real_set_box(rs: int, box) -> None:
    bx = np.ascontiguousarray(box, dtype=np.float64).reshape(9)
    check(load_library().pme_real_set_box(_vp(rs), bx.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))


def pme_real_reserve(rs: int, n: int) -> None:
    check(load_library().pme_real_reserve(_vp(rs), int(n)))


def pme_real_enqueue(rs: int, pos, q, forces, accumulate: bool = False, ev_dev=None) -> None:
    """Asynchronous real-space evaluation; ev_dev (8 doubles, device) receives E_real, E_self, virial[6]."""
    n = int(q.shape[0])
    check(load_library().pme_real_enqueue(_vp(rs), _vp(_f32(pos, (3,), "pos")), _vp(_f32(q, (), "q")), n,
                                          _vp(_f32(forces, (3,), "forces")), int(bool(accumulate)), _vp(_ptr(ev_dev))))


def pme_real_compute(rs: int, pos, q, forces) -> tuple[float, float, np.ndarray]:
    """Synchronous real-space evaluation on CUDA tensors; returns (E_real, E_self, virial[6])."""
    n = int(q.shape[0])
    er, es = ctypes.c_double(), ctypes.c_double()
    vir = (ctypes.c_double * 6)()
    check(load_library().pme_real_compute(_vp(rs), _vp(_f32(pos, (3,), "pos")), _vp(_f32(q, (), "q")), n,
                                          _vp(_f32(forces, (3,), "forces")), ctypes.byref(er), ctypes.byref(es), vir))
    return er.value, es.value, np.array(vir[:])


def pme_real_destroy(rs: int) -> None:
    if rs:
        load_library().pme_real_destroy(_vp(rs))


def pme_set_influence_path(plan: int, path: int) -> None:
    check(load_library().pme_set_influence_path(_vp(plan), int(path)))


def pme_get_influence_path(plan: int) -> int:
    return int(load_library().pme_get_influence_path(_vp(plan)))


def pme_slab_create(K, p: int, beta: float, box, nranks: int, rank: int, stream=None) -> int:
    Kc = (ctypes.c_int * 3)(*[int(k) for k in K])
    bx = np.ascontiguousarray(box, dtype=np.float64).reshape(9)
    out = _vp()
    check(load_library().pme_slab_create(Kc, int(p), float(beta), bx.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                         int(nranks), int(rank), _vp(_stream_handle(stream)), ctypes.byref(out)))
    return out.value


def pme_slab_layout(slab: int) -> dict:
    pl, cl, b = (ctypes.c_int * 2)(), (ctypes.c_int * 2)(), _i64()
    check(load_library().pme_slab_layout(_vp(slab), pl, cl, ctypes.byref(b)))
    return {"planes": (pl[0], pl[1]), "columns": (cl[0], cl[1]), "block_values": b.value}


def pme_slab_stage1(slab: int, pos, q, send) -> None:
    check(load_library().pme_slab_stage1(_vp(slab), _vp(_f32(pos, (3,), "pos")), _vp(_f32(q, (), "q")),
                                         int(q.shape[0]), _vp(_ptr(send))))


def pme_slab_stage2(slab: int, recv, send, ev_dev=None) -> None:
    check(load_library().pme_slab_stage2(_vp(slab), _vp(_ptr(recv)), _vp(_ptr(send)), _vp(_ptr(ev_dev))))


def pme_slab_stage3(slab: int, recv, pos, q, forces) -> None:
    check(load_library().pme_slab_stage3(_vp(slab), _vp(_ptr(recv)), _vp(_f32(pos, (3,), "pos")),
                                         _vp(_f32(q, (), "q")), int(q.shape[0]), _vp(_f32(forces, (3,), "forces"))))


def pme_slab_sync(slab: int) -> int:
    return check(load_library().pme_slab_sync(_vp(slab)))


def pme_slab_destroy(slab: int) -> None:
    if slab:
        load_library().pme_slab_destroy(_vp(slab))


def pme_debug_fail_alloc(nth: int) -> None:
    """Make the nth library allocation from now on fail (0 disarms); for tests."""
    check(load_library().pme_debug_fail_alloc(int(nth)))


def pme_strerror(status: int) -> str:
    return load_library().pme_strerror(int(status)).decode()


# ---------------------------------------------------------------------------------------------------------
# convenience wrapper


class Plan:
    """Owns a pme_plan: Plan(K, p, beta, box, stream=None)."""

    def __init__(self, K, p: int, beta: float, box, stream=None):
        self.K = tuple(int(k) for k in K)
        self.p = int(p)
        self.beta = float(beta)
        self.handle = pme_create(self.K, self.p, self.beta, box, stream)

    def compute(self, pos, q, forces=None):
        import torch

        if forces is None:
            forces = torch.empty_like(pos)
        e, vir = pme_compute(self.handle, pos, q, forces)
        return forces, e, vir

    def enqueue(self, pos, q, forces, ev_dev=None):
        pme_enqueue(self.handle, pos, q, forces, ev_dev)

    def close(self):
        if self.handle:
            pme_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
