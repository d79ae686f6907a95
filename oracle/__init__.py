"""FP64 CPU oracle for the reciprocal-space SPME evaluation (ctypes wrapper over ``spme_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()`` and by bench.py's
``cpu_baseline`` and ``--impl reference`` legs. The library in ``paper_2009_12617_gb300`` never imports
it, and the two share no code.

Parity status of each function (what pins it is in tests/test_oracle_pins.py):
  bspline, bspline_deriv   pinned: closed-form cubic, partition of unity, symmetry, exact node values
  spread                   pinned: charge sum, exact node weights, brute-force image sum on tiny meshes
  dft3                     pinned: non-separable DFT on tiny meshes, Parseval, numpy FFT
  bmod2, influence         pinned: closed-form p = 4 modulus; convergence of SPME to Ewald
  spme (E, virial, F)      pinned: Ewald convergence, NaCl Madelung constant, finite differences of E
                           (positions and strain), phi identity, one-cell translation invariance
  ewald_recip/real/self    pinned: independent numpy Ewald, Madelung constant at two beta values, FD forces;
                           real-space virial by central differences of the energy under strain;
  ewald_real_rows          pinned: equals ewald_real's forces and per-atom energies row by row
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spme_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle_spme.so")
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (strict IEEE: -O2, no fast-math). Returns the library path."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        base = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-fno-fast-math", "-ffp-contract=off", "-o", tmp, _SRC]
        # OpenMP where the compiler has it (results do not depend on the thread count); serial otherwise
        r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:] + ["-lm"], capture_output=True, text=True)
        if r.returncode != 0:
            subprocess.check_call(base + ["-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        L = _lib
        L.oracle_recip.argtypes = [_dp, _dp, _dp]
        L.oracle_recip.restype = ctypes.c_int
        L.oracle_bspline.argtypes = [ctypes.c_int, ctypes.c_double]
        L.oracle_bspline.restype = ctypes.c_double
        L.oracle_bspline_deriv.argtypes = [ctypes.c_int, ctypes.c_double]
        L.oracle_bspline_deriv.restype = ctypes.c_double
        L.oracle_scaled_coords.argtypes = [ctypes.c_int64, _dp, _ip, _dp, _dp]
        L.oracle_spread.argtypes = [ctypes.c_int64, _dp, _dp, _ip, ctypes.c_int, _dp, _dp]
        L.oracle_dft3.argtypes = [_ip, ctypes.c_int, _dp, _dp, _dp, _dp]
        L.oracle_dft3_full.argtypes = [_ip, ctypes.c_int, _dp, _dp, _dp, _dp]
        L.oracle_bmod2.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.oracle_bmod2.restype = ctypes.c_double
        L.oracle_influence.argtypes = [_ip, ctypes.c_int, ctypes.c_double, _dp, _dp]
        L.oracle_spme.argtypes = [ctypes.c_int64, _dp, _dp, _ip, ctypes.c_int, ctypes.c_double, _dp, _dp, _dp,
                                  _dp, _dp, _dp, _dp]
        L.oracle_spme.restype = ctypes.c_int
        L.oracle_ewald_recip.argtypes = [ctypes.c_int64, _dp, _dp, ctypes.c_double, _dp, ctypes.c_double, _dp,
                                         _dp, _dp]
        L.oracle_ewald_recip.restype = ctypes.c_int
        L.oracle_ewald_real.argtypes = [ctypes.c_int64, _dp, _dp, ctypes.c_double, _dp, ctypes.c_double, _dp,
                                        _dp, _dp]
        L.oracle_ewald_real.restype = ctypes.c_int
        L.oracle_ewald_real_rows.argtypes = [ctypes.c_int64, _dp, _dp, ctypes.c_double, _dp, ctypes.c_double,
                                             ctypes.c_int64, ctypes.POINTER(ctypes.c_int64), _dp, _dp]
        L.oracle_ewald_real_rows.restype = ctypes.c_int
        L.oracle_ewald_self.argtypes = [ctypes.c_int64, _dp, ctypes.c_double]
        L.oracle_ewald_self.restype = ctypes.c_double
        L.oracle_set_threads.argtypes = [ctypes.c_int]
        L.oracle_max_threads.restype = ctypes.c_int
        _lib.oracle_set_threads(1)  # single-threaded unless a caller asks for more (set_threads)
    return _lib


def set_threads(n: int) -> int:
    """Threads for the parallel loops (OpenMP build); results are identical for any count. Returns the
    count now in effect (1 when the oracle was built without OpenMP)."""
    L = _load()
    L.oracle_set_threads(int(n))
    return int(L.oracle_max_threads())


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def _d(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _k(K) -> ctypes.Array:
    K = tuple(int(k) for k in K)
    return (ctypes.c_int * 3)(*K)


def recip(box):
    """(a*, V): a*[alpha] is the reciprocal vector with a*_alpha . a_beta = delta_alpha,beta."""
    box = _d(box).reshape(9)
    out = np.zeros(9)
    vol = ctypes.c_double()
    if _load().oracle_recip(_p(box), _p(out), ctypes.byref(vol)) != 0:
        raise ValueError("singular box")
    return out.reshape(3, 3), vol.value


def bspline(p: int, x: float) -> float:
    """Cardinal B-spline M_p(x) by the two-term recursion."""
    return _load().oracle_bspline(int(p), float(x))


def bspline_deriv(p: int, x: float) -> float:
    """M_p'(x) = M_{p-1}(x) - M_{p-1}(x - 1)."""
    return _load().oracle_bspline_deriv(int(p), float(x))


def scaled_coords(pos, K, box) -> np.ndarray:
    """u = K_alpha frac(a*_alpha . r) per atom, shape (n, 3)."""
    pos = _d(pos).reshape(-1, 3)
    box = _d(box).reshape(9)
    out = np.zeros_like(pos)
    _load().oracle_scaled_coords(pos.shape[0], _p(pos), _k(K), _p(box), _p(out))
    return out


def spread(pos, q, K, p, box) -> np.ndarray:
    """Charge mesh Q, shape K (row-major, k3 fastest)."""
    pos = _d(pos).reshape(-1, 3)
    q = _d(q).reshape(-1)
    box = _d(box).reshape(9)
    Q = np.zeros(tuple(K))
    _load().oracle_spread(pos.shape[0], _p(pos), _p(q), _k(K), int(p), _p(box), _p(Q))
    return Q


def dft3(x, sign: int = +1, full: bool = False) -> np.ndarray:
    """Direct 3D DFT sum_k x(k) exp(sign 2 pi i m.k/K); separable unless full=True."""
    x = np.asarray(x)
    K = x.shape
    re = _d(x.real)
    im = _d(x.imag) if np.iscomplexobj(x) else np.zeros(K)
    o_re = np.zeros(K)
    o_im = np.zeros(K)
    fn = _load().oracle_dft3_full if full else _load().oracle_dft3
    fn(_k(K), int(sign), _p(re), _p(im), _p(o_re), _p(o_im))
    return o_re + 1j * o_im


def bmod2(K: int, p: int, m: int) -> float:
    """|b(m)|^2 of one dimension."""
    return _load().oracle_bmod2(int(K), int(p), int(m))


def influence(K, p, beta, box) -> np.ndarray:
    """B(m) C(m) on the full mesh of m, shape K."""
    box = _d(box).reshape(9)
    BC = np.zeros(tuple(K))
    _load().oracle_influence(_k(K), int(p), float(beta), _p(box), _p(BC))
    return BC


def spme(pos, q, K, p, beta, box, want_mesh: bool = False) -> dict:
    """Reciprocal-space SPME: {'energy', 'virial' (xx,yy,zz,xy,xz,yz), 'forces' (n,3)}.

    want_mesh adds 'Q' and 'phi' (mesh arrays) and 'e_phi' = 1/2 sum Q phi.
    """
    pos = _d(pos).reshape(-1, 3)
    q = _d(q).reshape(-1)
    box = _d(box).reshape(9)
    n = pos.shape[0]
    e = ctypes.c_double()
    ephi = ctypes.c_double()
    vir = np.zeros(6)
    F = np.zeros((n, 3))
    Q = np.zeros(tuple(K)) if want_mesh else None
    phi = np.zeros(tuple(K)) if want_mesh else None
    rc = _load().oracle_spme(n, _p(pos), _p(q), _k(K), int(p), float(beta), _p(box), ctypes.byref(e), _p(vir),
                             _p(F), _p(Q) if want_mesh else None, _p(phi) if want_mesh else None,
                             ctypes.byref(ephi))
    if rc != 0:
        raise ValueError("invalid SPME arguments")
    out = {"energy": e.value, "virial": vir, "forces": F}
    if want_mesh:
        out.update(Q=Q, phi=phi, e_phi=ephi.value)
    return out


def ewald_mcut(beta: float, tol: float = 1e-16) -> float:
    """|m| cutoff with exp(-pi^2 m^2 / beta^2) < tol."""
    return beta * np.sqrt(-np.log(tol)) / np.pi


def ewald_recip(pos, q, beta, box, mcut: float | None = None) -> dict:
    """Brute-force Ewald reciprocal sum: {'energy', 'virial', 'forces'}."""
    pos = _d(pos).reshape(-1, 3)
    q = _d(q).reshape(-1)
    box = _d(box).reshape(9)
    mcut = ewald_mcut(beta) if mcut is None else mcut
    e = ctypes.c_double()
    vir = np.zeros(6)
    F = np.zeros_like(pos)
    if _load().oracle_ewald_recip(pos.shape[0], _p(pos), _p(q), float(beta), _p(box), float(mcut), ctypes.byref(e),
                                  _p(vir), _p(F)) != 0:
        raise ValueError("singular box")
    return {"energy": e.value, "virial": vir, "forces": F}


def ewald_real(pos, q, beta, box, rcut: float | None = None) -> dict:
    """Real-space Ewald sum over images within rcut (default beta * rcut = 6): {'energy', 'forces', 'virial'}."""
    pos = _d(pos).reshape(-1, 3)
    q = _d(q).reshape(-1)
    box = _d(box).reshape(9)
    rcut = 6.0 / beta if rcut is None else rcut
    e = ctypes.c_double()
    F = np.zeros_like(pos)
    vir = np.zeros(6)
    if _load().oracle_ewald_real(pos.shape[0], _p(pos), _p(q), float(beta), _p(box), float(rcut), ctypes.byref(e),
                                 _p(F), _p(vir)) != 0:
        raise ValueError("singular box")
    return {"energy": e.value, "forces": F, "virial": vir}


def ewald_real_rows(pos, q, beta, box, rows, rcut: float | None = None) -> dict:
    """Real-space sum for the listed atoms only: {'e' (per row: sum_j q_i q_j erfc/r), 'forces' (rows, 3)}."""
    pos = _d(pos).reshape(-1, 3)
    q = _d(q).reshape(-1)
    box = _d(box).reshape(9)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    rcut = 6.0 / beta if rcut is None else rcut
    e = np.zeros(len(rows))
    F = np.zeros((len(rows), 3))
    if _load().oracle_ewald_real_rows(pos.shape[0], _p(pos), _p(q), float(beta), _p(box), float(rcut), len(rows),
                                      rows.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _p(e), _p(F)) != 0:
        raise ValueError("singular box")
    return {"e": e, "forces": F}


def ewald_self(q, beta) -> float:
    """-(beta/sqrt(pi)) sum q^2."""
    q = _d(q).reshape(-1)
    return _load().oracle_ewald_self(q.shape[0], _p(q), float(beta))
