"""Shared test helpers: error metrics, the CPU emulation build of the stage bodies, GPU fixtures."""
import ctypes
import os
import subprocess

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
EMU_SRC = os.path.join(ROOT, "tests", "emu", "emu_driver.cpp")
EMU_LIB = os.path.join(ROOT, "tests", "emu", "_build", "libpme_emu.so")

# Tolerances against the FP64 oracle at the same K, p, beta (FP32 arithmetic on the GPU path):
E_REL_TOL = 1e-6        # |E - E_oracle| / |E_oracle|
F_RMS_TOL = 1e-5        # RMS |F - F_oracle| / RMS |F_oracle|
V_TOL = 1e-5            # max |Pi - Pi_oracle| / max |Pi_oracle|
# Charge mesh: each contribution q theta1 theta2 theta3 carries a few FP32 roundings (relative 2^-24 each),
# so the pointwise bound is |Q - Q_oracle|(k) <= Q_TOL * Qabs(k), Qabs = the mesh spread from |q| (about
# 16 units of 2^-24). A bound relative to max |Q| would fail wherever opposite charges cancel.
Q_TOL = 1e-6
PHI_TOL = 1e-5          # max |phi - phi_oracle| / max |phi_oracle|


def rel_energy(e, e_ref):
    return abs(e - e_ref) / abs(e_ref)


def rms_force(F, F_ref):
    F = np.asarray(F, dtype=np.float64)
    return float(np.sqrt(np.mean((F - F_ref) ** 2) / np.mean(F_ref ** 2)))


def rel_virial(v, v_ref):
    return float(np.max(np.abs(np.asarray(v) - v_ref)) / np.max(np.abs(v_ref)))


def build_emu(force=False):
    srcs = [EMU_SRC] + [os.path.join(ROOT, "paper_2009_12617_gb300", "csrc", f)
                        for f in ("common.cuh", "fft.cuh", "stages.cuh", "host_tables.h")]
    if force or not os.path.exists(EMU_LIB) or any(os.path.getmtime(s) > os.path.getmtime(EMU_LIB) for s in srcs):
        os.makedirs(os.path.dirname(EMU_LIB), exist_ok=True)
        tmp = EMU_LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-DPME_HOST_EMULATION",
                               "-ffp-contract=off", "-I/usr/local/cuda/include", "-x", "c++", EMU_SRC, "-o", tmp])
        os.replace(tmp, EMU_LIB)
    lib = ctypes.CDLL(EMU_LIB)
    dp, fp = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_float)
    lib.emu_spme.argtypes = [ctypes.c_int64, fp, fp, ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_double, dp,
                             ctypes.c_int, ctypes.c_int, fp, dp, ctypes.POINTER(ctypes.c_longlong), fp, ctypes.c_int]
    lib.emu_spme.restype = ctypes.c_int
    return lib


def emu_spme(lib, pos, q, K, p, beta, box, cap=0, repeat=1, tile_log=0):
    """Run the emulated pipeline; returns (status, forces, ev[7], mesh int64, phi float32)."""
    pos = np.ascontiguousarray(pos, np.float32)
    q = np.ascontiguousarray(q, np.float32)
    n = len(q)
    F = np.zeros((n, 3), np.float32)
    ev = np.zeros(7)
    g = np.zeros(tuple(K), np.int64)
    phi = np.zeros(tuple(K), np.float32)
    bx = np.ascontiguousarray(box, np.float64).reshape(9)
    dp, fp = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_float)
    st = lib.emu_spme(n, pos.ctypes.data_as(fp), q.ctypes.data_as(fp), (ctypes.c_int * 3)(*K), p, beta,
                      bx.ctypes.data_as(dp), cap, repeat, F.ctypes.data_as(fp), ev.ctypes.data_as(dp),
                      g.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)), phi.ctypes.data_as(fp), tile_log)
    return st, F, ev, g, phi


def mesh_error_ok(mesh_fixed, Q_ref, Qabs_ref, tol=Q_TOL):
    """Pointwise check of the fixed-point mesh (int64, scale 2^40) against the oracle's Q."""
    err = np.abs(np.asarray(mesh_fixed, dtype=np.float64) * 2.0 ** -40 - Q_ref)
    # plus the fixed-point quantum: each contribution is rounded to a multiple of 2^-40
    bound = tol * Qabs_ref + 256 * 2.0 ** -40
    return bool(np.all(err <= bound)), float((err / bound).max())
