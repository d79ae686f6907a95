"""AddressSanitizer sweep of the emulated stage bodies (run by tests/test_emulation_asan.py in a child process
with libasan preloaded; not part of the library).

Every buffer the emulation hands to a stage body is a std::vector of exactly the size the library allocates on
the device, so any out-of-range index in bin, spread (tile and overflow paths), the three FFT passes, the
influence pass, the two energy-reduction levels or gather stops the process with an ASan report. The cases
cover every supported order, meshes from 8 to 128 points per dimension with ragged tiles (sizes not multiples of
the tile edge), atoms inside and far outside the cell, empty systems, tiny bucket capacities that force the
overflow path, both tile edges, and one system with every atom in a single tile.
"""
import ctypes
import os
import sys

import numpy as np


def main(lib_path):
    lib = ctypes.CDLL(lib_path)
    dp, fp = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_float)
    lib.emu_spme.argtypes = [ctypes.c_int64, fp, fp, ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_double,
                             dp, ctypes.c_int, ctypes.c_int, fp, dp, ctypes.POINTER(ctypes.c_longlong), fp,
                             ctypes.c_int]
    lib.emu_spme.restype = ctypes.c_int
    lib.emu_set_k1_pieces.argtypes = [ctypes.c_int]

    def run(pos, q, K, p, box, cap, tile_log):
        pos = np.ascontiguousarray(pos, np.float32)
        q = np.ascontiguousarray(q, np.float32)
        n = len(q)
        F = np.zeros((n, 3), np.float32)
        ev = np.zeros(7)
        g = np.zeros(tuple(K), np.int64)
        phi = np.zeros(tuple(K), np.float32)
        bx = np.ascontiguousarray(box, np.float64).reshape(9)
        st = lib.emu_spme(n, pos.ctypes.data_as(fp), q.ctypes.data_as(fp), (ctypes.c_int * 3)(*K), p, 0.34,
                          bx.ctypes.data_as(dp), cap, 2, F.ctypes.data_as(fp), ev.ctypes.data_as(dp),
                          g.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)), phi.ctypes.data_as(fp), tile_log)
        if st != 0:
            raise SystemExit(f"status {st} for K={K} p={p} n={n} cap={cap} tile_log={tile_log}")

    rng = np.random.default_rng(0)
    L = np.array([20.0, 23.0, 26.0])
    box = np.diag(L)
    cases = 0
    meshes = [(8, 8, 8), (10, 12, 18), (16, 18, 20), (24, 30, 36), (40, 48, 50), (54, 60, 64), (72, 80, 90),
              (96, 100, 108), (120, 128, 8), (128, 128, 128)]
    for K in meshes:
        for p in (4, 5, 6, 8):
            if p > min(K):
                continue
            n = int(rng.integers(0, 400))
            pos = (rng.random((n, 3)) * 3 - 1) * L  # inside the cell and up to one cell outside on each side
            q = rng.normal(size=n)
            for cap, tile_log in ((0, 0), (32, 3), (0, 4)):
                run(pos, q, K, p, box, cap, tile_log)
                cases += 1
            # the k1 axis cut into the most pieces the library may choose (widths floor / ceil of K1 / pieces)
            lib.emu_set_k1_pieces(2 * ((K[0] + 7) // 8))
            run(pos, q, K, p, box, 0, 3)
            lib.emu_set_k1_pieces(0)
            cases += 1
    # empty system and every atom in one tile (all of them on the overflow path)
    run(np.zeros((0, 3)), np.zeros(0), (32, 32, 32), 4, np.diag([20.0] * 3), 0, 0)
    pos = np.full((300, 3), 5.0) + rng.random((300, 3)) * 0.1
    run(pos, rng.normal(size=300), (32, 32, 32), 4, np.diag([20.0] * 3), 0, 0)
    # triclinic cell
    tri = np.array([[20.0, 0, 0], [4.0, 22.0, 0], [-3.0, 5.0, 24.0]])
    pos = rng.random((250, 3)) @ tri
    run(pos, rng.normal(size=250), (24, 30, 32), 6, tri, 0, 0)
    print(f"asan sweep ok: {cases + 3} cases")


if __name__ == "__main__":
    main(sys.argv[1])
