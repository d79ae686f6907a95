"""The library's stage bodies, compiled for the CPU with one thread per CTA (tests/emu), against the FP64
oracle: checks the index arithmetic, FFT plumbing, influence table and reductions without a GPU. The
tolerances are the ones the GPU parity tests use."""
import ctypes

import numpy as np
import pytest

from paper_2009_12617_gb300 import workloads as wl

from helpers import (E_REL_TOL, F_RMS_TOL, PHI_TOL, V_TOL, build_emu, emu_spme, mesh_error_ok, rel_energy,
                     rel_virial, rms_force)


@pytest.fixture(scope="module")
def emu():
    return build_emu()


CASES = [
    ((32, 32, 32), 4),   # the 2048-atom parity workload
    ((20, 24, 30), 6),   # radix 5 / 3 / mixed, ragged tiles
    ((32, 40, 48), 8),
    ((10, 12, 18), 4),   # small ragged meshes (tiles of 8 with tails of 2, 4, 2)
    ((8, 8, 8), 8),      # the p - 1 halo wraps onto the same tile
    ((24, 30, 40), 5),   # odd order: unequal support halves, the m = K/2 modulus reading
    ((10, 12, 16), 5),
]


@pytest.mark.parametrize("K,p", CASES)
def test_emulated_pipeline_matches_oracle(oracle_mod, emu, K, p):
    s = wl.parity_system()
    n = 2048 if min(K) >= 20 else 300
    pos, q = s.pos[:n], s.q[:n].copy()
    q[-1] -= q.sum()  # keep the subset neutral
    st, F, ev, mesh, phi = emu_spme(emu, pos, q, K, p, 0.34, s.box)
    assert st == 0
    r = oracle_mod.spme(pos.astype(float), q.astype(float), K, p, 0.34, s.box, want_mesh=True)
    assert rel_energy(ev[0], r["energy"]) < E_REL_TOL
    assert rms_force(F, r["forces"]) < F_RMS_TOL
    assert rel_virial(ev[1:], r["virial"]) < V_TOL
    ok, worst = mesh_error_ok(mesh, r["Q"], oracle_mod.spread(pos.astype(float), np.abs(q.astype(float)), K, p, s.box))
    assert ok, worst
    assert np.abs(phi - r["phi"]).max() < PHI_TOL * np.abs(r["phi"]).max()


def test_emulated_triclinic(oracle_mod, emu):
    s = wl.parity_system()
    box = np.array([[27.4, 0, 0], [3.1, 26.0, 0], [-2.0, 4.0, 28.0]])
    st, F, ev, _, _ = emu_spme(emu, s.pos, s.q, (30, 32, 36), 6, 0.34, box)
    r = oracle_mod.spme(s.pos.astype(float), s.q.astype(float), (30, 32, 36), 6, 0.34, box)
    assert st == 0
    assert rel_energy(ev[0], r["energy"]) < E_REL_TOL
    assert rms_force(F, r["forces"]) < F_RMS_TOL
    assert rel_virial(ev[1:], r["virial"]) < V_TOL


def test_emulated_overflow_path_and_repeat(oracle_mod, emu):
    """Tiny bucket capacity sends most atoms down the overflow path: mesh, forces and energies match the
    tile path bit for bit, and repeated evaluations agree (every counter and the int64 mesh are reset by
    their consumers; status 0x100 flags a leftover)."""
    s = wl.parity_system()
    st1, F1, ev1, m1, _ = emu_spme(emu, s.pos, s.q, (32, 32, 32), 4, 0.34, s.box, cap=32, repeat=1)
    st2, F2, ev2, m2, _ = emu_spme(emu, s.pos, s.q, (32, 32, 32), 4, 0.34, s.box, cap=0, repeat=3)
    assert st1 == 0 and st2 == 0
    assert np.array_equal(m1, m2)
    # an atom's force has the same bits on the overflow path and on the tile path
    assert np.array_equal(F1, F2) and np.array_equal(ev1, ev2)
    r = oracle_mod.spme(s.pos.astype(float), s.q.astype(float), (32, 32, 32), 4, 0.34, s.box)
    for F, ev in ((F1, ev1), (F2, ev2)):
        assert rel_energy(ev[0], r["energy"]) < E_REL_TOL
        assert rms_force(F, r["forces"]) < F_RMS_TOL


def test_emulated_results_do_not_depend_on_tiling(emu):
    """8^3 and 16^3 tiles give bit-identical meshes, forces and energies (tiling only reorders exact sums)."""
    s = wl.parity_system()
    _, F8, ev8, m8, _ = emu_spme(emu, s.pos, s.q, (32, 40, 48), 6, 0.34, s.box, tile_log=3)
    _, F16, ev16, m16, _ = emu_spme(emu, s.pos, s.q, (32, 40, 48), 6, 0.34, s.box, tile_log=4)
    assert np.array_equal(m8, m16)
    assert np.array_equal(F8, F16) and np.array_equal(ev8, ev16)


@pytest.mark.parametrize("K,p,tile_log,pieces", [((32, 40, 48), 4, 3, (5, 7, 8)), ((30, 32, 36), 5, 3, (5, 6, 8)),
                                                 ((32, 40, 48), 6, 4, (3, 4))])
def test_emulated_k1_pieces_do_not_change_results(emu, oracle_mod, K, p, tile_log, pieces):
    """Cutting the k1 axis into more, thinner tile pieces (widths floor / ceil of K1 / pieces, as the
    library does to balance tiles over the SMs) gives the default tiling's mesh, forces and energies bit
    for bit; the default matches the oracle."""
    s = wl.parity_system()
    emu.emu_set_k1_pieces.argtypes = [ctypes.c_int]
    emu.emu_set_k1_pieces(0)
    _, F0, ev0, m0, _ = emu_spme(emu, s.pos, s.q, K, p, 0.34, s.box, tile_log=tile_log)
    r = oracle_mod.spme(s.pos.astype(float), s.q.astype(float), K, p, 0.34, s.box)
    assert rel_energy(ev0[0], r["energy"]) < E_REL_TOL and rms_force(F0, r["forces"]) < F_RMS_TOL
    try:
        for n in pieces:
            emu.emu_set_k1_pieces(n)
            st, F, ev, m, _ = emu_spme(emu, s.pos, s.q, K, p, 0.34, s.box, tile_log=tile_log)
            assert st == 0
            assert np.array_equal(m, m0), n
            assert np.array_equal(F, F0) and np.array_equal(ev, ev0), n
    finally:
        emu.emu_set_k1_pieces(0)


def test_emulated_mesh_permutation_invariant(emu):
    """The fixed-point mesh does not depend on the order the atoms are given in."""
    s = wl.parity_system()
    perm = np.random.default_rng(3).permutation(s.n)
    _, F1, ev1, m1, _ = emu_spme(emu, s.pos, s.q, (32, 32, 32), 4, 0.34, s.box)
    _, F2, ev2, m2, _ = emu_spme(emu, s.pos[perm], s.q[perm], (32, 32, 32), 4, 0.34, s.box)
    assert np.array_equal(m1, m2)
    assert ev1[0] == ev2[0]
    assert np.array_equal(F1[perm], F2)


def test_emulated_invalid_inputs(emu):
    s = wl.parity_system()
    pos = s.pos.copy()
    pos[5, 1] = np.nan
    st, F, _, _, _ = emu_spme(emu, pos, s.q, (32, 32, 32), 4, 0.34, s.box)
    assert st & 1 and np.isnan(F[5]).all()
    q = s.q.copy()
    q[:] = 3000.0  # sum |q| = 6.1e6 e > 2^22
    st, _, _, _, _ = emu_spme(emu, s.pos, q, (32, 32, 32), 4, 0.34, s.box)
    assert st & 2


def test_emulated_odd_order_paths_bit_identical(oracle_mod, emu):
    """p = 5 (support halves of 3 and 2 planes): the overflow path equals the tile path bit for bit, and 8^3
    and 16^3 tiles agree bit for bit; all match the oracle."""
    s = wl.parity_system()
    K = (30, 32, 36)
    _, Ft, evt, mt, _ = emu_spme(emu, s.pos, s.q, K, 5, 0.34, s.box, tile_log=3)
    _, Fo, evo, mo, _ = emu_spme(emu, s.pos, s.q, K, 5, 0.34, s.box, cap=32, tile_log=3)
    _, F16, ev16, m16, _ = emu_spme(emu, s.pos, s.q, K, 5, 0.34, s.box, tile_log=4)
    for F, ev, m in ((Fo, evo, mo), (F16, ev16, m16)):
        assert np.array_equal(m, mt) and np.array_equal(F, Ft) and np.array_equal(ev, evt)
    r = oracle_mod.spme(s.pos.astype(float), s.q.astype(float), K, 5, 0.34, s.box)
    assert rel_energy(evt[0], r["energy"]) < E_REL_TOL
    assert rms_force(Ft, r["forces"]) < F_RMS_TOL
    assert rel_virial(evt[1:], r["virial"]) < V_TOL


def test_spread_layout_banks(emu):
    """Spreading region layouts, checked from the bank rule (word w sits in bank w mod 32): with p = 4 and 8^3
    tiles one warp takes one atom, lane (jA, j2, j3) = (lane / 16, lane / 4 mod 4, lane mod 4) adding the
    points (jA, j2, j3) and (jA + 2, j2, j3) below the atom's highest support point, and at each step the 32
    lanes must hit 32 distinct banks wherever the atom lies; otherwise two threads split an atom's planes
    into halves half_planes = ceil(p / 2) planes apart, which must sit 16 banks apart. Every region fits its
    padded array, rounded to 4 ints so the record arrays after it stay 16-byte aligned."""
    import ctypes
    emu.emu_spread_layout.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    for p in (4, 5, 6, 8):
        for tlog in (3, 4):
            out = (ctypes.c_int * 4)()
            emu.emu_spread_layout(p, tlog, out)
            rs, pl, vol, warp = list(out)
            R = (1 << tlog) + p - 1
            assert rs >= R and pl >= R * rs and vol >= R * pl and vol % 4 == 0
            assert warp == (p == 4 and tlog == 3)
            if warp:
                for base in range(64):  # the atom's highest support point, any bank alignment
                    for step in (0, 2):  # planes jA and jA + 2
                        banks = {(base - ((ja + step) * pl + j2 * rs + j3)) % 32
                                 for ja in range(2) for j2 in range(4) for j3 in range(4)}
                        assert len(banks) == 32, (p, tlog, base, step)
            else:
                assert rs == R
                assert ((p + 1) // 2 * pl) % 32 == 16
