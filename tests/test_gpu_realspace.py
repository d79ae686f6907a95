"""GPU real-space and self terms against the FP64 oracle, through the C ABI.

Real-space energy, forces and virial at the same tolerances as the reciprocal part (relative energy 1e-6,
RMS force 1e-5 of RMS force, virial 1e-5 of max |Pi|); the self term to FP64 rounding; the full Ewald sum
(GPU SPME reciprocal part + GPU real space + GPU self term) reproduces the NaCl Madelung constant; at the
paper-sized system (65536 atoms) the forces of sampled atoms match the oracle's per-atom sum.
"""
import math

import numpy as np
import pytest

from paper_2009_12617_gb300 import workloads as wl

from helpers import E_REL_TOL, F_RMS_TOL, V_TOL, rel_energy, rel_virial, rms_force

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pme():
    from paper_2009_12617_gb300 import build
    from paper_2009_12617_gb300 import pme as p

    build.build_library()
    p.load_library()
    return p


def gpu_real(pme, pos, q, box, beta, rcut):
    dev = torch.device("cuda:0")
    P = torch.from_numpy(np.ascontiguousarray(pos, np.float32)).to(dev)
    Q = torch.from_numpy(np.ascontiguousarray(q, np.float32)).to(dev)
    F = torch.full_like(P, float("nan"))
    rs = pme.pme_real_create(box, beta, rcut)
    try:
        er, es, vir = pme.pme_real_compute(rs, P, Q, F)
    finally:
        pme.pme_real_destroy(rs)
    return er, es, vir, F.cpu().numpy()


TRI = np.array([[27.4, 0, 0], [3.1, 26.0, 0], [-2.0, 4.0, 28.0]])


@pytest.mark.parametrize("case", ["rc9", "rc_wide", "triclinic"])
def test_real_space_parity(pme, oracle_mod, case):
    """2048 water-like atoms: a 9 A cutoff (3 cells per axis), a cutoff of 6/beta = 17.6 A wider than half the
    cell (one cell, 27 images), and a triclinic cell."""
    s = wl.parity_system()
    box, rcut = {"rc9": (s.box, 9.0), "rc_wide": (s.box, 6.0 / 0.34), "triclinic": (TRI, 9.0)}[case]
    er, es, vir, F = gpu_real(pme, s.pos, s.q, box, 0.34, rcut)
    pos64, q64 = s.pos.astype(np.float64), s.q.astype(np.float64)
    oracle_mod.set_threads(16)
    try:
        r = oracle_mod.ewald_real(pos64, q64, 0.34, box, rcut=rcut)
    finally:
        oracle_mod.set_threads(1)
    assert rel_energy(er, r["energy"]) < E_REL_TOL, (er, r["energy"])
    assert rms_force(F, r["forces"]) < F_RMS_TOL
    assert rel_virial(vir, r["virial"]) < V_TOL
    assert es == pytest.approx(oracle_mod.ewald_self(q64, 0.34), rel=1e-13)


def test_real_space_bit_exact_repeat_wrap_and_permutation(pme, oracle_mod):
    """Repeats give the same bits; a permutation of the atoms gives the same energy and forces within FP32
    rounding of the summation order; atoms given far outside the cell (periodic images, rounded to FP32 there)
    match the oracle on the same FP32 inputs."""
    s = wl.parity_system()
    a = gpu_real(pme, s.pos, s.q, s.box, 0.34, 9.0)
    b = gpu_real(pme, s.pos, s.q, s.box, 0.34, 9.0)
    assert a[0] == b[0] and np.array_equal(a[2], b[2]) and np.array_equal(a[3], b[3])
    perm = np.random.default_rng(3).permutation(s.n)
    d = gpu_real(pme, s.pos[perm], s.q[perm], s.box, 0.34, 9.0)
    assert rel_energy(d[0], a[0]) < 1e-6
    assert rms_force(d[3][np.argsort(perm)], a[3].astype(np.float64)) < 1e-5
    shift = np.array([3 * 27.4, -5 * 27.4, 40 * 27.4])
    far = (s.pos[:600] + shift).astype(np.float32)
    c = gpu_real(pme, far, s.q[:600], s.box, 0.34, 9.0)
    r = oracle_mod.ewald_real(far.astype(np.float64), s.q[:600].astype(np.float64), 0.34, s.box, rcut=9.0)
    assert rel_energy(c[0], r["energy"]) < E_REL_TOL
    assert rms_force(c[3], r["forces"]) < F_RMS_TOL
    assert rel_virial(c[2], r["virial"]) < V_TOL


def test_empty_and_invalid(pme, oracle_mod):
    er, es, vir, _ = gpu_real(pme, np.zeros((0, 3), np.float32), np.zeros(0, np.float32), np.eye(3) * 20.0, 0.34, 9.0)
    assert er == 0.0 and es == 0.0 and np.all(vir == 0.0)
    s = wl.parity_system()
    pos = s.pos.copy()
    pos[11, 1] = np.nan
    with pytest.raises(pme.PMEError) as ei:
        gpu_real(pme, pos, s.q, s.box, 0.34, 9.0)
    assert ei.value.status == pme.PME_EINVAL
    with pytest.raises(pme.PMEError) as ei:
        pme.pme_real_create(s.box, 0.34, 200.0)  # more than four cell widths
    assert ei.value.status == pme.PME_EUNSUPPORTED


def test_full_ewald_madelung_on_gpu(pme):
    """NaCl rock salt (a = 5.64 A, 2x2x2 conventional cells, 64 ions): GPU SPME reciprocal energy + GPU real
    space + GPU self term = -M N_pairs / (a/2) with the Madelung constant M = 1.747565."""
    import os

    golden = os.path.join(os.path.dirname(__file__), "golden", "madelung_nacl.txt")
    vals = dict(ln.split() for ln in open(golden) if ln.strip() and not ln.startswith("#"))
    M, a, cells = float(vals["M"]), float(vals["a_angstrom"]), int(vals["cells"])
    pos, q, box = wl.rocksalt(a, cells)
    beta = 0.9
    dev = torch.device("cuda:0")
    P = torch.from_numpy(pos.astype(np.float32)).to(dev)
    Q = torch.from_numpy(q.astype(np.float32)).to(dev)
    F = torch.empty_like(P)
    plan = pme.pme_create((32, 32, 32), 6, beta, box)
    try:
        e_rec, _ = pme.pme_compute(plan, P, Q, F)
    finally:
        pme.pme_destroy(plan)
    er, es, _, Fr = gpu_real(pme, pos, q, box, beta, 6.0 / beta)
    tot = e_rec + er + es
    assert -tot * (a / 2) / (len(q) / 2) == pytest.approx(M, abs=1e-6)
    assert np.abs(Fr).max() < 1e-4  # the lattice is force-free by symmetry


def test_accumulate_onto_reciprocal_forces(pme):
    """pme_real_enqueue with accumulate adds the real-space forces onto the reciprocal forces written by
    pme_enqueue on the same stream; ev_dev receives E_real, E_self and the virial."""
    s = wl.parity_system()
    dev = torch.device("cuda:0")
    P = torch.from_numpy(s.pos).to(dev)
    Q = torch.from_numpy(s.q).to(dev)
    stream = torch.cuda.Stream(dev)
    plan = pme.pme_create(s.K, s.p, s.beta, s.box, stream=stream)
    rs = pme.pme_real_create(s.box, s.beta, 9.0, stream=stream)
    try:
        F_rec, F_real, F_sum = torch.empty_like(P), torch.empty_like(P), torch.empty_like(P)
        pme.pme_compute(plan, P, Q, F_rec)
        er, es, vir = pme.pme_real_compute(rs, P, Q, F_real)
        ev = torch.zeros(7, dtype=torch.float64, device=dev)
        ev8 = torch.zeros(8, dtype=torch.float64, device=dev)
        with torch.cuda.stream(stream):
            pme.pme_enqueue(plan, P, Q, F_sum, ev)
            pme.pme_real_enqueue(rs, P, Q, F_sum, accumulate=True, ev_dev=ev8)
        pme.pme_sync(plan)
        assert torch.equal(F_sum, F_rec + F_real)
        assert ev8[0].item() == er and ev8[1].item() == es and np.array_equal(ev8[2:].cpu().numpy(), vir)
    finally:
        pme.pme_real_destroy(rs)
        pme.pme_destroy(plan)


def test_real_space_full_size_sampled_atoms(pme, oracle_mod):
    """65536 atoms, 86.9 A, 9 A cutoff: the forces of 24 sampled atoms against the oracle's per-atom sum."""
    s = wl.headline_system()
    er, es, vir, F = gpu_real(pme, s.pos, s.q, s.box, 0.34, 9.0)
    rows = np.random.default_rng(5).choice(s.n, 24, replace=False)
    oracle_mod.set_threads(16)
    try:
        r = oracle_mod.ewald_real_rows(s.pos.astype(np.float64), s.q.astype(np.float64), 0.34, s.box, rows, rcut=9.0)
    finally:
        oracle_mod.set_threads(1)
    assert rms_force(F[rows], r["forces"]) < F_RMS_TOL
    assert es == pytest.approx(oracle_mod.ewald_self(s.q.astype(np.float64), 0.34), rel=1e-11)  # FP64 sum order
    assert math.isfinite(er) and np.all(np.isfinite(vir))
