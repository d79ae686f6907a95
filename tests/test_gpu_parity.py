"""GPU parity: the CUDA pipeline, called through the C ABI, against the FP64 oracle on the same seeded inputs.

Tolerances (tests/helpers.py): relative energy 1e-6, RMS force 1e-5 of RMS force, virial 1e-5 of max |Pi|,
charge mesh pointwise within 1e-6 of the |q| mesh plus the 2^-40 quantum, phi 1e-5 of max |phi|; the
fixed-point mesh bit-exact run to run and under any permutation of the atoms.
"""
import numpy as np
import pytest

from paper_2009_12617_gb300 import workloads as wl

from helpers import (E_REL_TOL, F_RMS_TOL, PHI_TOL, V_TOL, mesh_error_ok, rel_energy, rel_virial, rms_force)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pmelib():
    from paper_2009_12617_gb300 import build, pme

    build.build_library()
    pme.load_library()
    assert torch.cuda.is_available()
    return pme


def gpu_eval(pme, plan, pos, q, K=None, taps=False):
    dev = torch.device("cuda:0")
    pos_d = torch.from_numpy(np.ascontiguousarray(pos, np.float32)).to(dev)
    q_d = torch.from_numpy(np.ascontiguousarray(q, np.float32)).to(dev)
    F = torch.full_like(pos_d, float("nan"))
    mesh = torch.zeros(tuple(K), dtype=torch.int64, device=dev) if taps else None
    phi = torch.zeros(tuple(K), dtype=torch.float32, device=dev) if taps else None
    E, vir = pme.pme_compute_debug(plan, pos_d, q_d, F, mesh, phi)
    out = {"energy": E, "virial": vir, "forces": F.cpu().numpy()}
    if taps:
        out["mesh"] = mesh.cpu().numpy()
        out["phi"] = phi.cpu().numpy()
    return out


def check_against_oracle(oracle_mod, g, pos, q, K, p, beta, box, taps=True):
    r = oracle_mod.spme(np.asarray(pos, np.float64), np.asarray(q, np.float64), K, p, beta, box, want_mesh=taps)
    assert rel_energy(g["energy"], r["energy"]) < E_REL_TOL, (g["energy"], r["energy"])
    assert rms_force(g["forces"], r["forces"]) < F_RMS_TOL
    assert rel_virial(g["virial"], r["virial"]) < V_TOL
    if taps:
        Qabs = oracle_mod.spread(np.asarray(pos, np.float64), np.abs(np.asarray(q, np.float64)), K, p, box)
        ok, worst = mesh_error_ok(g["mesh"], r["Q"], Qabs)
        assert ok, worst
        assert np.abs(g["phi"] - r["phi"]).max() < PHI_TOL * np.abs(r["phi"]).max()
    return r


def test_parity_config1(pmelib, oracle_mod):
    """2048 atoms (682 water-like triplets + one ion pair), 27.4 A cubic box, 32^3, p = 4, beta = 0.34."""
    s = wl.parity_system()
    plan = pmelib.pme_create(s.K, s.p, s.beta, s.box)
    try:
        g = gpu_eval(pmelib, plan, s.pos, s.q, s.K, taps=True)
        check_against_oracle(oracle_mod, g, s.pos, s.q, s.K, s.p, s.beta, s.box)
    finally:
        pmelib.pme_destroy(plan)


SHAPES = [((8, 10, 12), 4), ((16, 18, 20), 6), ((24, 30, 32), 8), ((36, 40, 48), 4), ((50, 54, 60), 6),
          ((64, 72, 80), 4), ((90, 96, 100), 4), ((108, 120, 128), 6), ((40, 40, 40), 8), ((8, 8, 8), 8),
          ((96, 80, 128), 6), ((128, 128, 128), 4), ((30, 32, 36), 5), ((64, 64, 64), 5), ((50, 48, 54), 5)]


@pytest.mark.parametrize("K,p", SHAPES, ids=[f"{K[0]}x{K[1]}x{K[2]}_p{p}" for K, p in SHAPES])
def test_parity_mesh_shapes(pmelib, oracle_mod, K, p):
    """Every radix-2/3/5 length from 8 to 128 in some dimension, ragged tiles, orders 4, 5, 6 and 8 (odd p: the
    m = K/2 modulus reading); register (lane-plan) and shared-memory transform paths, specialised and general
    kernels."""
    L = np.array(K, dtype=float) * 1.1
    box = np.diag(L)
    n = 3000
    rng = np.random.default_rng(sum(K) + p)
    pos = (rng.random((n, 3)) * L).astype(np.float32)
    q = rng.normal(size=n)
    q -= q.mean()
    q = q.astype(np.float32)
    plan = pmelib.pme_create(K, p, 0.34, box)
    try:
        g = gpu_eval(pmelib, plan, pos, q, K, taps=True)
        check_against_oracle(oracle_mod, g, pos, q, K, p, 0.34, box)
    finally:
        pmelib.pme_destroy(plan)


def test_parity_triclinic(pmelib, oracle_mod):
    s = wl.parity_system()
    box = np.array([[27.4, 0, 0], [3.1, 26.0, 0], [-2.0, 4.0, 28.0]])
    plan = pmelib.pme_create((30, 32, 36), 6, 0.34, box)
    try:
        g = gpu_eval(pmelib, plan, s.pos, s.q, (30, 32, 36), taps=True)
        check_against_oracle(oracle_mod, g, s.pos, s.q, (30, 32, 36), 6, 0.34, box)
    finally:
        pmelib.pme_destroy(plan)


def test_parity_full_size_headline(pmelib, oracle_mod):
    """65536 atoms, 86.9 A, 64^3, p = 4 (the paper-sized system), every output against the oracle."""
    s = wl.headline_system()
    plan = pmelib.pme_create(s.K, s.p, s.beta, s.box)
    try:
        g = gpu_eval(pmelib, plan, s.pos, s.q, s.K, taps=True)
        check_against_oracle(oracle_mod, g, s.pos, s.q, s.K, s.p, s.beta, s.box)
    finally:
        pmelib.pme_destroy(plan)


def test_parity_full_size_large(pmelib, oracle_mod):
    """262144 atoms, 137.9 A, 128^3, p = 6: energy, virial, all forces and both meshes."""
    s = wl.large_system()
    plan = pmelib.pme_create(s.K, s.p, s.beta, s.box)
    try:
        g = gpu_eval(pmelib, plan, s.pos, s.q, s.K, taps=True)
        check_against_oracle(oracle_mod, g, s.pos, s.q, s.K, s.p, s.beta, s.box)
    finally:
        pmelib.pme_destroy(plan)


SPLIT_CASES = [("parity", (1, 2)), ("headline", (1, 2, 4)), ("large", (1, 2))]


@pytest.mark.parametrize("name,splits", SPLIT_CASES, ids=[c[0] for c in SPLIT_CASES])
def test_slab_split_bit_identical(pmelib, name, splits):
    """The slab stages split over clusters of 2 or 4 CTAs (distributed shared memory) give the one-CTA
    results bit for bit: forces, energy, virial and the potential mesh (32^3, 64^3 p=4, 128^3 p=6); a
    forward / inverse mix too."""
    s = {"parity": wl.parity_system, "headline": wl.headline_system, "large": wl.large_system}[name]()
    out = []
    try:
        for cs in splits:
            pmelib.pme_set_slab_split(cs)
            plan = pmelib.pme_create(s.K, s.p, s.beta, s.box)
            try:
                out.append(gpu_eval(pmelib, plan, s.pos, s.q, s.K, taps=True))
            finally:
                pmelib.pme_destroy(plan)
    finally:
        pmelib.pme_set_slab_split(1)
    for o in out[1:]:
        assert o["energy"] == out[0]["energy"]
        assert np.array_equal(o["virial"], out[0]["virial"])
        assert np.array_equal(o["forces"], out[0]["forces"])
        assert np.array_equal(o["phi"], out[0]["phi"])
        assert np.array_equal(o["mesh"], out[0]["mesh"])
    pmelib.pme_set_slab_split(2, 1)
    try:
        plan = pmelib.pme_create(s.K, s.p, s.beta, s.box)
        try:
            o = gpu_eval(pmelib, plan, s.pos, s.q, s.K)
        finally:
            pmelib.pme_destroy(plan)
    finally:
        pmelib.pme_set_slab_split(1)
    assert o["energy"] == out[0]["energy"] and np.array_equal(o["forces"], out[0]["forces"])
    with pytest.raises(Exception):
        pmelib.pme_set_slab_split(3)


def test_mesh_bit_exact_repeat_and_permutation(pmelib):
    """The int64 charge mesh is bit-identical over repeated runs and any input order; so is everything
    downstream (no floating-point atomics anywhere)."""
    s = wl.headline_system()
    plan = pmelib.pme_create(s.K, s.p, s.beta, s.box)
    try:
        g0 = gpu_eval(pmelib, plan, s.pos, s.q, s.K, taps=True)
        for _ in range(3):
            g = gpu_eval(pmelib, plan, s.pos, s.q, s.K, taps=True)
            assert np.array_equal(g["mesh"], g0["mesh"])
            assert g["energy"] == g0["energy"] and np.array_equal(g["virial"], g0["virial"])
            assert np.array_equal(g["forces"], g0["forces"])
        perm = np.random.default_rng(9).permutation(s.n)
        gp = gpu_eval(pmelib, plan, s.pos[perm], s.q[perm], s.K, taps=True)
        assert np.array_equal(gp["mesh"], g0["mesh"])
        assert gp["energy"] == g0["energy"]
        assert np.array_equal(gp["forces"], g0["forces"][perm])
    finally:
        pmelib.pme_destroy(plan)


def test_empty_single_and_wrapped(pmelib, oracle_mod):
    box = np.diag([20.0, 21.0, 22.0])
    plan = pmelib.pme_create((20, 24, 24), 4, 0.34, box)
    try:
        g = gpu_eval(pmelib, plan, np.zeros((0, 3), np.float32), np.zeros(0, np.float32))
        assert g["energy"] == 0.0 and np.all(g["virial"] == 0.0)
        one = np.array([[3.3, 4.4, 5.5]], np.float32)
        g = gpu_eval(pmelib, plan, one, np.array([1.0], np.float32))
        r = oracle_mod.spme(one.astype(float), [1.0], (20, 24, 24), 4, 0.34, box)
        assert rel_energy(g["energy"], r["energy"]) < E_REL_TOL
        # positions far outside the cell are wrapped (images of the parity system)
        s = wl.parity_system()
        shift = np.array([3 * 20.0, -5 * 21.0, 40 * 22.0], np.float32)
        far = (s.pos[:500] + shift).astype(np.float32)  # the same FP32 inputs go to both sides
        g = gpu_eval(pmelib, plan, far, s.q[:500])
        r = oracle_mod.spme(far.astype(float), s.q[:500].astype(float), (20, 24, 24), 4, 0.34, box)
        assert rel_energy(g["energy"], r["energy"]) < E_REL_TOL
        assert rms_force(g["forces"], r["forces"]) < F_RMS_TOL
    finally:
        pmelib.pme_destroy(plan)


def test_clustered_atoms_use_overflow_path(pmelib, oracle_mod):
    """Every atom inside one spread tile: the tile's bucket overflows and the global-memory paths run."""
    rng = np.random.default_rng(21)
    box = np.diag([30.0, 30.0, 30.0])
    pos = (10.0 + rng.random((4000, 3)) * 1.5).astype(np.float32)
    q = rng.normal(size=4000)
    q -= q.mean()
    q = q.astype(np.float32)
    plan = pmelib.pme_create((32, 32, 32), 4, 0.34, box)
    try:
        g = gpu_eval(pmelib, plan, pos, q, (32, 32, 32), taps=True)
        check_against_oracle(oracle_mod, g, pos, q, (32, 32, 32), 4, 0.34, box)
    finally:
        pmelib.pme_destroy(plan)


def test_host_pointer_path(pmelib, oracle_mod):
    s = wl.parity_system()
    plan = pmelib.pme_create(s.K, s.p, s.beta, s.box)
    try:
        F, E, vir = pmelib.pme_compute_host(plan, s.pos, s.q)
        r = oracle_mod.spme(s.pos.astype(float), s.q.astype(float), s.K, s.p, s.beta, s.box)
        assert rel_energy(E, r["energy"]) < E_REL_TOL
        assert rms_force(F, r["forces"]) < F_RMS_TOL
        assert rel_virial(vir, r["virial"]) < V_TOL
    finally:
        pmelib.pme_destroy(plan)


def test_host_pointer_path_pinned_graph(pmelib):
    """Page-locked host arrays take the recorded-graph path: its results equal the pageable path's bit for
    bit, new positions in the same arrays are picked up on replay, and a box change re-records the graph."""
    torch = pytest.importorskip("torch")
    s = wl.parity_system()
    n = s.n
    pos_t = torch.empty((n, 3), dtype=torch.float32).pin_memory()
    q_t = torch.empty(n, dtype=torch.float32).pin_memory()
    f_t = torch.empty((n, 3), dtype=torch.float32).pin_memory()
    P, Q, F = pos_t.numpy(), q_t.numpy(), f_t.numpy()
    Q[:] = s.q
    plan = pmelib.pme_create(s.K, s.p, s.beta, s.box)
    try:
        L = float(s.box[0, 0])
        frames = [s.pos.astype(np.float32)]
        for step in range(2):
            frames.append(wl.jitter(frames[-1], L, 7, step).astype(np.float32))
        for box_scale in (1.0, 1.02):
            if box_scale != 1.0:
                pmelib.pme_set_box(plan, s.box * box_scale)
            for fr in frames:
                P[:] = fr
                _, E1, v1 = pmelib.pme_compute_host(plan, P, Q, F)
                F1 = F.copy()
                F2, E2, v2 = pmelib.pme_compute_host(plan, fr.copy(), s.q.copy())  # pageable: plain path
                assert E1 == E2
                assert np.array_equal(F1, F2)
                assert np.array_equal(v1, v2)
    finally:
        pmelib.pme_destroy(plan)


def test_compute_repeated_calls(pmelib):
    """Repeated synchronous calls with the same device arrays are replayed from a recorded graph: results
    equal a fresh plan's bit for bit, new values in the same arrays are picked up, and a box change and a
    launch-mode change are honoured."""
    torch = pytest.importorskip("torch")
    s = wl.parity_system()
    dev = torch.device("cuda", 0)
    L = float(s.box[0, 0])
    frames = [s.pos.astype(np.float32)]
    for step in range(3):
        frames.append(wl.jitter(frames[-1], L, 11, step).astype(np.float32))
    pos = torch.from_numpy(frames[0]).to(dev)
    q = torch.from_numpy(s.q.astype(np.float32)).to(dev)
    F = torch.empty_like(pos)
    plan = pmelib.pme_create(s.K, s.p, s.beta, s.box)
    try:
        for box_scale, mode in ((1.0, 2), (1.03, 2), (1.03, 0)):
            if box_scale != 1.0:
                pmelib.pme_set_box(plan, s.box * box_scale)
            pmelib.pme_set_launch_mode(mode)
            for fr in frames:
                pos.copy_(torch.from_numpy(fr))
                for _ in range(3):  # eager, recorded, replayed
                    E, v = pmelib.pme_compute(plan, pos, q, F)
                    fresh = pmelib.pme_create(s.K, s.p, s.beta, s.box * box_scale)
                    try:
                        F2 = torch.empty_like(pos)
                        E2, v2 = pmelib.pme_compute(fresh, pos, q, F2)
                    finally:
                        pmelib.pme_destroy(fresh)
                    assert E == E2
                    assert np.array_equal(v, v2)
                    assert torch.equal(F, F2)
    finally:
        pmelib.pme_set_launch_mode(2)
        pmelib.pme_destroy(plan)


def test_enqueue_in_cuda_graph(pmelib):
    """pme_enqueue allocates nothing after pme_reserve, so a torch CUDA graph can capture it; replays give
    the synchronous result bit for bit."""
    s = wl.parity_system()
    stream = torch.cuda.Stream()
    plan = pmelib.pme_create(s.K, s.p, s.beta, s.box, stream=stream)
    try:
        pos = torch.from_numpy(s.pos).cuda()
        q = torch.from_numpy(s.q).cuda()
        F_ref = torch.empty_like(pos)
        with torch.cuda.stream(stream):
            E_ref, vir_ref = pmelib.pme_compute(plan, pos, q, F_ref)
            pmelib.pme_reserve(plan, s.n)
            F = torch.empty_like(pos)
            ev = torch.zeros(7, dtype=torch.float64, device="cuda")
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=stream):
                pmelib.pme_enqueue(plan, pos, q, F, ev)
            for _ in range(3):
                graph.replay()
            pmelib.pme_sync(plan)
        assert torch.equal(F, F_ref)
        assert ev[0].item() == E_ref and np.array_equal(ev[1:].cpu().numpy(), vir_ref)
    finally:
        pmelib.pme_destroy(plan)


def test_set_box(pmelib, oracle_mod):
    s = wl.parity_system()
    plan = pmelib.pme_create(s.K, s.p, s.beta, s.box)
    try:
        box2 = s.box * 1.03
        pmelib.pme_set_box(plan, box2)
        g = gpu_eval(pmelib, plan, s.pos, s.q)
        r = oracle_mod.spme(s.pos.astype(float), s.q.astype(float), s.K, s.p, s.beta, box2)
        assert rel_energy(g["energy"], r["energy"]) < E_REL_TOL
        assert rms_force(g["forces"], r["forces"]) < F_RMS_TOL
    finally:
        pmelib.pme_destroy(plan)


def test_invalid_inputs_report_and_recover(pmelib, oracle_mod):
    s = wl.parity_system()
    plan = pmelib.pme_create(s.K, s.p, s.beta, s.box)
    try:
        pos = s.pos.copy()
        pos[7, 2] = np.inf
        with pytest.raises(pmelib.PMEError) as ei:
            gpu_eval(pmelib, plan, pos, s.q)
        assert ei.value.status == pmelib.PME_EINVAL
        q = np.full(s.n, 3000.0, np.float32)  # sum |q| = 6.1e6 e >= 2^22
        with pytest.raises(pmelib.PMEError) as ei:
            gpu_eval(pmelib, plan, s.pos, q)
        assert ei.value.status == pmelib.PME_EOVERFLOW
        # the plan is still usable and exact afterwards
        g = gpu_eval(pmelib, plan, s.pos, s.q)
        r = oracle_mod.spme(s.pos.astype(float), s.q.astype(float), s.K, s.p, s.beta, s.box)
        assert rel_energy(g["energy"], r["energy"]) < E_REL_TOL
    finally:
        pmelib.pme_destroy(plan)


def test_headline_trajectory_every_100th_frame(pmelib, oracle_mod):
    """The paper-sized system over 1000 successive frames, each jittered by N(0, 0.01 A) from the one before
    (cumulative, wrapped): every frame is evaluated on device arrays through the synchronous entry point
    (its recorded-graph replay after the first two calls), and frames 0, 100, ..., 900 are compared with the
    FP64 oracle on the same FP32 positions at the energy, force and virial tolerances."""
    s = wl.headline_system()
    L = float(s.box[0, 0])
    dev = torch.device("cuda:0")
    pos = torch.from_numpy(s.pos).to(dev)
    q = torch.from_numpy(s.q).to(dev)
    F = torch.empty_like(pos)
    plan = pmelib.pme_create(s.K, s.p, s.beta, s.box)
    try:
        cur = s.pos
        for f in range(1000):
            pos.copy_(torch.from_numpy(cur))
            E, V = pmelib.pme_compute(plan, pos, q, F)
            if f % 100 == 0:
                r = oracle_mod.spme(cur.astype(np.float64), s.q.astype(np.float64), s.K, s.p, s.beta, s.box)
                assert rel_energy(E, r["energy"]) < E_REL_TOL, (f, E, r["energy"])
                assert rms_force(F.cpu().numpy(), r["forces"]) < F_RMS_TOL, f
                assert rel_virial(V, r["virial"]) < V_TOL, f
            cur = wl.jitter(cur, L, 77, f)
    finally:
        pmelib.pme_destroy(plan)


def test_enqueue_host_double_buffered(pmelib):
    """pme_enqueue_host on two sets of page-locked arrays kept in flight alternately: every frame's forces,
    energy, virial and status equal the synchronous host-array call's bit for bit; pageable arrays are
    refused."""
    s = wl.parity_system()
    n = s.n
    L = float(s.box[0, 0])
    frames = [s.pos.astype(np.float32)]
    for step in range(9):
        frames.append(wl.jitter(frames[-1], L, 19, step).astype(np.float32))
    bufs = []
    for _ in range(2):
        P = torch.empty((n, 3), dtype=torch.float32).pin_memory().numpy()
        Q = torch.empty(n, dtype=torch.float32).pin_memory().numpy()
        F = torch.empty((n, 3), dtype=torch.float32).pin_memory().numpy()
        R = torch.empty(8, dtype=torch.float64).pin_memory().numpy()
        Q[:] = s.q
        bufs.append((P, Q, F, R))
    stream = torch.cuda.Stream()
    plan = pmelib.pme_create(s.K, s.p, s.beta, s.box, stream=stream)
    ref = pmelib.pme_create(s.K, s.p, s.beta, s.box)
    try:
        tickets = [None, None]
        got = [None] * len(frames)
        for i, fr in enumerate(frames + [None, None]):
            slot = i % 2
            if tickets[slot] is not None:  # the evaluation of frame i - 2: wait for its ticket, read it
                pmelib.pme_host_wait(plan, tickets[slot])
                P, Q, F, R = bufs[slot]
                got[i - 2] = (F.copy(), R.copy())
                tickets[slot] = None
            if fr is None:
                continue
            P, Q, F, R = bufs[slot]
            P[:] = fr
            R[:] = np.nan
            F[:] = np.nan
            tickets[slot] = pmelib.pme_enqueue_host(plan, P, Q, F, R)
            assert tickets[slot] == i
        pmelib.pme_sync(plan)
        with pytest.raises(pmelib.PMEError):
            pmelib.pme_host_wait(plan, len(frames))  # not issued
        for i, fr in enumerate(frames):
            F2, E2, V2 = pmelib.pme_compute_host(ref, fr.copy(), s.q.copy())
            F, R = got[i]
            assert R[7] == 0.0 and R[0] == E2 and np.array_equal(R[1:7], V2) and np.array_equal(F, F2), i
        with pytest.raises(pmelib.PMEError) as ei:
            pmelib.pme_enqueue_host(plan, frames[0].copy(), s.q.copy(), np.empty((n, 3), np.float32), np.zeros(8))
        assert ei.value.status == pmelib.PME_EINVAL
    finally:
        pmelib.pme_destroy(ref)
        pmelib.pme_destroy(plan)
