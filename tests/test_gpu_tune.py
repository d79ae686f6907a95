"""GPU tests of the autotuner: every candidate configuration gives bit-identical results, the tuner picks one
of them and persists it, batches tune their strategy, and a batch follows its plans when they change.
"""
import json

import numpy as np
import pytest

from paper_2009_12617_gb300 import workloads as wl

from helpers import E_REL_TOL, F_RMS_TOL, rel_energy, rms_force

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pme():
    from paper_2009_12617_gb300 import build
    from paper_2009_12617_gb300 import pme as p

    build.build_library()
    p.load_library()
    return p


def _dev(s):
    dev = torch.device("cuda:0")
    return torch.from_numpy(s.pos).to(dev), torch.from_numpy(s.q).to(dev)


SYSTEMS = {"headline": lambda: wl.headline_system(), "large": lambda: wl.large_system(),
           "noncubic": lambda: wl.System(*_noncubic())}


def _noncubic():
    K = (50, 54, 48)
    L = np.array(K, dtype=float) * 1.05
    pos, q = wl.water_box(8000, float(L.min()), 91)
    pos = (pos / float(L.min()) * L).astype(np.float32)
    return pos, q, np.diag(L), K, 6, 0.34


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_every_tiling_candidate_is_bit_identical(pme, oracle_mod, name):
    """Tile edges 8 and 16, CTA sizes 128 and 256 (and 512 with 16^3 tiles): energy, virial and forces equal
    the default's bit for bit; the default matches the oracle."""
    s = SYSTEMS[name]()
    P, Q = _dev(s)
    plan = pme.pme_create(s.K, s.p, s.beta, s.box)
    try:
        F0 = torch.empty_like(P)
        E0, V0 = pme.pme_compute(plan, P, Q, F0)
        for edge in (8, 16):
            for nt in ((128, 256) if edge == 8 else (128, 256, 512)):
                pme.pme_plan_set_tiling(plan, edge, nt)
                assert pme.pme_plan_get_tiling(plan) == (edge, nt)
                F = torch.full_like(P, float("nan"))
                for _ in range(2):  # eager, then recorded graph
                    E, V = pme.pme_compute(plan, P, Q, F)
                    assert E == E0 and np.array_equal(V, V0) and torch.equal(F, F0), (edge, nt)
        if name != "large":
            r = oracle_mod.spme(s.pos.astype(np.float64), s.q.astype(np.float64), s.K, s.p, s.beta, s.box)
            assert rel_energy(E0, r["energy"]) < E_REL_TOL
            assert rms_force(F0.cpu().numpy(), r["forces"]) < F_RMS_TOL
    finally:
        pme.pme_destroy(plan)


def test_autotune_picks_and_persists(pme, tmp_path):
    s = wl.headline_system()
    P, Q = _dev(s)
    cache = tmp_path / "tune.json"
    pme.pme_tune_cache(str(cache))
    try:
        plan = pme.pme_create(s.K, s.p, s.beta, s.box)
        try:
            F0 = torch.empty_like(P)
            E0, V0 = pme.pme_compute(plan, P, Q, F0)
            F = torch.empty_like(P)
            res = pme.pme_autotune(plan, P, Q, F, reps=20)
            assert res["candidates"] == 5 and res["rejected"] == 0 and res["from_cache"] == 0
            assert (res["tile_edge"], res["tile_threads"]) in ((8, 0), (16, 0), (8, 128), (8, 256), (16, 256),
                                                                (16, 512))
            assert 0 < res["us_per_eval"] <= res["default_us"]
            assert pme.pme_plan_get_tiling(plan) == (res["tile_edge"], res["tile_threads"])
            E, V = pme.pme_compute(plan, P, Q, F)
            assert E == E0 and np.array_equal(V, V0) and torch.equal(F, F0)
        finally:
            pme.pme_destroy(plan)
        entries = json.loads(cache.read_text())["entries"]
        assert len(entries) == 1 and entries[0]["K"] == list(s.K) and entries[0]["p"] == s.p
        assert entries[0]["tile_edge"] == res["tile_edge"] and entries[0]["tile_threads"] == res["tile_threads"]
        # a new process would read the file: force a reload and tune a fresh plan from the cache
        pme.pme_tune_cache(str(cache))
        plan = pme.pme_create(s.K, s.p, s.beta, s.box)
        try:
            r2 = pme.pme_autotune(plan, P, Q, F, reps=5)
            assert r2["from_cache"] == 1 and (r2["tile_edge"], r2["tile_threads"]) == (res["tile_edge"], res["tile_threads"])
            E, V = pme.pme_compute(plan, P, Q, F)
            assert E == E0 and torch.equal(F, F0)
        finally:
            pme.pme_destroy(plan)
    finally:
        pme.pme_tune_cache(None)


def test_batch_autotune_and_refresh(pme):
    """A batch of 12 uneven systems tunes its strategy and tile CTA size and still equals every system's single
    evaluation bit for bit; after a plan's tiling and another plan's cell change underneath it, the batch
    re-reads them and equals the new single-system results."""
    dev = torch.device("cuda:0")
    systems = wl.batch_systems(count=12, seed=7)
    plans = [pme.pme_create(s.K, s.p, s.beta, s.box) for s in systems]
    try:
        singles = []
        for s, pl in zip(systems, plans):
            P, Q = _dev(s)
            F = torch.empty_like(P)
            E, V = pme.pme_compute(pl, P, Q, F)
            singles.append((F.cpu().numpy(), E, V))
        ns = [s.n for s in systems]
        pos = torch.from_numpy(np.concatenate([s.pos for s in systems])).to(dev)
        q = torch.from_numpy(np.concatenate([s.q for s in systems])).to(dev)
        F = torch.empty_like(pos)
        ev = torch.zeros((len(systems), 7), dtype=torch.float64, device=dev)
        b = pme.pme_batch_create(plans, ns)
        try:
            strategy, us = pme.pme_batch_autotune(b, pos, q, F, ev, reps=5)
            assert strategy in (pme.PME_BATCH_GROUPED, pme.PME_BATCH_PERSISTENT) and us > 0
            assert pme.pme_batch_get_strategy(b) == strategy
            pme.pme_batch_enqueue(b, pos, q, F, ev)
            pme.pme_batch_sync(b)
            Fh, evh = F.cpu().numpy(), ev.cpu().numpy()
            off = 0
            for i, (Fs, Es, Vs) in enumerate(singles):
                assert evh[i, 0] == Es and np.array_equal(evh[i, 1:], Vs)
                assert np.array_equal(Fh[off:off + ns[i]], Fs)
                off += ns[i]
            # change two plans underneath the batch
            pme.pme_plan_set_tiling(plans[3], 8, 128 if pme.pme_plan_get_tiling(plans[3])[1] == 256 else 256)
            box5 = systems[5].box * 1.02
            pme.pme_set_box(plans[5], box5)
            pme.pme_batch_enqueue(b, pos, q, F, ev)
            pme.pme_batch_sync(b)
            Fh, evh = F.cpu().numpy(), ev.cpu().numpy()
            off5 = sum(ns[:5])
            fresh = pme.pme_create(systems[5].K, systems[5].p, systems[5].beta, box5)
            try:
                P5, Q5 = _dev(systems[5])
                F5 = torch.empty_like(P5)
                E5, V5 = pme.pme_compute(fresh, P5, Q5, F5)
            finally:
                pme.pme_destroy(fresh)
            assert evh[5, 0] == E5 and np.array_equal(evh[5, 1:], V5)
            assert np.array_equal(Fh[off5:off5 + ns[5]], F5.cpu().numpy())
            off3 = sum(ns[:3])
            assert evh[3, 0] == singles[3][1] and np.array_equal(Fh[off3:off3 + ns[3]], singles[3][0])
        finally:
            pme.pme_batch_destroy(b)
    finally:
        for pl in plans:
            pme.pme_destroy(pl)
