"""GPU tests of batched evaluation (grouped stage launches; the persistent work-list kernel, in normal
operation and behind the stall hook) and the serving loop.

Each system's result in a batch or a served mix must equal its result alone (pme_compute) within the
parity tolerances; the work decomposition of a system is the same in every launch, so the results are
expected to be bit-identical, which the tests also check.
"""
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


@pytest.fixture(scope="module")
def systems(pme):
    """12 uneven water-like boxes (atom counts log-uniform in [1024, 32768]; meshes 32..64), each with its
    own plan and its single-system result."""
    dev = torch.device("cuda:0")
    out = []
    for s in wl.batch_systems(count=12, seed=7):
        plan = pme.pme_create(s.K, s.p, s.beta, s.box)
        pos = torch.from_numpy(s.pos).to(dev)
        q = torch.from_numpy(s.q).to(dev)
        F = torch.empty_like(pos)
        E, V = pme.pme_compute(plan, pos, q, F)
        out.append(dict(sys=s, plan=plan, pos=pos, q=q, F=F.cpu().numpy(), E=E, V=V))
    yield out
    for o in out:
        pme.pme_destroy(o["plan"])


def packed(systems):
    pos = torch.cat([o["pos"] for o in systems])
    q = torch.cat([o["q"] for o in systems])
    return pos, q, [o["sys"].n for o in systems]


def check_same(o, F, E, V, exact):
    assert rel_energy(E, o["E"]) < E_REL_TOL
    assert rms_force(F, o["F"].astype(np.float64)) < F_RMS_TOL
    assert rel_virial(V, o["V"]) < V_TOL
    if exact:
        assert E == o["E"] and np.array_equal(V, o["V"]) and np.array_equal(F, o["F"])


def test_batch_matches_single_systems(pme, systems, oracle_mod):
    pos, q, ns = packed(systems)
    F = torch.full_like(pos, float("nan"))
    ev = torch.zeros((len(systems), 7), dtype=torch.float64, device="cuda:0")
    b = pme.pme_batch_create([o["plan"] for o in systems], ns)
    try:
        for rep in range(3):  # graph replays reuse and reset every counter
            pme.pme_batch_enqueue(b, pos, q, F, ev)
            pme.pme_batch_sync(b)
            Fh, evh = F.cpu().numpy(), ev.cpu().numpy()
            off = 0
            for i, o in enumerate(systems):
                check_same(o, Fh[off:off + ns[i]], evh[i, 0], evh[i, 1:], exact=True)
                off += ns[i]
        # and the batch agrees with the oracle on one system
        s = systems[0]["sys"]
        r = oracle_mod.spme(s.pos.astype(float), s.q.astype(float), s.K, s.p, s.beta, s.box)
        assert rel_energy(evh[0, 0], r["energy"]) < E_REL_TOL
        assert rms_force(Fh[:ns[0]], r["forces"]) < F_RMS_TOL
    finally:
        pme.pme_batch_destroy(b)


def test_batch_persistent_strategy_matches_single_systems(pme, systems, oracle_mod):
    """The persistent work-list kernel (one launch for all 12 uneven systems, entries waiting only on their
    own system's previous stage) in normal operation: every system equals its single evaluation bit for bit
    over graph replays, one system matches the oracle, and switching back to grouped launches re-records."""
    pos, q, ns = packed(systems)
    F = torch.full_like(pos, float("nan"))
    ev = torch.zeros((len(systems), 7), dtype=torch.float64, device="cuda:0")
    b = pme.pme_batch_create([o["plan"] for o in systems], ns)
    try:
        assert pme.pme_batch_get_strategy(b) == pme.PME_BATCH_GROUPED
        pme.pme_batch_set_strategy(b, pme.PME_BATCH_PERSISTENT)
        assert pme.pme_batch_get_strategy(b) == pme.PME_BATCH_PERSISTENT
        for rep in range(3):  # replays: the last CTA out resets every counter of the work list
            F.fill_(float("nan"))
            pme.pme_batch_enqueue(b, pos, q, F, ev)
            pme.pme_batch_sync(b)
            Fh, evh = F.cpu().numpy(), ev.cpu().numpy()
            off = 0
            for i, o in enumerate(systems):
                check_same(o, Fh[off:off + ns[i]], evh[i, 0], evh[i, 1:], exact=True)
                off += ns[i]
        s = systems[5]["sys"]
        r = oracle_mod.spme(s.pos.astype(float), s.q.astype(float), s.K, s.p, s.beta, s.box)
        off = sum(ns[:5])
        assert rel_energy(evh[5, 0], r["energy"]) < E_REL_TOL
        assert rms_force(Fh[off:off + ns[5]], r["forces"]) < F_RMS_TOL
        assert rel_virial(evh[5, 1:], r["virial"]) < V_TOL
        pme.pme_batch_set_strategy(b, pme.PME_BATCH_GROUPED)
        F.fill_(float("nan"))
        pme.pme_batch_enqueue(b, pos, q, F, ev)
        pme.pme_batch_sync(b)
        assert np.array_equal(F.cpu().numpy(), Fh) and np.array_equal(ev.cpu().numpy(), evh)
        with pytest.raises(pme.PMEError):
            pme.pme_batch_set_strategy(b, 7)
    finally:
        pme.pme_batch_destroy(b)


def test_batch_new_pointers_recapture(pme, systems):
    sub = systems[:4]
    pos, q, ns = packed(sub)
    b = pme.pme_batch_create([o["plan"] for o in sub], ns)
    try:
        for _ in range(2):  # fresh output buffers each time: the launch is re-recorded
            F = torch.empty_like(pos)
            ev = torch.zeros((len(sub), 7), dtype=torch.float64, device="cuda:0")
            pme.pme_batch_enqueue(b, pos, q, F, ev)
            pme.pme_batch_sync(b)
            off = 0
            for i, o in enumerate(sub):
                check_same(o, F.cpu().numpy()[off:off + ns[i]], ev[i, 0].item(), ev[i, 1:].cpu().numpy(), exact=True)
                off += ns[i]
    finally:
        pme.pme_batch_destroy(b)


def test_batch_rejects_shared_plan_and_mixed_order(pme, systems):
    p0 = systems[0]["plan"]
    with pytest.raises(pme.PMEError) as ei:
        pme.pme_batch_create([p0, p0], [10, 10])
    assert ei.value.status == pme.PME_EINVAL
    other = pme.pme_create((32, 32, 32), 6, 0.34, np.eye(3) * 30.0)
    try:
        with pytest.raises(pme.PMEError) as ei:
            pme.pme_batch_create([p0, other], [10, 10])
        assert ei.value.status == pme.PME_EINVAL
    finally:
        pme.pme_destroy(other)


def test_batch_stuck_dependency_times_out_and_recovers(pme, systems):
    """Test hook: one list entry waits on a counter nothing advances. The bounded wait gives up after 50 ms,
    the launch ends, pme_batch_sync reports PME_ETIMEOUT, and the next launch is correct again."""
    sub = systems[:3]
    pos, q, ns = packed(sub)
    F = torch.empty_like(pos)
    ev = torch.zeros((len(sub), 7), dtype=torch.float64, device="cuda:0")
    b = pme.pme_batch_create([o["plan"] for o in sub], ns)
    try:
        pme.pme_batch_debug_stall(b, True, 50_000_000)
        pme.pme_batch_enqueue(b, pos, q, F, ev)
        with pytest.raises(pme.PMEError) as ei:
            pme.pme_batch_sync(b)
        assert ei.value.status == pme.PME_ETIMEOUT
        pme.pme_batch_debug_stall(b, False)
        pme.pme_batch_enqueue(b, pos, q, F, ev)
        pme.pme_batch_sync(b)
        off = 0
        for i, o in enumerate(sub):
            check_same(o, F.cpu().numpy()[off:off + ns[i]], ev[i, 0].item(), ev[i, 1:].cpu().numpy(), exact=True)
            off += ns[i]
    finally:
        pme.pme_batch_destroy(b)


def test_server_results_same_alone_and_in_mix(pme, systems):
    """Every system submitted twice (so requests on one plan queue behind each other) into a server whose
    waves mix all systems; each result equals the system's result alone."""
    srv = pme.pme_server_create(1 << 34, 64)
    try:
        tickets = []
        for rep in range(2):
            for o in systems:
                F = torch.full_like(o["pos"], float("nan"))
                t = pme.pme_submit(srv, o["plan"], o["pos"], o["q"], F)
                assert t is not None
                tickets.append((o, F, t))
        for o, F, t in tickets:
            assert pme.pme_poll(srv, t, block=True) == pme.PME_OK
            check_same(o, F.cpu().numpy(), t.energy.value, np.array(t.virial[:]), exact=True)
        st = pme.pme_server_stats(srv)
        assert st["completed"] == len(tickets) and st["waves"] >= 2 and st["p99_us"] >= st["p50_us"] > 0
    finally:
        pme.pme_server_destroy(srv)


def test_server_admission_limits(pme, systems):
    o = systems[0]
    nbytes = pme.pme_plan_device_bytes(o["plan"])
    srv = pme.pme_server_create(nbytes - 1, 4)  # budget below one plan
    try:
        F = torch.empty_like(o["pos"])
        with pytest.raises(pme.PMEError) as ei:
            pme.pme_submit(srv, o["plan"], o["pos"], o["q"], F)
        assert ei.value.status == pme.PME_ENOMEM
    finally:
        pme.pme_server_destroy(srv)
    srv = pme.pme_server_create(nbytes, 2)  # one plan at a time, two slots
    try:
        outs = [torch.empty_like(o["pos"]) for _ in range(3)]
        t1 = pme.pme_submit(srv, o["plan"], o["pos"], o["q"], outs[0])
        t2 = pme.pme_submit(srv, o["plan"], o["pos"], o["q"], outs[1])
        assert t1 is not None and t2 is not None
        assert pme.pme_submit(srv, o["plan"], o["pos"], o["q"], outs[2]) is None  # PME_EAGAIN: slots full
        for t, F in ((t1, outs[0]), (t2, outs[1])):
            assert pme.pme_poll(srv, t, block=True) == pme.PME_OK
            check_same(o, F.cpu().numpy(), t.energy.value, np.array(t.virial[:]), exact=True)
    finally:
        pme.pme_server_destroy(srv)


def _shaped_systems(pme, specs, seed0):
    """Water-like boxes with the given (n, K, p); rectangular cells so every mesh spacing is about 1 A."""
    dev = torch.device("cuda:0")
    out = []
    for i, (n, K, p) in enumerate(specs):
        L = np.array(K, dtype=float) * 1.05
        pos, q = wl.water_box(n, float(L.min()), seed0 + i)
        pos = (pos / float(L.min()) * L).astype(np.float32)  # stretch the cubic box onto the cell
        box = np.diag(L)
        plan = pme.pme_create(K, p, 0.34, box)
        P = torch.from_numpy(pos).to(dev)
        Q = torch.from_numpy(q).to(dev)
        F = torch.empty_like(P)
        E, V = pme.pme_compute(plan, P, Q, F)
        out.append(dict(sys=wl.System(pos, q, box, K, p, 0.34), plan=plan, pos=P, q=Q, F=F.cpu().numpy(), E=E, V=V))
    return out


def test_batch_mixed_shapes_bit_identical(pme, oracle_mod):
    """Groups of equal and unequal mesh shapes, including lengths without a register plan (30, 36, 50, 54)
    and non-cubic meshes, which run the general kernels: every system equals its single evaluation bit for
    bit, repeatedly."""
    specs = [(3000, (32, 32, 32), 6), (2500, (32, 32, 32), 6), (4000, (30, 36, 40), 6), (3500, (30, 36, 40), 6),
             (5000, (50, 54, 48), 6), (2000, (24, 24, 24), 6), (6000, (40, 40, 40), 6)]
    syst = _shaped_systems(pme, specs, 300)
    try:
        pos, q, ns = packed(syst)
        F = torch.full_like(pos, float("nan"))
        ev = torch.zeros((len(syst), 7), dtype=torch.float64, device="cuda:0")
        b = pme.pme_batch_create([o["plan"] for o in syst], ns)
        try:
            for _ in range(2):
                pme.pme_batch_enqueue(b, pos, q, F, ev)
                pme.pme_batch_sync(b)
                Fh, evh = F.cpu().numpy(), ev.cpu().numpy()
                off = 0
                for i, o in enumerate(syst):
                    check_same(o, Fh[off:off + ns[i]], evh[i, 0], evh[i, 1:], exact=True)
                    off += ns[i]
        finally:
            pme.pme_batch_destroy(b)
        s = syst[4]["sys"]  # a shape on the general path, against the oracle
        r = oracle_mod.spme(s.pos.astype(float), s.q.astype(float), s.K, s.p, s.beta, s.box)
        assert rel_energy(syst[4]["E"], r["energy"]) < E_REL_TOL
        assert rms_force(syst[4]["F"], r["forces"]) < F_RMS_TOL
    finally:
        for o in syst:
            pme.pme_destroy(o["plan"])


def test_server_mixed_orders_and_shapes(pme):
    """Waves that mix B-spline orders and mesh shapes (each shape a group of its own): every result equals
    the system's single evaluation bit for bit."""
    specs = [(3000, (32, 32, 32), 4), (3000, (32, 32, 32), 6), (2500, (24, 30, 36), 8), (4000, (40, 40, 40), 4),
             (3500, (36, 36, 36), 6)]
    syst = _shaped_systems(pme, specs, 400)
    srv = pme.pme_server_create(1 << 34, 64)
    try:
        tickets = []
        for rep in range(3):
            for o in syst:
                F = torch.full_like(o["pos"], float("nan"))
                t = pme.pme_submit(srv, o["plan"], o["pos"], o["q"], F)
                assert t is not None
                tickets.append((o, F, t))
        for o, F, t in tickets:
            assert pme.pme_poll(srv, t, block=True) == pme.PME_OK
            check_same(o, F.cpu().numpy(), t.energy.value, np.array(t.virial[:]), exact=True)
    finally:
        pme.pme_server_destroy(srv)
        for o in syst:
            pme.pme_destroy(o["plan"])


def test_batch_and_server_odd_order(pme, oracle_mod):
    """p = 5 systems through grouped and persistent batches and the server: bit-identical to their single
    evaluations, which match the oracle."""
    specs = [(3000, (32, 32, 32), 5), (2500, (32, 32, 32), 5), (4000, (30, 36, 40), 5)]
    syst = _shaped_systems(pme, specs, 500)
    try:
        s = syst[2]["sys"]
        r = oracle_mod.spme(s.pos.astype(float), s.q.astype(float), s.K, s.p, s.beta, s.box)
        assert rel_energy(syst[2]["E"], r["energy"]) < E_REL_TOL
        assert rms_force(syst[2]["F"], r["forces"]) < F_RMS_TOL
        pos, q, ns = packed(syst)
        F = torch.full_like(pos, float("nan"))
        ev = torch.zeros((len(syst), 7), dtype=torch.float64, device="cuda:0")
        b = pme.pme_batch_create([o["plan"] for o in syst], ns)
        try:
            for strategy in (pme.PME_BATCH_GROUPED, pme.PME_BATCH_PERSISTENT):
                pme.pme_batch_set_strategy(b, strategy)
                pme.pme_batch_enqueue(b, pos, q, F, ev)
                pme.pme_batch_sync(b)
                Fh, evh = F.cpu().numpy(), ev.cpu().numpy()
                off = 0
                for i, o in enumerate(syst):
                    check_same(o, Fh[off:off + ns[i]], evh[i, 0], evh[i, 1:], exact=True)
                    off += ns[i]
        finally:
            pme.pme_batch_destroy(b)
        srv = pme.pme_server_create(1 << 34, 16)
        try:
            tickets = []
            for o in syst:
                Fo = torch.full_like(o["pos"], float("nan"))
                tickets.append((o, Fo, pme.pme_submit(srv, o["plan"], o["pos"], o["q"], Fo)))
            for o, Fo, t in tickets:
                assert pme.pme_poll(srv, t, block=True) == pme.PME_OK
                check_same(o, Fo.cpu().numpy(), t.energy.value, np.array(t.virial[:]), exact=True)
        finally:
            pme.pme_server_destroy(srv)
    finally:
        for o in syst:
            pme.pme_destroy(o["plan"])
