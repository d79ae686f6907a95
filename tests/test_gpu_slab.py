"""Slab decomposition on the GPU (pme_slab_*): P ranks of one system run on one GPU one after another (no
kernel waits on another rank; the all-to-alls are block transpositions of device buffers), and the summed
forces, energy and virial must equal the undivided evaluation within FP32 rounding and the FP64 oracle
within the parity tolerances."""
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


def run_slabs(pme, s, P, reps=2):
    dev = torch.device("cuda:0")
    pos = torch.from_numpy(s.pos).to(dev)
    q = torch.from_numpy(s.q).to(dev)
    slabs = [pme.pme_slab_create(s.K, s.p, s.beta, s.box, P, r) for r in range(P)]
    try:
        lay = [pme.pme_slab_layout(h) for h in slabs]
        B = lay[0]["block_values"]
        for _ in range(reps):  # a second evaluation checks that every counter and mesh plane was reset
            sends = [torch.zeros(P * B * 2, dtype=torch.float32, device=dev) for _ in range(P)]
            for r, h in enumerate(slabs):
                pme.pme_slab_stage1(h, pos, q, sends[r])
            recvs = [torch.cat([sends[r].view(P, 2 * B)[t] for r in range(P)]) for t in range(P)]
            evs = [torch.zeros(7, dtype=torch.float64, device=dev) for _ in range(P)]
            sends2 = [torch.zeros_like(x) for x in sends]
            for r, h in enumerate(slabs):
                pme.pme_slab_stage2(h, recvs[r], sends2[r], evs[r])
            recvs2 = [torch.cat([sends2[r].view(P, 2 * B)[t] for r in range(P)]) for t in range(P)]
            Fs = [torch.full_like(pos, float("nan")) for _ in range(P)]
            for r, h in enumerate(slabs):
                pme.pme_slab_stage3(h, recvs2[r], pos, q, Fs[r])
            for h in slabs:
                pme.pme_slab_sync(h)
            F = sum(f.double() for f in Fs).cpu().numpy()
            ev = sum(evs).cpu().numpy()
        return F, ev, lay
    finally:
        for h in slabs:
            pme.pme_slab_destroy(h)


CASES = [("parity", 2), ("parity", 3), ("p6", 4), ("headline", 2), ("headline", 4)]


@pytest.mark.parametrize("name,P", CASES, ids=[f"{n}_P{P}" for n, P in CASES])
def test_slab_ranks_match_undivided_and_oracle(pme, oracle_mod, name, P):
    if name == "parity":
        s = wl.parity_system()
    elif name == "p6":
        b = wl.parity_system()
        s = wl.System(b.pos, b.q, b.box, (32, 40, 48), 6, 0.34)
    else:
        s = wl.headline_system()
    F, ev, lay = run_slabs(pme, s, P)
    assert lay[0]["planes"][0] == 0 and lay[-1]["planes"][1] == s.K[0]
    dev = torch.device("cuda:0")
    pos = torch.from_numpy(s.pos).to(dev)
    q = torch.from_numpy(s.q).to(dev)
    plan = pme.pme_create(s.K, s.p, s.beta, s.box)
    try:
        F1 = torch.empty_like(pos)
        E1, V1 = pme.pme_compute(plan, pos, q, F1)
    finally:
        pme.pme_destroy(plan)
    assert rel_energy(ev[0], E1) < 1e-6 and rms_force(F, F1.cpu().numpy().astype(np.float64)) < 1e-6
    assert rel_virial(ev[1:], V1) < 1e-6
    oracle_mod.set_threads(16)
    try:
        r = oracle_mod.spme(s.pos.astype(np.float64), s.q.astype(np.float64), s.K, s.p, s.beta, s.box)
    finally:
        oracle_mod.set_threads(1)
    assert rel_energy(ev[0], r["energy"]) < E_REL_TOL
    assert rms_force(F, r["forces"]) < F_RMS_TOL
    assert rel_virial(ev[1:], r["virial"]) < V_TOL
