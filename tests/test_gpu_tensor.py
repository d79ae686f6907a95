"""The tensor-core influence stage (pme_set_influence_path(PME_INFLUENCE_TENSOR), K1 = 128): the k1 transforms
as split-BF16 matrix products on tcgen05. Energy, virial and forces against the FP64 oracle at the parity
tolerances, and against the FP32 path; repeat evaluations bit-identical; K1 != 128 refused."""
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


def _small():
    K = (128, 32, 40)
    L = np.array([110.0, 28.0, 35.0])
    rng = np.random.default_rng(77)
    pos = (rng.random((3000, 3)) * L).astype(np.float32)
    q = rng.normal(size=3000)
    q = (q - q.mean()).astype(np.float32)
    return wl.System(pos, q, np.diag(L), K, 4, 0.34)


@pytest.mark.parametrize("name", ["small", "large"])
def test_tensor_influence_matches_oracle(pme, oracle_mod, name):
    s = _small() if name == "small" else wl.large_system()
    dev = torch.device("cuda:0")
    P = torch.from_numpy(s.pos).to(dev)
    Q = torch.from_numpy(s.q).to(dev)
    plan = pme.pme_create(s.K, s.p, s.beta, s.box)
    try:
        F32 = torch.empty_like(P)
        E32, V32 = pme.pme_compute(plan, P, Q, F32)
        pme.pme_set_influence_path(plan, pme.PME_INFLUENCE_TENSOR)
        assert pme.pme_get_influence_path(plan) == pme.PME_INFLUENCE_TENSOR
        Ft = torch.full_like(P, float("nan"))
        Et, Vt = pme.pme_compute(plan, P, Q, Ft)
        for _ in range(2):  # recorded graph, then replay: the same bits
            F2 = torch.full_like(P, float("nan"))
            E2, V2 = pme.pme_compute(plan, P, Q, F2)
            assert E2 == Et and np.array_equal(V2, Vt) and torch.equal(F2, Ft)
        oracle_mod.set_threads(16)
        try:
            r = oracle_mod.spme(s.pos.astype(np.float64), s.q.astype(np.float64), s.K, s.p, s.beta, s.box)
        finally:
            oracle_mod.set_threads(1)
        Fh = Ft.cpu().numpy()
        assert rel_energy(Et, r["energy"]) < E_REL_TOL, (Et, r["energy"], E32)
        assert rms_force(Fh, r["forces"]) < F_RMS_TOL
        assert rel_virial(Vt, r["virial"]) < V_TOL
        assert rel_energy(Et, E32) < E_REL_TOL and rms_force(Fh, F32.cpu().numpy().astype(np.float64)) < F_RMS_TOL
        pme.pme_set_influence_path(plan, pme.PME_INFLUENCE_FP32)
        F3 = torch.empty_like(P)
        E3, V3 = pme.pme_compute(plan, P, Q, F3)
        assert E3 == E32 and np.array_equal(V3, V32) and torch.equal(F3, F32)
    finally:
        pme.pme_destroy(plan)


def test_tensor_influence_refused_off_k128(pme):
    s = wl.parity_system()
    plan = pme.pme_create(s.K, s.p, s.beta, s.box)
    try:
        with pytest.raises(pme.PMEError) as ei:
            pme.pme_set_influence_path(plan, pme.PME_INFLUENCE_TENSOR)
        assert ei.value.status == pme.PME_EUNSUPPORTED
    finally:
        pme.pme_destroy(plan)
