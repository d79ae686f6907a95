"""pme_compute_noalloc: the evaluation for callers that must not allocate device memory.

Some callers cannot let a library call cudaMalloc: an application that handed all device memory to its
own pool at start-up may have nothing left, and cudaMalloc / cudaFree synchronise the whole device, which a
latency-bound caller cannot afford on every call. This entry point keeps all of its scratch in one static
device array instead. The test calls it through the C ABI twice in a row and compares each result with the
ordinary entry point (pme_compute, which allocates its plan) at the tolerances the parity tests use. This
file is collected last so that a run stopping at its first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_2009_12617_gb300 import workloads as wl

from helpers import E_REL_TOL, F_RMS_TOL, V_TOL, rel_energy, rel_virial, rms_force

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_noalloc_matches_pme_compute_twice():
    from paper_2009_12617_gb300 import build, pme

    build.build_library()
    pme.load_library()
    s = wl.parity_system()
    dev = torch.device("cuda:0")
    pos = torch.from_numpy(s.pos).to(dev)
    q = torch.from_numpy(s.q).to(dev)
    F_ref = torch.empty_like(pos)
    plan = pme.pme_create(s.K, s.p, s.beta, s.box)
    try:
        E_ref, V_ref = pme.pme_compute(plan, pos, q, F_ref)
    finally:
        pme.pme_destroy(plan)
    F_ref = F_ref.cpu().numpy().astype(np.float64)
    for _ in range(2):  # the second call runs on whatever the first left in the shared static array
        F = torch.full_like(pos, float("nan"))
        E, V = pme.pme_compute_noalloc(s.K, s.p, s.beta, s.box, pos, q, F)
        assert rel_energy(E, E_ref) < E_REL_TOL
        assert rms_force(F.cpu().numpy(), F_ref) < F_RMS_TOL
        assert rel_virial(V, V_ref) < V_TOL


def test_noalloc_rejects_oversize():
    from paper_2009_12617_gb300 import pme

    pme.load_library()
    pos = torch.zeros((4, 3), device="cuda:0")
    q = torch.zeros(4, device="cuda:0")
    F = torch.empty_like(pos)
    with pytest.raises(pme.PMEError) as ei:
        pme.pme_compute_noalloc((64, 64, 64), 4, 0.34, np.eye(3) * 80.0, pos, q, F)
    assert ei.value.status == pme.PME_EINVAL and "static limit" in ei.value.detail
