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


def _case(name):
    """(K, p, beta, box, pos, q) of one allocation-free test case, all within the static limits."""
    if name.startswith("parity"):
        s = wl.parity_system()
        return s.K, int(name[-1]), s.beta, s.box, s.pos, s.q
    rng = np.random.default_rng(31)
    if name == "noncubic":
        K = (24, 30, 40)
        box = np.diag(np.array(K, float) * 1.1)
        pos = (rng.random((3000, 3)) * np.diag(box)).astype(np.float32)
    elif name == "triclinic":
        K = (30, 32, 32)
        box = np.array([[27.4, 0, 0], [3.1, 26.0, 0], [-2.0, 4.0, 28.0]])
        pos = wl.parity_system().pos
    elif name == "overflow":  # every atom in one tile: the bucket overflows, global-memory paths run
        K = (32, 32, 32)
        box = np.diag([30.0, 30.0, 30.0])
        pos = (10.0 + rng.random((4000, 3)) * 1.5).astype(np.float32)
    else:  # empty
        K, box, pos = (32, 32, 32), np.diag([27.4] * 3), np.zeros((0, 3), np.float32)
    q = rng.normal(size=len(pos))
    q = (q - q.mean()).astype(np.float32) if len(pos) else q.astype(np.float32)
    p = 6 if name == "triclinic" else 4
    return K, p, 0.34, box, np.ascontiguousarray(pos, np.float32), q


CASES = ["parity_p4", "parity_p6", "parity_p8", "noncubic", "triclinic", "overflow", "empty"]


@pytest.mark.parametrize("name", CASES)
def test_noalloc_matches_pme_compute_twice(name):
    from paper_2009_12617_gb300 import build, pme

    build.build_library()
    pme.load_library()
    K, p, beta, box, pos_h, q_h = _case(name)
    dev = torch.device("cuda:0")
    pos = torch.from_numpy(pos_h).to(dev)
    q = torch.from_numpy(q_h).to(dev)
    F_ref = torch.empty_like(pos)
    plan = pme.pme_create(K, p, beta, box)
    try:
        E_ref, V_ref = pme.pme_compute(plan, pos, q, F_ref)
    finally:
        pme.pme_destroy(plan)
    F_ref = F_ref.cpu().numpy().astype(np.float64)
    for _ in range(2):  # the second call runs on whatever the first left in the shared static array
        F = torch.full_like(pos, float("nan"))
        E, V = pme.pme_compute_noalloc(K, p, beta, box, pos, q, F)
        if name == "empty":
            assert E == 0.0 and np.all(V == 0.0) and E_ref == 0.0
            continue
        assert rel_energy(E, E_ref) < E_REL_TOL
        assert rms_force(F.cpu().numpy(), F_ref) < F_RMS_TOL
        assert rel_virial(V, V_ref) < V_TOL


def test_noalloc_rejects_mismatched_arrays():
    from paper_2009_12617_gb300 import pme

    pme.load_library()
    s = wl.parity_system()
    pos = torch.from_numpy(s.pos).cuda()
    q = torch.from_numpy(s.q[:-1]).cuda()
    with pytest.raises(ValueError):
        pme.pme_compute_noalloc(s.K, s.p, s.beta, s.box, pos, q, torch.empty_like(pos))


def test_noalloc_rejects_oversize():
    from paper_2009_12617_gb300 import pme

    pme.load_library()
    pos = torch.zeros((4, 3), device="cuda:0")
    q = torch.zeros(4, device="cuda:0")
    F = torch.empty_like(pos)
    with pytest.raises(pme.PMEError) as ei:
        pme.pme_compute_noalloc((64, 64, 64), 4, 0.34, np.eye(3) * 80.0, pos, q, F)
    assert ei.value.status == pme.PME_EINVAL and "static limit" in ei.value.detail
