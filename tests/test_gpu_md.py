"""The device-resident multi-step loop (pme_run_steps) against the same steps driven from the host.

Each host step calls the synchronous entry points (reciprocal and, when used, real space), adds the forces and
applies v += (F * inv_mass) * dt, x += v * dt with one FP32 rounding per operation; the device loop must give
the same positions, velocities, forces and per-step energies bit for bit. Chunks of 32 steps replay one
recorded graph, so 70 steps exercise the replay and the directly launched remainder.
"""
import numpy as np
import pytest

from paper_2009_12617_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pme():
    from paper_2009_12617_gb300 import build
    from paper_2009_12617_gb300 import pme as p

    build.build_library()
    p.load_library()
    return p


def _state(s, seed):
    rng = np.random.default_rng(seed)
    vel = (rng.normal(size=(s.n, 3)) * 0.01).astype(np.float32)
    inv_mass = np.where(s.q < 0, 1.0 / 16.0, 1.0).astype(np.float32)  # oxygen-like and hydrogen-like
    return vel, inv_mass


@pytest.mark.parametrize("with_real", [False, True])
def test_run_steps_matches_host_loop(pme, with_real):
    s = wl.parity_system()
    dev = torch.device("cuda:0")
    vel0, im = _state(s, 3)
    dt = np.float32(0.002)
    steps = 70
    stream = torch.cuda.Stream(dev)
    plan = pme.pme_create(s.K, s.p, s.beta, s.box, stream=stream)
    rs = pme.pme_real_create(s.box, s.beta, 9.0, stream=stream) if with_real else 0
    try:
        with torch.cuda.stream(stream):  # torch work and the library share the plan stream
            # host-driven reference
            pos = torch.from_numpy(s.pos.copy()).to(dev)
            vel = torch.from_numpy(vel0.copy()).to(dev)
            q = torch.from_numpy(s.q).to(dev)
            invm = torch.from_numpy(im).to(dev)
            F, Fr = torch.empty_like(pos), torch.empty_like(pos)
            ref_ev = []
            for _ in range(steps):
                E, V = pme.pme_compute(plan, pos, q, F)
                row = [E, *V]
                if with_real:
                    er, es, vr = pme.pme_real_compute(rs, pos, q, Fr)
                    F = F + Fr
                    row += [er, es, *vr]
                else:
                    row += [0.0] * 8
                ref_ev.append(row)
                vel = vel + (F * invm[:, None]) * dt
                pos = pos + vel * dt
            torch.cuda.synchronize()
            # the same on the device, one call
            pos_d = torch.from_numpy(s.pos.copy()).to(dev)
            vel_d = torch.from_numpy(vel0.copy()).to(dev)
            F_d = torch.empty_like(pos_d)
            ev = torch.full((steps, 15), float("nan"), dtype=torch.float64, device=dev)
            pme.pme_run_steps(plan, pos_d, vel_d, q, F_d, float(dt), steps, rs=rs, inv_mass=invm, ev_steps=ev)
            pme.pme_sync(plan)
            assert torch.equal(pos_d, pos) and torch.equal(vel_d, vel) and torch.equal(F_d, F)
            assert np.array_equal(ev.cpu().numpy(), np.array(ref_ev))
            # a second call continues from where the first ended (graph replayed, counter reset)
            ev2 = torch.zeros((5, 15), dtype=torch.float64, device=dev)
            pme.pme_run_steps(plan, pos_d, vel_d, q, F_d, float(dt), 5, rs=rs, inv_mass=invm, ev_steps=ev2)
            pme.pme_sync(plan)
            for k in range(5):
                E, _ = pme.pme_compute(plan, pos, q, F)
                if with_real:
                    pme.pme_real_compute(rs, pos, q, Fr)
                    F = F + Fr
                assert ev2[k, 0].item() == E
                vel = vel + (F * invm[:, None]) * dt
                pos = pos + vel * dt
            assert torch.equal(pos_d, pos) and torch.equal(vel_d, vel)
    finally:
        if rs:
            pme.pme_real_destroy(rs)
        pme.pme_destroy(plan)
