"""Slab decomposition of one system (the paper's distributed FFT with two all-to-all corner turns), run by the
CPU emulation of the library's stage bodies: P ranks each own k1 planes and influence-stage columns; their
three stages with the exchanges in between must give the energy, virial and forces of the undivided
evaluation and of the FP64 oracle. First with P virtual ranks in one process (the exchange a transposition
of blocks), then with two gloo processes exchanging through torch.distributed.all_to_all_single."""
import ctypes
import os
import socket

import numpy as np
import pytest

from paper_2009_12617_gb300 import workloads as wl

from helpers import E_REL_TOL, F_RMS_TOL, V_TOL, build_emu, emu_spme, rel_energy, rel_virial, rms_force

_fp = ctypes.POINTER(ctypes.c_float)
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def _bind(lib):
    lib.emu_slab_create.restype = ctypes.c_void_p
    lib.emu_slab_create.argtypes = [ctypes.c_int64, _ip, ctypes.c_int, ctypes.c_double, _dp, ctypes.c_int, ctypes.c_int]
    lib.emu_slab_destroy.argtypes = [ctypes.c_void_p]
    lib.emu_slab_layout.restype = ctypes.c_int64
    lib.emu_slab_layout.argtypes = [ctypes.c_void_p, _ip, _ip]
    lib.emu_slab_stage1.argtypes = [ctypes.c_void_p, ctypes.c_int64, _fp, _fp, _fp]
    lib.emu_slab_stage2.argtypes = [ctypes.c_void_p, _fp, _fp, _dp]
    lib.emu_slab_stage3.argtypes = [ctypes.c_void_p, _fp, _fp]
    return lib


class Rank:
    """One rank's emulated slab state."""

    def __init__(self, lib, s, P, r):
        self.lib = lib
        self.pos = np.ascontiguousarray(s.pos, np.float32)
        self.q = np.ascontiguousarray(s.q, np.float32)
        bx = np.ascontiguousarray(s.box, np.float64).reshape(9)
        self.h = lib.emu_slab_create(len(self.q), (ctypes.c_int * 3)(*s.K), s.p, s.beta, bx.ctypes.data_as(_dp), P, r)
        assert self.h
        pl, cl = (ctypes.c_int * 2)(), (ctypes.c_int * 2)()
        self.block = int(lib.emu_slab_layout(self.h, pl, cl))
        self.planes, self.cols = tuple(pl), tuple(cl)
        self.P = P

    def stage1(self):
        send = np.zeros(self.P * self.block * 2, np.float32)
        assert self.lib.emu_slab_stage1(self.h, len(self.q), self.pos.ctypes.data_as(_fp), self.q.ctypes.data_as(_fp),
                                        send.ctypes.data_as(_fp)) == 0
        return send

    def stage2(self, recv):
        send = np.zeros_like(recv)
        ev = np.zeros(7)
        self.lib.emu_slab_stage2(self.h, recv.ctypes.data_as(_fp), send.ctypes.data_as(_fp), ev.ctypes.data_as(_dp))
        return send, ev

    def stage3(self, recv):
        F = np.zeros((len(self.q), 3), np.float32)
        assert self.lib.emu_slab_stage3(self.h, recv.ctypes.data_as(_fp), F.ctypes.data_as(_fp)) == 0
        return F

    def close(self):
        self.lib.emu_slab_destroy(self.h)


def _all_to_all(sends, block):
    """recv of rank s = the s-th block of every rank's send, in rank order."""
    P = len(sends)
    blk = [x.reshape(P, 2 * block) for x in sends]
    return [np.ascontiguousarray(np.concatenate([blk[r][s] for r in range(P)])) for s in range(P)]


@pytest.fixture(scope="module")
def emu():
    return _bind(build_emu())


@pytest.mark.parametrize("K,p,P", [((32, 32, 32), 4, 2), ((30, 32, 36), 5, 3), ((32, 40, 48), 6, 4), ((24, 30, 40), 4, 5)])
def test_virtual_ranks_match_undivided_and_oracle(emu, oracle_mod, K, p, P):
    s = wl.parity_system()
    s = wl.System(s.pos, s.q, s.box, K, p, 0.34)
    ranks = [Rank(emu, s, P, r) for r in range(P)]
    try:
        # the planes and the columns are each partitioned exactly once
        assert ranks[0].planes[0] == 0 and ranks[-1].planes[1] == K[0]
        assert all(ranks[r].planes[1] == ranks[r + 1].planes[0] for r in range(P - 1))
        assert ranks[0].cols[0] == 0 and ranks[-1].cols[1] == K[1] * (K[2] // 2 + 1)
        assert all(ranks[r].cols[1] == ranks[r + 1].cols[0] for r in range(P - 1))
        recv = _all_to_all([rk.stage1() for rk in ranks], ranks[0].block)
        out = [rk.stage2(recv[r]) for r, rk in enumerate(ranks)]
        ev = sum(o[1] for o in out)
        recv2 = _all_to_all([o[0] for o in out], ranks[0].block)
        F = sum(rk.stage3(recv2[r]).astype(np.float64) for r, rk in enumerate(ranks))
    finally:
        for rk in ranks:
            rk.close()
    st, F1, ev1, _, _ = emu_spme(emu, s.pos, s.q, K, p, 0.34, s.box)
    assert st == 0
    assert rel_energy(ev[0], ev1[0]) < 1e-6 and rms_force(F, F1.astype(np.float64)) < 1e-6
    r = oracle_mod.spme(s.pos.astype(float), s.q.astype(float), K, p, 0.34, s.box)
    assert rel_energy(ev[0], r["energy"]) < E_REL_TOL
    assert rms_force(F, r["forces"]) < F_RMS_TOL
    assert rel_virial(ev[1:], r["virial"]) < V_TOL


def _free_port():
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        return so.getsockname()[1]


def _gloo_rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        lib = _bind(build_emu())
        s = wl.parity_system()
        rk = Rank(lib, s, world, rank)
        try:
            send = torch.from_numpy(rk.stage1())
            recv = torch.empty_like(send)
            dist.all_to_all_single(recv, send)
            send2, ev = rk.stage2(recv.numpy())
            recv2 = torch.empty(send2.shape, dtype=torch.float32)
            dist.all_to_all_single(recv2, torch.from_numpy(send2))
            F = torch.from_numpy(rk.stage3(recv2.numpy()).astype(np.float64))
            evt = torch.from_numpy(ev)
            dist.all_reduce(F)
            dist.all_reduce(evt)
            q.put((rank, F.numpy(), evt.numpy()))
        finally:
            rk.close()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_exchange_through_torch_distributed(emu, oracle_mod):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_gloo_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=300) for _ in procs), key=lambda o: o[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    F, ev = out[0][1], out[0][2]
    assert np.array_equal(F, out[1][1]) and np.array_equal(ev, out[1][2])
    s = wl.parity_system()
    r = oracle_mod.spme(s.pos.astype(float), s.q.astype(float), s.K, s.p, s.beta, s.box)
    assert rel_energy(ev[0], r["energy"]) < E_REL_TOL
    assert rms_force(F, r["forces"]) < F_RMS_TOL
    assert rel_virial(ev[1:], r["virial"]) < V_TOL
