"""Reciprocal-space SPME in FP64 with numpy's FFT (pocketfft): a CPU context baseline, not the oracle.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: timed by bench.py beside the oracle and checked
against the oracle by tests/test_oracle_pins.py. The library in ``paper_2009_12617_gb300`` never imports it.

It evaluates the same standard SPME sums as ``spme_oracle.c`` (cardinal B-splines of order p on the mesh,
forward 3D FFT, multiply by B(m) C(m), energy and virial over the full spectrum, inverse FFT, forces from
the B-spline derivatives), but with array operations and a fast transform instead of the oracle's plain
loops and direct DFT, so its time shows what an ordinary vectorised FP64 CPU implementation costs.

Sign convention: the oracle's forward transform is sum_k Q(k) exp(+2 pi i m.k/K); numpy's fftn uses the
opposite sign, which only maps m to -m. |Qhat|^2 and the B C product are even in m on orthogonal cells,
and the potential is phi(k) = K1 K2 K3 ifftn(B C fftn(Q)) with B C taken at -m, which is what is done.
"""
from __future__ import annotations

import numpy as np


def _bspline(w: np.ndarray, p: int) -> tuple[np.ndarray, np.ndarray]:
    """theta[j] = M_p(w + j) and dtheta[j] = M_p'(w + j), j < p, for w in [0, 1): arrays (n, p)."""
    n = w.shape[0]
    th = np.zeros((n, p))
    th[:, 0] = w
    th[:, 1] = 1.0 - w  # M_2(w + j), j = 0, 1
    dth = None
    for order in range(3, p + 1):
        if order == p:  # M_p' (w + j) = M_{p-1}(w + j) - M_{p-1}(w + j - 1)
            prev = th[:, :p - 1]
            dth = np.zeros((n, p))
            dth[:, 0] = prev[:, 0]
            dth[:, 1:p - 1] = prev[:, 1:] - prev[:, :-1]
            dth[:, p - 1] = -prev[:, p - 2]
        new = np.zeros((n, p))
        for j in range(order):
            x = w + j
            a = th[:, j] if j < order - 1 else 0.0
            b = th[:, j - 1] if j >= 1 else 0.0
            new[:, j] = (x * a + (order - x) * b) / (order - 1)
        th = new
    if dth is None:  # p == 2
        dth = np.stack([np.ones(n), -np.ones(n)], axis=1)
    return th, dth


def moduli(K: int, p: int) -> np.ndarray:
    """|b(m)|^2 = 1 / |sum_{k<=p-2} M_p(k+1) exp(2 pi i m k / K)|^2 for m < K."""
    knots, _ = _bspline(np.zeros(1), p)  # M_p(j), j < p
    Mk = np.append(knots[0], 0.0)[1:p]   # M_p(1..p-1)
    m = np.arange(K)[:, None]
    k = np.arange(p - 1)[None, :]
    z = (Mk[None, :] * np.exp(2j * np.pi * ((m * k) % K) / K)).sum(axis=1)
    return 1.0 / np.abs(z) ** 2


class Plan:
    """Tables of one (K, p, beta, box): B C on the full mesh at -m, the reciprocal vectors, |m'|^2 terms."""

    def __init__(self, K, p: int, beta: float, box):
        self.K = tuple(int(k) for k in K)
        self.p = int(p)
        box = np.asarray(box, dtype=np.float64).reshape(3, 3)
        self.recip = np.linalg.inv(box).T  # rows a*_alpha
        self.vol = abs(np.linalg.det(box))
        mt = [np.where(2 * np.arange(k) <= k, np.arange(k), np.arange(k) - k) for k in self.K]
        M1, M2, M3 = np.meshgrid(*mt, indexing="ij")
        mv = M1[..., None] * self.recip[0] + M2[..., None] * self.recip[1] + M3[..., None] * self.recip[2]
        m2n = (mv ** 2).sum(-1)
        m2n[0, 0, 0] = 1.0
        B = np.einsum("i,j,k->ijk", *[moduli(k, self.p) for k in self.K])
        fac = np.pi ** 2 / beta ** 2
        BC = B * np.exp(-fac * m2n) / (np.pi * self.vol * m2n)
        BC[0, 0, 0] = 0.0
        self.BC = BC
        f = 2.0 * (1.0 + fac * m2n) / m2n
        # virial factor per component (xx, yy, zz, xy, xz, yz): delta_ab - f m'_a m'_b
        pairs = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
        self.vfac = np.stack([(1.0 if a == b else 0.0) - f * mv[..., a] * mv[..., b] for a, b in pairs])
        # B C at -m (numpy's forward transform evaluates the oracle's Qhat at -m)
        self.BCneg = np.roll(np.flip(BC, axis=(0, 1, 2)), shift=1, axis=(0, 1, 2))

    def evaluate(self, pos, q) -> dict:
        K, p = self.K, self.p
        pos = np.asarray(pos, dtype=np.float64).reshape(-1, 3)
        q = np.asarray(q, dtype=np.float64).reshape(-1)
        s = pos @ self.recip.T
        s -= np.floor(s)
        u = s * np.array(K, dtype=np.float64)
        base = np.floor(u).astype(np.int64)
        w = u - base
        th, dth, idx = [], [], []
        for al in range(3):
            t, dt = _bspline(w[:, al], p)
            th.append(t)
            dth.append(dt)
            idx.append(np.mod(base[:, al, None] - np.arange(p)[None, :], K[al]))
        # spreading: Q(k) += q theta1 theta2 theta3 at k = base - j
        flat = (idx[0][:, :, None, None] * K[1] + idx[1][:, None, :, None]) * K[2] + idx[2][:, None, None, :]
        wts = q[:, None, None, None] * th[0][:, :, None, None] * th[1][:, None, :, None] * th[2][:, None, None, :]
        Q = np.bincount(flat.ravel(), weights=wts.ravel(), minlength=K[0] * K[1] * K[2]).reshape(K)
        Qh = np.fft.fftn(Q)
        e_m = 0.5 * self.BCneg * (Qh.real ** 2 + Qh.imag ** 2)
        E = float(e_m.sum())
        vfac_neg = np.roll(np.flip(self.vfac, axis=(1, 2, 3)), shift=1, axis=(1, 2, 3))
        virial = (vfac_neg * e_m[None]).reshape(6, -1).sum(axis=1)
        phi = np.fft.ifftn(self.BCneg * Qh).real * (K[0] * K[1] * K[2])
        ph = phi.ravel()[flat]
        g1 = (dth[0][:, :, None, None] * th[1][:, None, :, None] * th[2][:, None, None, :] * ph).sum(axis=(1, 2, 3))
        g2 = (th[0][:, :, None, None] * dth[1][:, None, :, None] * th[2][:, None, None, :] * ph).sum(axis=(1, 2, 3))
        g3 = (th[0][:, :, None, None] * th[1][:, None, :, None] * dth[2][:, None, None, :] * ph).sum(axis=(1, 2, 3))
        g = np.stack([g1, g2, g3], axis=1) * np.array(K, dtype=np.float64)
        F = -q[:, None] * (g @ self.recip)
        return {"energy": E, "virial": virial, "forces": F}


def spme(pos, q, K, p, beta, box) -> dict:
    """One evaluation, tables included."""
    return Plan(K, p, beta, box).evaluate(pos, q)
