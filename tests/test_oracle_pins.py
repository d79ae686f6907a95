"""Pins for the FP64 oracle against what the mathematics fixes (no GPU).

The paper prints no worked example for its SPME pipeline (it validates against OpenMM, Sec. I), so each
oracle function is pinned to closed forms, textbook special cases, invariants, brute force on tiny
inputs and the NaCl Madelung constant. Each pin is chosen so a plausible mistake fails it: a dropped
1/(pi V) or B-spline modulus (Ewald convergence, Madelung), a sign or index error in the forces or virial
(finite differences), a transposed reciprocal matrix (triclinic Ewald comparison), a wrong frequency
aliasing (Ewald convergence).
"""
import math
import os

import numpy as np
import pytest

from paper_2009_12617_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------------------------------------
# B-splines


def _m4_closed(x):
    """Textbook piecewise cubic B-spline on [0, 4]."""
    if x <= 0 or x >= 4:
        return 0.0
    if x < 1:
        return x ** 3 / 6
    if x < 2:
        return (-3 * x ** 3 + 12 * x ** 2 - 12 * x + 4) / 6
    if x < 3:
        return (3 * x ** 3 - 24 * x ** 2 + 60 * x - 44) / 6
    return (4 - x) ** 3 / 6


def _mp_truncated_power(p, x):
    """Cardinal B-spline by the truncated-power formula (1/(p-1)!) sum_k (-1)^k C(p,k) (x-k)_+^(p-1)."""
    return sum((-1) ** k * math.comb(p, k) * max(x - k, 0.0) ** (p - 1) for k in range(p + 1)) / math.factorial(
        p - 1)


def test_bspline_cubic_closed_form(oracle_mod):
    for x in np.linspace(-0.5, 4.5, 401):
        assert oracle_mod.bspline(4, x) == pytest.approx(_m4_closed(x), abs=1e-13)


@pytest.mark.parametrize("p", [2, 3, 4, 5, 6, 7, 8])
def test_bspline_truncated_power(oracle_mod, p):
    for x in np.linspace(0.013, p - 0.013, 97):
        assert oracle_mod.bspline(p, x) == pytest.approx(_mp_truncated_power(p, x), abs=1e-12)


@pytest.mark.parametrize("p", [3, 4, 5, 6, 8])
def test_bspline_partition_of_unity_and_symmetry(oracle_mod, p):
    for w in np.linspace(0.0, 0.999, 37):
        s = sum(oracle_mod.bspline(p, w + j) for j in range(p))
        ds = sum(oracle_mod.bspline_deriv(p, w + j) for j in range(p))
        assert s == pytest.approx(1.0, abs=1e-14)
        assert ds == pytest.approx(0.0, abs=1e-14)
        assert oracle_mod.bspline(p, w + 0.5) == pytest.approx(oracle_mod.bspline(p, p - w - 0.5), abs=1e-15)


@pytest.mark.parametrize("p", [4, 6])
def test_bspline_derivative_matches_finite_difference(oracle_mod, p):
    h = 1e-6
    for x in np.linspace(0.1, p - 0.1, 53):
        fd = (oracle_mod.bspline(p, x + h) - oracle_mod.bspline(p, x - h)) / (2 * h)
        assert oracle_mod.bspline_deriv(p, x) == pytest.approx(fd, abs=1e-8)


def test_bspline_node_values_golden(oracle_mod):
    with open(os.path.join(GOLDEN, "bspline_nodes.txt")) as f:
        rows = [list(map(int, ln.split())) for ln in f if ln.strip() and not ln.startswith("#")]
    for row in rows:
        p, num, den = row[0], row[1:-1], row[-1]
        assert len(num) == p - 1
        for k, nk in enumerate(num, start=1):
            assert oracle_mod.bspline(p, k) == pytest.approx(nk / den, abs=1e-15)


# ---------------------------------------------------------------------------------------------------------
# Charge spreading


def test_spread_node_atom_exact_weights(oracle_mod):
    """An atom on a mesh node (w = 0) has weights M_4(j) = 0, 1/6, 2/3, 1/6 on nodes base - j."""
    L, K = 10.0, (10, 12, 14)
    box = np.diag([L, L, L])
    node = np.array([3, 5, 7])
    pos = (node / np.array(K) * L)[None, :]
    Q = oracle_mod.spread(pos, [2.0], K, 4, box)
    w = np.array([0.0, 1 / 6, 2 / 3, 1 / 6])
    expect = np.zeros(K)
    for a in range(4):
        for b in range(4):
            for c in range(4):
                expect[(node[0] - a) % K[0], (node[1] - b) % K[1], (node[2] - c) % K[2]] += 2.0 * w[a] * w[b] * w[c]
    np.testing.assert_allclose(Q, expect, atol=1e-15)


def test_spread_charge_sum_and_periodic_images(oracle_mod):
    """Sum of Q equals the total charge; on a mesh smaller than p the image sum wraps onto itself."""
    rng = np.random.default_rng(0)
    L = 7.0
    box = np.diag([L, L, L])
    pos = rng.random((5, 3)) * L
    q = rng.normal(size=5)
    for K in [(3, 3, 3), (5, 4, 6), (8, 8, 8)]:
        Q = oracle_mod.spread(pos, q, K, 4, box)
        assert Q.sum() == pytest.approx(q.sum(), abs=1e-13)
        # brute-force image sum of eq. (3) for this tiny mesh
        u = oracle_mod.scaled_coords(pos, K, box)
        Qb = np.zeros(K)
        for i in range(5):
            wts = []
            for al in range(3):
                wa = np.zeros(K[al])
                for k in range(K[al]):
                    for nimg in range(-6, 7):
                        wa[k] += oracle_mod.bspline(4, u[i, al] - k - nimg * K[al])
                wts.append(wa)
            Qb += q[i] * np.einsum("a,b,c->abc", *wts)
        np.testing.assert_allclose(Q, Qb, atol=1e-13)


# ---------------------------------------------------------------------------------------------------------
# DFT


def test_dft_separable_equals_full_and_numpy(oracle_mod):
    rng = np.random.default_rng(1)
    x = rng.normal(size=(4, 6, 5)) + 1j * rng.normal(size=(4, 6, 5))
    for sign in (+1, -1):
        a = oracle_mod.dft3(x, sign)
        b = oracle_mod.dft3(x, sign, full=True)
        np.testing.assert_allclose(a, b, atol=1e-11)
    # numpy's fftn uses exp(-2 pi i ...): sign -1
    np.testing.assert_allclose(oracle_mod.dft3(x, -1), np.fft.fftn(x), atol=1e-11)
    np.testing.assert_allclose(oracle_mod.dft3(x, +1), np.fft.ifftn(x) * x.size, atol=1e-11)


def test_dft_parseval(oracle_mod):
    rng = np.random.default_rng(2)
    Q = rng.normal(size=(8, 10, 12))
    F = oracle_mod.dft3(Q, +1)
    assert np.sum(np.abs(F) ** 2) == pytest.approx(Q.size * np.sum(Q ** 2), rel=1e-12)


# ---------------------------------------------------------------------------------------------------------
# Moduli


@pytest.mark.parametrize("K", [8, 10, 32, 40, 64])
def test_bmod_closed_forms(oracle_mod, K):
    """p = 4: |sum M4(k+1) e^{i k t}|^2 = ((2 + cos t)/3)^2; p = 6: ((66 + 52 cos t + 2 cos 2t)/120)^2."""
    for m in range(K):
        t = 2 * math.pi * m / K
        assert oracle_mod.bmod2(K, 4, m) == pytest.approx(1.0 / ((2 + math.cos(t)) / 3) ** 2, rel=1e-13)
        d6 = (66 + 52 * math.cos(t) + 2 * math.cos(2 * t)) / 120
        assert oracle_mod.bmod2(K, 6, m) == pytest.approx(1.0 / d6 ** 2, rel=1e-13)


# ---------------------------------------------------------------------------------------------------------
# Ewald comparison terms: an independent numpy implementation


def _np_ewald_recip(pos, q, beta, box, mcut):
    recip = np.linalg.inv(box)  # columns are a*_alpha
    V = abs(np.linalg.det(box))
    nmax = [int(math.ceil(mcut * np.linalg.norm(box[a]))) for a in range(3)]
    ms = np.array([(a, b, c) for a in range(-nmax[0], nmax[0] + 1) for b in range(-nmax[1], nmax[1] + 1)
                   for c in range(-nmax[2], nmax[2] + 1) if (a, b, c) != (0, 0, 0)], dtype=float)
    mv = ms @ recip.T
    m2 = np.sum(mv ** 2, axis=1)
    keep = m2 <= mcut ** 2
    mv, m2 = mv[keep], m2[keep]
    f = np.exp(-math.pi ** 2 * m2 / beta ** 2) / m2
    S = np.exp(2j * math.pi * pos @ mv.T).T @ q  # (nm,)
    E = np.sum(f * np.abs(S) ** 2) / (2 * math.pi * V)
    ph = np.exp(2j * math.pi * pos @ mv.T)  # (n, nm)
    # F_j = -dE/dr_j ;  dE/dr_j = (1/(2 pi V)) sum f 2 Re(conj(S) q_j 2 pi i m' e^{i th_j})
    dS = (np.conj(S)[None, :] * 1j * ph).real  # (n, nm)
    F = -(q[:, None] * (2.0 / V)) * ((dS * f[None, :]) @ mv)
    e_m = f * np.abs(S) ** 2 / (2 * math.pi * V)
    fac = 2 * (1 + math.pi ** 2 * m2 / beta ** 2) / m2
    vir = np.zeros(6)
    pairs = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    for k, (a, b) in enumerate(pairs):
        vir[k] = np.sum(e_m * ((1.0 if a == b else 0.0) - fac * mv[:, a] * mv[:, b]))
    return E, F, vir


def _np_ewald_real(pos, q, beta, box, rcut):
    from scipy.special import erfc

    E = 0.0
    F = np.zeros_like(pos)
    V = np.zeros(6)
    rinv = np.linalg.inv(box)
    nmax = [int(math.ceil(rcut * np.linalg.norm(rinv[:, a]))) + 1 for a in range(3)]
    shifts = np.array([(a, b, c) for a in range(-nmax[0], nmax[0] + 1) for b in range(-nmax[1], nmax[1] + 1)
                       for c in range(-nmax[2], nmax[2] + 1)], dtype=float) @ box
    for i in range(len(q)):
        d = pos[i][None, None, :] - pos[None, :, :] + shifts[:, None, :]  # (ns, n, 3)
        r = np.linalg.norm(d, axis=2)
        mask = (r <= rcut) & (r > 0)
        rr = np.where(mask, r, 1.0)
        e = np.where(mask, q[i] * q[None, :] * erfc(beta * rr) / rr, 0.0)
        E += 0.5 * e.sum()
        s = np.where(mask, q[i] * q[None, :] * (erfc(beta * rr) / rr + 2 * beta / math.sqrt(math.pi)
                                                 * np.exp(-beta ** 2 * rr ** 2)) / rr ** 2, 0.0)
        F[i] = np.sum(s[:, :, None] * d, axis=(0, 1))
        for k, (a, b) in enumerate([(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]):
            V[k] += 0.5 * np.sum(s * d[:, :, a] * d[:, :, b])
    return E, F, V


def _tri_box():
    return np.array([[9.0, 0.0, 0.0], [2.1, 8.5, 0.0], [-1.3, 1.7, 10.2]])


@pytest.mark.parametrize("tri", [False, True])
def test_ewald_terms_match_independent_numpy(oracle_mod, tri):
    rng = np.random.default_rng(3)
    box = _tri_box() if tri else np.diag([9.0, 10.0, 11.0])
    n = 24
    pos = rng.random((n, 3)) @ box
    q = rng.normal(size=n)
    q -= q.mean()
    beta = 0.45
    mcut = oracle_mod.ewald_mcut(beta)
    E, F, V = _np_ewald_recip(pos, q, beta, box, mcut)
    r = oracle_mod.ewald_recip(pos, q, beta, box)
    assert r["energy"] == pytest.approx(E, rel=1e-12)
    np.testing.assert_allclose(r["forces"], F, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(r["virial"], V, rtol=1e-10, atol=1e-12)
    Er, Fr, Vr = _np_ewald_real(pos, q, beta, box, 6.0 / beta)
    rr = oracle_mod.ewald_real(pos, q, beta, box)
    assert rr["energy"] == pytest.approx(Er, rel=1e-12)
    np.testing.assert_allclose(rr["forces"], Fr, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(rr["virial"], Vr, rtol=1e-10, atol=1e-12)
    assert oracle_mod.ewald_self(q, beta) == pytest.approx(-beta / math.sqrt(math.pi) * np.sum(q ** 2), rel=1e-14)


def _madelung():
    with open(os.path.join(GOLDEN, "madelung_nacl.txt")) as f:
        vals = dict(ln.split() for ln in f if ln.strip() and not ln.startswith("#"))
    return float(vals["M"]), float(vals["a_angstrom"]), int(vals["cells"])


@pytest.mark.parametrize("beta", [0.7, 1.1])
def test_ewald_madelung(oracle_mod, beta):
    M, a, cells = _madelung()
    pos, q, box = wl.rocksalt(a, cells)
    tot = (oracle_mod.ewald_recip(pos, q, beta, box)["energy"] + oracle_mod.ewald_real(pos, q, beta, box)["energy"]
           + oracle_mod.ewald_self(q, beta))
    assert -tot * (a / 2) / (len(q) / 2) == pytest.approx(M, abs=1e-6)


def test_spme_madelung(oracle_mod):
    """E_rec(SPME) + E_dir + E_self reproduces the NaCl Madelung constant to 6 digits."""
    M, a, cells = _madelung()
    pos, q, box = wl.rocksalt(a, cells)
    beta = 0.9
    r = oracle_mod.spme(pos, q, (32, 32, 32), 6, beta, box)
    tot = r["energy"] + oracle_mod.ewald_real(pos, q, beta, box)["energy"] + oracle_mod.ewald_self(q, beta)
    assert -tot * (a / 2) / (len(q) / 2) == pytest.approx(M, abs=1e-6)
    # the NaCl lattice is a force-free equilibrium: every reciprocal force is set by symmetry to ~0
    assert np.abs(r["forces"]).max() < 1e-9


def _small_water(n=150, L=18.0, seed=5):
    pos, q = wl.water_box(n, L, seed)
    return pos.astype(np.float64), q.astype(np.float64), np.diag([L, L, L])


@pytest.mark.parametrize("p", [4, 6])
def test_spme_converges_to_ewald(oracle_mod, p):
    """SPME -> Ewald as the mesh is refined, with error falling at least like h^(p-1)."""
    pos, q, box = _small_water()
    beta = 0.34
    ref = oracle_mod.ewald_recip(pos, q, beta, box)
    Ks = (12, 24, 48) if p == 4 else (12, 24)
    errE, errF, errV = [], [], []
    for K in Ks:
        r = oracle_mod.spme(pos, q, (K, K, K), p, beta, box)
        errE.append(abs(r["energy"] - ref["energy"]) / abs(ref["energy"]))
        errF.append(np.sqrt(np.mean((r["forces"] - ref["forces"]) ** 2) / np.mean(ref["forces"] ** 2)))
        errV.append(np.max(np.abs(r["virial"] - ref["virial"])) / np.max(np.abs(ref["virial"])))
    for err in (errE, errF, errV):
        slopes = [math.log2(err[i] / err[i + 1]) for i in range(len(err) - 1)]
        assert min(slopes) >= p - 1, (err, slopes)
    assert errE[-1] < 1e-3 and errF[-1] < 1e-3


def test_spme_triclinic_converges_to_ewald(oracle_mod):
    """A triclinic cell: a transposed reciprocal matrix or wrong m' would not converge."""
    rng = np.random.default_rng(7)
    box = _tri_box()
    pos = rng.random((40, 3)) @ box
    q = rng.normal(size=40)
    q -= q.mean()
    beta = 0.4
    ref = oracle_mod.ewald_recip(pos, q, beta, box)
    r = oracle_mod.spme(pos, q, (36, 36, 40), 6, beta, box)
    assert r["energy"] == pytest.approx(ref["energy"], rel=1e-5)
    np.testing.assert_allclose(r["forces"], ref["forces"], atol=1e-4 * np.abs(ref["forces"]).max())
    np.testing.assert_allclose(r["virial"], ref["virial"], atol=1e-5 * np.abs(ref["virial"]).max())


@pytest.mark.parametrize("tri", [False, True])
def test_spme_forces_are_gradient(oracle_mod, tri):
    """F = -dE/dr by central differences (SPME forces are the exact gradient of SPME energy for p >= 3)."""
    rng = np.random.default_rng(11)
    box = _tri_box() if tri else np.diag([11.0, 12.0, 13.0])
    n = 12
    pos = rng.random((n, 3)) @ box
    q = rng.normal(size=n)
    q -= q.mean()
    K, p, beta = (16, 18, 20), 4, 0.4
    F = oracle_mod.spme(pos, q, K, p, beta, box)["forces"]
    h = 1e-5
    for i in range(0, n, 3):
        for d in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[i, d] += h
            pm[i, d] -= h
            fd = -(oracle_mod.spme(pp, q, K, p, beta, box)["energy"] - oracle_mod.spme(pm, q, K, p, beta, box)["energy"]) / (2 * h)
            assert F[i, d] == pytest.approx(fd, rel=1e-6, abs=1e-9)


@pytest.mark.parametrize("tri", [False, True])
def test_spme_virial_is_strain_derivative(oracle_mod, tri):
    """Pi_ab = -dE/d eps_ab under r -> (I+eps) r, a -> (I+eps) a at fixed fractional coordinates."""
    rng = np.random.default_rng(13)
    box = _tri_box() if tri else np.diag([11.0, 12.0, 13.0])
    n = 16
    frac = rng.random((n, 3))
    q = rng.normal(size=n)
    q -= q.mean()
    K, p, beta = (16, 16, 20), 4, 0.4
    vir = oracle_mod.spme(frac @ box, q, K, p, beta, box)["virial"]
    h = 1e-6
    pairs = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    for k, (a, b) in enumerate(pairs):
        es = []
        for sgn in (+1, -1):
            eps = np.zeros((3, 3))
            eps[a, b] = sgn * h
            T = np.eye(3) + eps
            bx = box @ T.T  # rows a_alpha -> (I + eps) a_alpha
            es.append(oracle_mod.spme(frac @ bx, q, K, p, beta, bx)["energy"])
        fd = -(es[0] - es[1]) / (2 * h)
        assert vir[k] == pytest.approx(fd, rel=1e-6, abs=1e-9), (k, vir[k], fd)


def test_spme_phi_identity_and_translation(oracle_mod):
    """E = 1/2 sum Q phi; shifting every atom by one mesh cell leaves E and F unchanged."""
    pos, q, box = _small_water(90, 15.0, 17)
    K, p, beta = (20, 24, 30), 4, 0.34
    r = oracle_mod.spme(pos, q, K, p, beta, box, want_mesh=True)
    assert r["e_phi"] == pytest.approx(r["energy"], rel=1e-12)
    for al in range(3):
        shift = box[al] / K[al]
        s = oracle_mod.spme(pos + shift, q, K, p, beta, box)
        assert s["energy"] == pytest.approx(r["energy"], rel=1e-11)
        np.testing.assert_allclose(s["forces"], r["forces"], atol=1e-11 * np.abs(r["forces"]).max())
    # a whole-cell shift (a periodic image) changes nothing either
    s = oracle_mod.spme(pos + box[0] - 2 * box[2], q, K, p, beta, box)
    assert s["energy"] == pytest.approx(r["energy"], rel=1e-11)


def test_spme_empty_and_single_charge(oracle_mod):
    box = np.diag([10.0, 10.0, 10.0])
    r = oracle_mod.spme(np.zeros((0, 3)), np.zeros(0), (8, 8, 8), 4, 0.3, box)
    assert r["energy"] == 0.0 and np.all(r["virial"] == 0.0)
    # a lone charge: E_rec is a positive self-interaction that does not depend on where it sits
    e0 = oracle_mod.spme([[1.0, 2.0, 3.0]], [1.0], (16, 16, 16), 6, 0.3, box)["energy"]
    e1 = oracle_mod.spme([[4.2, 7.1, 0.3]], [1.0], (16, 16, 16), 6, 0.3, box)["energy"]
    assert e0 > 0 and e1 == pytest.approx(e0, rel=1e-4)


def test_oracle_results_do_not_depend_on_thread_count(oracle_mod):
    """The OpenMP loops give each output to one thread with the serial loop's operations in order: energy,
    virial, forces and both meshes are bit-identical for 1 and 4 threads (Ewald real-space sum too)."""
    s = wl.parity_system()
    try:
        oracle_mod.set_threads(1)
        r1 = oracle_mod.spme(s.pos, s.q, s.K, 6, s.beta, s.box, want_mesh=True)
        e1 = oracle_mod.ewald_real(s.pos[:400], s.q[:400], 0.34, s.box)
        oracle_mod.set_threads(4)
        r4 = oracle_mod.spme(s.pos, s.q, s.K, 6, s.beta, s.box, want_mesh=True)
        e4 = oracle_mod.ewald_real(s.pos[:400], s.q[:400], 0.34, s.box)
    finally:
        oracle_mod.set_threads(1)
    assert r1["energy"] == r4["energy"] and np.array_equal(r1["virial"], r4["virial"])
    assert np.array_equal(r1["forces"], r4["forces"]) and np.array_equal(r1["phi"], r4["phi"])
    assert np.array_equal(r1["Q"], r4["Q"])
    assert e1["energy"] == e4["energy"] and np.array_equal(e1["forces"], e4["forces"])


@pytest.mark.parametrize("K,p,tri", [((32, 32, 32), 4, False), ((30, 32, 36), 6, False), ((30, 32, 36), 6, True)])
def test_numpy_fft_baseline_matches_oracle(oracle_mod, K, p, tri):
    """The FP64 numpy-FFT context baseline (timed beside the oracle) evaluates the same sums: it agrees with
    the direct-DFT oracle to FP64 rounding in energy, forces and virial, orthogonal and triclinic."""
    from oracle import numpy_spme

    s = wl.parity_system()
    box = np.array([[27.4, 0, 0], [3.1, 26.0, 0], [-2.0, 4.0, 28.0]]) if tri else s.box
    r = oracle_mod.spme(s.pos, s.q, K, p, s.beta, box)
    x = numpy_spme.spme(s.pos, s.q, K, p, s.beta, box)
    assert abs(x["energy"] - r["energy"]) <= 1e-12 * abs(r["energy"])
    assert np.abs(x["forces"] - r["forces"]).max() <= 1e-12 * np.abs(r["forces"]).max()
    assert np.abs(x["virial"] - r["virial"]).max() <= 1e-12 * np.abs(r["virial"]).max()


@pytest.mark.parametrize("tri", [False, True])
def test_ewald_real_virial_and_forces_are_derivatives(oracle_mod, tri):
    """Real-space term: Pi_ab = -dE/d eps_ab (strain at fixed fractional coordinates) and F = -dE/dr, by
    central differences, with beta * rcut = 6 so no pair crosses the cutoff discontinuously."""
    rng = np.random.default_rng(29)
    box = _tri_box() if tri else np.diag([9.0, 10.0, 11.0])
    n = 20
    frac = rng.random((n, 3))
    q = rng.normal(size=n)
    q -= q.mean()
    beta = 0.55
    r = oracle_mod.ewald_real(frac @ box, q, beta, box)
    h = 1e-6
    pairs = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    for k, (a, b) in enumerate(pairs):
        es = []
        for sgn in (+1, -1):
            eps = np.zeros((3, 3))
            eps[a, b] = sgn * h
            bx = box @ (np.eye(3) + eps).T
            es.append(oracle_mod.ewald_real(frac @ bx, q, beta, bx)["energy"])
        fd = -(es[0] - es[1]) / (2 * h)
        assert r["virial"][k] == pytest.approx(fd, rel=1e-6, abs=1e-8), (k, r["virial"][k], fd)
    pos = frac @ box
    for i in (0, 7):
        for d in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[i, d] += h
            pm[i, d] -= h
            fd = -(oracle_mod.ewald_real(pp, q, beta, box)["energy"] - oracle_mod.ewald_real(pm, q, beta, box)["energy"]) / (2 * h)
            assert r["forces"][i, d] == pytest.approx(fd, rel=1e-6, abs=1e-8)


def test_ewald_real_rows_match_full_sum(oracle_mod):
    """The per-atom form (used to check single atoms of large systems) reproduces the full real-space sum:
    its forces row by row, and 1/2 sum_i e_i = E_real."""
    rng = np.random.default_rng(41)
    box = _tri_box()
    pos = rng.random((30, 3)) @ box
    q = rng.normal(size=30)
    q -= q.mean()
    full = oracle_mod.ewald_real(pos, q, 0.5, box, rcut=7.0)
    rows = oracle_mod.ewald_real_rows(pos, q, 0.5, box, np.arange(30), rcut=7.0)
    np.testing.assert_allclose(rows["forces"], full["forces"], rtol=1e-13, atol=1e-14)
    assert 0.5 * rows["e"].sum() == pytest.approx(full["energy"], rel=1e-13)


@pytest.mark.parametrize("K", [8, 16, 30])
def test_bmod_odd_order(oracle_mod, K):
    """p = 5: the denominator |sum M5(k+1) e^{i k t}|^2 = |(1 + 11 e^{it} + 11 e^{2it} + e^{3it}) / 24|^2 has
    the closed form ((2 cos(3t/2) + 22 cos(t/2)) / 24)^2 (knot values 1/24, 11/24, 11/24, 1/24); it vanishes
    at t = pi (m = K/2), where the modulus takes the mean of the two neighbouring denominators."""
    def den(t):
        return ((2 * math.cos(1.5 * t) + 22 * math.cos(0.5 * t)) / 24) ** 2

    for m in range(K):
        t = 2 * math.pi * m / K
        if 2 * m == K:
            want = 1.0 / (0.5 * (den(2 * math.pi * (m - 1) / K) + den(2 * math.pi * (m + 1) / K)))
        else:
            want = 1.0 / den(t)
        assert oracle_mod.bmod2(K, 5, m) == pytest.approx(want, rel=1e-12), m
    # the knot values are symmetric, so the alternating sum (t = pi) is exactly zero
    assert abs(den(math.pi)) < 1e-30


def test_spme_odd_order_converges_and_forces_are_gradient(oracle_mod):
    """p = 5 on a water-like box: SPME -> Ewald with slope >= p - 1 in energy and forces as the mesh doubles,
    and the forces are -dE/dr by central differences (the m = K/2 modulus reading keeps E smooth)."""
    pos, q, box = _small_water()
    beta = 0.34
    ref = oracle_mod.ewald_recip(pos, q, beta, box)
    errE, errF = [], []
    for K in (12, 24, 48):
        r = oracle_mod.spme(pos, q, (K, K, K), 5, beta, box)
        errE.append(abs(r["energy"] - ref["energy"]) / abs(ref["energy"]))
        errF.append(np.sqrt(np.mean((r["forces"] - ref["forces"]) ** 2) / np.mean(ref["forces"] ** 2)))
    for err in (errE, errF):
        slopes = [math.log2(err[i] / err[i + 1]) for i in range(len(err) - 1)]
        assert min(slopes) >= 4, (err, slopes)
    K = (16, 18, 20)
    r = oracle_mod.spme(pos, q, K, 5, beta, box)
    h = 1e-5
    for i in (0, 31):
        for d in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[i, d] += h
            pm[i, d] -= h
            fd = -(oracle_mod.spme(pp, q, K, 5, beta, box)["energy"] - oracle_mod.spme(pm, q, K, 5, beta, box)["energy"]) / (2 * h)
            assert r["forces"][i, d] == pytest.approx(fd, rel=1e-6, abs=1e-9)
