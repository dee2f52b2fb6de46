"""Pins of the oracle's single-crystal Born-von Karman one-phonon kernel (CPU only).

Dispersion: closed forms at the X point, numpy's symmetric eigen-solver (library routine) on
random wave vectors, lattice periodicity, inversion symmetry and the linear acoustic limit.
Kernel: energy and momentum conservation of every sampled event, and its mean weight for a
given outgoing direction against a brute-force integral of the double-differential cross
section over Ef (delta function smeared over a fine grid, thermal factor written as
(coth(hw/2kT) +- 1)/2 as in the paper's supplement S4).
"""
import math

import numpy as np
import pytest

import mcv_inputs as mi
import oracle

HBAR, QE, KB, AMU = 1.054571817e-34, 1.602176634e-19, 1.380649e-23, 1.66053906660e-27
M_N = 1.67492749804e-27
C_EV = 0.5 * M_N / (QE * 1e-3)
C_KV = M_N / HBAR * 1e-10
A = 4.05
WL = mi.config3()
BONDS = np.array([[1, 1, 0], [1, -1, 0], [1, 0, 1], [1, 0, -1], [0, 1, 1], [0, 1, -1]], float)


def dynmat(q, phi=10.0, mass=27 * AMU, a=A):
    """Force-constant model restated: 12 nearest neighbours (a/2)(+-1,+-1,0) etc., central
    springs: D = phi/M sum (1 - cos q.delta) d d^T (1/s^2), q in 1/A."""
    q = np.atleast_2d(q)
    D = np.zeros((q.shape[0], 3, 3))
    for n in BONDS:
        c = 2.0 * phi / mass * (1 - np.cos(0.5 * a * (q @ n))) * 0.5
        D += c[:, None, None] * np.outer(n, n)[None]
    return D


def hw_of(lam):
    return HBAR * np.sqrt(np.maximum(lam, 0)) / (QE * 1e-3)


def test_x_point_closed_forms():
    hw, _ = oracle.bvk_modes(WL, [2 * math.pi / A, 0, 0])
    t = HBAR * math.sqrt(4 * 10.0 / (27 * AMU)) / (QE * 1e-3)
    l = HBAR * math.sqrt(8 * 10.0 / (27 * AMU)) / (QE * 1e-3)
    np.testing.assert_allclose(hw, [t, t, l], rtol=1e-12)
    assert abs(l - 27.80) < 0.01 and abs(t - 19.66) < 0.01


def test_modes_against_numpy_eigh():
    rng = np.random.default_rng(11)
    for q in rng.uniform(-3, 3, size=(200, 3)):
        hw, ev = oracle.bvk_modes(WL, q)
        lam, vec = np.linalg.eigh(dynmat(q)[0])
        np.testing.assert_allclose(hw, hw_of(lam), rtol=1e-9, atol=1e-9)
        gaps = np.diff(lam) / lam.max()
        for b in range(3):
            isolated = (b == 0 or gaps[b - 1] > 1e-6) and (b == 2 or gaps[b] > 1e-6)
            if isolated:
                assert abs(abs(ev[:, b] @ vec[:, b]) - 1) < 1e-8
        np.testing.assert_allclose(ev.T @ ev, np.eye(3), atol=1e-8)


def test_periodicity_inversion_acoustic_limit():
    rng = np.random.default_rng(12)
    G = [2 * math.pi / A * np.array(v, float) for v in ((1, 1, 1), (2, 0, 0), (1, -1, 1), (0, 2, 2))]
    for q in rng.uniform(-2, 2, size=(50, 3)):
        h0, _ = oracle.bvk_modes(WL, q)
        for g in G:
            h1, _ = oracle.bvk_modes(WL, q + g)
            np.testing.assert_allclose(h1, h0, rtol=1e-9, atol=1e-9)
        h2, _ = oracle.bvk_modes(WL, -q)
        np.testing.assert_allclose(h2, h0, rtol=1e-12, atol=1e-12)
    d = np.array([0.3, 0.5, 0.81])
    d /= np.linalg.norm(d)
    h1, _ = oracle.bvk_modes(WL, 1e-4 * d)
    h2, _ = oracle.bvk_modes(WL, 2e-4 * d)
    np.testing.assert_allclose(h2 / h1, 2.0, rtol=1e-6)


def _lab_to_crystal(v, rot):
    c, s = math.cos(rot), math.sin(rot)
    bx, by, bz = c * v[..., 0] - s * v[..., 2], v[..., 1], s * v[..., 0] + c * v[..., 2]
    return np.stack([bz, bx, by], -1)


def test_events_conserve_energy_and_momentum():
    rng = np.random.default_rng(13)
    ei = 50.0
    speed = math.sqrt(ei / C_EV)
    ki = C_KV * speed
    rot = math.radians(23.0)
    n_ok = 0
    for _ in range(400):
        out = oracle.kernel_bvk(WL, rot, speed, [0, 0, 1], rng.random(4))
        if not out["ok"]:
            continue
        ev = out["event"]
        kf = C_KV * out["speed"]
        Qlab = ki * np.array([0, 0, 1.0]) - kf * out["d"]
        assert abs(np.linalg.norm(Qlab) - ev["q"]) < 1e-9 * ev["q"]
        E = ei - C_EV * out["speed"] ** 2
        assert abs(E - ev["e"]) < 1e-9
        hw, _ = oracle.bvk_modes(WL, _lab_to_crystal(Qlab, rot))
        b, s = ev["mode"] % 3, (1 if ev["mode"] < 3 else -1)
        assert abs(E - s * hw[b]) < 1e-9 * max(1.0, abs(E))
        n_ok += 1
    assert n_ok > 100


def _brute_force_direction(df, rot, ei, n_grid=1_600_000):
    """sum over modes and roots of (kf/ki) e^{-2W} R_b N_s / |g'|, as the integral over Ef
    of the same integrand times a narrow box around g = 0."""
    speed = math.sqrt(ei / C_EV)
    ki = C_KV * speed
    kT = KB * 300.0 / (QE * 1e-3)
    w_max = 49.0
    ef = np.linspace(1e-6, ei + w_max, n_grid)
    dE = ef[1] - ef[0]
    kf = C_KV * np.sqrt(ef / C_EV)
    Q = ki * np.array([0, 0, 1.0])[None] - kf[:, None] * df[None]
    Qc = _lab_to_crystal(Q, rot)
    lam, vec = np.linalg.eigh(dynmat(Qc))
    hw = hw_of(lam)
    hb2m = HBAR**2 / (2 * 27 * AMU) * 1e20 / (QE * 1e-3)
    dw = np.exp(-np.sum(Qc**2, -1) * mi.Bvk().msd_A2 / 3)
    total = 0.0
    h = 0.02  # meV, width of the box standing in for the delta function
    for b in range(3):
        qe = np.einsum("ni,ni->n", Qc, vec[:, :, b])
        R = hb2m * qe**2 / np.maximum(hw[:, b], 1e-12)
        coth = 1 / np.tanh(hw[:, b] / (2 * kT))
        for s in (1, -1):
            N = 0.5 * (coth + s)
            g = ei - ef - s * hw[:, b]
            box = (np.abs(g) < h / 2) / h
            total += np.sum((kf / ki) * dw * R * N * box) * dE
    return total


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_kernel_mean_weight_against_brute_force(seed):
    rng = np.random.default_rng(seed)
    ei = 50.0
    speed = math.sqrt(ei / C_EV)
    rot = math.radians(rng.uniform(0, 180))
    u0, u1 = rng.random(2)
    # the oracle: exact average over the six modes and over the roots of each mode
    total = 0.0
    for m in range(6):
        u2 = (m + 0.5) / 6
        probe = oracle.kernel_bvk(WL, rot, speed, [0, 0, 1], [u0, u1, u2, 0.5])
        nr = int(probe["event"]["nroots"])
        for r in range(nr):
            out = oracle.kernel_bvk(WL, rot, speed, [0, 0, 1], [u0, u1, u2, (r + 0.5) / nr])
            if out["ok"]:
                total += out["factor"] / (6 * nr)
    ct = 2 * u0 - 1
    st = 2 * math.sqrt(u0 * (1 - u0))
    df = np.array([st * math.cos(2 * math.pi * u1), st * math.sin(2 * math.pi * u1), ct])
    ref = _brute_force_direction(df, rot, ei)
    assert total > 0
    assert abs(total - ref) < 3e-3 * ref, (total, ref)


# ---- accuracy near degenerate branches, against 40-digit arithmetic -------------------------
def _mp_dynmat(mp, q):
    coef = mp.mpf(10) / (27 * mp.mpf("1.66053906660e-27"))
    D = mp.zeros(3, 3)
    for n in BONDS:
        qd = mp.mpf(A) / 2 * sum(mp.mpf(q[i]) * int(n[i]) for i in range(3))
        c = coef * (1 - mp.cos(qd))
        for i in range(3):
            for j in range(3):
                D[i, j] += c * int(n[i]) * int(n[j])
    return D


def _mp_modes(mp, q):
    E, V = mp.eigsy(_mp_dynmat(mp, q))
    order = sorted(range(3), key=lambda k: E[k])
    lam = [E[k] for k in order]
    vec = [[V[i, k] for i in range(3)] for k in order]
    hbar, mev = mp.mpf("1.054571817e-34"), mp.mpf("1.602176634e-22")
    return [hbar * mp.sqrt(max(x, 0)) / mev for x in lam], lam, vec


def test_near_degenerate_branches_against_40_digit_reference():
    """Along [100] the two transverse branches coincide; slightly off that axis they are
    nearly degenerate (relative gaps 1e-2 .. 1e-7).  The eigenvalues must keep full relative
    accuracy, and each eigenvector its accuracy over the gap (the trigonometric cubic alone
    loses both there)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    base = np.array([2.1, 0.0, 0.0])
    for tilt in (1e-1, 1e-2, 1e-3, 1e-4):
        for direction in ([0, 1, 0], [0, 0.6, 0.8], [0, 1, 1]):
            q = base + tilt * np.array(direction, float)
            hw, ev = oracle.bvk_modes(WL, q)
            hw_ref, lam, vec = _mp_modes(mp, q)
            lmax = float(lam[2])
            for b in range(3):
                assert abs(hw[b] - float(hw_ref[b])) <= 1e-14 * float(hw_ref[2]) * float(hw_ref[2]) / max(float(hw_ref[b]), 1e-300) + 1e-15 * float(hw_ref[b]), (tilt, b)
                gap = min([abs(float(lam[b] - lam[k])) for k in range(3) if k != b])
                dot = abs(sum(ev[i, b] * float(vec[b][i]) for i in range(3)))
                assert 1.0 - dot <= (8e-16 * lmax / gap) ** 2 + 1e-15, (tilt, b, 1.0 - dot)


def _mp_factor(mp, speed, d, u, rot):
    """The one-phonon factor of one event in 40-digit arithmetic: the same sampling (u), the
    roots of g bracketed on the same 32 sub-intervals and solved to full precision."""
    hbar, mn, e = mp.mpf("1.054571817e-34"), mp.mpf("1.67492749804e-27"), mp.mpf("1.602176634e-19")
    kB, amu = mp.mpf("1.380649e-23"), mp.mpf("1.66053906660e-27")
    mevv2 = mn / 2 / (e * mp.mpf("1e-3"))
    kpv = mn / hbar * mp.mpf("1e-10")
    mev_j = 1 / (e * mp.mpf("1e-3"))
    M = 27 * amu
    coef = mp.mpf(10) / M
    c, sn = mp.cos(rot), mp.sin(rot)
    u = [mp.mpf(x) for x in u]
    d = [mp.mpf(x) for x in d]
    speed = mp.mpf(speed)
    ct = 2 * u[0] - 1
    st = 2 * mp.sqrt(u[0] * (1 - u[0]))
    ph = 2 * mp.pi * u[1]
    df = (st * mp.cos(ph), st * mp.sin(ph), ct)
    mode = min(max(int(mp.floor(6 * u[2])), 0), 5)
    b, s = mode % 3, (1 if mode < 3 else -1)
    Ei, ki = mevv2 * speed**2, kpv * speed

    def at(E):
        kf = kpv * mp.sqrt(E / mevv2)
        Q = [ki * d[i] - kf * df[i] for i in range(3)]
        bx, by, bz = c * Q[0] - sn * Q[2], Q[1], sn * Q[0] + c * Q[2]
        Qc = (bz, bx, by)
        Ev, V = mp.eigsy(_mp_dynmat(mp, Qc))
        k = sorted(range(3), key=lambda j: Ev[j])[b]
        hw = hbar * mp.sqrt(max(Ev[k], 0)) * mev_j
        return Ei - E - s * hw, hw, Qc, [V[i, k] for i in range(3)], kf

    wmax = hbar * mp.sqrt(24 * coef) * mev_j
    lo = 0 if s > 0 else Ei
    hi = Ei if s > 0 else Ei + wmax
    step = (hi - lo) / 32
    gk = [at(lo + k * step)[0] for k in range(33)]
    br = [k for k in range(32) if (gk[k] > 0) != (gk[k + 1] > 0)]
    pick = min(max(int(mp.floor(u[3] * len(br))), 0), len(br) - 1)
    kb = br[pick]
    Ef = mp.findroot(lambda E: at(E)[0], (lo + kb * step, lo + (kb + 1) * step),
                     solver="anderson")
    g, hw, Qc, ev, kf = at(Ef)
    gp = mp.diff(lambda E: at(E)[0], Ef)
    kT = kB * 300 * mev_j
    nB = 1 / (mp.exp(hw / kT) - 1)
    Ns = nB + 1 if s > 0 else nB
    qe = sum(Qc[i] * ev[i] for i in range(3))
    Q2 = sum(x * x for x in Qc)
    dw = mp.exp(-Q2 * mp.mpf(mi.Bvk().msd_A2) / 3)
    Rb = hbar**2 / (2 * M) * mp.mpf("1e20") * mev_j * qe * qe / hw
    return 6 * len(br) * (kf / ki) * dw * Rb * Ns / abs(gp)


def test_kernel_factor_against_40_digit_reference():
    """Sampled events of the crystal run (multiple scattering, 30 degrees): the oracle's
    factor agrees with the 40-digit evaluation within a few epsilon times the event's share
    of the condition estimate."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    wl = mi.config3(rot_deg=30.0, n=400)
    o = oracle.trace(wl, packets=True)
    pk = o["packets"]
    S = wl.max_orders + 1
    rng = np.random.default_rng(5)
    cand = [(i, k) for i in range(wl.n) for k in range(1, S) if pk["order"][i * S + k] >= 0]
    checked = 0
    for j in rng.choice(len(cand), 12, replace=False):
        i, k = cand[j]
        prev, cur = i * S + k - 1, i * S + k
        v = np.array([pk["vx"][prev], pk["vy"][prev], pk["vz"][prev]])
        sp = float(np.linalg.norm(v))
        u = np.concatenate([oracle.uniforms(wl.seed, wl.sim_id, i, k - 1, 1),
                            oracle.uniforms(wl.seed, wl.sim_id, i, k - 1, 2)])
        got = oracle.kernel_scatter(wl, mi.K_BVK, sp, v / sp, u)
        ref = _mp_factor(mp, sp, v / sp, u, mp.radians(30))
        err = abs(got["factor"] / float(ref) - 1.0)
        dk = pk["kappa"][cur] - pk["kappa"][prev]
        assert err <= 4 * 2.2e-16 * dk + 1e-15, (i, k, err, dk)
        checked += 1
    assert checked == 12


# ---- root bracketing against a dense scan ----------------------------------------------------
def _g_dense(ef, df, rot, ei, b, s):
    """g(Ef) = Ei - Ef - s hw_b(Q(Ef)) at many Ef (numpy eigh, branches ascending)."""
    speed = math.sqrt(ei / C_EV)
    ki = C_KV * speed
    kf = C_KV * np.sqrt(np.maximum(ef, 0.0) / C_EV)
    Q = ki * np.array([0, 0, 1.0])[None] - kf[:, None] * df[None]
    lam = np.linalg.eigvalsh(dynmat(_lab_to_crystal(Q, rot)))
    return ei - ef - s * hw_of(lam[:, b])


def test_roots_against_dense_scan():
    """The 32-sub-interval bracketing of g (section S4 single-crystal kernel, our reading):
    every root the oracle solves is a root of g found independently (dense scan with numpy's
    eigen-solver, refined by Brent's method) in the same sub-interval; a sub-interval holds
    an odd number of dense roots exactly when the oracle brackets one there; and the roots the
    bracketing cannot see (pairs inside one sub-interval) are rare."""
    brentq = pytest.importorskip("scipy.optimize").brentq
    rng = np.random.default_rng(21)
    ei = 50.0
    speed = math.sqrt(ei / C_EV)
    w_max = HBAR * math.sqrt(24 * 10.0 / (27 * AMU)) / (QE * 1e-3)
    n_dense, n_missed, n_checked = 0, 0, 0
    for _ in range(60):
        rot = math.radians(rng.uniform(0, 180))
        u0, u1 = rng.random(2)
        ct, st = 2 * u0 - 1, 2 * math.sqrt(u0 * (1 - u0))
        df = np.array([st * math.cos(2 * math.pi * u1), st * math.sin(2 * math.pi * u1), ct])
        for m in range(6):
            b, s = m % 3, (1 if m < 3 else -1)
            lo, hi = (0.0, ei) if s > 0 else (ei, ei + w_max)
            step = (hi - lo) / 32
            u2 = (m + 0.5) / 6
            nr = int(oracle.kernel_bvk(WL, rot, speed, [0, 0, 1], [u0, u1, u2, 0.5])
                     ["event"]["nroots"])
            # dense scan: 128 points per sub-interval, sub-interval ends included
            ef = lo + step * np.arange(32 * 128 + 1) / 128
            g = _g_dense(ef, df, rot, ei, b, s)
            roots = []
            for k in np.flatnonzero((g[:-1] > 0) != (g[1:] > 0)):
                f = lambda e: _g_dense(np.array([e]), df, rot, ei, b, s)[0]  # noqa: E731
                roots.append(brentq(f, ef[k], ef[k + 1], xtol=1e-13, rtol=1e-15))
            roots = np.array(roots)
            sub = np.minimum(((roots - lo) / step).astype(int), 31)
            bracketed = [k for k in range(32) if (g[128 * k] > 0) != (g[128 * (k + 1)] > 0)]
            assert len(bracketed) == nr, (rot, u0, u1, m, bracketed, nr)
            for k in range(32):
                assert (np.sum(sub == k) % 2 == 1) == (k in bracketed)
            n_dense += len(roots)
            n_missed += len(roots) - nr
            for r in range(nr):
                out = oracle.kernel_bvk(WL, rot, speed, [0, 0, 1], [u0, u1, u2, (r + 0.5) / nr])
                if not out["ok"]:
                    continue
                e_f = C_EV * out["speed"] ** 2
                cand = roots[sub == bracketed[r]]
                assert np.min(np.abs(cand - e_f)) < 1e-7, (e_f, cand)
                n_checked += 1
    assert n_checked > 200
    assert n_missed <= 0.01 * n_dense, (n_missed, n_dense)
