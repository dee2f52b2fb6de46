"""Pins of the oracle's incoherent phonon kernel (supplement S4: incoherent elastic with the
Debye-Waller factor, incoherent inelastic single-phonon, multi-phonon from the density of
states), CPU only.

  - The phonon tables: every A_n sums to 1, obeys detailed balance A_n(-E) = e^{-E/kT} A_n(E)
    bin by bin, has n times the mean and n times the variance of A_1 (moments of a
    convolution), and equals numpy's convolution of A_1 with A_{n-1}.
  - gamma_0 = int coth(E/2kT) Z(E)/E dE against scipy's adaptive quadrature of the continuous
    density of states the histogram samples (within the histogram's rectangle-rule error),
    for the vanadium-like density and for a Debye density; 2W = hbar^2 Q^2 gamma_0 / 2M.
  - The kernel's weighted (Q, E) tally of single scatters at a fixed incident energy equals
    the integral of (kf/ki) S(Q,E) dOmega/4pi over each (Q, E) block, channel by channel:
    elastic e^{-2W}, one-phonon 2W e^{-2W} A_1 (so proportional to Q^2 at small Q) and
    multi-phonon e^{-2W} sum_n (2W)^n/n! A_n (proportional to Q^4 at small Q); a dropped
    power of 2W or a wrong channel probability fails the z-tests.
  - Q = |ki - kf| and E = Ei - Ef of every scatter of a multiple-scattering run.
"""
import math

import numpy as np
import pytest

import mcv_inputs as mi
import oracle

integrate = pytest.importorskip("scipy.integrate")

# CODATA 2018 restated here, independently of the oracle
M_N, HBAR, QE, KB, U = 1.67492749804e-27, 1.054571817e-34, 1.602176634e-19, 1.380649e-23, 1.66053906660e-27
C_EV = 0.5 * M_N / (QE * 1e-3)      # meV per (m/s)^2
C_KV = M_N / HBAR * 1e-10           # 1/A per m/s
KT300 = KB * 300.0 / (QE * 1e-3)


def speed_of(e_mev):
    return math.sqrt(e_mev / C_EV)


@pytest.fixture(scope="module")
def vwl():
    return mi.vanadium_powder(n=1)


@pytest.fixture(scope="module")
def tables(vwl):
    return oracle.phonon_tables(vwl)


def test_phonon_tables_sum_rules_and_detailed_balance(vwl, tables):
    A, E = tables["A"], tables["E"]
    N = vwl.phonon.nmax
    mean1 = (A[0] * E).sum()
    var1 = (A[0] * E * E).sum() - mean1 ** 2
    for n in range(1, N + 1):
        a = A[n - 1]
        assert abs(a.sum() - 1.0) < 1e-12
        assert np.all(a >= 0.0)
        pos = E > 0
        neg = a[::-1][pos]          # A_n(-E) at the positive energies
        m = a[pos] > 1e-250
        np.testing.assert_allclose(neg[m], a[pos][m] * np.exp(-E[pos][m] / KT300), rtol=1e-11)
        mean = (a * E).sum()
        assert abs(mean - n * mean1) < 1e-10 * abs(n * mean1) + 1e-12
        var = (a * E * E).sum() - mean ** 2
        assert abs(var - n * var1) < 1e-9 * n * var1
    # A_1 has no mass at E = 0 nor beyond the highest mode
    J = vwl.phonon.z.size
    assert A[0][N * J] == 0.0 and np.all(A[0][np.abs(E) > J * vwl.phonon.de + 1e-9] == 0.0)


def test_multiphonon_tables_are_convolutions(vwl, tables):
    A = tables["A"]
    N, J = vwl.phonon.nmax, vwl.phonon.z.size
    c = N * J
    a1 = A[0][c - J: c + J + 1]
    for n in range(2, N + 1):
        prev = A[n - 2][c - (n - 1) * J: c + (n - 1) * J + 1]
        conv = np.convolve(a1, prev)
        got = A[n - 1][c - n * J: c + n * J + 1]
        assert np.abs(conv - got).max() <= 1e-14 * conv.max()


def _gamma0_quad(zfun, e_max, kT, de, f0):
    """gamma_0 of the continuous density zfun by adaptive quadrature, as a sum over the modes
    at j de (j >= 1) sees it: a rectangle rule whose only first-order term is the missing
    half of the end point E = 0, where the integrand tends to f0 (Euler-Maclaurin)."""
    norm = integrate.quad(zfun, 0.0, e_max, limit=400)[0]
    g = integrate.quad(lambda e: zfun(e) / (e * math.tanh(e / (2 * kT))) if e > 0 else f0,
                       0.0, e_max, limit=400)[0]
    return (g - 0.5 * de * f0) / norm


def test_gamma0_and_debye_waller_against_quadrature(vwl, tables):
    de, e_max = vwl.phonon.de, 40.0
    # the vanadium-like density as a continuous function (the histogram samples it at j de)
    def zv(e):
        g = lambda c, s: math.exp(-0.5 * ((e - c) / s) ** 2)
        z = (e / 20.0) ** 2 * math.exp(-(e / 24.0) ** 4) + 0.9 * g(22.0, 2.5) + 1.2 * g(35.0, 1.8)
        return z * min(max((e_max - e) / 2.0, 0.0), 1.0)
    # near E = 0 the density rises as (E/20)^2, so Z / (E tanh(E/2kT)) tends to 2kT/400
    g_ref = _gamma0_quad(zv, e_max, KT300, de, 2 * KT300 / 400.0)
    # the remaining rectangle-rule error is of order (de / 10 meV)^2
    assert abs(tables["gamma0"] - g_ref) < 3e-4 * g_ref, (tables["gamma0"], g_ref)
    hb2m = HBAR ** 2 / (2 * vwl.phonon.mass_u * U) * 1e20 / (QE * 1e-3)  # meV A^2
    assert abs(tables["c_w"] - hb2m * tables["gamma0"]) < 1e-12 * tables["c_w"]
    # a Debye density Z = 3 E^2 / E_D^3 up to E_D = 30 meV, on a fine grid
    ed, dd = 30.0, 0.05
    z = 3 * (dd * np.arange(1, int(ed / dd) + 1)) ** 2 / ed ** 3
    w = vwl.replace(phonon=mi.PhononDos(z=z, de=dd, mass_u=vwl.phonon.mass_u, nmax=2))
    t = oracle.phonon_tables(w)
    # a Debye density stops at E_D with a jump: its end point adds -de f(E_D)/2 as well
    fd = lambda e: 3 * e / (ed ** 3 * math.tanh(e / (2 * KT300)))
    g_d = _gamma0_quad(lambda e: 3 * e * e / ed ** 3, ed, KT300, dd, 6 * KT300 / ed ** 3)
    norm_shift = 0.5 * dd * 3 / ed  # the rectangle sum of Z counts half of Z(E_D) too much
    g_d = (g_d + 0.5 * dd * fd(ed)) / (1.0 + norm_shift)
    assert abs(t["gamma0"] - g_d) < 1e-4 * g_d, (t["gamma0"], g_d)


def _expected_block(ki, Ei, q0, q1, e0, e1, term, de, nq=24):
    """int over E in [e0, e1) and Q in [q0, q1) of term(Q, E) Q / (2 ki^2) over the
    kinematically allowed Q (midpoint rule, two E points per grid bin of width de)."""
    tot = 0.0
    ne = 2 * int(round((e1 - e0) / de))
    for e in e0 + (np.arange(ne) + 0.5) * (e1 - e0) / ne:
        if e >= Ei:
            continue
        kf = C_KV * speed_of(Ei - e)
        lo, hi = max(q0, abs(ki - kf)), min(q1, ki + kf)
        if hi <= lo:
            continue
        q = lo + (np.arange(nq) + 0.5) * (hi - lo) / nq
        tot += (term(q, e) * q / (2 * ki * ki)).sum() * (hi - lo) / nq * (e1 - e0) / ne
    return tot


def test_phonon_kernel_tally_reproduces_the_expansion(vwl, tables):
    """Single scatters at Ei = 100 meV: the weighted tally of each channel in (Q, E) blocks
    against the channel's term of S(Q,E), with A_n from the (separately pinned) tables."""
    ei = 100.0
    speed = speed_of(ei)
    ki = C_KV * speed
    rng = np.random.default_rng(11)
    Ntot = 150000
    d = np.array([0.0, 0.0, 1.0])
    rec = np.empty((Ntot, 4))
    for i in range(Ntot):
        out = oracle.kernel_scatter(vwl, mi.K_PHONON, speed, d, rng.random(4))
        if out is None:
            rec[i] = np.nan
            continue
        ev = out["event"]
        rec[i] = (ev["q"], ev["e"], out["factor"], ev["mode"])
        kf = ev["kf"]
        assert abs(ki * ki + kf * kf - 2 * ki * kf * (out["d"] @ d) - ev["q"] ** 2) < 1e-9
    rec = rec[~np.isnan(rec[:, 0])]
    cw, A, Eg = tables["c_w"], tables["A"], tables["E"]
    de, N = vwl.phonon.de, vwl.phonon.nmax
    p = vwl.phonon.p

    def a_density(n, e):
        # A_n's mass of the grid bin holding e, spread over the bin (width de)
        i = int(round(e / de)) + (A.shape[1] - 1) // 2
        return A[n - 1][i] / de

    terms = {1: lambda q, e: cw * q * q * np.exp(-cw * q * q) * a_density(1, e),
             2: lambda q, e: np.exp(-cw * q * q) * sum(
                 (cw * q * q) ** n / math.factorial(n) * a_density(n, e) for n in range(2, N + 1))}
    zs = {1: [], 2: []}
    qb, eb = 1.0, 16 * de   # blocks: 1/A in Q, sixteen grid bins in E (edges on bin edges)
    for ch in (1, 2):
        r = rec[rec[:, 3] == ch]
        for e0 in np.arange(-40.0, 80.0, eb) - de / 2:
            e1 = e0 + eb
            sel_e = (r[:, 1] >= e0) & (r[:, 1] < e1)
            for q0 in np.arange(0.0, 16.0, qb):
                q1 = q0 + qb
                sel = sel_e & (r[:, 0] >= q0) & (r[:, 0] < q1)
                tal = r[sel, 2].sum()
                var = (r[sel, 2] ** 2).sum()
                ex = Ntot * _expected_block(ki, ei, q0, q1, e0, e1, terms[ch], de)
                if ex <= 0 or sel.sum() < 30:
                    continue
                zs[ch].append((tal - ex) / math.sqrt(var))
    for ch in (1, 2):
        z = np.array(zs[ch])
        assert z.size > 40, (ch, z.size)
        assert np.abs(z).max() < 5.0 and 0.6 < (z ** 2).mean() < 1.5, (ch, np.abs(z).max(), (z ** 2).mean())
    # elastic channel: E = 0, Q = 2 ki sin(theta/2) over the sphere; tally per Q block
    r = rec[rec[:, 3] == 0]
    assert np.all(r[:, 1] == 0.0)
    z0 = []
    for q0 in np.arange(0.0, 2 * ki, 0.5):
        q1 = min(q0 + 0.5, 2 * ki)
        sel = (r[:, 0] >= q0) & (r[:, 0] < q1)
        q = q0 + (np.arange(200) + 0.5) * (q1 - q0) / 200
        ex = Ntot * (np.exp(-cw * q * q) * q / (2 * ki * ki)).sum() * (q1 - q0) / 200
        z0.append((r[sel, 2].sum() - ex) / math.sqrt((r[sel, 2] ** 2).sum()))
    z0 = np.array(z0)
    assert np.abs(z0).max() < 5.0 and 0.5 < (z0 ** 2).mean() < 1.6
    # channel shares
    for ch in range(3):
        k = int((rec[:, 3] == ch).sum())
        assert abs(k - p[ch] * Ntot) < 5 * math.sqrt(Ntot * p[ch] * (1 - p[ch])) + Ntot * 0.002


def test_phonon_event_kinematics_in_a_run():
    wl = mi.vanadium_powder(n=3000).replace(detector=None)
    r = oracle.trace(wl, events=True, hist=False)
    pk = r["packets"].reshape(wl.n, wl.max_orders + 1)
    ev = r["events"].reshape(wl.n, wl.max_orders)
    checked = 0
    for i in range(wl.n):
        for o in range(1, wl.max_orders + 1):
            e = ev[i, o - 1]
            if e["order"] != o or pk[i, o]["order"] != o or pk[i, o - 1]["order"] != o - 1:
                continue
            vi = np.array([pk[i, o - 1][k] for k in ("vx", "vy", "vz")])
            vf = np.array([pk[i, o][k] for k in ("vx", "vy", "vz")])
            qv = C_KV * vi - C_KV * vf
            assert abs(np.linalg.norm(qv) - e["q"]) < 1e-9 * max(e["q"], 1.0)
            assert abs(C_EV * (vi @ vi - vf @ vf) - e["e"]) < 1e-9
            assert e["kernel"] == mi.K_PHONON and e["entry"] == -1
            checked += 1
    assert checked > 1000
