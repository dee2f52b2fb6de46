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
