"""Pins of the oracle's coherent elastic powder kernel (supplement S4, the Debye-Scherrer
cross section), CPU only.

  - Bragg's law: every scatter leaves on the cone of an allowed reflection, |ki - kf| =
    2 pi / d_tau with kf = ki, i.e. lambda = 2 d sin(theta_B).
  - The reflection picked follows the per-atom Debye-Scherrer cross sections, written here
    as sigma_tau = lambda^2 d_tau w_tau / 2 (lambda^3 / (4 sin theta_B) with sin theta_B =
    lambda / 2d), chi-square over the reflections at several wavelengths.
  - The weight is the summed cross section over the kernel's nominal one, at every wavelength;
    it steps at the Bragg edges lambda = 2 d_tau and vanishes beyond the last (no scattering).
  - The azimuth about the incident direction is uniform.
  - The reflection list: spacings of an fcc lattice a / sqrt(h^2 + k^2 + l^2) with h, k, l of
    one parity, multiplicities summing to the number of lattice vectors in the shell.
"""
import math

import numpy as np
import pytest

import mcv_inputs as mi
import oracle

stats = pytest.importorskip("scipy.stats")

M_N, HBAR, QE = 1.67492749804e-27, 1.054571817e-34, 1.602176634e-19
C_EV = 0.5 * M_N / (QE * 1e-3)
C_KV = M_N / HBAR * 1e-10


def _speed_for_lambda(lam):
    return 2 * math.pi / lam / C_KV


@pytest.fixture(scope="module")
def wl():
    return mi.aluminium_powder(n=1)


def _scatter(wl, lam, u, d=(0.0, 0.0, 1.0)):
    return oracle.kernel_scatter(wl, mi.K_BRAGG, _speed_for_lambda(lam), np.array(d), u)


def test_fcc_reflection_list():
    br = mi.fcc_reflections(a=4.05, d_min=0.5)
    s2 = np.rint((4.05 / br.d) ** 2).astype(int)
    assert list(s2[:6]) == [3, 4, 8, 11, 12, 16]          # (111) (200) (220) (311) (222) (400)
    # multiplicities: (111) 8, (200) 6, (220) 12, (311) 24, (222) 8
    v0, b2 = 4.05 ** 3, (3.449e-13) ** 2 / 1e-24
    q = 2 * math.pi / br.d
    m = br.w * v0 * 4.0 / (16 * b2 * np.exp(-q * q * 0.053334 / 3.0))
    np.testing.assert_allclose(m[:5], [8, 6, 12, 24, 8], rtol=1e-12)
    assert np.all(np.diff(br.d) < 0)


@pytest.mark.parametrize("lam", [0.9, 1.5, 2.2, 4.2])
def test_bragg_law_and_reflection_probabilities(wl, lam):
    br = wl.bragg
    sig_k = wl.scatterers[0].kernels[0][1]
    allowed = br.d > lam / 2
    sig = lam ** 2 * br.d * br.w / 2.0
    sig = np.where(allowed, sig, 0.0)
    rng = np.random.default_rng(int(lam * 100))
    N = 20000 if allowed.any() else 200
    counts = np.zeros(br.d.size)
    ki = 2 * math.pi / lam
    phis = []
    for _ in range(N):
        out = _scatter(wl, lam, rng.random(4))
        if not allowed.any():
            assert out is None
            continue
        ev = out["event"]
        # the weight: the summed Debye-Scherrer cross section over the kernel's nominal one
        assert abs(out["factor"] - sig.sum() / sig_k) < 1e-12 * sig.sum() / sig_k
        assert abs(ev["kf"] - ki) < 1e-12 * ki and abs(ev["ki"] - ki) < 1e-12 * ki
        t = int(ev["mode"])
        assert allowed[t]
        assert abs(ev["q"] - 2 * math.pi / br.d[t]) < 1e-10 * ev["q"]
        # lambda = 2 d sin(theta_B), theta_B = half the angle between d_in and d_out
        c2t = float(out["d"][2])
        sin_tb = math.sqrt(max(0.0, (1 - c2t) / 2))
        assert abs(2 * br.d[t] * sin_tb - lam) < 1e-9 * lam
        counts[t] += 1
        phis.append(math.atan2(out["d"][1], out["d"][0]))
    if not allowed.any():
        return
    p = sig / sig.sum()
    use = p * N > 5
    chi2 = ((counts[use] - N * p[use]) ** 2 / (N * p[use])).sum()
    dof = int(use.sum()) - 1
    assert stats.chi2.sf(chi2, max(dof, 1)) > 1e-4, (chi2, dof)
    assert counts[~allowed].sum() == 0
    assert stats.kstest((np.array(phis) + math.pi) / (2 * math.pi), stats.uniform.cdf).pvalue > 1e-3


def test_bragg_edges(wl):
    br = wl.bragg
    rng = np.random.default_rng(3)
    for t in range(3):
        edge = 2 * br.d[t]
        below = _scatter(wl, edge * (1 - 1e-9), rng.random(4))
        above = _scatter(wl, edge * (1 + 1e-9), rng.random(4))
        sig_k = wl.scatterers[0].kernels[0][1]
        if t == 0:
            assert above is None            # beyond the last Bragg edge nothing scatters
        else:
            # crossing the edge of reflection t removes exactly its cross section
            lam = edge
            jump = lam ** 2 * br.d[t] * br.w[t] / 2.0 / sig_k
            assert abs((below["factor"] - above["factor"]) - jump) < 1e-6 * below["factor"]
        assert below is not None
