"""Pins of the oracle's synthetic source and of its kernel choice (CPU only).

The source (the stand-in for the beam simulation of the paper's section 3, first step) is
pinned by what its description fixes, independently of how the oracle writes it:
  - the incident energy is normal with mean Ei and standard deviation ei_rel_sigma * Ei
    (Kolmogorov-Smirnov test, and the sample mean and standard deviation within their
    statistical errors -- a FWHM read as a standard deviation is off by 2.35x);
  - the start point is uniform on the width x height rectangle centred on the beam axis in
    the plane z = -z0 (KS test against the uniform law, and the extremes reach the edges);
  - the horizontal and vertical divergence angles, atan(vx/vz) and atan(vy/vz), are each
    normal with standard deviation div_sigma_rad and independent of each other (KS tests,
    correlation, and the squared radial angle following the chi-square law with 2 degrees
    of freedom -- the same trigonometric function on both axes would correlate them);
  - the time is the flight from a source l1 upstream of the sample centre along the drawn
    direction: t = (l1 - z0) / vz for every neutron.
Kernel choice (section 2.4.2, a kernel composite; section 2.4.3, "selecting a kernel"):
in a scatterer with two kernels, kernel k is picked with probability sigma_k / (sigma_1 +
sigma_2) and the weight does not depend on the choice (binomial tests on the events).
"""
import math

import numpy as np
import pytest

import mcv_inputs as mi
import oracle

stats = pytest.importorskip("scipy.stats")

# CODATA 2018 restated here, independently of the oracle
M_N, QE = 1.67492749804e-27, 1.602176634e-19
C_EV = 0.5 * M_N / (QE * 1e-3)      # meV per (m/s)^2


def _beam_only(beam, n):
    """A workload without sample or detector: the order-0 packets are the incident beam."""
    return mi.Workload(name="beam", beam=beam, scatterers=[], detector=None, n=n, max_orders=0)


def _incident(beam, n, seed=0):
    wl = _beam_only(beam, n).replace(seed=seed)
    pk = oracle.trace(wl, packets=True, hist=False)["packets"]
    assert np.all(pk["order"] == 0)
    assert np.all(pk["w"] == 1.0)
    return pk


BEAM = mi.Beam(ei_mev=100.0, ei_rel_sigma=0.01, div_sigma_rad=0.005, width_m=0.05,
               height_m=0.03, z0_m=0.05, l1_m=11.6)
N_BEAM = 200_000


@pytest.fixture(scope="module")
def incident():
    return _incident(BEAM, N_BEAM)


def test_beam_energy_is_normal_with_the_stated_spread(incident):
    v2 = incident["vx"] ** 2 + incident["vy"] ** 2 + incident["vz"] ** 2
    e = C_EV * v2
    mu, sd = BEAM.ei_mev, BEAM.ei_rel_sigma * BEAM.ei_mev
    n = e.size
    assert abs(e.mean() - mu) < 4.0 * sd / math.sqrt(n)
    # standard error of a normal sample's standard deviation: sd / sqrt(2 n)
    assert abs(e.std(ddof=1) - sd) < 4.0 * sd / math.sqrt(2 * n)
    assert stats.kstest((e - mu) / sd, stats.norm.cdf).pvalue > 1e-3


def test_beam_footprint_is_uniform_on_the_rectangle(incident):
    x, y, z = incident["x"], incident["y"], incident["z"]
    assert np.all(z == -BEAM.z0_m)
    hw, hh = 0.5 * BEAM.width_m, 0.5 * BEAM.height_m
    assert np.all(np.abs(x) < hw) and np.all(np.abs(y) < hh)
    # the extremes of N uniform draws lie within ~width / N of the edges
    assert x.min() < -hw + 50 * BEAM.width_m / N_BEAM and x.max() > hw - 50 * BEAM.width_m / N_BEAM
    assert y.min() < -hh + 50 * BEAM.height_m / N_BEAM and y.max() > hh - 50 * BEAM.height_m / N_BEAM
    assert stats.kstest((x + hw) / BEAM.width_m, stats.uniform.cdf).pvalue > 1e-3
    assert stats.kstest((y + hh) / BEAM.height_m, stats.uniform.cdf).pvalue > 1e-3
    # the two coordinates are independent
    assert abs(np.corrcoef(x, y)[0, 1]) < 4.0 / math.sqrt(N_BEAM)


def test_beam_divergence_is_normal_per_axis_and_independent(incident):
    ax = np.arctan2(incident["vx"], incident["vz"])
    ay = np.arctan2(incident["vy"], incident["vz"])
    s = BEAM.div_sigma_rad
    for a in (ax, ay):
        assert abs(a.mean()) < 4.0 * s / math.sqrt(N_BEAM)
        assert abs(a.std(ddof=1) - s) < 4.0 * s / math.sqrt(2 * N_BEAM)
        assert stats.kstest(a / s, stats.norm.cdf).pvalue > 1e-3
    assert abs(np.corrcoef(ax, ay)[0, 1]) < 4.0 / math.sqrt(N_BEAM)
    assert abs(np.corrcoef(ax ** 2, ay ** 2)[0, 1]) < 4.0 / math.sqrt(N_BEAM)
    # (ax^2 + ay^2) / s^2 is chi-square with two degrees of freedom
    r2 = (ax ** 2 + ay ** 2) / s ** 2
    assert stats.kstest(r2, stats.chi2(2).cdf).pvalue > 1e-3
    # the direction is independent of the footprint and of the energy
    e = C_EV * (incident["vx"] ** 2 + incident["vy"] ** 2 + incident["vz"] ** 2)
    for a in (ax, ay):
        for b in (incident["x"], incident["y"], e):
            assert abs(np.corrcoef(a, b)[0, 1]) < 4.0 / math.sqrt(N_BEAM)


def test_beam_time_is_the_flight_from_the_source(incident):
    # the neutron left the source plane z = -l1 at t = 0 and moved along its direction to
    # the start plane z = -z0, i.e. over (l1 - z0) along z at speed vz
    t_ref = (BEAM.l1_m - BEAM.z0_m) / incident["vz"]
    np.testing.assert_allclose(incident["t"], t_ref, rtol=2e-15, atol=0)


def test_pencil_beam_is_exact():
    b = mi.Beam(ei_mev=60.0)
    pk = _incident(b, 1000)
    assert np.all(pk["x"] == 0.0) and np.all(pk["y"] == 0.0)
    assert np.all(pk["vx"] == 0.0) and np.all(pk["vy"] == 0.0)
    np.testing.assert_allclose(pk["vz"], math.sqrt(60.0 / C_EV), rtol=1e-15)
    np.testing.assert_allclose(pk["t"], (b.l1_m - b.z0_m) / math.sqrt(60.0 / C_EV), rtol=1e-15)


def test_beam_streams_differ_by_seed_and_sim():
    a = _incident(BEAM, 2000, seed=0)
    b = _incident(BEAM, 2000, seed=1)
    assert np.count_nonzero(a["x"] == b["x"]) == 0
    c = oracle.trace(_beam_only(BEAM, 2000).replace(sim_id=5), hist=False)["packets"]
    assert np.count_nonzero(a["x"] == c["x"]) == 0


# ---------------------------------------------------------------- kernel choice
def two_kernel_powder(n, sig_iso=1.5, sig_sqe=5.0, ei=100.0):
    return mi.powder_two_kernels(n, sig_iso, sig_sqe, ei)


@pytest.mark.parametrize("sig_iso,sig_sqe", [(1.5, 5.0), (4.0, 1.0)])
def test_kernel_choice_follows_the_cross_sections(sig_iso, sig_sqe):
    wl = two_kernel_powder(60_000, sig_iso, sig_sqe)
    ev = oracle.trace(wl, packets=False, events=True, hist=False)["events"]
    ev = ev[ev["order"] >= 1]
    first = ev[ev["order"] == 1]
    p_iso = sig_iso / (sig_iso + sig_sqe)
    # every scattering, first or later, picks the kernel with the same probability
    for sub in (first, ev):
        n = sub.size
        k = int((sub["kernel"] == mi.K_ISO).sum())
        assert k + int((sub["kernel"] == mi.K_SQE).sum()) == n
        assert abs(k - n * p_iso) < 4.5 * math.sqrt(n * p_iso * (1 - p_iso)) + 1, (k, n, p_iso)
    # the choice does not alter the weight: the scattered weight of the first order, before
    # the kernel's own factor, has the same distribution for both kernels
    # (the kernel's draws are independent of the scattering point, so keeping the events
    # whose kernel factor is not zero keeps that distribution)
    f = first[first["factor"] > 0]
    w_pre = f["w"] / f["factor"]
    a, b = w_pre[f["kernel"] == mi.K_ISO], w_pre[f["kernel"] == mi.K_SQE]
    assert stats.ks_2samp(a, b).pvalue > 1e-3


def test_single_kernel_is_always_chosen():
    wl = two_kernel_powder(5000).replace(scatterers=[mi.powder_sample()])
    ev = oracle.trace(wl, packets=False, events=True, hist=False)["events"]
    ev = ev[ev["order"] >= 1]
    assert ev.size > 0 and np.all(ev["kernel"] == mi.K_SQE)
