"""Pins of the oracle against what the paper and the mathematics fix (CPU only).

Each test checks the oracle against something other than itself: a library routine
(cuRAND's host Philox generator), closed forms (transmission, mean scatter weight, chord
lengths, truncated-exponential depth), an independent numpy quadrature (flat angular
distribution of the isotropic kernel), brute force (tube search over all tubes), kinematic
identities (Q = ki - kf, E = Ei - Ef), the kernel's defining density (weighted (Q,E) tally
reproduces S(Q,E) Q / 2ki^2), the paper-literal recursion (statistical agreement), and
central finite differences of the loss (gradient).
"""
import ctypes
import math
import os

import numpy as np
import pytest

import mcv_inputs as mi
import oracle

# CODATA 2018 restated here, independently of the oracle
M_N, HBAR, QE = 1.67492749804e-27, 1.054571817e-34, 1.602176634e-19
C_EV = 0.5 * M_N / (QE * 1e-3)      # meV per (m/s)^2
C_KV = M_N / HBAR * 1e-10           # 1/A per m/s
KT300 = 1.380649e-23 * 300.0 / (QE * 1e-3)


def speed_of(e_mev):
    return math.sqrt(e_mev / C_EV)


# ---------------------------------------------------------------- random numbers
def _curand():
    for name in ("libcurand.so", "libcurand.so.10",
                 os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "lib64",
                              "libcurand.so")):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    return None


def curand_host_philox(seed, offset, n_words):
    """cuRAND's host-side PHILOX4_32_10 generator (runs on the CPU, no GPU needed)."""
    cr = _curand()
    if cr is None:
        pytest.skip("libcurand not available")
    g = ctypes.c_void_p()
    assert cr.curandCreateGeneratorHost(ctypes.byref(g), 161) == 0  # PHILOX4_32_10
    assert cr.curandSetPseudoRandomGeneratorSeed(g, ctypes.c_ulonglong(seed)) == 0
    assert cr.curandSetGeneratorOffset(g, ctypes.c_ulonglong(offset)) == 0
    out = np.zeros(n_words, dtype=np.uint32)
    assert cr.curandGenerate(g, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n_words)) == 0
    cr.curandDestroyGenerator(g)
    return out


@pytest.mark.parametrize("seed", [0, 0x12345678, 0xFFFFFFFF_00000001, 0x0123456789ABCDEF])
def test_philox_matches_curand_host_generator(seed):
    # cuRAND's host generator emits, in its default ordering, the block with counter
    # (j // 65536, 0, j % 65536, 0) at position j, with key (seed_lo, seed_hi); the element
    # offset shifts j.  Compare blocks reaching all key words and counter words 0-2.
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for block0 in (0, 65536 * 3 + 5, 65536 * (2**32 + 7)):
        words = curand_host_philox(seed, 4 * block0, 4 * 24)
        for i in range(24):
            j = block0 + i
            ctr = [(j // 65536) & 0xFFFFFFFF, (j // 65536) >> 32, j % 65536, 0]
            assert list(oracle.philox(ctr, key)) == list(words[4 * i: 4 * i + 4]), (seed, j)


def test_philox_fourth_counter_word_is_mixed():
    a = oracle.philox([1, 2, 3, 0], [4, 5])
    b = oracle.philox([1, 2, 3, 1], [4, 5])
    assert np.count_nonzero(a != b) == 4


def test_uniform_mapping_and_uniformity():
    # orc_uniforms uses key (seed, sim) and counter (nid_lo, nid_hi, 4*(event+1)+block, 0);
    # the double is (53 bits + 1/2) 2^-53
    seed, sim, nid, ev, blk = 7, 3, (5 << 32) + 11, 2, 1
    w = oracle.philox([11, 5, 4 * (ev + 1) + blk, 0], [seed, sim])
    u = oracle.uniforms(seed, sim, nid, ev, blk)
    k0 = (int(w[0]) << 21) | (int(w[1]) >> 11)
    k1 = (int(w[2]) << 21) | (int(w[3]) >> 11)
    assert u[0] == (k0 + 0.5) / 2.0**53 and u[1] == (k1 + 0.5) / 2.0**53
    us = np.array([oracle.uniforms(0, 0, i, 0, 0) for i in range(20000)]).ravel()
    assert us.min() > 0.0 and us.max() < 1.0
    counts, _ = np.histogram(us, bins=50, range=(0, 1))
    exp = us.size / 50
    chi2 = ((counts - exp) ** 2 / exp).sum()
    assert chi2 < 100  # 49 dof; p ~ 1e-5 cut
    # successive draws are uncorrelated
    assert abs(np.corrcoef(us[0::2], us[1::2])[0, 1]) < 0.03


# ---------------------------------------------------------------- geometry
def _brute_chord(inside, r, d, smax=0.05, n=200001):
    s = np.linspace(0.0, smax, n)
    p = r[None, :] + s[:, None] * d[None, :]
    return inside(p).sum() * (s[1] - s[0])


def test_shape_chords_closed_forms():
    cyl = mi.Scatterer(mi.SOLID_CYL, (0.005, 0.02), 0.06, 0.0, [(mi.K_ISO, 1.0)])
    segs = oracle.shape_segments(cyl, [0, 0, -0.5], [0, 0, 1])
    assert len(segs) == 1 and abs(segs[0][1] - segs[0][0] - 0.01) < 1e-13
    assert abs(segs[0][0] - 0.495) < 1e-13
    b = 0.003
    segs = oracle.shape_segments(cyl, [b, 0, -0.5], [0, 0, 1])
    assert abs(segs[0][1] - segs[0][0] - 2 * math.sqrt(0.005**2 - b**2)) < 1e-13
    # top face clips a steep ray; start inside
    d = np.array([0.0, 0.6, 0.8])
    segs = oracle.shape_segments(cyl, [0, 0, 0], d)
    assert len(segs) == 1 and segs[0][0] == 0.0
    assert abs(segs[0][1] - min(0.01 / 0.6, 0.005 / 0.8)) < 1e-15
    hol = mi.Scatterer(mi.HOLLOW_CYL, (0.008, 0.010, 0.04), 0.06, 0.0, [(mi.K_ISO, 1.0)])
    segs = oracle.shape_segments(hol, [0, 0, -0.5], [0, 0, 1])
    assert len(segs) == 2
    assert all(abs((s1 - s0) - 0.002) < 1e-13 for s0, s1 in segs)
    blk = mi.Scatterer(mi.BLOCK, (0.02, 0.02, 0.02), 0.06, 0.0, [(mi.K_ISO, 1.0)],
                       rot_y=math.radians(45))
    segs = oracle.shape_segments(blk, [0, 0, -0.5], [0, 0, 1])
    assert abs(segs[0][1] - segs[0][0] - 0.02 * math.sqrt(2)) < 1e-13
    # a ray missing everything
    assert oracle.shape_segments(cyl, [0.01, 0, -0.5], [0, 0, 1]) == []


def test_shape_chords_brute_force():
    rng = np.random.default_rng(1)
    hol = mi.Scatterer(mi.HOLLOW_CYL, (0.008, 0.010, 0.04), 0.06, 0.0, [(mi.K_ISO, 1.0)])
    blk = mi.Scatterer(mi.BLOCK, (0.02, 0.015, 0.01), 0.06, 0.0, [(mi.K_ISO, 1.0)],
                       rot_y=0.3)

    def in_hollow(p):
        rho2 = p[:, 0] ** 2 + p[:, 2] ** 2
        return (rho2 < 0.010**2) & (rho2 > 0.008**2) & (np.abs(p[:, 1]) < 0.02)

    def in_block(p):
        c, s = math.cos(0.3), math.sin(0.3)
        xb = c * p[:, 0] - s * p[:, 2]
        zb = s * p[:, 0] + c * p[:, 2]
        return (np.abs(xb) < 0.01) & (np.abs(p[:, 1]) < 0.0075) & (np.abs(zb) < 0.005)

    for shape, inside in ((hol, in_hollow), (blk, in_block)):
        for _ in range(12):
            r = rng.uniform(-0.012, 0.012, 3) + np.array([0, 0, -0.025])
            d = rng.normal(size=3) * np.array([0.3, 0.3, 1.0]) + np.array([0, 0, 1.0])
            d /= np.linalg.norm(d)
            segs = oracle.shape_segments(shape, r, d)
            total = sum(s1 - s0 for s0, s1 in segs)
            assert abs(total - _brute_chord(inside, r, d)) < 2e-6


# ---------------------------------------------------------------- transmission & weights
def mu_tot_config1(speed):
    return 100.0 * 0.0603 * (5.0 + 0.23 * 2200.0 / speed)   # 1/m


def test_transmission_closed_form():
    wl = mi.config1(n=5000)
    r = oracle.trace(wl, packets=False, hist=False)
    T = math.exp(-mu_tot_config1(speed_of(60.0)) * 0.01)
    assert abs(r["tallies"][oracle.T_BEAMSTOP] / wl.n - T) < 1e-12 * T
    assert abs(T - 0.73308) < 1e-5   # mu_s = 0.3015 /cm, mu_abs(3388 m/s) = 0.009006 /cm


def test_mean_scatter_weight_closed_form():
    wl = mi.config1(n=200_000)
    r = oracle.trace(wl, packets=False, events=True, hist=False)
    ev = r["events"]
    w = ev["w"][ev["order"] == 1]
    assert w.size == wl.n
    mu = mu_tot_config1(speed_of(60.0))
    mus = 100.0 * 0.0603 * 5.0
    expect = mus / mu * (1 - math.exp(-mu * 0.01))
    assert abs(expect - 0.25918) < 1e-5
    assert abs(w.mean() - expect) < 5 * w.std() / math.sqrt(w.size)


def test_thin_sample_single_and_double_scattering():
    base = mi.config1(n=100_000)

    def run(scale, orders):
        s = base.scatterers[0]
        s2 = mi.Scatterer(s.kind, s.dims, s.n_per_A3, s.sig_abs_b * scale,
                          [(mi.K_ISO, 5.0 * scale)])
        wl = base.replace(scatterers=[s2], max_orders=orders)
        return oracle.trace(wl, hist=False)["packets"]

    pk = run(1e-3, 1)
    w1 = pk["w"][pk["order"] == 1].sum() / base.n
    musL = 100 * 0.0603 * 5e-3 * 0.01
    mutL = mu_tot_config1(speed_of(60.0)) * 1e-3 * 0.01
    assert abs(w1 / musL - 1) < 2 * mutL
    ratios = []
    for scale in (0.2, 0.1):
        pk = run(scale, 2)
        ratios.append(pk["w"][pk["order"] == 2].sum() / pk["w"][pk["order"] == 1].sum())
    # order-2 / order-1 scales like mu_s L in the thin limit
    assert 1.8 < ratios[0] / ratios[1] < 2.2


def test_no_orders_and_min_prob_and_empty():
    wl = mi.config1(n=1000).replace(max_orders=0)
    r = oracle.trace(wl)
    assert r["hist"].sum() == 0.0 and np.all(r["packets"]["order"] == 0)
    wl = mi.config1(n=1000).replace(min_prob=0.302)
    r = oracle.trace(wl)
    # every scattered weight is below mu_s L = 0.3015
    assert np.all(r["packets"]["order"] <= 0)
    wl = mi.config1(n=1000).replace(min_prob=0.29)
    r = oracle.trace(wl)
    assert np.any(r["packets"]["order"] == 1)
    wl = mi.config1(n=1000).replace(min_prob=1.5)
    r = oracle.trace(wl)
    assert np.all(r["packets"]["order"] == -1)  # even the incident packet is dropped
    r = oracle.trace(mi.config1(), n=0)
    assert r["hist"].sum() == 0.0 and r["packets"].size == 0


def test_additive_over_neutron_ranges():
    wl = mi.config2(n=3000).replace(detector=mi.tube_detector(n_tof=50))
    a = oracle.trace(wl, 0, 1000, packets=False)
    b = oracle.trace(wl, 1000, 2000, packets=False)
    c = oracle.trace(wl, 0, 3000, packets=False)
    np.testing.assert_allclose(a["hist"] + b["hist"], c["hist"], rtol=1e-13, atol=1e-300)
    np.testing.assert_allclose(a["tallies"] + b["tallies"], c["tallies"], rtol=1e-13)


# ---------------------------------------------------------------- isotropic kernel
def _gauss(n, a, b):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (b - a) * x + 0.5 * (b + a), 0.5 * (b - a) * w


def test_flat_angular_distribution_against_quadrature():
    """Per-pixel single-scattering intensity of the isotropic kernel (config 1) against a
    deterministic quadrature of  int dz mu_s e^{-mu (z + r)} int_pixel dOmega/4pi
    e^{-mu L_out(z, Omega)}  over the solid cylinder and each detector pixel."""
    # a strongly absorbing cylinder and a tall detector make the expected intensity vary
    # by a large factor across pixels, in both the angular and the vertical index
    base = mi.config1(n=300_000)
    s = base.scatterers[0]
    sig_abs = 30.0
    det = mi.Detector(kind=mi.DET_SURFACE, tof_min_s=4.2e-3, tof_max_s=4.8e-3, n_tof=60,
                      radius_m=3.0, height_m=6.0, n_phi=32, n_y=32)
    wl = base.replace(scatterers=[mi.Scatterer(s.kind, s.dims, s.n_per_A3, sig_abs, s.kernels)],
                      detector=det)
    res = oracle.trace(wl)
    pk = res["packets"]
    hit = pk[(pk["order"] == 1) & (pk["bin"] >= 0)]
    npix = det.n_pixels
    H = np.bincount(hit["pixel"], weights=hit["w_det"], minlength=npix)
    V = np.bincount(hit["pixel"], weights=hit["w_det"] ** 2, minlength=npix)
    assert abs(H.sum() - res["hist"].sum()) < 1e-9 * H.sum()
    # quadrature
    r0, h0, R, Hd = 0.005, 0.02, det.radius_m, det.height_m
    mu = 100.0 * 0.0603 * (5.0 + sig_abs * 2200.0 / speed_of(60.0))
    mus = 100 * 0.0603 * 5.0
    zq, zw = _gauss(16, -r0, r0)
    expect = np.zeros((det.n_phi, det.n_y))
    gp, gw = np.polynomial.legendre.leggauss(6)
    for ip in range(det.n_phi):
        p0 = -math.pi + ip * 2 * math.pi / det.n_phi
        phis = p0 + (gp + 1) * math.pi / det.n_phi
        wphi = gw * math.pi / det.n_phi
        for iy in range(det.n_y):
            y0 = -Hd / 2 + iy * Hd / det.n_y
            ys = y0 + (gp + 1) * 0.5 * Hd / det.n_y
            wy = gw * 0.5 * Hd / det.n_y
            Z, PH, Y = np.meshgrid(zq, phis, ys, indexing="ij")
            W = zw[:, None, None] * wphi[None, :, None] * wy[None, None, :]
            D = np.stack([R * np.sin(PH), Y, R * np.cos(PH) - Z], -1)
            dist = np.linalg.norm(D, axis=-1)
            u = D / dist[..., None]
            dOm = R * (R - Z * np.cos(PH)) / dist**3
            a = u[..., 0] ** 2 + u[..., 2] ** 2
            b = Z * u[..., 2]
            c = Z**2 - r0**2
            s_cyl = (-b + np.sqrt(b * b - a * c)) / a
            s_y = np.where(u[..., 1] != 0, (h0 / 2) / np.abs(u[..., 1] + 1e-300), np.inf)
            Lout = np.minimum(s_cyl, s_y)
            f = mus * np.exp(-mu * (Z + r0)) * np.exp(-mu * Lout) * dOm / (4 * math.pi)
            expect[ip, iy] = (W * f).sum()
    E = expect.ravel() * wl.n
    z = (H - E) / np.sqrt(np.maximum(V, 1e-30))
    assert np.abs(z).max() < 5.0
    assert 0.8 < (z**2).mean() < 1.25
    # the distribution is not flat in pixel space (solid angle and exit paths vary),
    # which is what makes this a check of the pixel mapping too
    Em = E.reshape(det.n_phi, det.n_y)
    assert Em.mean(1).max() / Em.mean(1).min() > 1.3 and Em.mean(0).max() / Em.mean(0).min() > 2.0


def test_event_kinematics_identities():
    """Q = |ki - kf| and E = Ei - Ef of every scatter, from the packet velocities."""
    wl = mi.config2(n=3000).replace(detector=None)
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
            assert abs(np.linalg.norm(qv) - e["q"]) < 1e-9 * e["q"]
            assert abs(C_EV * (vi @ vi - vf @ vf) - e["e"]) < 1e-9
            assert abs(C_KV * np.linalg.norm(vi) - e["ki"]) < 1e-12 * e["ki"]
            assert wl.sqe.e_min <= e["e"] <= min(wl.sqe.e_max, C_EV * (vi @ vi))
            checked += 1
    assert checked > 1000


def test_sqe_kernel_tally_reproduces_table():
    """Weighted (Q,E) tally of S(Q,E) scatters at fixed Ei equals S(Q,E) Q / (2 ki^2)."""
    table = mi.sqe_table()
    grid = mi.SqeGrid(table)
    wl = mi.config2(n=1).replace(sqe=grid)
    rng = np.random.default_rng(5)
    ei = 100.0
    speed = speed_of(ei)
    ki = C_KV * speed
    N = 60000
    qs, es, fs = np.empty(N), np.empty(N), np.empty(N)
    d = np.array([0.0, 0.0, 1.0])
    for i in range(N):
        out = oracle.kernel_scatter(wl, mi.K_SQE, speed, d, rng.random(4))
        if out is None:
            qs[i] = es[i] = fs[i] = np.nan
            continue
        ev = out["event"]
        qs[i], es[i], fs[i] = ev["q"], ev["e"], out["factor"]
        # scattering angle matches Q
        c2t = out["d"] @ d
        kf = ev["kf"]
        assert abs(ki * ki + kf * kf - 2 * ki * kf * c2t - ev["q"] ** 2) < 1e-9
    ok = ~np.isnan(fs)
    qs, es, fs = qs[ok], es[ok], fs[ok]
    bq, be = 10, 20   # coarse blocks of table bins
    dq, de = 12.0 / 200, 180.0 / 400
    tal = np.zeros((200 // bq, 400 // be))
    var = np.zeros_like(tal)
    iq = (qs / (dq * bq)).astype(int)
    ie = ((es + 90.0) / (de * be)).astype(int)
    np.add.at(tal, (iq, ie), fs)
    np.add.at(var, (iq, ie), fs**2)
    qc = (np.arange(200) + 0.5) * dq
    ec = -90.0 + (np.arange(400) + 0.5) * de
    S = table.astype(np.float64)
    expect_fine = S * qc[:, None] * dq * de / (2 * ki * ki)
    # second moment of the weight factor: F^2 times the sampling density 1/(dE dQ(E))
    kf_c = C_KV * np.sqrt(np.maximum(ei - ec, 1e-9) / C_EV)
    dQ_c = np.minimum(ki + kf_c, 12.0) - np.abs(ki - kf_c)
    m2_fine = (S * qc[:, None]) ** 2 * 180.0 * dQ_c[None, :] / (4 * ki**4) * dq * de
    zs = []
    for a in range(tal.shape[0]):
        for b in range(tal.shape[1]):
            q0, q1 = a * bq * dq, (a + 1) * bq * dq
            e0, e1 = -90 + b * be * de, -90 + (b + 1) * be * de
            inside = True
            for E in (e0, e1):
                kf = C_KV * speed_of(ei - E)
                if not (abs(ki - kf) <= q0 and q1 <= min(ki + kf, 12.0)):
                    inside = False
            if not inside:
                continue
            blk = (slice(a * bq, (a + 1) * bq), slice(b * be, (b + 1) * be))
            ex = expect_fine[blk].sum() * N
            vx = m2_fine[blk].sum() * N
            if vx <= 0.0:
                assert tal[a, b] == 0.0
                continue
            zs.append((tal[a, b] - ex) / math.sqrt(vx))
    zs = np.array(zs)
    assert zs.size > 50
    assert np.abs(zs).max() < 5 and 0.7 < (zs**2).mean() < 1.4


def test_sqe_table_detailed_balance():
    t = mi.sqe_table().astype(np.float64)
    e = -90 + (np.arange(400) + 0.5) * 0.45
    pos = e > 0
    m = (t[:, pos] > 1e-20) & (t[:, ~pos][:, ::-1] > 1e-30)
    ratio = np.where(m, t[:, ~pos][:, ::-1], 1.0) / np.where(m, t[:, pos], 1.0)
    expect = np.exp(-e[pos] / KT300)
    np.testing.assert_allclose(ratio[m], np.broadcast_to(expect, ratio.shape)[m], rtol=1e-5)


# ---------------------------------------------------------------- detector
def test_surface_detector_pixels_and_tof():
    wl = mi.config1()
    det = wl.detector
    speed = 3000.0
    for ip, iy in ((0, 0), (5, 17), (16, 31), (31, 3)):
        phi = -math.pi + (ip + 0.5) * 2 * math.pi / det.n_phi
        y = -0.5 + (iy + 0.5) / det.n_y
        D = np.array([3 * math.sin(phi), y, 3 * math.cos(phi)])
        dist = np.linalg.norm(D)
        out = oracle.detect(wl, [0, 0, 0], D / dist * speed, 1e-3, 0.7, 0.5)
        assert out["pixel"] == ip * det.n_y + iy
        assert abs(out["tof"] - (1e-3 + dist / speed)) < 1e-15
        assert out["w_det"] == 0.7
    # above the detector
    out = oracle.detect(wl, [0, 0, 0], [0, 3000.0, 100.0], 1e-3, 1.0, 0.5)
    assert out["bin"] == -1


def _tube_centres(det):
    period = det.tubes_per_pack * det.tube_pitch_m + det.pack_gap_m
    cent = []
    off = 0
    for row in range(det.n_rows):
        for p in range(det.packs[row]):
            for k in range(det.tubes_per_pack):
                phi = det.phi0_rad + (p * period + (k + 0.5) * det.tube_pitch_m) / det.radius_m
                cent.append((row, off + p, k, phi))
        off += det.packs[row]
    return cent


def test_tube_detector_known_rays():
    wl = mi.config2(n=1)
    det = wl.detector
    speed = speed_of(80.0)
    mu = 100 * det.he3_n_per_A3 * det.he3_sig_abs_b * 2200 / speed
    cents = _tube_centres(det)
    for idx in (0, 7, 8, 300, 312, 919):
        row, pack, k, phi = cents[idx]
        if row != 1:
            continue
        d = np.array([math.sin(phi), 0.0, math.cos(phi)])
        out = oracle.detect(wl, [0, 0, 0], d * speed, 0.0, 1.0, 0.5)
        assert out["pixel"] // det.pixels_per_tube == pack * det.tubes_per_pack + k
        assert out["pixel"] % det.pixels_per_tube == det.pixels_per_tube // 2
        L = 2 * det.tube_r_m
        assert abs(out["w_det"] - (1 - math.exp(-mu * L))) < 1e-13
        # depth: the truncated exponential at u = 1/2
        pabs = 1 - math.exp(-mu * L)
        x = -math.log(1 - 0.5 * pabs) / mu
        assert abs(out["tof"] - (det.radius_m - det.tube_r_m + x) / speed) < 1e-15
    # a ray through a pack gap misses
    period = det.tubes_per_pack * det.tube_pitch_m + det.pack_gap_m
    phi_gap = det.phi0_rad + (period * 3 - 0.5 * det.pack_gap_m) / det.radius_m
    out = oracle.detect(wl, [0, 0, 0], [math.sin(phi_gap) * 1000, 0, math.cos(phi_gap) * 1000],
                        0.0, 1.0, 0.5)
    assert out["bin"] == -1


def test_absorption_depth_mean():
    wl = mi.config2(n=1)
    det = wl.detector
    speed = speed_of(30.0)
    mu = 100 * det.he3_n_per_A3 * det.he3_sig_abs_b * 2200 / speed
    L = 2 * det.tube_r_m
    _, _, _, phi = _tube_centres(det)[39 * 8 + 100]
    d = np.array([math.sin(phi), 0.0, math.cos(phi)])
    us = (np.arange(4000) + 0.5) / 4000
    xs = [oracle.detect(wl, [0, 0, 0], d * speed, 0.0, 1.0, u)["tof"] * speed
          - (det.radius_m - det.tube_r_m) for u in us]
    expect = 1 / mu - L * math.exp(-mu * L) / (1 - math.exp(-mu * L))
    assert abs(np.mean(xs) - expect) < 1e-6 * expect + 1e-9


def test_tube_search_against_brute_force():
    """First tube hit by the oracle's candidate search == first tube of all 920."""
    wl = mi.config2(n=1)
    det = wl.detector
    cents = _tube_centres(det)
    R = det.radius_m
    rng = np.random.default_rng(3)
    n_ok = n_tot = n_edge = 0
    for _ in range(3000):
        r = rng.uniform(-0.01, 0.01, 3)
        d = rng.normal(size=3)
        d[1] *= 0.4
        d /= np.linalg.norm(d)
        best, best_in, best_out = None, np.inf, None
        for ti, (row, pack, k, phi) in enumerate(cents):
            cx, cz = R * math.sin(phi), R * math.cos(phi)
            ox, oz = r[0] - cx, r[2] - cz
            a = d[0] ** 2 + d[2] ** 2
            b = ox * d[0] + oz * d[2]
            c = ox * ox + oz * oz - det.tube_r_m**2
            disc = b * b - a * c
            if disc <= 0:
                continue
            s1, s2 = (-b - math.sqrt(disc)) / a, (-b + math.sqrt(disc)) / a
            ylo = det.row_y_m[row] - det.tube_len_m / 2
            yhi = ylo + det.tube_len_m
            t1, t2 = sorted(((ylo - r[1]) / d[1], (yhi - r[1]) / d[1]))
            si, so = max(s1, t1, 0.0), min(s2, t2)
            if so > si and si < best_in:
                best, best_in, best_out = ti, si, so
        out = oracle.detect(wl, r, d * 3000.0, 0.0, 1.0, 0.5)
        got = None if out["bin"] == -1 else out["pixel"] // det.pixels_per_tube
        exp = None if best is None else cents[best][1] * det.tubes_per_pack + cents[best][2]
        n_tot += 1
        if got == exp:
            n_ok += 1
            if got is not None:
                mu = 100 * det.he3_n_per_A3 * det.he3_sig_abs_b * 2200 / 3000.0
                assert abs(out["w_det"] - (1 - math.exp(-mu * (best_out - best_in)))) < 1e-9
        else:
            # the candidate search takes the row at the crossing of the tube-centre circle:
            # only rays crossing a row edge there may differ
            sR = (-(r[0] * d[0] + r[2] * d[2]) + math.sqrt((r[0] * d[0] + r[2] * d[2]) ** 2
                  - (d[0] ** 2 + d[2] ** 2) * (r[0] ** 2 + r[2] ** 2 - R * R))) / (d[0] ** 2 + d[2] ** 2)
            yR = r[1] + sR * d[1]
            edges = [y + s * det.tube_len_m / 2 for y in det.row_y_m for s in (-1, 1)]
            assert min(abs(yR - e) for e in edges) < 0.02
            n_edge += 1
    assert n_ok >= n_tot - 5 and n_tot - n_ok == n_edge


# ---------------------------------------------------------------- paper-literal recursion
def test_chain_rewrite_agrees_with_paper_recursion():
    """The bounded chain (scatter point over all segments ahead) and the paper's recursion
    (scatterM / interactM_path1 / interactM1: first segment only) estimate the same
    histogram; the unscattered beam-stop weight agrees neutron by neutron."""
    det = mi.tube_detector(n_tof=25, packs=(38, 39, 38), pixels_per_tube=128)
    base = mi.config2(n=1).replace(detector=det)
    nb, per = 16, 12_000
    hc, hp = [], []
    for b in range(nb):
        wl = base.replace(seed=100 + b, n=per)
        c = oracle.trace(wl, packets=False)
        p = oracle.trace_paper(wl)
        assert abs(c["tallies"][oracle.T_BEAMSTOP] - p["tallies"][oracle.T_BEAMSTOP]) < \
            1e-12 * c["tallies"][oracle.T_BEAMSTOP]
        # per pack (115 coarse bins)
        shape = (115, det.tubes_per_pack * det.pixels_per_tube * det.n_tof)
        hc.append(c["hist"].reshape(shape).sum(1))
        hp.append(p["hist"].reshape(shape).sum(1))
    hc, hp = np.array(hc), np.array(hp)
    mc, mp = hc.mean(0), hp.mean(0)
    se = np.sqrt(hc.var(0, ddof=1) / nb + hp.var(0, ddof=1) / nb)
    m = se > 0
    z = (mc[m] - mp[m]) / se[m]
    assert np.abs(z).max() < 5 and (z**2).mean() < 1.6
    tot_c, tot_p = hc.sum(1), hp.sum(1)
    zt = (tot_c.mean() - tot_p.mean()) / math.sqrt(tot_c.var(ddof=1) / nb + tot_p.var(ddof=1) / nb)
    assert abs(zt) < 4


# ---------------------------------------------------------------- gradient
def _grad_case(n=1500):
    det = mi.tube_detector(n_tof=40, packs=(38, 39, 38), pixels_per_tube=16)
    wl = mi.config2(n=n).replace(detector=det)
    tw = wl.replace(sqe=mi.SqeGrid(mi.sqe_table(omega_scale=1.05)), seed=1)
    ref = oracle.trace(tw, packets=False)["hist"]
    c = 1e4 / ref.sum()
    target = mi.poisson_target(ref, c, seed=2)
    return wl, target, c


def test_gradient_against_central_differences():
    wl, target, c = _grad_case()
    g = oracle.grad(wl, target, c)
    assert abs(g["loss"] - oracle.loss(wl, target, c)) < 1e-12 * g["loss"]
    # sigma_abs, sigma_s of the sample
    for i, name in ((0, "abs"), (1, "s")):
        s = wl.scatterers[0]
        v = s.sig_abs_b if i == 0 else s.kernels[0][1]
        h = 1e-4 * v
        ls = []
        for sgn in (1, -1):
            if i == 0:
                s2 = mi.Scatterer(s.kind, s.dims, s.n_per_A3, v + sgn * h, s.kernels)
            else:
                s2 = mi.Scatterer(s.kind, s.dims, s.n_per_A3, s.sig_abs_b, [(s.kernels[0][0], v + sgn * h)])
            ls.append(oracle.loss(wl.replace(scatterers=[s2]), target, c))
        fd = (ls[0] - ls[1]) / (2 * h)
        assert abs(fd - g["dsig"][i]) < 1e-3 * abs(fd), (name, fd, g["dsig"][i])
    # table entries with non-zero gradient
    rng = np.random.default_rng(3)
    dsq = g["dsqe"].ravel()
    nz = np.flatnonzero((np.abs(dsq) > 1e-3 * np.abs(dsq).max()) & (wl.sqe.table.ravel() > 0))
    for e in rng.choice(nz, size=8, replace=False):
        tab0 = wl.sqe.table
        vals = []
        for sgn in (1, -1):
            t = tab0.copy()
            t.ravel()[e] = np.float32(tab0.ravel()[e] * (1 + sgn * 1e-4))
            vals.append((float(t.ravel()[e]), oracle.loss(wl.replace(sqe=mi.SqeGrid(t)), target, c)))
        fd = (vals[0][1] - vals[1][1]) / (vals[0][0] - vals[1][0])
        an = g["dsqe"].ravel()[e]
        assert abs(fd - an) < 1e-3 * abs(an), (e, fd, an)


def test_gradient_zero_table_entry_continues_path():
    """The adjoint of an entry whose value is exactly 0 is still the derivative: paths are
    traced through the zero factor.  The loss is quadratic in one table entry (unless a path
    uses the entry twice), so a central difference around 0 with a large step is exact up to
    rounding (min_prob is lowered so that the negative weights of the lower point are kept)."""
    wl, target, c = _grad_case(n=6000)
    wl = wl.replace(min_prob=-1e300)
    g = oracle.grad(wl, target, c)
    dsq = g["dsqe"].ravel()
    # entries whose derivative stands above the rounding noise of the loss differences
    zero = np.flatnonzero((wl.sqe.table.ravel() == 0) & (np.abs(dsq) > 1e-7))
    assert zero.size > 0
    for e in zero[:3]:
        vals = []
        for sgn in (1, -1):
            t = wl.sqe.table.copy()
            t.ravel()[e] = np.float32(sgn * 0.1)
            vals.append((float(t.ravel()[e]), oracle.loss(wl.replace(sqe=mi.SqeGrid(t)), target, c)))
        fd = (vals[0][1] - vals[1][1]) / (vals[0][0] - vals[1][0])
        an = g["dsqe"].ravel()[e]
        assert abs(fd - an) < 1e-3 * abs(an), (e, fd, an)


def test_multi_tube_detector_absorbs_the_remainder():
    """The detector system as a composite of absorbing tubes (the paper's section 2.4.3): a
    packet running nearly along the tube ring crosses several candidate tubes; each absorbs
    1 - e^{-mu L} of the weight the earlier ones left, L the chord through it (computed here
    from the closest approach of the line to the tube axis), at a depth drawn from the
    truncated exponential."""
    import dataclasses
    det = dataclasses.replace(mi.tube_detector(), multi_tube=True)
    wl = mi.config2(n=1).replace(detector=det)
    R, rt = det.radius_m, det.tube_r_m
    period = det.tubes_per_pack * det.tube_pitch_m + det.pack_gap_m
    checked = 0
    cases = [(pack, tube, off, tilt) for pack in (10, 40, 77) for tube in (1, 4)
             for off, tilt in ((0.004, 0.02), (0.002, 0.01), (0.006, 0.03))]
    for pack, tube, off, tilt in cases:
        # a tube of row 1 (y = 0) and a ray just inside the ring, heading along it
        phic = det.phi0_rad + (pack * period + (tube + 0.5) * det.tube_pitch_m) / R
        phi0 = phic - 0.045
        rad = R - off
        r0 = np.array([rad * math.sin(phi0), 0.013, rad * math.cos(phi0)])
        tang = np.array([math.cos(phi0), 0.0, -math.sin(phi0)])
        d = tang + np.array([math.sin(phi0), 0.0, math.cos(phi0)]) * tilt
        d /= np.linalg.norm(d)
        speed = speed_of(50.0)
        u = np.array([0.3, 0.7, 0.5])
        hits = oracle.detect_multi(wl, r0, speed * d, 1e-3, 1.0, u)
        if len(hits) < 2:
            continue
        # the expected chain: the three candidates around where the ray leaves the ring
        sR = -(r0[0] * d[0] + r0[2] * d[2]) / (d[0] ** 2 + d[2] ** 2)
        a = d[0] ** 2 + d[2] ** 2
        cr = r0[0] * d[2] - r0[2] * d[0]
        sR += math.sqrt(R * R * a - cr * cr) / a
        P = r0 + sR * d
        arc = (math.atan2(P[0], P[2]) - det.phi0_rad) * R
        p = math.floor(arc / period)
        k = min(math.floor((arc - p * period) / det.tube_pitch_m), det.tubes_per_pack - 1)
        g = p * det.tubes_per_pack + k
        mu = 100 * det.he3_n_per_A3 * det.he3_sig_abs_b * 2200.0 / speed
        chords = []
        for c in (g - 1, g, g + 1):
            pc, tc = divmod(c, det.tubes_per_pack)
            ph = det.phi0_rad + (pc * period + (tc + 0.5) * det.tube_pitch_m) / R
            axis = np.array([R * math.sin(ph), R * math.cos(ph)])
            rel = np.array([r0[0], r0[2]]) - axis
            dh = np.array([d[0], d[2]])
            t_c = -(rel @ dh) / (dh @ dh)
            b2 = (rel @ rel) - (rel @ dh) ** 2 / (dh @ dh)
            if b2 >= rt * rt:
                continue
            half = math.sqrt((rt * rt - b2) / (dh @ dh))
            s_in, s_out = max(t_c - half, 0.0), t_c + half
            if s_out > s_in:
                chords.append((s_in, s_out, c))
        chords.sort()
        assert len(chords) == len(hits)
        left = 1.0
        for (s_in, s_out, c), (b, pix, tof, wd), ui in zip(chords, hits, u):
            pabs = -math.expm1(-mu * (s_out - s_in))
            assert abs(wd - left * pabs) < 1e-12 * left * pabs
            x = -math.log1p(-ui * pabs) / mu
            assert abs(tof - (1e-3 + (s_in + x) / speed)) < 1e-12 * tof
            assert pix // det.pixels_per_tube == (sum(det.packs[:1]) * det.tubes_per_pack + c)
            left *= 1 - pabs
        checked += 1
    assert checked >= 4, checked


def test_paper_recursion_with_multi_tube_detector_agrees_with_chain():
    """With the multi-tube detector the paper mode still estimates the chain's histogram:
    packets from the sample cross one tube (a single layer), so the remainder that goes on
    changes nothing beyond Monte Carlo error."""
    import dataclasses
    det = dataclasses.replace(mi.tube_detector(n_tof=25), multi_tube=True)
    base = mi.config2(n=1).replace(detector=det)
    tc, tp = [], []
    for b in range(8):
        wl = base.replace(seed=200 + b, n=8000)
        tc.append(oracle.trace(wl, packets=False)["tallies"][oracle.T_WDET])
        tp.append(oracle.trace_paper(wl)["tallies"][oracle.T_WDET])
    tc, tp = np.array(tc), np.array(tp)
    z = (tc.mean() - tp.mean()) / math.sqrt(tc.var(ddof=1) / 8 + tp.var(ddof=1) / 8)
    assert abs(z) < 4
