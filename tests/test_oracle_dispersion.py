"""Pins of the oracle's dispersion-surface kernel (supplement S4: S(Q) delta(E - E(Q)), with the
paper's example surface E(Q) = 2.5 sqrt(1 - (cos(4.4 Qx) cos(4.4 Qz))^2), S(Q) = 1), CPU only.

  - Energy conservation on the surface: for every scatter of a multiple-scattering run,
    Ei - Ef equals the paper's expression evaluated here (numpy, written as the paper prints
    it) at Q = ki - kf taken from the packet velocities and turned into the crystal frame.
  - The roots: against a dense scan of g(Ef) = Ei - Ef - E(Q(Ef)) (64 points per bracketing
    sub-interval), the kernel finds a root in exactly the sub-intervals where g changes sign,
    and its root is a root of the dense g to 1e-9 meV.
  - The weight n_roots (kf/ki) S / |g'| with g' from a central difference of the dense g.
"""
import math

import numpy as np
import pytest

import mcv_inputs as mi
import oracle

M_N, HBAR, QE = 1.67492749804e-27, 1.054571817e-34, 1.602176634e-19
C_EV = 0.5 * M_N / (QE * 1e-3)
C_KV = M_N / HBAR * 1e-10


def e_of_q(q):
    """The paper's example surface, as printed: 2.5*sqrt(1-(cos(4.4*Qx)*cos(4.4*Qz))^2)."""
    return 2.5 * np.sqrt(np.maximum(0.0, 1 - (np.cos(4.4 * q[..., 0]) * np.cos(4.4 * q[..., 2])) ** 2))


def crystal_frame(v, rot):
    """Lab vector in the frame of a crystal rotated by rot about +y ([100] along the beam and
    [001] vertical at zero rotation)."""
    c, s = math.cos(rot), math.sin(rot)
    bx, by, bz = c * v[..., 0] - s * v[..., 2], v[..., 1], s * v[..., 0] + c * v[..., 2]
    return np.stack([bz, bx, by], axis=-1)


def test_events_lie_on_the_dispersion_surface():
    rot = math.radians(30.0)
    wl = mi.dispersion_crystal(8000, rot_deg=30.0).replace(detector=None)
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
            q = crystal_frame(C_KV * vi - C_KV * vf, rot)
            de = C_EV * (vi @ vi - vf @ vf)
            assert abs(de - float(e_of_q(q))) < 1e-9, (de, float(e_of_q(q)))
            assert 0.0 <= de <= 2.5 + 1e-12
            checked += 1
    assert checked > 300


def _g_dense(ei, ki, di, df, efs, rot):
    kf = C_KV * np.sqrt(efs / C_EV)
    q = crystal_frame(ki * di[None, :] - kf[:, None] * df[None, :], rot)
    return ei - efs - e_of_q(q)


@pytest.mark.parametrize("rot_deg", [0.0, 30.0, 77.0])
def test_roots_and_weight_against_a_dense_scan(rot_deg):
    rot = math.radians(rot_deg)
    wl = mi.dispersion_crystal(1, rot_deg=rot_deg)
    rng = np.random.default_rng(int(rot_deg) + 1)
    ei = 7.5
    speed = math.sqrt(ei / C_EV)
    ki = C_KV * speed
    checked = multi = hidden = 0
    for t in range(800):
        # incident directions near the beam axis (first scatterings) and anywhere (later ones)
        di = rng.normal(size=3) * (0.05 if t % 2 else 1.0) + (np.array([0, 0, 1.0]) if t % 2 else 0)
        di /= np.linalg.norm(di)
        u = rng.random(4)
        out = oracle.kernel_scatter(wl, mi.K_DISP, speed, di, u)
        df = out["d"] if out is not None else None
        # the outgoing direction is drawn whatever the roots: recompute it from u
        ct, ph = 2 * u[0] - 1, 2 * math.pi * u[1]
        st = 2 * math.sqrt(u[0] * (1 - u[0]))
        dfu = np.array([st * math.cos(ph), st * math.sin(ph), ct])
        if df is not None:
            np.testing.assert_allclose(df, dfu, atol=1e-15)
        lo, hi = max(0.0, ei - 2.5), ei
        edges = lo + (hi - lo) * np.arange(33) / 32
        fine = lo + (hi - lo) * np.arange(32 * 64 + 1) / (32 * 64)
        g = _g_dense(ei, ki, di, dfu, fine, rot)
        ge = g[::64]
        brackets = [k for k in range(32) if (ge[k] > 0) != (ge[k + 1] > 0)]
        # sign changes of the dense scan inside sub-intervals whose ends agree (a hidden pair)
        for k in range(32):
            seg = g[64 * k: 64 * (k + 1) + 1] > 0
            if seg[0] == seg[-1] and np.any(seg != seg[0]):
                hidden += 1
        if out is None:
            assert not brackets
            continue
        ev = out["event"]
        assert ev["nroots"] == len(brackets)
        multi += len(brackets) > 1
        ef = ei - ev["e"]
        k = int((ef - lo) / ((hi - lo) / 32))
        assert min(abs(k - b) for b in brackets) <= 1
        gr = float(_g_dense(ei, ki, di, dfu, np.array([ef]), rot)[0])
        # |g| at the root within its rounding and the bisection's final width
        assert abs(gr) < 1e-9
        h = 1e-6
        gp = float((_g_dense(ei, ki, di, dfu, np.array([ef + h]), rot)[0] -
                    _g_dense(ei, ki, di, dfu, np.array([ef - h]), rot)[0]) / (2 * h))
        kf = C_KV * math.sqrt(ef / C_EV)
        expect = len(brackets) * (kf / ki) * 1.0 / abs(gp)
        assert abs(out["factor"] - expect) < 1e-6 * expect, (out["factor"], expect)
        checked += 1
    assert checked > 500 and multi > 0, (checked, multi)
    assert hidden == 0
