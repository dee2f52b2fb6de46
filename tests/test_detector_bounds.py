"""The tube system's sure-miss rule against the oracle's detector (CPU only).

The fused kernels count a scattered packet as missed, without tracing it through the
detector, when on its way out to the tube ring its height is already beyond every row or
its horizontal direction points away from the arc of tubes (bounds from the geometry,
section 2.4.3 "Ray tracing in a detector system"; margins 1 mm and 1 mrad; the sample's
radius sets how far a start point can shift the crossing angle).  This restates that rule
and checks, on packets drawn inside the sample with directions concentrated next to the
bounds, that the oracle's detector finds every packet the rule skips missing -- so the rule
never drops a detection -- and that the rule skips a substantial share of packets.  The
GPU side is pinned by the fused FP64 parity runs (equal detected and missed counts).
"""
import dataclasses
import math

import numpy as np
import pytest

import mcv_inputs as mi
import oracle


def _bounds(det, r_s):
    r_in = det.radius_m - det.tube_r_m - 1e-3
    top = max(y + 0.5 * det.tube_len_m for y in det.row_y_m) + 1e-3
    bot = min(y - 0.5 * det.tube_len_m for y in det.row_y_m) - 1e-3
    period = det.tubes_per_pack * det.tube_pitch_m + det.pack_gap_m
    widen = math.asin(r_s / r_in) + math.asin(det.tube_r_m / r_in) + 1e-3
    lo = det.phi0_rad - widen
    hi = det.phi0_rad + max(det.packs) * period / det.radius_m + widen
    if not hi - lo < math.pi - 0.01:  # the direction test is off for arcs near half a turn
        lo = hi = None
    return r_in, top, bot, lo, hi


def _surely_misses(b, r, d):
    r_in, top, bot, lo, hi = b
    lmin = r_in - (abs(r[0]) + abs(r[2]))
    assert lmin > 0
    # room left above (below) the start against the rise over the shortest path out
    a = top - r[1] if d[1] >= 0 else r[1] - bot
    if a <= 0 or a * a * (d[0] ** 2 + d[2] ** 2) < (d[1] * lmin) ** 2:
        return True
    if lo is None:
        return False
    return (d[0] * math.cos(lo) - d[2] * math.sin(lo) < 0 or
            d[2] * math.sin(hi) - d[0] * math.cos(hi) < 0)


def _directions(rng, n, b):
    """Unit vectors: half uniform on the sphere, half next to the height and arc bounds."""
    r_in, top, bot, lo, hi = b
    out = []
    for k in range(n):
        if k % 2 == 0:
            v = rng.normal(size=3)
        else:
            # elevation next to the height bound, or azimuth next to an arc end
            if lo is None or rng.random() < 0.5:
                phi = rng.uniform(-math.pi, math.pi)
                t = (top if rng.random() < 0.5 else bot) / r_in
                el = math.atan(t) + rng.normal(scale=0.01)
            else:
                phi = (lo if rng.random() < 0.5 else hi) + rng.normal(scale=0.01)
                el = rng.uniform(-0.4, 0.4)
            v = np.array([math.cos(el) * math.sin(phi), math.sin(el), math.cos(el) * math.cos(phi)])
        out.append(v / np.linalg.norm(v))
    return out


@pytest.mark.parametrize("packs", [(38, 39, 38), (20, 22, 20)])
def test_rule_never_skips_a_detection(packs):
    wl = mi.powder_in_can(n=1)
    det = dataclass_with_wide_window(wl.detector, packs)
    wl = wl.replace(detector=det)
    r_s = max(s.dims[1] for s in wl.scatterers)  # hollow cylinders: outer radius
    b = _bounds(det, r_s)
    rng = np.random.default_rng(8)
    speed = 4000.0
    n, skipped, detected = 6000, 0, 0
    for d in _directions(rng, n, b):
        # a start point inside the can's bounding cylinder
        a, rad = rng.uniform(0, 2 * math.pi), r_s * math.sqrt(rng.random())
        r = np.array([rad * math.sin(a), rng.uniform(-0.02, 0.02), rad * math.cos(a)])
        h = oracle.detect(wl, r, speed * d, 0.0, 1.0, 0.5)
        if h["bin"] >= 0:
            detected += 1
        if _surely_misses(b, r, d):
            skipped += 1
            assert h["bin"] == -1, (r, d, h)
    assert detected > 300
    assert b[3] is not None  # both arcs are under half a turn: the direction test is on
    assert skipped > 0.4 * n


def dataclass_with_wide_window(det, packs):
    return dataclasses.replace(det, tof_min_s=0.0, tof_max_s=1.0, packs=packs)
