"""Pin of the oracle's condition estimate (kappa) against 60-digit arithmetic (CPU only).

kappa sets the tolerance of every FP64 weight comparison (1e-12 + 1e-15 kappa), so it must
bound the rounding error a correct FP64 evaluation can make.  Here each emitted weight of
chains that scatter only in isotropic scatterers is evaluated again with mpmath at 60
digits from the same random numbers (the oracle's Philox uniforms, pinned elsewhere), with
the geometry, attenuation and scattering-point choice of section 2.4.3 restated, and the
oracle's own FP64 error must stay within kappa units of the FP64 epsilon.  The chains
with the largest kappa are checked together with a random sample: those are the points
close to a surface whose next chord is a tiny difference of large distances.
"""
import math

import numpy as np
import pytest

import mcv_inputs as mi
import oracle

mp = pytest.importorskip("mpmath")

EPS = 2.0 ** -52
M_N = "1.67492749804e-27"
Q_E = "1.602176634e-19"


def _cyl(R, r, d):
    a = d[0] ** 2 + d[2] ** 2
    if a == 0:
        return (-mp.inf, mp.inf) if r[0] ** 2 + r[2] ** 2 < R * R else None
    tc = -(r[0] * d[0] + r[2] * d[2]) / a
    cr = r[0] * d[2] - r[2] * d[0]
    g = R * R - cr * cr / a
    if g <= 0:
        return None
    h = mp.sqrt(g / a)
    return tc - h, tc + h


def _slab(half, p, dp):
    if dp == 0:
        return (-mp.inf, mp.inf) if abs(p) < half else None
    a, b = (-half - p) / dp, (half - p) / dp
    return min(a, b), max(a, b)


def _keep(lo, hi, out):
    lo = max(lo, 0)
    if hi > lo:
        out.append((lo, hi))


def _segments(sc, r, d):
    """Material intervals ahead of r along d (section 2.4.2 shapes, the hollow cylinder as a
    difference of two cylinders, the block rotated by rot_y about +y)."""
    dims = [mp.mpf(x) for x in sc.dims]
    out = []
    if sc.kind == mi.SOLID_CYL:
        c, y = _cyl(dims[0], r, d), _slab(dims[1] / 2, r[1], d[1])
        if c and y:
            _keep(max(c[0], y[0]), min(c[1], y[1]), out)
    elif sc.kind == mi.HOLLOW_CYL:
        c, y = _cyl(dims[1], r, d), _slab(dims[2] / 2, r[1], d[1])
        if c and y:
            lo, hi = max(c[0], y[0]), min(c[1], y[1])
            if hi > lo:
                i = _cyl(dims[0], r, d)
                if i:
                    _keep(lo, min(hi, i[0]), out)
                    _keep(max(lo, i[1]), hi, out)
                else:
                    _keep(lo, hi, out)
    else:
        c, s = mp.cos(mp.mpf(sc.rot_y)), mp.sin(mp.mpf(sc.rot_y))
        rb = [c * r[0] - s * r[2], r[1], s * r[0] + c * r[2]]
        db = [c * d[0] - s * d[2], d[1], s * d[0] + c * d[2]]
        lo, hi = -mp.inf, mp.inf
        for k in range(3):
            iv = _slab(dims[k] / 2, rb[k], db[k])
            if iv is None:
                return out
            lo, hi = max(lo, iv[0]), min(hi, iv[1])
        _keep(lo, hi, out)
    return out


def exact_weights(wl, nid, orders):
    """Emitted weights of one neutron's chain of `orders` scatterings at 60 digits
    (isotropic kernels only)."""
    with mp.workdps(60):
        def U(event, block):
            return [mp.mpf(float(x)) for x in oracle.uniforms(wl.seed, wl.sim_id, nid,
                                                              event, block)]
        b = wl.beam
        u = U(-1, 0)
        E = mp.mpf(b.ei_mev) * (1 + mp.mpf(b.ei_rel_sigma) * mp.sqrt(-2 * mp.log(u[0])) *
                                mp.cos(2 * mp.pi * u[1]))
        u = U(-1, 1)
        r = [(u[0] - mp.mpf(0.5)) * mp.mpf(b.width_m), (u[1] - mp.mpf(0.5)) * mp.mpf(b.height_m),
             -mp.mpf(b.z0_m)]
        u = U(-1, 2)
        rho = mp.sqrt(-2 * mp.log(u[0]))
        tx = mp.tan(mp.mpf(b.div_sigma_rad) * rho * mp.cos(2 * mp.pi * u[1]))
        ty = mp.tan(mp.mpf(b.div_sigma_rad) * rho * mp.sin(2 * mp.pi * u[1]))
        nrm = mp.sqrt(tx * tx + ty * ty + 1)
        d = [tx / nrm, ty / nrm, 1 / nrm]
        v = mp.sqrt(E / (mp.mpf(0.5) * mp.mpf(M_N) / (mp.mpf(Q_E) * mp.mpf("1e-3"))))

        def sig_s(sc):
            return sum(mp.mpf(k[1]) for k in sc.kernels)

        def mu_t(sc):
            return 100 * mp.mpf(sc.n_per_A3) * (sig_s(sc) + mp.mpf(sc.sig_abs_b) * 2200 / v)

        w = mp.mpf(1)
        out = []
        for o in range(orders + 1):
            seg = sorted(((a, e, j) for j, sc in enumerate(wl.scatterers)
                          for a, e in _segments(sc, r, d)), key=lambda t: t[0])
            tau = sum(mu_t(wl.scatterers[j]) * (e - a) for a, e, j in seg)
            L = sum(e - a for a, e, j in seg)
            out.append(w * mp.exp(-tau))
            if o == orders or not L > 0:
                break
            ell = U(o, 0)[0] * L
            acc, tau_pt = mp.mpf(0), mp.mpf(0)
            for i, (a, e, j) in enumerate(seg):
                mu = mu_t(wl.scatterers[j])
                if ell < acc + (e - a) or i == len(seg) - 1:
                    s_pt = a + (ell - acc)
                    tau_pt += mu * (ell - acc)
                    sc = wl.scatterers[j]
                    break
                acc += e - a
                tau_pt += mu * (e - a)
            assert sc.kernels[0][0] == mi.K_ISO and len(sc.kernels) == 1
            w = w * 100 * mp.mpf(sc.n_per_A3) * sig_s(sc) * L * mp.exp(-tau_pt)
            r = [r[k] + d[k] * s_pt for k in range(3)]
            uk = U(o, 1)
            st = 2 * mp.sqrt(uk[0] * (1 - uk[0]))
            d = [st * mp.cos(2 * mp.pi * uk[1]), st * mp.sin(2 * mp.pi * uk[1]), 2 * uk[0] - 1]
        return out


def _iso_block():
    return mi.Scatterer(kind=mi.BLOCK, dims=(0.02, 0.01, 0.03), n_per_A3=0.0603,
                        sig_abs_b=0.23, kernels=[(mi.K_ISO, 5.0)], rot_y=math.radians(30.0))


def _workloads():
    can = mi.powder_in_can(n=6000)
    return {
        # chains that stay in the can (the powder uses S(Q,E) and is left out)
        "can-100meV": (can, 1),
        "can-10meV": (mi.powder_in_can(n=6000, ei=10.0), 1),
        "solid-cylinder-5-orders": (mi.config1(n=4000).replace(max_orders=5), 0),
        "rotated-block": (can.replace(scatterers=[_iso_block()], n=4000), 0),
    }


@pytest.mark.parametrize("name", list(_workloads()))
def test_kappa_bounds_the_oracle_rounding_error(name):
    wl, iso = _workloads()[name]
    o = oracle.trace(wl, packets=True, events=True, hist=False, tallies=False)
    pk, ev = o["packets"], o["events"]
    S, M = wl.max_orders + 1, wl.max_orders
    order = pk["order"].reshape(wl.n, S)
    kappa = pk["kappa"].reshape(wl.n, S)
    scat = ev["scatterer"].reshape(wl.n, M)
    n_sc = (order >= 0).sum(1) - 1
    ok = np.array([n_sc[i] >= 1 and np.all(scat[i, :n_sc[i]] == iso) for i in range(wl.n)])
    cand = np.flatnonzero(ok)
    assert cand.size >= 100
    kmax = np.array([kappa[i, :n_sc[i] + 1].max() for i in cand])
    rng = np.random.default_rng(3)
    pick = np.unique(np.concatenate([cand[np.argsort(-kmax)[:40]],
                                     rng.choice(cand, 40, replace=False)]))
    worst_ratio, worst_err = 0.0, 0.0
    for i in pick:
        exact = exact_weights(wl, int(i), int(n_sc[i]))
        assert len(exact) == n_sc[i] + 1, (i, len(exact), n_sc[i])
        for k, x in enumerate(exact):
            if x == 0:
                continue
            err = abs(float((mp.mpf(float(pk["w"][i * S + k])) - x) / x)) / EPS
            worst_err = max(worst_err, err)
            worst_ratio = max(worst_ratio, err / kappa[i, k])
            assert err <= kappa[i, k], (int(i), k, err, kappa[i, k])
    # the sample holds ill-conditioned chains (errors far above a few units of epsilon)
    assert worst_err > 20.0, worst_err
