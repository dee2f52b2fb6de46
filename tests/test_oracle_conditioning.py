"""Pin of the oracle's condition estimate (kappa) against 60-digit arithmetic (CPU only).

kappa sets the tolerance of every FP64 weight comparison (1e-12 + 1e-15 kappa), so it must
bound the rounding error a correct FP64 evaluation can make.  Here each emitted weight of
chains through isotropic and powder S(Q,E) scatterers is evaluated again with mpmath at 60
digits from the same random numbers (the oracle's Philox uniforms, pinned elsewhere), with
the geometry, attenuation and scattering-point choice of section 2.4.3 and the S(Q,E)
kinematics of supplement S4 restated (the angle from the law of cosines, the azimuth about
the incoming direction), and the oracle's own FP64 error must stay within kappa units of
the FP64 epsilon.  The chains
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
HBAR = "1.054571817e-34"


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


def _rotate_about(d, c, s, phi):
    """Unit vector at polar angle (cos c, sin s) and azimuth phi about d, with the frame
    e1 = a x d / |a x d| (a the z axis, or the x axis when |d_z| >= 0.9), e2 = d x e1."""
    a = [0, 0, 1] if abs(float(d[2])) < 0.9 else [1, 0, 0]
    e1 = [a[1] * d[2] - a[2] * d[1], a[2] * d[0] - a[0] * d[2], a[0] * d[1] - a[1] * d[0]]
    n1 = mp.sqrt(sum(x * x for x in e1))
    e1 = [x / n1 for x in e1]
    e2 = [d[1] * e1[2] - d[2] * e1[1], d[2] * e1[0] - d[0] * e1[2], d[0] * e1[1] - d[1] * e1[0]]
    cp, sp = mp.cos(phi), mp.sin(phi)
    return [d[k] * c + (e1[k] * cp + e2[k] * sp) * s for k in range(3)]


def _sqe(wl, v, d, u, mev_per_v2, k_per_v):
    """Powder S(Q,E) kernel (supplement S4 form): E uniform on [e_lo, min(e_max, Ei)], Q
    uniform on [|ki - kf|, min(ki + kf, q_max)], the scattering angle from the law of
    cosines, azimuth 2 pi u2, weight S Q dE dQ / (2 ki^2); returns (speed, direction,
    factor, table entry)."""
    g = wl.sqe
    Ei = mev_per_v2 * v * v
    ki = k_per_v * v
    e_lo, e_hi = mp.mpf(g.e_min), min(mp.mpf(g.e_max), Ei)
    dE = e_hi - e_lo
    E = e_lo + u[0] * dE
    Ef = Ei - E
    vf = mp.sqrt(Ef / mev_per_v2)
    kf = k_per_v * vf
    q_lo, q_hi = abs(ki - kf), min(ki + kf, mp.mpf(g.q_max))
    dQ = q_hi - q_lo
    Q = q_lo + u[1] * dQ
    c = (ki * ki + kf * kf - Q * Q) / (2 * ki * kf)
    s = mp.sqrt(max(mp.mpf(0), 1 - c * c))
    nq, ne = g.table.shape
    fq = int(mp.floor(Q / (mp.mpf(g.q_max) / nq)))
    fe = int(mp.floor((E - mp.mpf(g.e_min)) / ((mp.mpf(g.e_max) - mp.mpf(g.e_min)) / ne)))
    entry = fq * ne + fe
    S = mp.mpf(float(g.table.reshape(-1)[entry]))
    d_out = _rotate_about(d, c, s, 2 * mp.pi * u[2])
    return vf, d_out, S * Q * dE * dQ / (2 * ki * ki), entry


def exact_weights(wl, nid, orders, entries=None):
    """Emitted weights of one neutron's chain of `orders` scatterings at 60 digits
    (isotropic and S(Q,E) kernels).  entries: the oracle's table entries per scattering;
    None is returned when a 60-digit draw falls in another bin (a rounding decision at a bin
    edge, not a weight error)."""
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
        mev_per_v2 = mp.mpf(0.5) * mp.mpf(M_N) / (mp.mpf(Q_E) * mp.mpf("1e-3"))
        k_per_v = mp.mpf(M_N) / mp.mpf(HBAR) * mp.mpf("1e-10")
        v = mp.sqrt(E / mev_per_v2)

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
            assert len(sc.kernels) == 1
            w = w * 100 * mp.mpf(sc.n_per_A3) * sig_s(sc) * L * mp.exp(-tau_pt)
            r = [r[k] + d[k] * s_pt for k in range(3)]
            uk = U(o, 1) + U(o, 2)
            if sc.kernels[0][0] == mi.K_ISO:
                st = 2 * mp.sqrt(uk[0] * (1 - uk[0]))
                d = [st * mp.cos(2 * mp.pi * uk[1]), st * mp.sin(2 * mp.pi * uk[1]),
                     2 * uk[0] - 1]
            else:
                assert sc.kernels[0][0] == mi.K_SQE
                v, d, factor, entry = _sqe(wl, v, d, uk, mev_per_v2, k_per_v)
                if entries is not None and entry != entries[o]:
                    return None
                w = w * factor
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
        # every chain: S(Q,E) scatterings in the powder, isotropic ones in the can
        "powder-sqe": (mi.config2(n=3000), None),
        "powder-in-can": (mi.powder_in_can(n=3000), None),
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
    ok = np.array([n_sc[i] >= 1 and (iso is None or np.all(scat[i, :n_sc[i]] == iso))
                   for i in range(wl.n)])
    entry = ev["entry"].reshape(wl.n, M)
    cand = np.flatnonzero(ok)
    assert cand.size >= 100
    kmax = np.array([kappa[i, :n_sc[i] + 1].max() for i in cand])
    rng = np.random.default_rng(3)
    pick = np.unique(np.concatenate([cand[np.argsort(-kmax)[:40]],
                                     rng.choice(cand, 40, replace=False)]))
    worst_ratio, worst_err, checked = 0.0, 0.0, 0
    for i in pick:
        exact = exact_weights(wl, int(i), int(n_sc[i]), entry[i])
        if exact is None:  # a draw on a table bin edge: another bin at 60 digits
            continue
        checked += 1
        assert len(exact) == n_sc[i] + 1, (i, len(exact), n_sc[i])
        for k, x in enumerate(exact):
            if x == 0:
                continue
            err = abs(float((mp.mpf(float(pk["w"][i * S + k])) - x) / x)) / EPS
            worst_err = max(worst_err, err)
            worst_ratio = max(worst_ratio, err / kappa[i, k])
            assert err <= kappa[i, k], (int(i), k, err, kappa[i, k])
    assert checked >= 0.9 * len(pick)
    # the sample holds ill-conditioned chains (errors far above a few units of epsilon)
    assert worst_err > 20.0, worst_err
