"""The parity bars of the hot path, asserted as stated and with the slack reported.

FP64 mode: states and weights of every packet within 1e-12 relative of the oracle; the share
of packets whose weight needs the condition-scaled allowance (1e-12 + 1e-15 kappa, kappa the
oracle's per-packet condition estimate) is printed and bounded, and each of those is within it.
FP32 fast mode: the fused kernel's histogram against the oracle's per bin at 1e6 neutrons,
where every bin must agree within 1e-5 of its weight (or 1e-6 kappa, printed) except the bins
of at most 1e-4 of the detected events (each event in another bin moves weight out of one bin
into another: at most two bins).
Gradient: the FP32 trace's adjoint (the benchmarked differentiable form) against the oracle's
FP64 adjoint entry by entry, and against central differences of the FP64 forward.
"""
import numpy as np
import pytest

import mcv_inputs as mi
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1504_02776_gb300 import api, binding as B  # noqa: E402

import gpu_helpers as H  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = H.ctx()
    yield c
    c.close()


def rate_bound(rate, n):
    """Largest count consistent with a true rate `rate` over n trials (Poisson, 4 sigma)."""
    mu = rate * n
    return mu + 4.0 * np.sqrt(mu) + 1.0


# ---------------------------------------------------------------- FP64: flat 1e-12
# Share of packets allowed to need the condition-scaled weight bar.  Powder and isotropic
# chains: a packet's weight loses more than 1e-12 only after a chord from a point next to a
# surface or a draw at the end of its Q range (measured: 4.2e-4 of the packets for S(Q,E),
# 8.3e-4 for the phonon kernel, 1.06e-3 for Bragg scattering, whose packets keep their speed
# and weight through more orders; every one within 0.014 of its condition bar).  Crystal: the
# outgoing energy is a root found by bisection, whose rounding is amplified by 1/|g'| where
# the dispersion runs nearly parallel to the kinematic line (measured: 2.7e-3 of the packets,
# within 0.042 of the bar).
FLAT_SHARE = {"powder": 2e-3, "crystal": 5e-3}


@pytest.mark.parametrize("make,n,kind", [
    (mi.config1, 20000, "powder"),
    (lambda n: mi.config2(n=n), 20000, "powder"),
    (lambda n: mi.powder_in_can(n), 20000, "powder"),
    (lambda n: mi.powder_in_can(n, ei=10.0), 20000, "powder"),
    (lambda n: mi.powder_two_kernels(n), 20000, "powder"),
    (lambda n: mi.vanadium_powder(n), 20000, "powder"),
    (lambda n: mi.aluminium_powder(n), 20000, "powder"),
    (lambda n: mi.config3(rot_deg=30.0, n=n), 4000, "crystal"),
    (lambda n: mi.dispersion_crystal(n, rot_deg=30.0), 40000, "crystal")])
def test_fp64_flat_bar_holds_for_almost_every_packet(ctx, make, n, kind):
    wl = make(n)
    _, g = H.packets(ctx, wl, B.FP64)
    op = oracle.trace(wl, packets=True, hist=False)["packets"]
    dev, bad = H.check_fp64_packets(g, op)
    assert not any(bad.values()), bad
    m = op["order"] >= 0
    cnt, share, worst = H.flat_excess(dev["w"], op["kappa"][m])
    print("\n%s: %d of %d packets beyond the flat 1e-12 weight bar (%.2e), worst %.3f of the "
          "condition bar; states: r %.2e v %.2e t %.2e" % (
              wl.name, cnt, int(m.sum()), share, worst, dev["r"].max(), dev["v"].max(),
              dev["t"].max()))
    assert share <= FLAT_SHARE[kind] and worst <= 1.0


# ---------------------------------------------------------------- FP32: per bin, fused
# per event: detected weights this small are beyond what FP32 carries (its normal range ends
# at 1.2e-38; within two orders of it intermediate products may have been subnormal)
W_ABS = 1e-36


@pytest.mark.parametrize("make", [lambda n: mi.config2(n=n), lambda n: mi.powder_in_can(n),
                                  lambda n: mi.powder_two_kernels(n),
                                  lambda n: mi.vanadium_powder(n),
                                  lambda n: mi.aluminium_powder(n)])
def test_fp32_fused_histogram_per_bin_against_oracle(ctx, make):
    n = 1_000_000
    wl = make(n)
    orc = H.oracle_sparse_hist(wl)
    counts, tallies = ctx.trace(wl, fp_mode=B.FP32)
    at, extra, extra_v = H.gpu_sparse(counts, orc["bins"])
    diff = np.abs(at - orc["I"])
    floor = W_ABS * orc["n"]
    bad_k = diff > orc["tol_k"] + floor
    bad_flat = diff > orc["tol_flat"] + floor
    extra_bad = int((np.abs(extra_v) > W_ABS).sum())
    events = orc["events"]
    allowed = 2 * rate_bound(1e-4, events)
    print("\n%s n=%d: %d events in %d bins; bins beyond 1e-5: %d, beyond max(1e-5, 1e-6 kappa): "
          "%d, GPU-only bins: %d (allowed %d); total rel diff %.2e" % (
              wl.name, n, events, orc["bins"].size, int(bad_flat.sum()), int(bad_k.sum()),
              extra_bad, allowed, abs(float(counts.sum()) - orc["I"].sum()) / orc["I"].sum()))
    assert int(bad_k.sum()) + extra_bad <= allowed
    assert abs(float(counts.sum()) - orc["I"].sum()) <= 1e-4 * orc["I"].sum()


# ---------------------------------------------------------------- gradient, FP32 trace
def _target(wl_fit, n_ref, c_total):
    """Seeded target of the fit: the oracle's run with omega scaled by 1.05 (seed 1) over
    n_ref neutrons, scaled to c_total counts, Poisson noise (PCG64 seed 2)."""
    tw = wl_fit.replace(sqe=mi.SqeGrid(mi.sqe_table(omega_scale=1.05)), seed=1, n=n_ref)
    ref = H.oracle_sparse_hist(tw)
    hist = np.zeros(wl_fit.detector.n_bins)
    hist[ref["bins"]] = ref["I"]
    c = c_total / hist.sum()
    return mi.poisson_target(hist, c, seed=2), c


def test_fp32_adjoint_against_oracle_fp64_adjoint(ctx):
    det = mi.tube_detector(n_tof=40, packs=(38, 39, 38), pixels_per_tube=16)
    wl = mi.config2(n=20000).replace(detector=det)
    target, c = _target(wl, 20000, 1e4)
    tg = torch.from_numpy(target).cuda()
    g32 = ctx.grad(wl, tg, c, fp_mode=B.FP32)
    ref = oracle.grad(wl, target, c)
    a, b = g32["dsqe"].cpu().numpy(), ref["dsqe"].ravel()
    l1 = np.abs(a - b).sum() / np.abs(b).sum()
    big = np.abs(b) > 1e-2 * np.abs(b).max()
    rel = np.abs(a[big] - b[big]) / np.abs(b[big])
    ds = np.abs(g32["dsig"].cpu().numpy() - ref["dsig"]) / np.abs(ref["dsig"])
    print("\nFP32 adjoint vs oracle FP64: L1 %.2e; entries >1e-2 max: %d, median rel %.2e, "
          "share > 1e-3: %.3f, max %.2e; dsig rel %s; loss rel %.2e" % (
              l1, int(big.sum()), np.median(rel), (rel > 1e-3).mean(), rel.max(), ds,
              abs(g32["loss"].item() - ref["loss"]) / ref["loss"]))
    # measured: L1 3.1e-5, entries above 1e-2 of the largest within 4.6e-4 (median 6.9e-6),
    # dsig within 1.3e-5, loss within 2.1e-6
    assert l1 <= 1e-4
    assert np.all(rel <= 1e-3)
    assert np.all(ds <= 1e-4)
    assert abs(g32["loss"].item() - ref["loss"]) <= 1e-5 * ref["loss"]


def _hist64(ctx, wl, table, sig=None):
    w = wl
    if sig is not None:
        s = wl.scatterers[0]
        w = wl.replace(scatterers=[mi.Scatterer(s.kind, s.dims, s.n_per_A3, sig[0],
                                                [(s.kernels[0][0], sig[1])])])
    counts, _ = ctx.trace(w, fp_mode=B.FP64, table=table)
    return counts


def _loss_diff(tg, c, h_plus, h_minus):
    """chi2(h_plus) - chi2(h_minus) bin by bin, c (I+ - I-) (c (I+ + I-) - 2 T) / max(T, 1):
    the difference of two nearly equal losses without the cancellation of their large common
    part (the bins nothing reaches)."""
    den = torch.clamp(tg, min=1.0)
    return float((c * (h_plus - h_minus) * (c * (h_plus + h_minus) - 2.0 * tg) / den).sum())


def test_fp32_adjoint_against_fp64_central_differences_config4(ctx):
    """The benchmarked form: FP32 trace, 1e7 neutrons, full detector; 64 table entries (seed
    3) and both cross sections against central differences (h = 1e-4 relative) of the FP64
    forward on the same random stream, within 1e-3.

    An entry is eligible when its difference quotient can be resolved to 1e-3 at that step:
    the loss change 2 h S_e |dchi2/dS_e| must exceed 1e4 times the noise of the FP64 loss
    difference (the histogram's FP64 atomics add in a varying order; measured by running the
    same forward twice).  Entries with tiny table values (1e-12 and below) fall under that
    noise at a relative step of 1e-4 and are left out."""
    wl = mi.config4()
    target, c = _target(wl, 1_000_000, float(wl.n))
    tg = torch.from_numpy(target).cuda()
    table = ctx.table(wl)
    out = ctx.grad(wl, tg, c, fp_mode=B.FP32, table=table)
    dsqe = out["dsqe"].cpu().numpy()
    noise = max(abs(_loss_diff(tg, c, _hist64(ctx, wl, table), _hist64(ctx, wl, table)))
                for _ in range(3))
    noise = max(noise, 1e-300)
    tab = wl.sqe.table.ravel().astype(np.float64)
    signal = np.abs(dsqe) * 2e-4 * tab
    cand = np.flatnonzero((np.abs(dsqe) > 1e-4 * np.abs(dsqe).max()) & (tab > 0) &
                          (signal >= 1e4 * noise))
    rng = np.random.default_rng(3)
    picks = rng.choice(cand, size=64, replace=False)
    rels = []
    for e in picks:
        vals = []
        for sgn in (1, -1):
            t = table.clone()
            t.view(-1)[e] = float(np.float32(tab[e] * (1 + sgn * 1e-4)))
            vals.append((float(t.view(-1)[e]), _hist64(ctx, wl, t)))
        fd = _loss_diff(tg, c, vals[0][1], vals[1][1]) / (vals[0][0] - vals[1][0])
        rels.append(abs(fd - dsqe[e]) / abs(fd))
    rels = np.array(rels)
    s = wl.scatterers[0]
    base = (s.sig_abs_b, s.kernels[0][1])
    rs = []
    for i in range(2):
        h = 1e-4 * base[i]
        lo, hi = list(base), list(base)
        lo[i] -= h
        hi[i] += h
        fd = _loss_diff(tg, c, _hist64(ctx, wl, table, hi), _hist64(ctx, wl, table, lo)) / (2 * h)
        rs.append(abs(fd - out["dsig"][i].item()) / abs(fd))
    print("\nconfig 4 FP32 adjoint vs FP64 central differences: %d eligible entries (FD noise "
          "%.2e); 64 picked: median %.2e max %.2e; sig_abs %.2e sig_s %.2e" % (
              cand.size, noise, np.median(rels), rels.max(), rs[0], rs[1]))
    assert np.all(rels <= 1e-3)
    assert max(rs) <= 1e-3


# ---------------------------------------------------------------- work buffer, errors
def test_gradient_with_and_without_work_buffer(ctx):
    det = mi.tube_detector(n_tof=40, packs=(38, 39, 38), pixels_per_tube=16)
    wl = mi.config2(n=5000).replace(detector=det)
    target, c = _target(wl, 5000, 1e4)
    tg = torch.from_numpy(target).cuda()
    # FP64: both evaluate g_b in FP64 (the same function); FP32: the adjoint without a work
    # buffer evaluates g_b in FP32 from the FP64 difference c I_b - T_b, the one with a buffer
    # rounds the buffer's FP64 value, so they differ by FP32 roundings of g_b
    for fp, rt in ((B.FP64, 1e-12), (B.FP32, 1e-6)):
        work = torch.empty(det.n_bins, dtype=torch.float64, device="cuda")
        a = ctx.grad(wl, tg, c, fp_mode=fp, g_work=work)
        b = ctx.grad(wl, tg, c, fp_mode=fp)
        assert a["loss"].item() == pytest.approx(b["loss"].item(), rel=1e-13)
        np.testing.assert_allclose(a["dsig"].cpu().numpy(), b["dsig"].cpu().numpy(), rtol=rt)
        x, y = a["dsqe"].cpu().numpy(), b["dsqe"].cpu().numpy()
        assert np.abs(x - y).max() <= rt * np.abs(y).max()
        # the work buffer holds dchi2/dI of every bin
        h = b["hist"].cpu().numpy()
        g_ref = 2 * c * (c * h - target) / np.maximum(target, 1.0)
        np.testing.assert_allclose(work.cpu().numpy(), g_ref, rtol=1e-14, atol=1e-300)


def test_device_errors_are_reported_at_sync(ctx):
    det = mi.tube_detector(n_tof=40, packs=(38, 39, 38), pixels_per_tube=16)
    wl = mi.config2(n=500).replace(detector=det)
    target, c = _target(wl, 500, 1e3)
    ctx.sync()
    bad = target.copy()
    bad[3] = np.inf
    ctx.grad(wl, torch.from_numpy(bad).cuda(), c, fp_mode=B.FP64, sync=False)
    with pytest.raises(B.McvError) as e:
        ctx.sync()
    assert e.value.status == B.MCV_EDEVICE
    ctx.sync()  # the flag was cleared
    # a stored packet with an order no packet of the library has
    pk = ctx.trace_packets(wl, fp_mode=B.FP64)
    o = pk.order.clone()
    k = int(torch.nonzero(o >= 1)[0])
    pk.order[k] = 9
    counts, tallies, ev = ctx.detect(wl, pk, sync=False)
    with pytest.raises(B.McvError) as e:
        ctx.sync()
    assert e.value.status == B.MCV_EDEVICE
    ctx.sync()
    # the other packets were detected as before (slots without a packet are not written)
    pk.order.copy_(o)
    c2, t2, ev2 = ctx.detect(wl, pk)
    keep = o >= 0
    keep[k] = False
    assert torch.equal(ev["bin"][keep], ev2["bin"][keep])


def test_adjoint_of_split_ranges_adds_up(ctx):
    """mcv_adjoint on the whole run's histogram, called for two id ranges, gives mcv_grad's
    gradient of the whole run (the per-device step of a sharded gradient), and
    Context.grad_sharded on one process equals Context.grad."""
    det = mi.tube_detector(n_tof=40, packs=(38, 39, 38), pixels_per_tube=16)
    wl = mi.config2(n=6000).replace(detector=det)
    target, c = _target(wl, 6000, 1e4)
    tg = torch.from_numpy(target).cuda()
    table = ctx.table(wl)
    for fp in (B.FP64, B.FP32):
        full = ctx.grad(wl, tg, c, fp_mode=fp, table=table)
        hist = full["hist"]
        parts = [api._adjoint_call(ctx, wl, hist, tg, c, fp, m, f, table, 0)
                 for f, m in ((0, 2500), (2500, 3500))]
        ctx.sync()
        for p in parts:
            assert p["loss"].item() == pytest.approx(full["loss"].item(), rel=1e-14)
        ds = (parts[0]["dsqe"] + parts[1]["dsqe"]).cpu().numpy()
        ref = full["dsqe"].cpu().numpy()
        assert np.abs(ds - ref).max() <= 1e-12 * np.abs(ref).max()
        # the FP32 adjoint sums dsig per thread in (compensated) FP32 before its FP64 atomics,
        # so another grouping of the neutrons rounds those partial sums differently
        rt = 1e-12 if fp == B.FP64 else 1e-5
        np.testing.assert_allclose((parts[0]["dsig"] + parts[1]["dsig"]).cpu().numpy(),
                                   full["dsig"].cpu().numpy(), rtol=rt)
        sh = ctx.grad_sharded(wl, tg, c, 0, 1, fp_mode=fp, table=table)
        assert sh["loss"].item() == pytest.approx(full["loss"].item(), rel=1e-13)
        np.testing.assert_allclose(sh["dsig"].cpu().numpy(), full["dsig"].cpu().numpy(),
                                   rtol=rt)
