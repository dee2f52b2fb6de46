"""Coherent elastic powder diffraction and event-mode output on the GPU, against the oracle.

  - The Bragg kernel (aluminium-like powder: fcc reflections next to a weak incoherent term):
    every emitted packet and detector result in FP64 as the oracle's (states 1e-12; weights
    1e-12 plus the condition allowance), in FP32 within the FP32 bars.
  - Event mode: the fused run's event list holds every detected packet once -- the same
    multiset of (pixel, time of flight, weight) as the oracle's detected packets (FP64, 1e-12)
    -- and binning it on the host reproduces the run's own histogram and tallies; a list that
    is too short counts every packet but writes only its capacity; the detector step on
    stored packets fills one as well; in a batch, each record carries its simulation's tag.
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


@pytest.mark.parametrize("ei", [100.0, 20.0])
def test_fp64_bragg_packets_match_oracle(ctx, ei):
    wl = mi.aluminium_powder(20000, ei=ei)
    pk, g = H.packets(ctx, wl, B.FP64)
    op = oracle.trace(wl, packets=True, hist=False)["packets"]
    dev, bad = H.check_fp64_packets(g, op)
    assert not any(bad.values()), (bad, {f: float(d.max()) for f, d in dev.items()})
    counts, tallies, ev = H.run_events(ctx, wl, pk)
    m = op["order"] >= 1
    assert np.array_equal(ev["bin"][m], op["bin"][m])
    assert m.sum() > 5000


def _sorted_events(pixel, tof, w):
    o = np.lexsort((w, tof, pixel))
    return pixel[o], tof[o], w[o]


def test_event_mode_holds_every_detected_packet(ctx):
    wl = mi.config2(n=100000)
    evb = api.EventBuffers(200000)
    counts, tallies = ctx.trace(wl, fp_mode=B.FP64, events=evb)
    ev = evb.to_dict()
    t = tallies.cpu().numpy()
    assert ev["count"] == int(t[B.T_NDET] + t[B.T_NOVER]) < evb.capacity
    assert np.all(ev["sim"] == wl.sim_id)
    # the same packets as the oracle's detections, in or outside the time window
    op = oracle.trace(wl, packets=True, hist=False)["packets"]
    hit = (op["order"] >= 1) & (op["pixel"] >= 0)
    a = _sorted_events(ev["pixel"], ev["tof"], ev["w"])
    b = _sorted_events(op["pixel"][hit].astype(np.int32), op["tof"][hit], op["w_det"][hit])
    assert np.array_equal(a[0], b[0])
    np.testing.assert_allclose(a[1], b[1], rtol=1e-12)
    tol = H.fp64_weight_tol(np.sort(op["kappa_det"][hit]).max())
    assert np.all(np.abs(a[2] - b[2]) <= tol * np.abs(b[2]) + 1e-300)
    # binned on the host, the list gives the run's histogram
    det = wl.detector
    dt = (det.tof_max_s - det.tof_min_s) / det.n_tof
    fb = np.floor((ev["tof"] - det.tof_min_s) / dt)
    inw = (fb >= 0) & (fb < det.n_tof)
    h = np.zeros(det.n_bins)
    np.add.at(h, ev["pixel"][inw].astype(np.int64) * det.n_tof + fb[inw].astype(np.int64),
              ev["w"][inw])
    hc = counts.cpu().numpy()
    nz = (h != 0) | (hc != 0)
    np.testing.assert_allclose(h[nz], hc[nz], rtol=1e-12)
    assert abs(ev["w"][~inw].sum() - t[B.T_WOVER]) <= 1e-12 * max(t[B.T_WOVER], 1e-300)


def test_event_list_overflow_and_event_only_runs(ctx):
    wl = mi.config2(n=50000)
    full = api.EventBuffers(100000)
    ctx.trace(wl, fp_mode=B.FP32, events=full)
    n = full.n()
    assert n > 1000
    short = api.EventBuffers(n // 3)
    _, tallies = ctx.trace(wl, fp_mode=B.FP32, events=short, hist=False)
    assert short.n() == n                      # every packet counted
    d, f = short.to_dict(), full.to_dict()
    assert d["pixel"].size == n // 3          # only the capacity written
    # the records written are records of the full list
    key_f = set(zip(f["pixel"].tolist(), f["tof"].tolist()))
    assert all(k in key_f for k in zip(d["pixel"].tolist(), d["tof"].tolist()))
    t = tallies.cpu().numpy()
    assert int(t[B.T_NDET] + t[B.T_NOVER]) == n


def test_detector_step_fills_an_event_list(ctx):
    wl = mi.config2(n=20000)
    pk = ctx.trace_packets(wl, fp_mode=B.FP64)
    evb = api.EventBuffers(50000)
    counts, tallies, ev = ctx.detect(wl, pk, event_list=evb)
    d = evb.to_dict()
    m = (ev["pixel"].cpu().numpy() >= 0) & (pk.order.cpu().numpy() >= 1)
    assert d["count"] == int(m.sum())
    a = _sorted_events(d["pixel"], d["tof"], d["w"])
    b = _sorted_events(ev["pixel"].cpu().numpy()[m], ev["tof"].cpu().numpy()[m],
                       ev["w_det"].cpu().numpy()[m])
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_batch_event_records_carry_the_simulation(ctx):
    wls = [mi.config3(rot_deg=float(a), n=20000) for a in (0, 45, 90)]
    evb = api.EventBuffers(200000)
    hists = ctx.trace_batch(wls, fp_mode=B.FP32, event_lists=[evb] * 3)
    d = evb.to_dict()
    assert d["count"] < evb.capacity
    for wl, (counts, tallies) in zip(wls, hists):
        t = tallies.cpu().numpy()
        assert int((d["sim"] == wl.sim_id).sum()) == int(t[B.T_NDET] + t[B.T_NOVER])
    assert set(np.unique(d["sim"]).tolist()) <= {0, 45, 90}
