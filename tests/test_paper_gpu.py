"""The paper's recursive estimator on the GPU (MCV_EST_PAPER), against the oracle's paper mode.

The random numbers of every packet are keyed by its place in the tree of interactions, so
the GPU's depth-first walk and the oracle's breadth-first walk draw the same numbers and
produce the same packets: the FP64 tallies' counts are equal and their sums agree to 1e-11;
the histograms agree bin by bin to 1e-12 but for the bins holding packets whose weights went
through ill-conditioned steps (near-tangent chords, crystal eigenvectors; the ulp differences
of the transcendental functions are amplified there).  The chain estimator bounds those per
packet with its condition estimate; the paper mode carries none, so its bar is the measured
one with margin: at most 3% of the bins beyond 1e-12 (0.6% to 2.2% measured), none beyond
1e-8 (1.7e-9 measured).  FP32 runs give the oracle's counts within 1e-3 (every transmitted
packet is clipped on its parent's line, so no rounding creates packets).  The multi-tube detector (the weight a tube leaves goes on) is checked the same way on
packets that cross several tubes, and the estimator agrees with the bounded chain within
Monte Carlo error.
"""
import dataclasses
import math

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


def _cases():
    multi = dataclasses.replace(mi.tube_detector(), multi_tube=True)
    return [("config1", mi.config1(20000)),
            ("powder", mi.config2(n=20000)),
            ("powder-multi-tube", mi.config2(n=20000).replace(detector=multi)),
            ("can", mi.powder_in_can(20000)),
            ("crystal", mi.config3(rot_deg=30.0, n=3000))]


@pytest.mark.parametrize("name,wl", _cases())
def test_fp64_paper_estimator_matches_the_oracle(ctx, name, wl):
    counts, tallies = ctx.trace(wl, fp_mode=B.FP64, estimator=B.EST_PAPER)
    ref = oracle.trace_paper(wl)
    t, to = tallies.cpu().numpy(), ref["tallies"]
    for gi, oi in ((B.T_NDET, oracle.T_NDET), (B.T_NOVER, oracle.T_NOVER),
                   (B.T_NMISS, oracle.T_NMISS), (B.T_NHIT, oracle.T_NHIT)):
        assert t[gi] == to[oi], (name, gi, t[gi], to[oi])
    for gi, oi in ((B.T_BEAMSTOP, oracle.T_BEAMSTOP), (B.T_WDET, oracle.T_WDET)):
        assert abs(t[gi] - to[oi]) <= 1e-11 * abs(to[oi]), (name, gi, t[gi], to[oi])
    hc, ho = counts.cpu().numpy(), ref["hist"]
    nz = (hc != 0) | (ho != 0)
    assert nz.sum() > 100
    rel = np.abs(hc[nz] - ho[nz]) / np.maximum(np.abs(ho[nz]), 1e-300)
    share = float((rel > 1e-12).mean())
    print("\n%s: %d bins, largest relative difference %.2e, share beyond 1e-12 %.2e"
          % (name, int(nz.sum()), rel.max(), share))
    assert share <= 3e-2
    assert np.all(rel <= 1e-8)


def test_fp32_paper_estimator_against_the_oracle(ctx):
    wl = mi.config2(n=100000)
    counts, tallies = ctx.trace(wl, fp_mode=B.FP32, estimator=B.EST_PAPER)
    to = oracle.trace_paper(wl)["tallies"]
    t = tallies.cpu().numpy()
    print("\nFP32 paper: WDET %.8g / %.8g, NDET %d / %d" % (t[B.T_WDET], to[oracle.T_WDET],
                                                          t[B.T_NDET], to[oracle.T_NDET]))
    assert abs(t[B.T_WDET] - to[oracle.T_WDET]) <= 1e-4 * to[oracle.T_WDET]
    assert abs(t[B.T_BEAMSTOP] - to[oracle.T_BEAMSTOP]) <= 1e-5 * to[oracle.T_BEAMSTOP]
    assert abs(t[B.T_NDET] - to[oracle.T_NDET]) <= 1e-3 * to[oracle.T_NDET] + 3


def test_fp32_paper_histogram_per_bin(ctx):
    """The FP32 paper estimator's histogram against the oracle's paper mode.  Weight moves
    between bins mostly with the hollow shell; the explanation the measurements point to: in
    the paper's recursion every segment a ray crosses is an interaction, and in FP32 a ray
    that grazes the shell's inner surface can cross the wall as one segment or as two, after
    which the tree below and the node-keyed random numbers of its packets differ.  Measured (2e5 neutrons): on the powder
    shell 1.55e-3 of the weight moves between bins (L1 / total; half of it in bins below
    1e-30, where FP32 weights underflow), with the isotropic kernel on the same shell
    2.7e-4, on config 1's solid cylinder at two orders 1.5e-5 -- against 3.2e-5 for the
    chain on the powder.  Bars: L1 3e-3 on the shell, 1e-4 on the solid cylinder, the
    total detected weight within 1e-5 on both."""
    for wl, l1_bar in ((mi.config2(n=200000), 3e-3), (mi.config1(200000).replace(max_orders=2), 1e-4)):
        counts, tallies = ctx.trace(wl, fp_mode=B.FP32, estimator=B.EST_PAPER)
        ref = oracle.trace_paper(wl)
        hc, ho = counts.cpu().numpy(), ref["hist"]
        l1 = np.abs(hc - ho).sum() / np.abs(ho).sum()
        print("\nFP32 paper %s: L1 / total %.3g, total %.3g" % (wl.name, l1, abs(hc.sum() / ho.sum() - 1)))
        assert l1 <= l1_bar
        assert abs(hc.sum() - ho.sum()) <= 1e-5 * ho.sum()


def test_paper_estimator_agrees_with_the_chain(ctx):
    """Both estimators of the same histogram (config 2 at 2e6 neutrons in 8 batches)."""
    base = mi.config2(n=250000)
    wp, wc = [], []
    for b in range(8):
        wl = base.replace(seed=300 + b)
        _, tp = ctx.trace(wl, fp_mode=B.FP32, estimator=B.EST_PAPER)
        _, tc = ctx.trace(wl, fp_mode=B.FP32)
        wp.append(tp[B.T_WDET].item())
        wc.append(tc[B.T_WDET].item())
    wp, wc = np.array(wp), np.array(wc)
    z = (wp.mean() - wc.mean()) / math.sqrt(wp.var(ddof=1) / 8 + wc.var(ddof=1) / 8)
    print("\npaper vs chain detected weight: %.6g vs %.6g (z = %.2f)" % (wp.mean(), wc.mean(), z))
    assert abs(z) < 4


def test_paper_estimator_event_list(ctx):
    """Event mode with the paper's estimator: one record per detected packet (in or outside
    the time window), and binned on the host the records give the run's histogram."""
    wl = mi.config2(n=20000)
    evb = api.EventBuffers(200000)
    counts, tallies = ctx.trace(wl, fp_mode=B.FP64, estimator=B.EST_PAPER, events=evb)
    ev = evb.to_dict()
    t = tallies.cpu().numpy()
    assert ev["count"] == int(t[B.T_NDET] + t[B.T_NOVER]) < evb.capacity
    assert np.all(ev["sim"] == wl.sim_id)
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
    # and the same run without a list gives the same histogram
    c2, _ = ctx.trace(wl, fp_mode=B.FP64, estimator=B.EST_PAPER)
    np.testing.assert_allclose(c2.cpu().numpy()[nz], hc[nz], rtol=1e-12)


def test_paper_estimator_rejects_what_it_cannot_do(ctx):
    wl = mi.config2(n=10)
    table = ctx.table(wl)
    sample = api.sample_struct(wl, B.FP64, table, B.EST_PAPER)
    counts, tallies = ctx.new_hist(wl.detector)
    pk = api.NeutronBuffers(10 * (wl.max_orders + 1), B.FP64)
    with pytest.raises(B.McvError) as e:
        B.mcv_trace_sample(ctx.handle, sample, api.beam_struct(wl.beam), None, 0, 0, 0, 10,
                           api.detector_struct(wl.detector),
                           B.Hist(counts.data_ptr(), tallies.data_ptr()), pk.struct())
    assert e.value.status == B.MCV_EINVAL
    sample.estimator = 7
    with pytest.raises(B.McvError):
        B.mcv_trace_sample(ctx.handle, sample, api.beam_struct(wl.beam), None, 0, 0, 0, 10,
                           api.detector_struct(wl.detector),
                           B.Hist(counts.data_ptr(), tallies.data_ptr()), None)
