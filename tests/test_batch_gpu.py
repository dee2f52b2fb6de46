"""Batched launches (mcv_batch_*, mcv_trace_batch): many simulations in one persistent
launch, checked against one-simulation-per-launch runs of the same simulations (the same
per-neutron arithmetic, so histograms agree up to the order of the FP64 additions) and
against the oracle."""
import ctypes as C
import dataclasses

import numpy as np
import pytest
import torch

import gpu_helpers as H
import mcv_inputs as mi
import oracle
from paper_1504_02776_gb300 import binding as B

pytestmark = pytest.mark.gpu

# a smaller tube system (19 packs x 8 tubes x 32 pixels, 200 tof bins) for the small cases
SMALL_DET = mi.tube_detector(n_tof=200, packs=(6, 7, 6), pixels_per_tube=32)
ANGLES = [0, 17, 45, 90, 137, 180]


@pytest.fixture(scope="module")
def ctx():
    return H.ctx()


def _crystal_sims(counts):
    sims = mi.config3_batch(orientations=ANGLES, detector=SMALL_DET)
    return [w.replace(n=n) for w, n in zip(sims, counts)]


def _sweep_sims(count_scale=2e-4):
    return mi.config5(count_scale=count_scale, detector=SMALL_DET)


def _np(pair):
    return pair[0].cpu().numpy(), pair[1].cpu().numpy()


def _same_sums(a, b, rtol=1e-12):
    """Equal up to the order of FP64 additions of the same positive contributions."""
    return np.all(np.abs(a - b) <= rtol * np.abs(b))


# FP32: the batched and the single-launch kernels are compiled separately, so an event's
# last bits (and rarely its bin) may differ; at most 1e-4 of the events may change bin, each
# change moving its weight out of one bin and into another
FP32_MOVED = 2e-4

COUNT_TALLIES = (B.T_NDET, B.T_NOVER, B.T_NMISS, B.T_NHIT, B.T_NEMIT)
WEIGHT_TALLIES = (B.T_BEAMSTOP, B.T_WDET, B.T_WOVER)


def _check_same(batch_pair, single_pair):
    hb, tb = _np(batch_pair)
    hs, ts = _np(single_pair)
    assert _same_sums(hb, hs), float(np.max(np.abs(hb - hs)))
    assert np.array_equal(tb[list(COUNT_TALLIES)], ts[list(COUNT_TALLIES)]), (tb, ts)
    assert _same_sums(tb[list(WEIGHT_TALLIES)], ts[list(WEIGHT_TALLIES)])


def test_fp64_crystal_batch_matches_single_launches(ctx):
    sims = _crystal_sims([3000, 1, 2500, 0, 4000, 777])
    hists = ctx.trace_batch(sims, fp_mode=B.FP64)
    for wl, pair in zip(sims, hists):
        single = ctx.trace(wl, fp_mode=B.FP64)
        _check_same(pair, single)
    # the simulation without neutrons leaves its histogram untouched
    assert not hists[3][0].any() and not hists[3][1].any()


def test_fp32_sweep_batch_matches_single_launches(ctx):
    sims = _sweep_sims()
    b = ctx.batch(sims, fp_mode=B.FP32)
    b.run(sync=True)
    total = 0.0
    moved = 0.0
    for wl, pair in zip(sims, b.hists):
        hb, tb = _np(pair)
        hs, ts = _np(ctx.trace(wl, fp_mode=B.FP32))
        total += hs.sum()
        moved += np.abs(hb - hs).sum()
        assert abs(tb[B.T_NDET] - ts[B.T_NDET]) <= max(1, 1e-4 * ts[B.T_NDET])
    assert moved <= FP32_MOVED * total, (moved, total)
    b.close()


def test_fp64_batch_matches_oracle(ctx):
    # the lowest and highest incident energies of the sweep (own time windows) and two crystal
    # orientations, all on one detector geometry
    sweep = mi.config5(count_scale=1e-9, detector=SMALL_DET)
    sims = [sweep[0].replace(n=400), sweep[-1].replace(n=400)]
    sims += [w.replace(n=300) for w in mi.config3_batch(orientations=[30, 137],
                                                        detector=SMALL_DET)]
    hists = ctx.trace_batch(sims, fp_mode=B.FP64)
    for wl, pair in zip(sims, hists):
        h, t = _np(pair)
        orc = oracle.trace(wl, packets=True)
        op = orc["packets"]
        m = op["order"] >= 1
        tol = H.hist_tolerance(op[m], h.size)
        assert np.all(np.abs(h - orc["hist"]) <= tol + 1e-15 * np.abs(orc["hist"])), wl.name
        assert t[B.T_NDET] == orc["tallies"][oracle.T_NDET], wl.name


def test_batch_in_cuda_graph(ctx):
    sims = _sweep_sims(count_scale=5e-5)
    b = ctx.batch(sims, fp_mode=B.FP32)
    b.run(sync=True)
    ref = [_np(p) for p in b.hists]
    for c, t in b.hists:
        c.zero_()
        t.zero_()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            b.run()
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    for c, t in b.hists:  # capture does not run the work
        assert not c.any() and not t.any()
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    ctx.sync()
    for (hr, tr), pair in zip(ref, b.hists):
        h, t = _np(pair)
        assert _same_sums(h, 2.0 * hr)
        assert np.array_equal(t[list(COUNT_TALLIES)], 2.0 * tr[list(COUNT_TALLIES)])
    b.close()


def test_tuner_keeps_histograms_and_picks_a_candidate(ctx):
    sims = _crystal_sims([20000, 5000, 30000, 100, 8000, 12000])
    b = ctx.batch(sims, fp_mode=B.FP32)
    shape = b.tune(trial_neutrons=40000)
    for c, t in b.hists:
        assert not c.any() and not t.any()
    assert shape["chunk"] in (512, 1024, 2048, 4096, 8192)
    assert 1 <= shape["blocks_per_sm"] <= 16
    b.run(sync=True)
    for wl, pair in zip(sims, b.hists):
        hb, tb = _np(pair)
        hs, ts = _np(ctx.trace(wl, fp_mode=B.FP32))
        assert abs(tb[B.T_NDET] - ts[B.T_NDET]) <= max(1, 1e-4 * ts[B.T_NDET])
        assert np.abs(hb - hs).sum() <= FP32_MOVED * hs.sum()
    b.close()


def test_batch_argument_errors(ctx):
    from paper_1504_02776_gb300 import api
    det = api.detector_struct(SMALL_DET)
    with pytest.raises(B.McvError) as e:
        B.mcv_trace_batch(ctx.handle, [], det, B.FP32)
    assert e.value.status == B.MCV_EINVAL
    sims = _crystal_sims([10] * 6)
    # time window with tof_max <= tof_min
    bad = [w.replace(detector=dataclasses.replace(SMALL_DET, tof_min_s=5e-3, tof_max_s=4e-3))
           for w in sims[:1]]
    with pytest.raises(B.McvError) as e:
        ctx.trace_batch(bad, fp_mode=B.FP32)
    assert e.value.status == B.MCV_EINVAL
    # a sample whose fp_mode differs from the batch's
    wl = sims[0]
    sample = api.sample_struct(wl, B.FP64)
    beam = api.beam_struct(wl.beam)
    counts, tallies = ctx.new_hist(wl.detector)
    sim = B.Sim(C.pointer(sample), C.pointer(beam), 0, 0, 0, 10, 0.0, 0.0,
                B.Hist(counts.data_ptr(), tallies.data_ptr()))
    with pytest.raises(B.McvError) as e:
        B.mcv_trace_batch(ctx.handle, [sim], det, B.FP32)
    assert e.value.status == B.MCV_EINVAL
    # detector geometries must agree
    with pytest.raises(ValueError):
        ctx.trace_batch([sims[0], sims[1].replace(detector=mi.tube_detector())])


def test_allocation_failure_is_reported_and_the_context_stays_usable(ctx):
    """MCV_ENOMEM: the tuner's scratch histogram for 117,760 pixels x 1e7 time bins (9.4 TB)
    cannot be allocated; the call fails before any launch, and the context then traces as
    before (CUDA's record of the failed allocation is cleared)."""
    det = dataclasses.replace(mi.tube_detector(), n_tof=10_000_000)
    wl = mi.config2(n=1000).replace(detector=det)
    tiny = (torch.zeros(16, dtype=torch.float64, device="cuda"),
            torch.zeros(B.MCV_NTALLY, dtype=torch.float64, device="cuda"))
    b = ctx.batch([wl], fp_mode=B.FP32, hists=[tiny])
    with pytest.raises(B.McvError) as e:
        b.tune(trial_neutrons=1000)
    assert e.value.status == B.MCV_ENOMEM
    assert "scratch" in str(e.value)
    b.close()
    assert not tiny[0].any() and not tiny[1].any()
    ctx.sync()
    h, t = _np(ctx.trace(mi.config1(2000), fp_mode=B.FP64))
    assert t[B.T_NHIT] > 0 and t[B.T_NDET] > 0


def _free_bytes():
    free, _ = torch.cuda.mem_get_info()
    return free


def test_fullsize_crystal_batch_sampled_orientations(ctx):
    """The batched single-crystal run at full size -- 181 orientations x 2e6 neutrons, one
    117,760 x 1000 FP64 histogram each (170 GB) -- against single launches of sampled
    orientations."""
    sims = mi.config3_batch()
    nb = sims[0].detector.n_bins
    need = (len(sims) + 2) * nb * 8 + (8 << 30)
    if _free_bytes() < need:
        pytest.skip("needs %.0f GB of free device memory" % (need / 1e9))
    hists = [(torch.zeros(nb, dtype=torch.float64, device="cuda"),
              torch.zeros(B.MCV_NTALLY, dtype=torch.float64, device="cuda")) for _ in sims]
    b = ctx.batch(sims, fp_mode=B.FP32, hists=hists)
    b.run(sync=True)
    for k in (0, 77, 180):
        hb, tb = _np(hists[k])
        hs, ts = _np(ctx.trace(sims[k], fp_mode=B.FP32))
        assert abs(tb[B.T_NDET] - ts[B.T_NDET]) <= max(1, 1e-4 * ts[B.T_NDET])
        assert np.abs(hb - hs).sum() <= FP32_MOVED * hs.sum()
        assert tb[B.T_NEMIT] == ts[B.T_NEMIT]
    b.close()
    del hists
    torch.cuda.empty_cache()


def test_fullsize_sweep_batch_sampled_simulations(ctx):
    """The uneven incident-energy sweep at full size (64 simulations, 1e5..1e8 neutrons each,
    one full histogram each) against single launches of sampled simulations."""
    sims = mi.config5()
    nb = sims[0].detector.n_bins
    need = (len(sims) + 2) * nb * 8 + (8 << 30)
    if _free_bytes() < need:
        pytest.skip("needs %.0f GB of free device memory" % (need / 1e9))
    b = ctx.batch(sims, fp_mode=B.FP32)
    b.run(sync=True)
    for k in (0, 31, 63):
        hb, tb = _np(b.hists[k])
        hs, ts = _np(ctx.trace(sims[k], fp_mode=B.FP32))
        assert abs(tb[B.T_NDET] - ts[B.T_NDET]) <= max(1, 1e-4 * ts[B.T_NDET])
        assert np.abs(hb - hs).sum() <= FP32_MOVED * hs.sum()
    b.close()
    torch.cuda.empty_cache()
