"""The full-size powder run (1e8 neutrons, 117,760 pixels x 1000 tof bins) in the launch
configuration the benchmark times, checked on sampled neutrons the oracle computes one by
one: the histogram of the full range minus the histogram of the range without a block of
k neutrons is exactly the contribution of that block (up to FP64 summation rounding)."""
import numpy as np
import pytest

import mcv_inputs as mi
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1504_02776_gb300 import binding as B  # noqa: E402

import gpu_helpers as H  # noqa: E402

N = 100_000_000


@pytest.fixture(scope="module")
def ctx():
    c = H.ctx()
    yield c
    c.close()


@pytest.mark.parametrize("fp_mode", [B.FP32, B.FP64])
def test_full_size_block_contribution(ctx, fp_mode):
    wl = mi.config2(n=N)
    table = ctx.table(wl)
    a, k = 61_234_567, 3000
    full, tf = ctx.trace(wl, fp_mode=fp_mode, table=table)
    cut, tc = ctx.new_hist(wl.detector)
    ctx.trace(wl, fp_mode=fp_mode, n=a, table=table, counts=cut, tallies=tc)
    ctx.trace(wl, fp_mode=fp_mode, n=N - a - k, first_id=a + k, table=table, counts=cut,
              tallies=tc)
    diff = (full - cut).cpu().numpy()
    # the two FP64 histograms add their events in other orders: rounding of the full bin
    noise_b = 1e-13 * np.abs(full.cpu().numpy())
    del full, cut
    torch.cuda.empty_cache()
    ref = oracle.trace(wl, first_id=a, n=k, packets=True)
    pk = ref["packets"]
    hit = pk["bin"] >= 0
    bins = pk["bin"][hit]
    expect = np.zeros(diff.size)
    np.add.at(expect, bins, pk["w_det"][hit])
    # outside the block's bins only rounding noise remains
    mask = np.zeros(diff.size, dtype=bool)
    mask[bins] = True
    noise = (np.abs(diff) - noise_b)[~mask].max()
    assert noise <= 0.0, noise
    got = diff[mask]
    want = expect[mask]
    if fp_mode == B.FP64:
        tol = H.hist_tolerance(pk[pk["order"] >= 1], diff.size)[mask] + noise_b[mask]
        bad = int((np.abs(got - want) > tol + 1e-13 * np.abs(want)).sum())
        assert bad == 0, bad
    else:
        # FP32: weights within max(1e-5, 1e-6 kappa) (weights below the FP32 range aside); a
        # flipped event moves its weight to another bin and shows up as two mismatches
        tol = H.hist_tolerance(pk[pk["order"] >= 1], diff.size, fp=32)[mask] + noise_b[mask]
        keep = want >= 1e-25
        bad = int((np.abs(got - want) > tol + 1e-6 * np.abs(want))[keep].sum())
        assert bad <= 2 * (1e-4 * int(hit.sum()) + 4 * np.sqrt(1e-4 * int(hit.sum())) + 1), bad
    n_events = int(hit.sum())
    assert n_events > 200
    # the tallies add up the same way
    t = (tf - tc).cpu().numpy()
    if fp_mode == B.FP64:
        assert t[B.T_NDET] == ref["tallies"][oracle.T_NDET]
    else:
        # FP32 weights below its range (~1e-38) underflow to zero and end those histories
        sure = int((hit & (pk["w_det"] >= 1e-30)).sum())
        maybe = int((hit & (pk["w_det"] >= 1e-46)).sum())
        assert sure - 2 <= t[B.T_NDET] <= maybe + 2, (t[B.T_NDET], sure, maybe)
    if fp_mode == B.FP64:
        assert abs(t[B.T_BEAMSTOP] - ref["tallies"][oracle.T_BEAMSTOP]) <= 1e-6 * k
