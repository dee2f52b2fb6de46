"""mcv_grad_noalloc, the gradient entry point for callers that cannot allocate device memory
(graph capture, someone else's memory pool, a locked-down allocator): it must give what
mcv_grad gives, call after call, with its work buffer in the library's fixed device array.
Collected last so that a failure here does not hide the other tests."""
import ctypes as C
import gc

import numpy as np
import pytest

import mcv_inputs as mi
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1504_02776_gb300 import api, binding as B  # noqa: E402


def _case(n=3000):
    det = mi.tube_detector(n_tof=40, packs=(38, 39, 38), pixels_per_tube=16)
    wl = mi.config2(n=n).replace(detector=det)
    tw = wl.replace(sqe=mi.SqeGrid(mi.sqe_table(omega_scale=1.05)), seed=1)
    ref = oracle.trace(tw, packets=False)["hist"]
    c = 1e4 / ref.sum()
    return wl, mi.poisson_target(ref, c, seed=2), c


def _noalloc(wl, table, target, c, fp_mode):
    sample = api.sample_struct(wl, fp_mode, table)
    det = api.detector_struct(wl.detector)
    nb = wl.detector.n_bins
    counts = torch.empty(nb, dtype=torch.float64, device="cuda")
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    dsqe = torch.empty(wl.sqe.table.size, dtype=torch.float64, device="cuda")
    dsig = torch.empty(2, dtype=torch.float64, device="cuda")
    hist = B.Hist(counts.data_ptr(), None)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    B.mcv_grad_noalloc(sample, api.beam_struct(wl.beam), det, wl.seed, wl.sim_id, 0, wl.n,
                       C.c_void_p(target.data_ptr()), c, 0, hist, C.c_void_p(loss.data_ptr()),
                       C.c_void_p(dsqe.data_ptr()), C.c_void_p(dsig.data_ptr()), stream)
    torch.cuda.synchronize()
    return {"loss": loss, "dsqe": dsqe, "dsig": dsig, "hist": counts}


@pytest.mark.parametrize("fp_mode", [B.FP64, B.FP32])
def test_noalloc_gradient_matches_mcv_grad_twice(fp_mode):
    wl, target, c = _case()
    ctx = api.Context(0)
    tg = torch.from_numpy(target).cuda()
    table = ctx.table(wl)
    ref = ctx.grad(wl, tg, c, fp_mode=fp_mode, table=table)
    # the no-allocation call reads dchi2/dI from its work array; mcv_grad without one
    # evaluates it per packet, in FP32 in the FP32 mode: they differ by FP32 roundings there
    rt = 1e-10 if fp_mode == B.FP64 else 1e-6
    for _ in range(2):
        out = _noalloc(wl, table, tg, c, fp_mode)
        assert abs(out["loss"].item() - ref["loss"].item()) <= 1e-12 * ref["loss"].item()
        np.testing.assert_allclose(out["hist"].cpu().numpy(), ref["hist"].cpu().numpy(),
                                   rtol=1e-12, atol=1e-300)
        np.testing.assert_allclose(out["dsig"].cpu().numpy(), ref["dsig"].cpu().numpy(),
                                   rtol=rt)
        a, b = out["dsqe"].cpu().numpy(), ref["dsqe"].cpu().numpy()
        assert np.abs(a - b).max() <= rt * np.abs(b).max()
    ctx.close()


def test_noalloc_allocates_nothing():
    """After a first call (which loads the kernels), further calls leave both torch's
    allocator and the device's free memory exactly as they were."""
    wl, target, c = _case(n=2000)
    tg = torch.from_numpy(target).cuda()
    table = torch.from_numpy(wl.sqe.table).cuda()
    _noalloc(wl, table, tg, c, B.FP32)
    torch.cuda.synchronize()
    outs = [_noalloc(wl, table, tg, c, B.FP32) for _ in range(2)]  # output buffers first
    torch.cuda.synchronize()
    # tensors left by earlier tests must not be freed in between: collect them now and keep
    # the collector off while measuring
    gc.collect()
    gc.disable()
    try:
        _measure_noalloc(wl, table, tg, c, outs)
    finally:
        gc.enable()


def _measure_noalloc(wl, table, tg, c, outs):
    before = (torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0])
    sample = api.sample_struct(wl, B.FP32, table)
    det = api.detector_struct(wl.detector)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for o in outs:
        hist = B.Hist(o["hist"].data_ptr(), None)
        B.mcv_grad_noalloc(sample, api.beam_struct(wl.beam), det, wl.seed, wl.sim_id, 0, wl.n,
                           C.c_void_p(tg.data_ptr()), c, 0, hist,
                           C.c_void_p(o["loss"].data_ptr()), C.c_void_p(o["dsqe"].data_ptr()),
                           C.c_void_p(o["dsig"].data_ptr()), stream)
    torch.cuda.synchronize()
    after = (torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0])
    assert after == before, (before, after)
    B.mcv_sync(None, stream)


def test_noalloc_reports_device_errors_at_sync():
    """A target bin that is not a finite count >= 0 is found by the loss kernel on the device;
    the error word keeps it until mcv_sync(NULL, stream) reports it, and is clear afterwards."""
    wl, target, c = _case(n=1000)
    bad = target.copy()
    bad[7] = -1.0
    table = torch.from_numpy(wl.sqe.table).cuda()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    B.mcv_sync(None, stream)  # nothing pending
    _noalloc(wl, table, torch.from_numpy(bad).cuda(), c, B.FP64)
    # a later valid call does not hide the earlier error
    _noalloc(wl, table, torch.from_numpy(target).cuda(), c, B.FP64)
    with pytest.raises(B.McvError) as e:
        B.mcv_sync(None, stream)
    assert e.value.status == B.MCV_EDEVICE
    B.mcv_sync(None, stream)  # cleared
    bad[7] = float("nan")
    _noalloc(wl, table, torch.from_numpy(bad).cuda(), c, B.FP64)
    with pytest.raises(B.McvError) as e:
        B.mcv_sync(None, stream)
    assert e.value.status == B.MCV_EDEVICE
    B.mcv_sync(None, stream)


def test_noalloc_rejects_histograms_beyond_its_buffer():
    wl = mi.config2(n=10)  # 117,760 x 1000 bins, more than the fixed buffer holds
    table = torch.from_numpy(wl.sqe.table).cuda()
    sample = api.sample_struct(wl, B.FP64, table)
    det = api.detector_struct(wl.detector)
    one = torch.zeros(4, dtype=torch.float64, device="cuda")
    hist = B.Hist(one.data_ptr(), None)
    p = C.c_void_p(one.data_ptr())
    with pytest.raises(B.McvError) as e:
        B.mcv_grad_noalloc(sample, api.beam_struct(wl.beam), det, 0, 0, 0, 10, p, 1.0, 0, hist,
                           p, p, p)
    assert e.value.status == B.MCV_EINVAL
