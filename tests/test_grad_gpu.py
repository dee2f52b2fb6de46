"""Adjoint gradient (mcv_grad) on the GPU: against the oracle's FP64 adjoint, against
central finite differences of the GPU forward on the same random stream, and through the
torch.autograd.Function."""
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


def small_case(n=3000):
    det = mi.tube_detector(n_tof=40, packs=(38, 39, 38), pixels_per_tube=16)
    wl = mi.config2(n=n).replace(detector=det)
    tw = wl.replace(sqe=mi.SqeGrid(mi.sqe_table(omega_scale=1.05)), seed=1)
    ref = oracle.trace(tw, packets=False)["hist"]
    c = 1e4 / ref.sum()
    return wl, mi.poisson_target(ref, c, seed=2), c


def test_fp64_adjoint_matches_oracle(ctx):
    wl, target, c = small_case()
    tg = torch.from_numpy(target).cuda()
    out = ctx.grad(wl, tg, c, fp_mode=B.FP64)
    ref = oracle.grad(wl, target, c)
    assert abs(out["loss"].item() - ref["loss"]) <= 1e-11 * ref["loss"]
    np.testing.assert_allclose(out["hist"].cpu().numpy(), ref["hist"], rtol=1e-11, atol=1e-300)
    np.testing.assert_allclose(out["dsig"].cpu().numpy(), ref["dsig"], rtol=1e-10)
    d, r = out["dsqe"].cpu().numpy(), ref["dsqe"].ravel()
    scale = np.abs(r).max()
    assert np.abs(d - r).max() <= 1e-10 * scale
    nz = np.abs(r) > 1e-6 * scale
    np.testing.assert_allclose(d[nz], r[nz], rtol=1e-9)


def _gpu_loss(ctx, wl, tg, c, table, sig=None):
    w = wl
    if sig is not None:
        s = wl.scatterers[0]
        w = wl.replace(scatterers=[mi.Scatterer(s.kind, s.dims, s.n_per_A3, sig[0],
                                                [(s.kernels[0][0], sig[1])])])
    counts, _ = ctx.trace(w, fp_mode=B.FP64, table=table)
    den = torch.clamp(tg, min=1.0)
    return float((((c * counts - tg) ** 2) / den).sum())


def test_fp64_adjoint_matches_central_differences(ctx):
    """64 random table entries with non-zero gradient plus both cross sections, full
    117,760-pixel detector, FP64 trace, h = 1e-4 relative."""
    n = 200_000
    wl = mi.config2(n=n)
    tw = wl.replace(sqe=mi.SqeGrid(mi.sqe_table(omega_scale=1.05)), seed=1)
    ref = oracle.trace(tw, packets=False)["hist"]
    c = 1e6 / ref.sum()
    target = mi.poisson_target(ref, c, seed=2)
    tg = torch.from_numpy(target).cuda()
    table = ctx.table(wl)
    out = ctx.grad(wl, tg, c, fp_mode=B.FP64, table=table)
    dsqe = out["dsqe"].cpu().numpy()
    rng = np.random.default_rng(3)
    tab = wl.sqe.table.ravel()
    cand = np.flatnonzero((np.abs(dsqe) > 1e-4 * np.abs(dsqe).max()) & (tab > 0))
    picks = rng.choice(cand, size=64, replace=False)
    bad = []
    for e in picks:
        vals = []
        for sgn in (1, -1):
            t = table.clone()
            t.view(-1)[e] = float(np.float32(tab[e] * (1 + sgn * 1e-4)))
            vals.append((float(t.view(-1)[e]), _gpu_loss(ctx, wl, tg, c, t)))
        fd = (vals[0][1] - vals[1][1]) / (vals[0][0] - vals[1][0])
        if abs(fd - dsqe[e]) > 1e-3 * abs(dsqe[e]):
            bad.append((int(e), fd, float(dsqe[e])))
    assert not bad, bad[:5]
    s = wl.scatterers[0]
    base = (s.sig_abs_b, s.kernels[0][1])
    for i in range(2):
        h = 1e-4 * base[i]
        lo, hi = list(base), list(base)
        lo[i] -= h
        hi[i] += h
        fd = (_gpu_loss(ctx, wl, tg, c, table, hi) - _gpu_loss(ctx, wl, tg, c, table, lo)) / (2 * h)
        an = out["dsig"][i].item()
        assert abs(fd - an) <= 1e-3 * abs(fd), (i, fd, an)


def test_fp32_trace_gradient_close_to_fp64(ctx):
    wl, target, c = small_case(20000)
    tg = torch.from_numpy(target).cuda()
    g64 = ctx.grad(wl, tg, c, fp_mode=B.FP64)
    g32 = ctx.grad(wl, tg, c, fp_mode=B.FP32)
    a, b = g32["dsqe"].cpu().numpy(), g64["dsqe"].cpu().numpy()
    big = np.abs(b) > 1e-2 * np.abs(b).max()
    rel = np.abs(a[big] - b[big]) / np.abs(b[big])
    assert np.median(rel) < 1e-4 and (rel > 1e-2).mean() < 0.02
    np.testing.assert_allclose(g32["dsig"].cpu().numpy(), g64["dsig"].cpu().numpy(), rtol=1e-2)


def test_autograd_function_backward(ctx):
    wl, target, c = small_case(3000)
    tg = torch.from_numpy(target).cuda()
    table = ctx.table(wl).requires_grad_(True)
    s = wl.scatterers[0]
    sa = torch.tensor(s.sig_abs_b, dtype=torch.float64, requires_grad=True)
    ss = torch.tensor(s.kernels[0][1], dtype=torch.float64, requires_grad=True)
    loss = api.chi2_loss(ctx, wl, table, sa, ss, tg, c, fp_mode=B.FP64)
    loss.backward()
    ref = ctx.grad(wl, tg, c, fp_mode=B.FP64)
    assert abs(loss.item() - ref["loss"].item()) <= 1e-12 * ref["loss"].item()
    np.testing.assert_allclose(table.grad.cpu().numpy().ravel(),
                               ref["dsqe"].cpu().numpy().astype(np.float32), rtol=1e-6)
    assert abs(sa.grad.item() - ref["dsig"][0].item()) <= 1e-12 * abs(ref["dsig"][0].item())
    assert abs(ss.grad.item() - ref["dsig"][1].item()) <= 1e-12 * abs(ref["dsig"][1].item())
