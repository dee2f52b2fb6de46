"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI and bring the
results back as numpy arrays in the oracle's layout."""
import numpy as np

FIELDS = ("x", "y", "z", "vx", "vy", "vz", "t", "w")


def ctx():
    from paper_1504_02776_gb300 import api
    return api.Context(0)


def packets(c, wl, fp_mode, n=None, first_id=0, beam_in=None):
    pk = c.trace_packets(wl, fp_mode=fp_mode, n=n, first_id=first_id, beam_in=beam_in)
    return pk, pk.to_dict()


def compare_packets(gpu, orc, rtol=None):
    """Relative deviation of each packet's state over the slots both sides filled:
    position |dr| / max(|r|, 1 cm), velocity |dv| / |v|, time |dt| / t, weight |dw| / w."""
    assert np.array_equal(gpu["order"], orc["order"]), "packet orders differ"
    m = orc["order"] >= 0
    assert np.array_equal(gpu["id"][m], orc["nid"][m])
    g = {f: gpu[f][m].astype(np.float64) for f in FIELDS}
    o = {f: orc[f][m] for f in FIELDS}
    dr = np.sqrt(sum((g[f] - o[f]) ** 2 for f in ("x", "y", "z")))
    rr = np.sqrt(sum(o[f] ** 2 for f in ("x", "y", "z")))
    dv = np.sqrt(sum((g[f] - o[f]) ** 2 for f in ("vx", "vy", "vz")))
    vv = np.sqrt(sum(o[f] ** 2 for f in ("vx", "vy", "vz")))
    ow = np.where(o["w"] == 0, 1.0, np.abs(o["w"]))
    return {"r": dr / np.maximum(rr, 1e-2), "v": dv / vv, "t": np.abs(g["t"] - o["t"]) / o["t"],
            "w": np.abs(g["w"] - o["w"]) / ow}


def run_events(c, wl, pk):
    counts, tallies, ev = c.detect(wl, pk, events=True)
    return counts, tallies, {k: v.cpu().numpy() for k, v in ev.items()}


# FP64 mode: relative agreement of states to 1e-12; weights to 1e-12 plus the rounding
# amplification of the packet's history (kappa, the oracle's condition estimate) times a
# few units of the FP64 epsilon.
RT64 = 1e-12
EPS64_K = 1e-15


def fp64_weight_tol(kappa):
    return RT64 + EPS64_K * kappa


def hist_tolerance(packets, n_bins, fp=64):
    """Per-bin tolerance of a histogram, from the oracle's detected packets."""
    hit = packets["bin"] >= 0
    b = packets["bin"][hit]
    w = packets["w_det"][hit]
    k = packets["kappa_det"][hit]
    tol = np.zeros(n_bins)
    if fp == 64:
        np.add.at(tol, b, w * fp64_weight_tol(k))
    else:
        np.add.at(tol, b, w * np.maximum(1e-5, 1e-6 * k))
    return tol


def check_fp64_packets(gpu, orc):
    dev = compare_packets(gpu, orc)
    m = orc["order"] >= 0
    k = orc["kappa"][m]
    bad = {f: int((dev[f] > RT64).sum()) for f in ("r", "v", "t")}
    bad["w"] = int((dev["w"] > fp64_weight_tol(k)).sum())
    return dev, bad


def flat_excess(dev_w, kappa, flat=RT64):
    """Packets whose weight deviation exceeds the flat bar: count, share, and the largest
    deviation over the condition-scaled bar (<= 1 when every one of them is explained by the
    rounding amplification of its history)."""
    beyond = dev_w > flat
    worst = float((dev_w[beyond] / fp64_weight_tol(kappa[beyond])).max()) if beyond.any() else 0.0
    return int(beyond.sum()), float(beyond.mean()) if dev_w.size else 0.0, worst


def oracle_sparse_hist(wl, n=None, chunk=200_000):
    """The oracle's detected events of a run, traced in chunks of neutron ids: per bin the
    summed detected weight, the summed weight * max(1e-5, 1e-6 kappa_det) (the FP32 bar of
    its events), the summed weight * 1e-5 (the flat FP32 bar) and the event count."""
    import oracle
    n = wl.n if n is None else n
    bins, w, kd = [], [], []
    for first in range(0, n, chunk):
        m = min(chunk, n - first)
        pk = oracle.trace(wl, first_id=first, n=m, packets=True, hist=False)["packets"]
        hit = (pk["order"] >= 1) & (pk["bin"] >= 0)
        bins.append(pk["bin"][hit])
        w.append(pk["w_det"][hit])
        kd.append(pk["kappa_det"][hit])
    b = np.concatenate(bins)
    w = np.concatenate(w)
    kd = np.concatenate(kd)
    ub, inv = np.unique(b, return_inverse=True)
    return {"bins": ub,
            "I": np.bincount(inv, weights=w, minlength=ub.size),
            "tol_k": np.bincount(inv, weights=w * np.maximum(1e-5, 1e-6 * kd), minlength=ub.size),
            "tol_flat": np.bincount(inv, weights=w * 1e-5, minlength=ub.size),
            "n": np.bincount(inv, minlength=ub.size),
            "events": int(b.size)}


def gpu_sparse(counts, bins):
    """Values of a device histogram at `bins` and its own non-zero bins outside them."""
    import torch
    idx = torch.from_numpy(bins).to(counts.device)
    at = counts[idx].cpu().numpy() if bins.size else np.zeros(0)
    nz = torch.nonzero(counts).flatten().cpu().numpy()
    extra = np.setdiff1d(nz, bins, assume_unique=False)
    return at, extra, counts[torch.from_numpy(extra).to(counts.device)].cpu().numpy() if extra.size else np.zeros(0)
