"""Python access to the oracle (TEST INFRASTRUCTURE ONLY).

The oracle is a plain single-threaded FP64 C++ restatement of MCViNE's ray-tracing method
(liboracle.so, built from oracle.cpp).  Only the tests, the smoke check and the CPU
baseline leg of the benchmark may use it; the product path never imports this package.
This module only marshals arguments: every step of the method runs in oracle.cpp.

Parity unpinned: the absolute normalisation of the kernels against measured data.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None

PACKET_DTYPE = np.dtype([
    ("nid", np.int64), ("order", np.int32), ("pixel", np.int32),
    ("x", np.float64), ("y", np.float64), ("z", np.float64),
    ("vx", np.float64), ("vy", np.float64), ("vz", np.float64),
    ("t", np.float64), ("w", np.float64), ("tof", np.float64), ("w_det", np.float64),
    ("bin", np.int64), ("kappa", np.float64), ("kappa_det", np.float64)], align=True)

EVENT_DTYPE = np.dtype([
    ("nid", np.int64), ("order", np.int32), ("kernel", np.int32), ("scatterer", np.int32),
    ("entry", np.int32), ("q", np.float64), ("e", np.float64), ("ki", np.float64),
    ("kf", np.float64), ("factor", np.float64), ("w", np.float64),
    ("nroots", np.int32), ("mode", np.int32), ("qvec", np.float64, (3,))], align=True)

T_BEAMSTOP, T_WDET, T_WOVER, T_NDET, T_NOVER, T_NMISS, T_NHIT, T_NPACK0 = range(8)
NTALLY = T_NPACK0 + 8


class Scat(C.Structure):
    _fields_ = [("kind", C.c_int), ("dims", C.c_double * 3), ("rot_y", C.c_double),
                ("n_per_A3", C.c_double), ("sig_abs_b", C.c_double), ("nk", C.c_int),
                ("ktype", C.c_int * 2), ("ksig_b", C.c_double * 2)]


class Config(C.Structure):
    _fields_ = [
        ("ei_mev", C.c_double), ("ei_rel_sigma", C.c_double), ("div_sigma_rad", C.c_double),
        ("width_m", C.c_double), ("height_m", C.c_double), ("z0_m", C.c_double),
        ("l1_m", C.c_double),
        ("n_scat", C.c_int), ("scat", Scat * 4), ("max_orders", C.c_int),
        ("min_prob", C.c_double),
        ("sqe", C.POINTER(C.c_float)), ("nq", C.c_int), ("ne", C.c_int),
        ("q_max", C.c_double), ("e_min", C.c_double), ("e_max", C.c_double),
        ("bvk_phi_Nm", C.c_double), ("bvk_mass_u", C.c_double), ("bvk_a_A", C.c_double),
        ("bvk_msd_A2", C.c_double), ("temperature_K", C.c_double),
        ("dos_z", C.POINTER(C.c_double)), ("dos_n", C.c_int), ("dos_de", C.c_double),
        ("phonon_mass_u", C.c_double), ("phonon_nmax", C.c_int), ("phonon_p", C.c_double * 3),
        ("refl_d", C.POINTER(C.c_double)), ("refl_w", C.POINTER(C.c_double)), ("n_refl", C.c_int),
        ("det_multi_tube", C.c_int),
        ("disp_amp", C.c_double), ("disp_c", C.c_double), ("disp_s0", C.c_double),
        ("det_kind", C.c_int), ("det_radius_m", C.c_double), ("det_height_m", C.c_double),
        ("n_phi", C.c_int), ("n_y", C.c_int), ("n_rows", C.c_int), ("packs", C.c_int * 3),
        ("row_y_m", C.c_double * 3), ("tubes_per_pack", C.c_int),
        ("pixels_per_tube", C.c_int), ("tube_r_m", C.c_double), ("tube_len_m", C.c_double),
        ("tube_pitch_m", C.c_double), ("pack_gap_m", C.c_double), ("phi0_rad", C.c_double),
        ("he3_n_per_A3", C.c_double), ("he3_sig_abs_b", C.c_double),
        ("tof_min_s", C.c_double), ("tof_max_s", C.c_double), ("n_tof", C.c_int),
        ("seed", C.c_uint32), ("sim_id", C.c_uint32)]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        P = C.c_void_p
        L.orc_philox4x32_10.argtypes = [P, P, P]
        L.orc_uniforms.argtypes = [C.c_uint32, C.c_uint32, C.c_int64, C.c_int, C.c_int, P]
        L.orc_shape_segments.argtypes = [P, P, P, P, P]
        L.orc_shape_segments.restype = C.c_int
        L.orc_kernel_scatter.argtypes = [P, C.c_int, C.c_double, P, P, P, P, P, P]
        L.orc_kernel_scatter.restype = C.c_int
        L.orc_detect.argtypes = [P, P, P, C.c_double, C.c_double, C.c_double, P, P, P]
        L.orc_detect.restype = C.c_int64
        L.orc_trace.argtypes = [P, C.c_int64, C.c_int64, P, P, P, P]
        L.orc_trace.restype = C.c_int
        L.orc_trace_paper.argtypes = [P, C.c_int64, C.c_int64, P, P]
        L.orc_trace_paper.restype = C.c_int
        L.orc_detect_multi.argtypes = [P, P, P, C.c_double, C.c_double, P, P, P, P, P]
        L.orc_detect_multi.restype = C.c_int
        L.orc_n_pixels.argtypes = [P]
        L.orc_n_pixels.restype = C.c_int64
        L.orc_grad.argtypes = [P, C.c_int64, C.c_int64, P, C.c_double, C.c_int, P, P, P, P]
        L.orc_grad.restype = C.c_int
        L.orc_adjoint.argtypes = [P, C.c_int64, C.c_int64, P, P, C.c_double, C.c_int, P, P, P]
        L.orc_adjoint.restype = C.c_int
        L.orc_loss.argtypes = [P, C.c_int64, C.c_int64, P, C.c_double, P, P]
        L.orc_loss.restype = C.c_int
        L.orc_phonon_tables.argtypes = [P, P, P, P, C.c_int64]
        L.orc_phonon_tables.restype = C.c_int
        L.orc_bvk_modes.argtypes = [P, P, P, P]
        L.orc_kernel_bvk.argtypes = [P, C.c_double, C.c_double, P, P, P, P, P, P]
        L.orc_kernel_bvk.restype = C.c_int
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def make_config(wl):
    """orc_config from an mcv_inputs.Workload (keeps the table alive on the struct)."""
    c = Config()
    b = wl.beam
    c.ei_mev, c.ei_rel_sigma, c.div_sigma_rad = b.ei_mev, b.ei_rel_sigma, b.div_sigma_rad
    c.width_m, c.height_m, c.z0_m, c.l1_m = b.width_m, b.height_m, b.z0_m, b.l1_m
    c.n_scat = len(wl.scatterers)
    for j, s in enumerate(wl.scatterers):
        d = list(s.dims) + [0.0] * (3 - len(s.dims))
        c.scat[j].kind = s.kind
        c.scat[j].dims[:] = d
        c.scat[j].rot_y = s.rot_y
        c.scat[j].n_per_A3 = s.n_per_A3
        c.scat[j].sig_abs_b = s.sig_abs_b
        c.scat[j].nk = len(s.kernels)
        for k, (kt, ks) in enumerate(s.kernels):
            c.scat[j].ktype[k] = kt
            c.scat[j].ksig_b[k] = ks
    c.max_orders, c.min_prob = wl.max_orders, wl.min_prob
    if wl.sqe is not None:
        tab = np.ascontiguousarray(wl.sqe.table, dtype=np.float32)
        c._sqe_keep = tab
        c.sqe = tab.ctypes.data_as(C.POINTER(C.c_float))
        c.nq, c.ne = tab.shape
        c.q_max, c.e_min, c.e_max = wl.sqe.q_max, wl.sqe.e_min, wl.sqe.e_max
    if wl.bvk is not None:
        v = wl.bvk
        c.bvk_phi_Nm, c.bvk_mass_u, c.bvk_a_A = v.phi_Nm, v.mass_u, v.a_A
        c.bvk_msd_A2, c.temperature_K = v.msd_A2, v.temperature_K
    ph = getattr(wl, "phonon", None)
    if ph is not None:
        if wl.bvk is not None and wl.bvk.temperature_K != ph.temperature_K:
            raise ValueError("one temperature per sample")
        z = np.ascontiguousarray(ph.z, dtype=np.float64)
        c._dos_keep = z
        c.dos_z = z.ctypes.data_as(C.POINTER(C.c_double))
        c.dos_n, c.dos_de = z.size, ph.de
        c.phonon_mass_u, c.phonon_nmax = ph.mass_u, ph.nmax
        c.phonon_p[:] = list(ph.p)
        c.temperature_K = ph.temperature_K
    dp = getattr(wl, "dispersion", None)
    if dp is not None:
        c.disp_amp, c.disp_c, c.disp_s0 = dp.amp_mev, dp.c_A, dp.s0
    br = getattr(wl, "bragg", None)
    if br is not None:
        d = np.ascontiguousarray(br.d, dtype=np.float64)
        w = np.ascontiguousarray(br.w, dtype=np.float64)
        c._refl_keep = (d, w)
        c.refl_d = d.ctypes.data_as(C.POINTER(C.c_double))
        c.refl_w = w.ctypes.data_as(C.POINTER(C.c_double))
        c.n_refl = d.size
    det = wl.detector
    if det is not None:
        c.det_kind = det.kind
        c.det_radius_m, c.det_height_m = det.radius_m, det.height_m
        c.n_phi, c.n_y, c.n_rows = det.n_phi, det.n_y, det.n_rows
        c.packs[:] = list(det.packs) + [0] * (3 - len(det.packs))
        c.row_y_m[:] = list(det.row_y_m) + [0.0] * (3 - len(det.row_y_m))
        c.tubes_per_pack, c.pixels_per_tube = det.tubes_per_pack, det.pixels_per_tube
        c.tube_r_m, c.tube_len_m = det.tube_r_m, det.tube_len_m
        c.tube_pitch_m, c.pack_gap_m, c.phi0_rad = det.tube_pitch_m, det.pack_gap_m, det.phi0_rad
        c.he3_n_per_A3, c.he3_sig_abs_b = det.he3_n_per_A3, det.he3_sig_abs_b
        c.tof_min_s, c.tof_max_s, c.n_tof = det.tof_min_s, det.tof_max_s, det.n_tof
        c.det_multi_tube = int(getattr(det, "multi_tube", False))
    c.seed, c.sim_id = wl.seed, wl.sim_id
    return c


def philox(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(o))
    return o


def uniforms(seed, sim_id, nid, event, block):
    u = np.zeros(2)
    lib().orc_uniforms(seed, sim_id, nid, event, block, _ptr(u))
    return u


def shape_segments(scatterer, r, d):
    wl_scat = Scat()
    dims = list(scatterer.dims) + [0.0] * (3 - len(scatterer.dims))
    wl_scat.kind = scatterer.kind
    wl_scat.dims[:] = dims
    wl_scat.rot_y = scatterer.rot_y
    sa, sb = np.zeros(2), np.zeros(2)
    r = np.asarray(r, dtype=np.float64)
    d = np.asarray(d, dtype=np.float64)
    n = lib().orc_shape_segments(C.byref(wl_scat), _ptr(r), _ptr(d), _ptr(sa), _ptr(sb))
    return [(sa[i], sb[i]) for i in range(n)]


def kernel_scatter(wl, ktype, speed, d, u):
    cfg = make_config(wl)
    d = np.asarray(d, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    d_out = np.zeros(3)
    sp, fac = C.c_double(), C.c_double()
    ev = np.zeros(1, dtype=EVENT_DTYPE)
    ok = lib().orc_kernel_scatter(C.byref(cfg), ktype, speed, _ptr(d), _ptr(u), C.byref(sp),
                                  _ptr(d_out), C.byref(fac), _ptr(ev))
    if not ok:
        return None
    return {"speed": sp.value, "d": d_out, "factor": fac.value, "event": ev[0]}


def detect(wl, r, v, t, w, u_det):
    cfg = make_config(wl)
    r = np.asarray(r, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    pix, tof, wd = C.c_int32(), C.c_double(), C.c_double()
    b = lib().orc_detect(C.byref(cfg), _ptr(r), _ptr(v), t, w, u_det, C.byref(pix),
                         C.byref(tof), C.byref(wd))
    return {"bin": b, "pixel": pix.value, "tof": tof.value, "w_det": wd.value}


def detect_multi(wl, r, v, t, w, u):
    """The multi-tube detector on one packet: a list of (bin, pixel, tof, w_det)."""
    cfg = make_config(wl)
    r = np.asarray(r, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    pix = np.zeros(3, dtype=np.int32)
    tof, wd = np.zeros(3), np.zeros(3)
    b = np.zeros(3, dtype=np.int64)
    k = lib().orc_detect_multi(C.byref(cfg), _ptr(r), _ptr(v), t, w, _ptr(u), _ptr(pix),
                               _ptr(tof), _ptr(wd), _ptr(b))
    return [(int(b[i]), int(pix[i]), float(tof[i]), float(wd[i])) for i in range(k)]


def trace(wl, first_id=0, n=None, packets=True, events=False, hist=True, tallies=True):
    """Chain-mode tracer: per-packet records, per-scatter events, histogram, tallies."""
    n = wl.n if n is None else n
    cfg = make_config(wl)
    slots = wl.max_orders + 1
    pk = np.zeros(n * slots, dtype=PACKET_DTYPE) if packets else None
    ev = np.zeros(n * max(wl.max_orders, 1), dtype=EVENT_DTYPE) if events else None
    h = None
    if hist and wl.detector is not None:
        h = np.zeros(wl.detector.n_bins)
    t = np.zeros(NTALLY) if tallies else None
    rc = lib().orc_trace(C.byref(cfg), first_id, n, _ptr(pk), _ptr(ev), _ptr(h), _ptr(t))
    if rc:
        raise ValueError("oracle rejected the configuration")
    return {"packets": pk, "events": ev, "hist": h, "tallies": t}


def trace_paper(wl, first_id=0, n=None):
    """Paper-literal recursive estimator: histogram and tallies."""
    n = wl.n if n is None else n
    cfg = make_config(wl)
    h = np.zeros(wl.detector.n_bins) if wl.detector is not None else None
    t = np.zeros(NTALLY)
    rc = lib().orc_trace_paper(C.byref(cfg), first_id, n, _ptr(h), _ptr(t))
    if rc:
        raise ValueError("oracle rejected the configuration")
    return {"hist": h, "tallies": t}


def grad(wl, target, scale_c, first_id=0, n=None, gs=0):
    """Chi-squared loss, forward histogram, d loss / d S(Q,E), d loss / d (sig_abs, sig_s)."""
    n = wl.n if n is None else n
    cfg = make_config(wl)
    target = np.ascontiguousarray(target, dtype=np.float64)
    h = np.zeros(wl.detector.n_bins)
    loss = C.c_double()
    dsqe = np.zeros(wl.sqe.table.size if wl.sqe is not None else 1)
    dsig = np.zeros(2)
    rc = lib().orc_grad(C.byref(cfg), first_id, n, _ptr(target), scale_c, gs, _ptr(h),
                        C.byref(loss), _ptr(dsqe), _ptr(dsig))
    if rc:
        raise ValueError("oracle rejected the configuration")
    shape = wl.sqe.table.shape if wl.sqe is not None else (1,)
    return {"hist": h, "loss": loss.value, "dsqe": dsqe.reshape(shape), "dsig": dsig}


def adjoint(wl, hist, target, scale_c, first_id=0, n=None, gs=0):
    """Loss of the whole run's histogram `hist` and the gradient of neutrons
    first_id..first_id+n-1 (the share of one part of a split run)."""
    n = wl.n if n is None else n
    cfg = make_config(wl)
    hist = np.ascontiguousarray(hist, dtype=np.float64)
    target = np.ascontiguousarray(target, dtype=np.float64)
    out = C.c_double()
    dsqe = np.zeros(wl.sqe.table.size if wl.sqe is not None else 1)
    dsig = np.zeros(2)
    rc = lib().orc_adjoint(C.byref(cfg), first_id, n, _ptr(hist), _ptr(target), scale_c, gs,
                           C.byref(out), _ptr(dsqe), _ptr(dsig))
    if rc:
        raise ValueError("oracle rejected the configuration")
    shape = wl.sqe.table.shape if wl.sqe is not None else (1,)
    return {"loss": out.value, "dsqe": dsqe.reshape(shape), "dsig": dsig}


def loss(wl, target, scale_c, first_id=0, n=None):
    n = wl.n if n is None else n
    cfg = make_config(wl)
    target = np.ascontiguousarray(target, dtype=np.float64)
    h = np.zeros(wl.detector.n_bins)
    out = C.c_double()
    rc = lib().orc_loss(C.byref(cfg), first_id, n, _ptr(target), scale_c, _ptr(h),
                        C.byref(out))
    if rc:
        raise ValueError("oracle rejected the configuration")
    return out.value


def bvk_modes(wl, q):
    """Phonon energies (meV, ascending) and eigenvectors (columns) at q (1/A, crystal frame)."""
    cfg = make_config(wl)
    q = np.asarray(q, dtype=np.float64)
    hw, ev = np.zeros(3), np.zeros(9)
    lib().orc_bvk_modes(C.byref(cfg), _ptr(q), _ptr(hw), _ptr(ev))
    return hw, ev.reshape(3, 3)


def kernel_bvk(wl, rot_y, speed, d, u):
    cfg = make_config(wl)
    d = np.asarray(d, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    d_out = np.zeros(3)
    sp, fac = C.c_double(), C.c_double()
    ev = np.zeros(1, dtype=EVENT_DTYPE)
    ok = lib().orc_kernel_bvk(C.byref(cfg), rot_y, speed, _ptr(d), _ptr(u), C.byref(sp),
                              _ptr(d_out), C.byref(fac), _ptr(ev))
    return {"ok": bool(ok), "speed": sp.value, "d": d_out, "factor": fac.value, "event": ev[0]}


def phonon_tables(wl):
    """gamma_0 (1/meV), c_w (2W = c_w Q^2, A^2) and A_n (n = 1..n_max) as masses on the grid
    E = i de, i = -n_max J..n_max J (rows n - 1) of the workload's phonon kernel."""
    cfg = make_config(wl)
    g0, cw = C.c_double(), C.c_double()
    N, J = wl.phonon.nmax, wl.phonon.z.size
    M = 2 * N * J + 1
    a = np.zeros(N * M)
    m = lib().orc_phonon_tables(C.byref(cfg), C.byref(g0), C.byref(cw), _ptr(a), a.size)
    if m != M:
        raise ValueError("oracle rejected the phonon kernel")
    return {"gamma0": g0.value, "c_w": cw.value, "A": a.reshape(N, M),
            "E": np.arange(-N * J, N * J + 1) * wl.phonon.de}
