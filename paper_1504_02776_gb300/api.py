"""Torch-facing layer over the C ABI: builds the mcv.h structures from workload descriptions
(mcv_inputs) and owns the device buffers of a run.  Marshalling only: the ray tracing,
the detector and the histogram all run in libmcv.so's kernels.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import binding as B


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def beam_struct(beam):
    return B.BeamParams(beam.ei_mev, beam.ei_rel_sigma, beam.div_sigma_rad, beam.width_m,
                        beam.height_m, beam.z0_m, beam.l1_m)


def detector_struct(det):
    d = B.Detector()
    d.kind = det.kind
    d.radius_m, d.height_m = det.radius_m, det.height_m
    d.n_phi, d.n_y, d.n_rows = det.n_phi, det.n_y, det.n_rows
    d.packs[:] = list(det.packs) + [0] * (3 - len(det.packs))
    d.row_y_m[:] = list(det.row_y_m) + [0.0] * (3 - len(det.row_y_m))
    d.tubes_per_pack, d.pixels_per_tube = det.tubes_per_pack, det.pixels_per_tube
    d.tube_r_m, d.tube_len_m, d.tube_pitch_m = det.tube_r_m, det.tube_len_m, det.tube_pitch_m
    d.pack_gap_m, d.phi0_rad = det.pack_gap_m, det.phi0_rad
    d.he3_n_per_A3, d.he3_sig_abs_b = det.he3_n_per_A3, det.he3_sig_abs_b
    d.tof_min_s, d.tof_max_s, d.n_tof = det.tof_min_s, det.tof_max_s, det.n_tof
    d.multi_tube = int(getattr(det, "multi_tube", False))
    return d


def phonon_struct(ph, stream=None):
    """mcv_phonon of a workload's phonon density of states, its tables built by the library
    (mcv_phonon_build) into a device tensor; returns (struct, tensor) -- keep the tensor."""
    import numpy as np
    z = np.ascontiguousarray(ph.z, dtype=np.float64)
    p = B.Phonon()
    p.n_modes, p.n_max = z.size, ph.nmax
    p.de_mev, p.mass_u, p.temperature_K = ph.de, ph.mass_u, ph.temperature_K
    p.p[:] = list(ph.p)
    nbytes = B.mcv_phonon_table_bytes(p.n_modes, p.n_max)
    if nbytes <= 0:
        raise ValueError("bad phonon table size")
    tables = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    B.mcv_phonon_build(z.ctypes.data_as(C.c_void_p), p, C.c_void_p(tables.data_ptr()), nbytes,
                       _stream() if stream is None else stream)
    return p, tables


_PHONON_CACHE = {}


def phonon_for(ph):
    """The (struct, device tables) of a PhononDos, built once per description."""
    import numpy as np
    key = (np.asarray(ph.z, dtype=np.float64).tobytes(), ph.de, ph.mass_u, ph.nmax,
           tuple(ph.p), ph.temperature_K, torch.cuda.current_device())
    if key not in _PHONON_CACHE:
        _PHONON_CACHE[key] = phonon_struct(ph)
    return _PHONON_CACHE[key]


_BRAGG_CACHE = {}


def bragg_for(br):
    """(mcv_bragg struct, device tables) of a reflection list, built once per description."""
    import numpy as np
    d = np.ascontiguousarray(br.d, dtype=np.float64)
    w = np.ascontiguousarray(br.w, dtype=np.float64)
    key = (d.tobytes(), w.tobytes(), torch.cuda.current_device())
    if key not in _BRAGG_CACHE:
        b = B.Bragg()
        nbytes = B.mcv_bragg_table_bytes(d.size)
        if nbytes <= 0:
            raise ValueError("bad reflection count")
        tables = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        B.mcv_bragg_build(d.ctypes.data_as(C.c_void_p), w.ctypes.data_as(C.c_void_p), d.size, b,
                          C.c_void_p(tables.data_ptr()), nbytes, _stream())
        _BRAGG_CACHE[key] = (b, tables)
    return _BRAGG_CACHE[key]


class EventBuffers:
    """Caller-owned device arrays of an event list (mcv_event_list) with `capacity` records."""

    def __init__(self, capacity, device="cuda"):
        self.capacity = capacity
        self.pixel = torch.empty(capacity, dtype=torch.int32, device=device)
        self.sim = torch.empty(capacity, dtype=torch.int32, device=device)
        self.tof = torch.empty(capacity, dtype=torch.float64, device=device)
        self.w = torch.empty(capacity, dtype=torch.float64, device=device)
        self.count = torch.zeros(1, dtype=torch.int64, device=device)
        self._struct = B.EventList(self.pixel.data_ptr(), self.sim.data_ptr(), self.tof.data_ptr(),
                                   self.w.data_ptr(), capacity, self.count.data_ptr())

    def struct(self):
        return self._struct

    def n(self):
        return int(self.count.item())

    def to_dict(self):
        m = min(self.n(), self.capacity)
        return {"pixel": self.pixel[:m].cpu().numpy(), "sim": self.sim[:m].cpu().numpy(),
                "tof": self.tof[:m].cpu().numpy(), "w": self.w[:m].cpu().numpy(),
                "count": self.n()}


def sample_struct(wl, fp_mode, table=None, estimator=B.EST_CHAIN):
    """mcv_sample from a workload; `table` is the device FP32 S(Q,E) tensor (if any); the
    phonon kernel's tables are built on the device once per description (phonon_for)."""
    s = B.Sample()
    s.n_scatterers = len(wl.scatterers)
    for j, sc in enumerate(wl.scatterers):
        t = s.scat[j]
        t.shape = sc.kind
        t.dims[:] = list(sc.dims) + [0.0] * (3 - len(sc.dims))
        t.rot_y_rad = sc.rot_y
        t.n_per_A3, t.sig_abs_b = sc.n_per_A3, sc.sig_abs_b
        t.n_kernels = len(sc.kernels)
        for k, (kt, ks) in enumerate(sc.kernels):
            t.kernel[k] = kt
            t.kernel_sig_b[k] = ks
    s.max_orders, s.min_prob, s.fp_mode = wl.max_orders, wl.min_prob, fp_mode
    s.estimator = estimator
    if wl.sqe is not None:
        if table is None:
            raise ValueError("the S(Q,E) table must be on the device")
        s.sqe.table = table.data_ptr()
        s.sqe.nq, s.sqe.ne = wl.sqe.nq, wl.sqe.ne
        s.sqe.q_max, s.sqe.e_min, s.sqe.e_max = wl.sqe.q_max, wl.sqe.e_min, wl.sqe.e_max
    if wl.bvk is not None:
        v = wl.bvk
        s.bvk.phi_Nm, s.bvk.mass_u, s.bvk.a_A = v.phi_Nm, v.mass_u, v.a_A
        s.bvk.msd_A2, s.bvk.temperature_K = v.msd_A2, v.temperature_K
    if getattr(wl, "phonon", None) is not None:
        ph, _ = phonon_for(wl.phonon)
        C.memmove(C.addressof(s.phonon), C.addressof(ph), C.sizeof(ph))
    if getattr(wl, "bragg", None) is not None:
        br, _ = bragg_for(wl.bragg)
        C.memmove(C.addressof(s.bragg), C.addressof(br), C.sizeof(br))
    dp = getattr(wl, "dispersion", None)
    if dp is not None:
        s.dispersion.amp_mev, s.dispersion.c_A, s.dispersion.s0 = dp.amp_mev, dp.c_A, dp.s0
    return s


class NeutronBuffers:
    """Caller-owned SoA device arrays for `n` packet slots."""

    def __init__(self, n, fp_mode, device="cuda"):
        dt = torch.float32 if fp_mode == B.FP32 else torch.float64
        self.n = n
        self.fp_mode = fp_mode
        mk = lambda: torch.empty(n, dtype=dt, device=device)
        self.x, self.y, self.z, self.vx, self.vy, self.vz, self.w = (mk() for _ in range(7))
        self.t = torch.empty(n, dtype=torch.float64, device=device)
        self.id = torch.empty(n, dtype=torch.int64, device=device)
        self.order = torch.full((n,), -1, dtype=torch.int32, device=device)

    def struct(self):
        return B.Neutrons(*(t.data_ptr() for t in (self.x, self.y, self.z, self.vx, self.vy,
                                                    self.vz, self.t, self.w, self.id,
                                                    self.order)), self.n)

    def to_dict(self):
        return {k: getattr(self, k).cpu().numpy() for k in
                ("x", "y", "z", "vx", "vy", "vz", "t", "w", "id", "order")}


class Context:
    """One mcv_ctx on one CUDA device."""

    def __init__(self, device=0):
        torch.cuda.set_device(device)
        self.device = device
        self.handle = B.mcv_create(device)

    def close(self):
        if self.handle is not None:
            B.mcv_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sync(self):
        B.mcv_sync(self.handle, _stream())

    # ---- forward path --------------------------------------------------------------
    def table(self, wl):
        if wl.sqe is None:
            return None
        return torch.from_numpy(wl.sqe.table).to("cuda", non_blocking=False).contiguous()

    def new_hist(self, det):
        counts = torch.zeros(det.n_bins, dtype=torch.float64, device="cuda")
        tallies = torch.zeros(B.MCV_NTALLY, dtype=torch.float64, device="cuda")
        return counts, tallies

    def trace(self, wl, fp_mode=B.FP64, n=None, first_id=0, table=None, counts=None,
              tallies=None, beam_in=None, sync=True, events=None, hist=True,
              estimator=B.EST_CHAIN):
        """Fused path: source -> sample -> detector -> histogram; returns (counts, tallies).
        events: an EventBuffers that receives every detected packet as well (event mode);
        hist=False with events: no histogram, only the tallies and the event list;
        estimator=B.EST_PAPER: the paper's recursive estimator instead of the chain."""
        n = wl.n if n is None else n
        if table is None:
            table = self.table(wl)
        if counts is None and tallies is None:
            if hist:
                counts, tallies = self.new_hist(wl.detector)
            else:
                tallies = torch.zeros(B.MCV_NTALLY, dtype=torch.float64, device="cuda")
        sample = sample_struct(wl, fp_mode, table, estimator)
        det = detector_struct(wl.detector)
        hist = B.Hist(_ptr(counts), _ptr(tallies),
                      C.pointer(events.struct()) if events is not None else None)
        inp = beam_in.struct() if beam_in is not None else None
        B.mcv_trace_sample(self.handle, sample, beam_struct(wl.beam), inp, wl.seed, wl.sim_id,
                           first_id, n, det, hist, None, _stream())
        if sync:
            self.sync()
        return counts, tallies

    def trace_packets(self, wl, fp_mode=B.FP64, n=None, first_id=0, table=None, beam_in=None,
                      tallies=None, sync=True):
        """Unfused sample step: every emitted packet into n*(max_orders+1) slots."""
        n = wl.n if n is None else n
        if table is None:
            table = self.table(wl)
        pk = NeutronBuffers(n * (wl.max_orders + 1), fp_mode)
        sample = sample_struct(wl, fp_mode, table)
        hist = B.Hist(None, _ptr(tallies)) if tallies is not None else None
        inp = beam_in.struct() if beam_in is not None else None
        B.mcv_trace_sample(self.handle, sample, beam_struct(wl.beam), inp, wl.seed, wl.sim_id,
                           first_id, n, None, hist, pk.struct(), _stream())
        if sync:
            self.sync()
        return pk

    def beam(self, wl, fp_mode=B.FP64, n=None, first_id=0, sync=True):
        n = wl.n if n is None else n
        out = NeutronBuffers(n, fp_mode)
        B.mcv_beam(self.handle, beam_struct(wl.beam), fp_mode, wl.seed, wl.sim_id, first_id, n,
                   out.struct(), _stream())
        if sync:
            self.sync()
        return out

    def detect(self, wl, packets, counts=None, tallies=None, events=True, sync=True,
               event_list=None):
        """Detector step on stored packets; returns (counts, tallies, events dict).
        event_list: an EventBuffers that receives every detected packet (event mode)."""
        det = detector_struct(wl.detector)
        if counts is None and tallies is None:
            counts, tallies = self.new_hist(wl.detector)
        ev = None
        evs = None
        if events:
            n = packets.n
            ev = {"pixel": torch.empty(n, dtype=torch.int32, device="cuda"),
                  "tof": torch.empty(n, dtype=torch.float64, device="cuda"),
                  "w_det": torch.empty(n, dtype=torch.float64, device="cuda"),
                  "bin": torch.empty(n, dtype=torch.int64, device="cuda")}
            evs = B.Events(*(ev[k].data_ptr() for k in ("pixel", "tof", "w_det", "bin")))
        hist = B.Hist(_ptr(counts), _ptr(tallies),
                      C.pointer(event_list.struct()) if event_list is not None else None)
        B.mcv_detect(self.handle, det, packets.fp_mode, packets.struct(), wl.seed, wl.sim_id,
                     hist, evs, _stream())
        if sync:
            self.sync()
        return counts, tallies, ev


# ---- batched launches ------------------------------------------------------------------
def _batch_detector(workloads):
    """The shared detector geometry of a batch (time windows may differ per simulation)."""
    import dataclasses
    key = lambda d: {k: v for k, v in dataclasses.asdict(d).items()
                     if k not in ("tof_min_s", "tof_max_s")}
    d0 = workloads[0].detector
    for wl in workloads[1:]:
        if key(wl.detector) != key(d0):
            raise ValueError("the simulations of a batch share one detector geometry")
    return d0


def _batch_sims(ctx, workloads, fp_mode, hists, first_ids, tables, event_lists=None):
    """mcv_sim entries for the workloads; returns (sims, structs kept alive, hists)."""
    keep = []
    sims = []
    if hists is None:
        hists = [ctx.new_hist(wl.detector) for wl in workloads]
    for k, wl in enumerate(workloads):
        table = None
        if wl.sqe is not None:
            key = id(wl.sqe.table)
            if key not in tables:
                tables[key] = ctx.table(wl)
            table = tables[key]
        sample = sample_struct(wl, fp_mode, table)
        beam = beam_struct(wl.beam)
        keep += [sample, beam]
        counts, tallies = hists[k]
        first = 0 if first_ids is None else first_ids[k]
        ev = None
        if event_lists is not None and event_lists[k] is not None:
            ev = C.pointer(event_lists[k].struct())
            keep.append(ev)
        sims.append(B.Sim(C.pointer(sample), C.pointer(beam), wl.seed, wl.sim_id, first, wl.n,
                          wl.detector.tof_min_s, wl.detector.tof_max_s,
                          B.Hist(_ptr(counts), _ptr(tallies), ev)))
    return sims, keep, hists


class Batch:
    """Simulations that share one detector geometry, traced by one persistent launch
    (mcv_batch_create / mcv_batch_run).  Each workload brings its sample, beam, neutron
    count, random stream (seed, sim_id) and time window (its detector's tof_min_s,
    tof_max_s).  `hists`: one (counts, tallies) pair of device tensors per workload,
    accumulated into; None allocates zeroed ones (self.hists)."""

    def __init__(self, ctx, workloads, fp_mode=B.FP32, hists=None, first_ids=None):
        self.ctx = ctx
        self.workloads = list(workloads)
        self.tables = {}
        self.det = detector_struct(_batch_detector(self.workloads))
        sims, self._keep, self.hists = _batch_sims(ctx, self.workloads, fp_mode, hists,
                                                   first_ids, self.tables)
        self.handle = B.mcv_batch_create(ctx.handle, sims, self.det, fp_mode)

    def run(self, sync=False):
        B.mcv_batch_run(self.handle, _stream())
        if sync:
            self.ctx.sync()

    def tune(self, trial_neutrons=0):
        B.mcv_batch_tune(self.handle, trial_neutrons, _stream())
        return self.shape()

    def shape(self):
        return B.mcv_batch_shape(self.handle)

    def close(self):
        if getattr(self, "handle", None) is not None:
            B.mcv_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _trace_batch(self, workloads, fp_mode=B.FP32, hists=None, first_ids=None, sync=True,
                 event_lists=None):
    """One-shot batched launch (mcv_trace_batch); returns the (counts, tallies) pairs.
    event_lists: one EventBuffers (or None) per workload; several may be the same object."""
    det = detector_struct(_batch_detector(workloads))
    tables = {}
    sims, keep, hists = _batch_sims(self, workloads, fp_mode, hists, first_ids, tables,
                                    event_lists)
    B.mcv_trace_batch(self.handle, sims, det, fp_mode, _stream())
    if sync:
        self.sync()
    del keep
    return hists


Context.trace_batch = _trace_batch
Context.batch = lambda self, workloads, fp_mode=B.FP32, hists=None, first_ids=None: Batch(
    self, workloads, fp_mode, hists, first_ids)


def _grad_call(c, wl, target, scale_c, fp_mode, n, first_id, table, sig_abs, sig_s,
               grad_scatterer, counts=None, g_work=None):
    """mcv_grad with the cross sections of `grad_scatterer` replaced by sig_abs, sig_s (the
    kernels' cross sections scaled together).  g_work (optional): a tensor of n_bins doubles
    that receives dchi2/dI of every bin; without it the adjoint evaluates dchi2/dI only where
    its packets land."""
    sample = sample_struct(wl, fp_mode, table)
    sc = sample.scat[grad_scatterer]
    if sig_abs is not None:
        sc.sig_abs_b = float(sig_abs)
    if sig_s is not None:
        total = sum(sc.kernel_sig_b[k] for k in range(sc.n_kernels))
        for k in range(sc.n_kernels):
            sc.kernel_sig_b[k] = sc.kernel_sig_b[k] * float(sig_s) / total
    nb = wl.detector.n_bins
    if counts is None:
        counts = torch.empty(nb, dtype=torch.float64, device="cuda")
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    dsqe = torch.empty(wl.sqe.table.size if wl.sqe is not None else 1, dtype=torch.float64,
                       device="cuda")
    dsig = torch.empty(2, dtype=torch.float64, device="cuda")
    hist = B.Hist(_ptr(counts), None)
    B.mcv_grad(c.handle, sample, beam_struct(wl.beam), detector_struct(wl.detector), wl.seed,
               wl.sim_id, first_id, n, _ptr(target), float(scale_c), grad_scatterer, hist,
               _ptr(g_work), _ptr(loss), _ptr(dsqe), _ptr(dsig), _stream())
    return {"loss": loss, "dsqe": dsqe, "dsig": dsig, "hist": counts, "g": g_work}


def _grad_method(self, wl, target, scale_c, fp_mode=B.FP64, n=None, first_id=0, table=None,
                 grad_scatterer=0, sync=True, counts=None, g_work=None):
    """Chi-squared loss of the simulated histogram and its adjoint gradient (FP64 outputs)."""
    n = wl.n if n is None else n
    if table is None:
        table = self.table(wl)
    out = _grad_call(self, wl, target, scale_c, fp_mode, n, first_id, table, None, None,
                     grad_scatterer, counts, g_work)
    if sync:
        self.sync()
    return out


Context.grad = _grad_method


class Chi2Loss(torch.autograd.Function):
    """loss = chi2(I(table, sig_abs, sig_s), target) with the hand-written adjoint kernel as
    its backward.  `table` is the FP32 S(Q,E) tensor on the device; sig_abs and sig_s are
    0-d tensors (barn) of scatterer `grad_scatterer`."""

    @staticmethod
    def forward(fctx, table, sig_abs, sig_s, run):
        c, wl, target, scale_c, fp_mode, n, first_id, gs = run
        out = _grad_call(c, wl, target, scale_c, fp_mode, n, first_id, table.detach().contiguous(),
                         sig_abs.item(), sig_s.item(), gs)
        fctx.save_for_backward(out["dsqe"], out["dsig"])
        fctx.shapes = (table.shape, table.dtype, sig_abs.dtype, sig_s.dtype)
        return out["loss"][0].to(torch.float64)

    @staticmethod
    def backward(fctx, grad_out):
        dsqe, dsig = fctx.saved_tensors
        shape, tdt, adt, sdt = fctx.shapes
        g_table = (grad_out * dsqe).reshape(shape).to(tdt)
        return g_table, (grad_out * dsig[0]).to(adt), (grad_out * dsig[1]).to(sdt), None


def chi2_loss(ctx, wl, table, sig_abs, sig_s, target, scale_c, fp_mode=B.FP32, n=None,
              first_id=0, grad_scatterer=0):
    n = wl.n if n is None else n
    run = (ctx, wl, target, scale_c, fp_mode, n, first_id, grad_scatterer)
    return Chi2Loss.apply(table, sig_abs, sig_s, run)


def _adjoint_call(c, wl, hist, target, scale_c, fp_mode, n, first_id, table, grad_scatterer):
    """mcv_adjoint: loss of the whole run's histogram `hist`, gradient of this id range."""
    sample = sample_struct(wl, fp_mode, table)
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    dsqe = torch.empty(wl.sqe.table.size if wl.sqe is not None else 1, dtype=torch.float64,
                       device="cuda")
    dsig = torch.empty(2, dtype=torch.float64, device="cuda")
    B.mcv_adjoint(c.handle, sample, beam_struct(wl.beam), detector_struct(wl.detector), wl.seed,
                  wl.sim_id, first_id, n, _ptr(hist), _ptr(target), float(scale_c),
                  grad_scatterer, None, _ptr(loss), _ptr(dsqe), _ptr(dsig), _stream())
    return {"loss": loss, "dsqe": dsqe, "dsig": dsig}


def _grad_sharded(self, wl, target, scale_c, rank, world, fp_mode=B.FP32, n_total=None,
                  table=None, grad_scatterer=0, group=None, sync=True):
    """The chi-squared loss and gradient of a run of n_total neutrons (default wl.n) split
    over the ranks of `group` (one GPU each, NCCL): this rank traces its share of the ids,
    the histograms are summed over the ranks, this rank's adjoint runs on the summed
    histogram, and the gradients are summed (shards.sharded_gradient)."""
    from . import shards
    n_total = wl.n if n_total is None else n_total
    if table is None:
        table = self.table(wl)
    hist = torch.zeros(wl.detector.n_bins, dtype=torch.float64, device="cuda")

    def forward(first, n, h):
        self.trace(wl, fp_mode=fp_mode, n=n, first_id=first, table=table, counts=h,
                   tallies=None, sync=False)

    def adjoint(first, n, h):
        return _adjoint_call(self, wl, h, target, scale_c, fp_mode, n, first, table,
                             grad_scatterer)

    out = shards.sharded_gradient(forward, adjoint, hist, rank, world, n_total, group=group)
    if sync:
        self.sync()
    return out


Context.grad_sharded = _grad_sharded
