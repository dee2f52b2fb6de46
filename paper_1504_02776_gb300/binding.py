"""Python binding of libmcv.so: ctypes mirrors of include/mcv.h and thin wrappers with the
same names.  Argument marshalling only -- every step of the ray tracing runs in the CUDA
kernels of the library.  PyTorch provides device memory and streams.

The library is loaded from this package folder; if it is missing the import fails (there is
no CPU fallback).
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmcv.so")

MCV_OK, MCV_EINVAL, MCV_ENOMEM, MCV_ECUDA, MCV_ETIMEOUT, MCV_EDEVICE = range(6)
MCV_MAX_SCATTERERS, MCV_MAX_TUBES_PER_ROW, MCV_NTALLY = 4, 512, 8
SHAPE_SOLID_CYL, SHAPE_HOLLOW_CYL, SHAPE_BLOCK = 0, 1, 2
KERNEL_ISO, KERNEL_SQE, KERNEL_BVK, KERNEL_PHONON, KERNEL_BRAGG, KERNEL_DISP = 0, 1, 2, 3, 4, 5
DET_NONE, DET_SURFACE, DET_TUBES = 0, 1, 2
FP64, FP32 = 0, 1
EST_CHAIN, EST_PAPER = 0, 1
(T_BEAMSTOP, T_WDET, T_WOVER, T_NDET, T_NOVER, T_NMISS, T_NHIT, T_NEMIT) = range(8)

STATUS_NAMES = {0: "MCV_OK", 1: "MCV_EINVAL", 2: "MCV_ENOMEM", 3: "MCV_ECUDA",
                4: "MCV_ETIMEOUT", 5: "MCV_EDEVICE"}


class McvError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class BeamParams(C.Structure):
    _fields_ = [("ei_mev", C.c_double), ("ei_rel_sigma", C.c_double),
                ("div_sigma_rad", C.c_double), ("width_m", C.c_double),
                ("height_m", C.c_double), ("z0_m", C.c_double), ("l1_m", C.c_double)]


class Scatterer(C.Structure):
    _fields_ = [("shape", C.c_int), ("dims", C.c_double * 3), ("rot_y_rad", C.c_double),
                ("n_per_A3", C.c_double), ("sig_abs_b", C.c_double), ("n_kernels", C.c_int),
                ("kernel", C.c_int * 2), ("kernel_sig_b", C.c_double * 2)]


class Sqe(C.Structure):
    _fields_ = [("table", C.c_void_p), ("nq", C.c_int), ("ne", C.c_int),
                ("q_max", C.c_double), ("e_min", C.c_double), ("e_max", C.c_double)]


class Bvk(C.Structure):
    _fields_ = [("phi_Nm", C.c_double), ("mass_u", C.c_double), ("a_A", C.c_double),
                ("msd_A2", C.c_double), ("temperature_K", C.c_double)]


class Phonon(C.Structure):
    _fields_ = [("tables", C.c_void_p), ("n_modes", C.c_int), ("n_max", C.c_int),
                ("de_mev", C.c_double), ("mass_u", C.c_double), ("temperature_K", C.c_double),
                ("p", C.c_double * 3), ("gamma0", C.c_double), ("c_w", C.c_double)]


class Bragg(C.Structure):
    _fields_ = [("tables", C.c_void_p), ("n", C.c_int)]


class Dispersion(C.Structure):
    _fields_ = [("amp_mev", C.c_double), ("c_A", C.c_double), ("s0", C.c_double)]


class Sample(C.Structure):
    _fields_ = [("n_scatterers", C.c_int), ("scat", Scatterer * MCV_MAX_SCATTERERS),
                ("max_orders", C.c_int), ("min_prob", C.c_double), ("fp_mode", C.c_int),
                ("sqe", Sqe), ("bvk", Bvk), ("phonon", Phonon), ("bragg", Bragg),
                ("dispersion", Dispersion), ("estimator", C.c_int)]


class Detector(C.Structure):
    _fields_ = [("kind", C.c_int), ("radius_m", C.c_double), ("height_m", C.c_double),
                ("n_phi", C.c_int), ("n_y", C.c_int), ("n_rows", C.c_int),
                ("packs", C.c_int * 3), ("row_y_m", C.c_double * 3),
                ("tubes_per_pack", C.c_int), ("pixels_per_tube", C.c_int),
                ("tube_r_m", C.c_double), ("tube_len_m", C.c_double),
                ("tube_pitch_m", C.c_double), ("pack_gap_m", C.c_double),
                ("phi0_rad", C.c_double), ("he3_n_per_A3", C.c_double),
                ("he3_sig_abs_b", C.c_double), ("tof_min_s", C.c_double),
                ("tof_max_s", C.c_double), ("n_tof", C.c_int), ("multi_tube", C.c_int)]


class Neutrons(C.Structure):
    _fields_ = [("x", C.c_void_p), ("y", C.c_void_p), ("z", C.c_void_p),
                ("vx", C.c_void_p), ("vy", C.c_void_p), ("vz", C.c_void_p),
                ("t", C.c_void_p), ("w", C.c_void_p), ("id", C.c_void_p),
                ("order", C.c_void_p), ("n", C.c_int64)]


class EventList(C.Structure):
    _fields_ = [("pixel", C.c_void_p), ("sim", C.c_void_p), ("tof", C.c_void_p),
                ("w", C.c_void_p), ("capacity", C.c_int64), ("count", C.c_void_p)]


class Hist(C.Structure):
    _fields_ = [("counts", C.c_void_p), ("tallies", C.c_void_p),
                ("events", C.POINTER(EventList))]


class Events(C.Structure):
    _fields_ = [("pixel", C.c_void_p), ("tof", C.c_void_p), ("w_det", C.c_void_p),
                ("bin", C.c_void_p)]


class Sim(C.Structure):
    _fields_ = [("sample", C.POINTER(Sample)), ("beam", C.POINTER(BeamParams)),
                ("seed", C.c_uint32), ("sim_id", C.c_uint32), ("first_id", C.c_int64),
                ("n", C.c_int64), ("tof_min_s", C.c_double), ("tof_max_s", C.c_double),
                ("hist", Hist)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libmcv.so is not built (run __graft_entry__.build() or "
                          "paper_1504_02776_gb300/build.py); there is no CPU fallback")
    L = C.CDLL(LIB_PATH)
    P, st = C.c_void_p, C.c_int
    L.mcv_create.argtypes = [C.c_int, C.POINTER(C.c_void_p)]
    L.mcv_destroy.argtypes = [P]
    L.mcv_last_error.restype = C.c_char_p
    L.mcv_sync.argtypes = [P, P]
    L.mcv_detector_pixels.argtypes = [P]
    L.mcv_detector_pixels.restype = C.c_int64
    L.mcv_zero.argtypes = [P, P, C.c_int64, P]
    L.mcv_beam.argtypes = [P, P, C.c_int, C.c_uint32, C.c_uint32, C.c_int64, C.c_int64, P, P]
    L.mcv_trace_sample.argtypes = [P, P, P, P, C.c_uint32, C.c_uint32, C.c_int64, C.c_int64,
                                   P, P, P, P]
    L.mcv_detect.argtypes = [P, P, C.c_int, P, C.c_uint32, C.c_uint32, P, P, P]
    L.mcv_grad.argtypes = [P, P, P, P, C.c_uint32, C.c_uint32, C.c_int64, C.c_int64, P,
                           C.c_double, C.c_int, P, P, P, P, P, P]
    L.mcv_adjoint.argtypes = [P, P, P, P, C.c_uint32, C.c_uint32, C.c_int64, C.c_int64, P, P,
                              C.c_double, C.c_int, P, P, P, P, P]
    L.mcv_grad_noalloc.argtypes = [P, P, P, C.c_uint32, C.c_uint32, C.c_int64, C.c_int64, P,
                                   C.c_double, C.c_int, P, P, P, P, P]
    L.mcv_bench_atomics.argtypes = [P, P, C.c_int64, C.c_int64, C.c_uint64, P]
    L.mcv_bragg_table_bytes.argtypes = [C.c_int]
    L.mcv_bragg_table_bytes.restype = C.c_int64
    L.mcv_bragg_build.argtypes = [P, P, C.c_int, P, P, C.c_int64, P]
    L.mcv_phonon_table_bytes.argtypes = [C.c_int, C.c_int]
    L.mcv_phonon_table_bytes.restype = C.c_int64
    L.mcv_phonon_build.argtypes = [P, P, P, C.c_int64, P]
    L.mcv_batch_create.argtypes = [P, P, C.c_int, P, C.c_int, C.POINTER(C.c_void_p)]
    L.mcv_batch_run.argtypes = [P, P]
    L.mcv_batch_tune.argtypes = [P, C.c_int64, P]
    L.mcv_batch_shape.argtypes = [P, C.POINTER(C.c_int64), C.POINTER(C.c_int),
                                  C.POINTER(C.c_int), C.POINTER(C.c_int64)]
    L.mcv_batch_destroy.argtypes = [P]
    L.mcv_trace_batch.argtypes = [P, P, C.c_int, P, C.c_int, P]
    for name in ("mcv_create", "mcv_destroy", "mcv_sync", "mcv_zero", "mcv_beam",
                 "mcv_trace_sample", "mcv_detect", "mcv_grad", "mcv_adjoint", "mcv_grad_noalloc",
                 "mcv_phonon_build", "mcv_bragg_build", "mcv_bench_atomics",
                 "mcv_batch_create", "mcv_batch_run", "mcv_batch_tune", "mcv_batch_shape",
                 "mcv_batch_destroy", "mcv_trace_batch"):
        getattr(L, name).restype = st
    return L


lib = _load()


def _check(status):
    if status != MCV_OK:
        raise McvError(status, lib.mcv_last_error().decode())


def _ref(s):
    return None if s is None else C.byref(s)


# ---- the C entry points, same names ------------------------------------------------------
def mcv_create(device=0):
    h = C.c_void_p()
    _check(lib.mcv_create(device, C.byref(h)))
    return h


def mcv_destroy(ctx):
    _check(lib.mcv_destroy(ctx))


def mcv_sync(ctx, stream=None):
    _check(lib.mcv_sync(ctx, stream))


def mcv_detector_pixels(det):
    return lib.mcv_detector_pixels(C.byref(det))


def mcv_zero(ctx, ptr, n, stream=None):
    _check(lib.mcv_zero(ctx, ptr, n, stream))


def mcv_beam(ctx, beam, fp_mode, seed, sim_id, first_id, n, out, stream=None):
    _check(lib.mcv_beam(ctx, C.byref(beam), fp_mode, seed, sim_id, first_id, n, C.byref(out),
                        stream))


def mcv_trace_sample(ctx, sample, beam, inp, seed, sim_id, first_id, n, det, hist, packets,
                     stream=None):
    _check(lib.mcv_trace_sample(ctx, C.byref(sample), _ref(beam), _ref(inp), seed, sim_id,
                                first_id, n, _ref(det), _ref(hist), _ref(packets), stream))


def mcv_detect(ctx, det, fp_mode, packets, seed, sim_id, hist, events, stream=None):
    _check(lib.mcv_detect(ctx, C.byref(det), fp_mode, C.byref(packets), seed, sim_id,
                          _ref(hist), _ref(events), stream))


def mcv_grad(ctx, sample, beam, det, seed, sim_id, first_id, n, target, scale_c,
             grad_scatterer, hist, g_work, loss, dsqe, dsig, stream=None):
    _check(lib.mcv_grad(ctx, C.byref(sample), C.byref(beam), C.byref(det), seed, sim_id,
                        first_id, n, target, scale_c, grad_scatterer, C.byref(hist), g_work,
                        loss, dsqe, dsig, stream))


def mcv_adjoint(ctx, sample, beam, det, seed, sim_id, first_id, n, hist, target, scale_c,
                grad_scatterer, g_work, loss, dsqe, dsig, stream=None):
    _check(lib.mcv_adjoint(ctx, C.byref(sample), C.byref(beam), C.byref(det), seed, sim_id,
                           first_id, n, hist, target, scale_c, grad_scatterer, g_work, loss,
                           dsqe, dsig, stream))


def mcv_grad_noalloc(sample, beam, det, seed, sim_id, first_id, n, target, scale_c,
                     grad_scatterer, hist, loss, dsqe, dsig, stream=None):
    """mcv_grad without a context and without a caller work buffer: for callers that cannot
    allocate device memory (the library keeps the work buffer in a fixed device array)."""
    _check(lib.mcv_grad_noalloc(C.byref(sample), C.byref(beam), C.byref(det), seed, sim_id,
                                first_id, n, target, scale_c, grad_scatterer, C.byref(hist),
                                loss, dsqe, dsig, stream))


def mcv_bench_atomics(ctx, hist, n_bins, n_adds, seed=0, stream=None):
    _check(lib.mcv_bench_atomics(ctx, hist, n_bins, n_adds, seed, stream))


def mcv_bragg_table_bytes(n):
    return lib.mcv_bragg_table_bytes(n)


def mcv_bragg_build(d_A, w, n, bragg, tables, nbytes, stream=None):
    """d_A, w: C double arrays (host); bragg: a Bragg struct (completed in place)."""
    _check(lib.mcv_bragg_build(d_A, w, n, C.byref(bragg), tables, nbytes, stream))


def mcv_phonon_table_bytes(n_modes, n_max):
    return lib.mcv_phonon_table_bytes(n_modes, n_max)


def mcv_phonon_build(dos_z, phonon, tables, nbytes, stream=None):
    """dos_z: a C double array (host); phonon: a Phonon struct (completed in place)."""
    _check(lib.mcv_phonon_build(dos_z, C.byref(phonon), tables, nbytes, stream))


def _sims(sims):
    arr = (Sim * len(sims))(*sims)
    return arr


def mcv_batch_create(ctx, sims, det, fp_mode):
    """sims: a sequence of Sim (their sample and beam pointers must stay valid for the call)."""
    h = C.c_void_p()
    _check(lib.mcv_batch_create(ctx, _sims(sims), len(sims), C.byref(det), fp_mode, C.byref(h)))
    return h


def mcv_batch_run(batch, stream=None):
    _check(lib.mcv_batch_run(batch, stream))


def mcv_batch_tune(batch, trial_neutrons=0, stream=None):
    _check(lib.mcv_batch_tune(batch, trial_neutrons, stream))


def mcv_batch_shape(batch):
    chunk, grid, items = C.c_int64(), C.c_int(), C.c_int64()
    bps = C.c_int()
    _check(lib.mcv_batch_shape(batch, C.byref(chunk), C.byref(bps), C.byref(grid),
                               C.byref(items)))
    return {"chunk": chunk.value, "blocks_per_sm": bps.value, "grid": grid.value,
            "n_items": items.value}


def mcv_batch_destroy(batch):
    _check(lib.mcv_batch_destroy(batch))


def mcv_trace_batch(ctx, sims, det, fp_mode, stream=None):
    _check(lib.mcv_trace_batch(ctx, _sims(sims), len(sims), C.byref(det), fp_mode, stream))
