#!/usr/bin/env python
"""Benchmark of the powder S(Q,E) run: 1e8 neutrons per GPU per step through a hollow
cylinder (up to 5 scattering orders) into a 117,760-pixel x 1000-bin FP64 histogram.

A step is one pass of the whole hot path: the source drawn in registers, the sample
assembly, the detector system and the histogram, all in one fused kernel (plus the kernel
that clears the histogram).  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

For N > 1 it is launched by torch.distributed.run; each rank simulates its own neutron-id
range (weak scaling, no collective in the timed region); after the timed region the ranks'
histograms and tallies are summed over NCCL (the run's result), timed on its own.
"""
import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "neutrons/s + fraction of roofline (1e8-n powder S(Q,E), 1×GB300) vs plain FP64 fwd"
WORKLOAD = ("powder S(Q,E), hollow cylinder r_out=1 cm wall 2 mm h=4 cm, Ei=100 meV +-1%, "
            "5 mrad, 5x5 cm beam, up to 5 scattering orders, 115 8-packs x 128 pixels "
            "(117,760) x 1000 tof bins FP64")
N_DEFAULT = 100_000_000

# Lane-op weight of one transcendental or square root: GB300's SFU issues 16 per clock per SM
# against 128 FP32/INT32 lanes.
XU_WEIGHT = 8.0


def load_opcount(name="powder_sqe"):
    """Operations per incident neutron of a workload, counted on an instrumented oracle run
    (oracle/opcount.py; the condition estimate compiled out): fp, int, xu per neutron, and per
    oracle function with its calls."""
    p = os.path.join(ROOT, "profiles", "opcount_%s.json" % name)
    try:
        with open(p) as f:
            return json.load(f)
    except (OSError, ValueError):
        return None


def load_executed():
    """Executed lane-instructions per neutron of the fused FP32 kernel (ncu
    smsp__thread_inst_executed.sum on the 1e7-neutron case), if taken on this source."""
    p = os.path.join(ROOT, "profiles", "wave_kernel_fp32_executed.json")
    try:
        with open(p) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    if d.get("csrc_hash") != csrc_hash():
        return None
    return d.get("lane_inst_per_neutron")


def maybe_fraction(wl):
    """Share of footprints inside the sure-miss bounds (uniform footprint): the bounds are
    the sample's radius / half height plus the sideways move over (z0 + r) at the largest
    divergence the uniforms can give (8.66 sigma), with a 1 % and 1 um margin."""
    def radius(s):
        if s.kind == 0:
            return s.dims[0]
        if s.kind == 1:
            return s.dims[1]
        return 0.5 * math.hypot(s.dims[0], s.dims[2])

    def half_height(s):
        return 0.5 * (s.dims[2] if s.kind == 1 else s.dims[1])

    r = max(radius(s) for s in wl.scatterers)
    hh = max(half_height(s) for s in wl.scatterers)
    b = wl.beam
    shift = (b.z0_m + r) * math.tan(8.66 * b.div_sigma_rad) * 1.01 + 1e-6
    fx = 1.0 if b.width_m <= 0 else min(1.0, 2 * (r + shift) / b.width_m)
    fy = 1.0 if b.height_m <= 0 else min(1.0, 2 * (hh + shift) / b.height_m)
    return fx * fy


def ops_per_neutron(opc, wl):
    """(all, conservative) lane-op equivalents per incident neutron: fp + int + XU_WEIGHT xu
    of the instrumented oracle run; the conservative figure leaves out, for the footprints
    the kernel proves to miss the sample, the two further source draws (Philox blocks and
    the divergence and energy arithmetic) that the oracle makes for every neutron."""
    pn = opc["per_neutron"]
    total = pn["fp"] + pn["int"] + XU_WEIGHT * pn["xu"]
    pf = opc["per_function"]
    ph, un = pf.get("orc_philox4x32_10"), pf.get("orc_uniforms")
    block_ops = 0.0
    if ph and un and ph[3] > 0:
        block_ops = (ph[0] + ph[1] + un[0] + un[1] + XU_WEIGHT * (ph[2] + un[2])) / ph[3]
    beam = next((v for k, v in pf.items() if "make_beam" in k), None)
    beam_rest = 0.0 if beam is None or beam[3] <= 0 else (beam[0] + beam[1] + XU_WEIGHT * beam[2]) / beam[3]
    skipped = (1.0 - maybe_fraction(wl)) * (2.0 * block_ops + beam_rest)
    return total, total - skipped


def csrc_hash():
    """Hash of the kernel sources and of the build script (its per-file compiler flags)."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1504_02776_gb300", "csrc")
    files = [os.path.join(d, f) for f in sorted(os.listdir(d))]
    files.append(os.path.join(ROOT, "paper_1504_02776_gb300", "build.py"))
    for p in files:
        with open(p, "rb") as fh:
            h.update(os.path.basename(p).encode() + fh.read())
    return h.hexdigest()[:16]


def load_traffic():
    """DRAM bytes per neutron of the trace kernel from the committed ncu summary, if it was
    taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "trace_fp32_powder_traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    if d.get("csrc_hash") != csrc_hash():
        return None
    return d.get("dram_bytes_per_neutron")


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        # nvidia-smi's start-up (driver queries) stalled host-device copies: the timed region
        # starts once it is sampling (3 s at most)
        t0 = time.monotonic()
        while not self.rows and time.monotonic() - t0 < 3.0 and self.proc.poll() is None:
            time.sleep(0.01)

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 8:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4)
                          if r[4 + i].lower() == "active"})
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "samples": len(self.rows),
                "reasons": reasons}


# ---- oracle timing (the CPU baseline and the reference arm) -------------------------------
def _oracle_shard(args):
    first, n = args
    import mcv_inputs as mi
    import oracle
    wl = mi.config2(n=n)
    t0 = time.perf_counter()
    oracle.trace(wl, first_id=first, n=n, packets=False, hist=True)
    return n, time.perf_counter() - t0


def oracle_throughput(per_worker, workers, first=0):
    """Neutrons/s of the oracle on `workers` host processes (spawned), each tracing its own
    id range of `per_worker` neutrons of the same workload."""
    import multiprocessing as mp
    ctxm = mp.get_context("spawn")
    with ctxm.Pool(workers) as pool:
        pool.map(_oracle_shard, [(first + 10**12 + i, 10) for i in range(workers)])  # warm
        t0 = time.perf_counter()
        res = pool.map(_oracle_shard, [(first + i * per_worker, per_worker)
                                       for i in range(workers)])
        wall = time.perf_counter() - t0
    n = sum(r[0] for r in res)
    return n / wall, n, wall


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    workers = os.cpu_count() or 1
    per = args.ref_per_worker
    vals = []
    for _ in range(args.warmup if args.warmup < 2 else 1):
        oracle_throughput(per // 10 or 1, workers)
    t0 = time.perf_counter()
    for k in range(args.steps):
        v, n, wall = oracle_throughput(per, workers, first=k * per * workers)
        vals.append(wall)
    total = time.perf_counter() - t0
    n_step = per * workers
    value = n_step * args.steps / sum(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "neutrons/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(vals) / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "neutrons_per_step": n_step,
                   "sample": "bounded sample of the 1e8-neutron workload"},
        "cpu_baseline": {"value": value, "unit": "neutrons/s", "cores": workers,
                         "kind": "oracle",
                         "sample": "%d neutrons per step (%d per process)" % (n_step, per)},
        "e2e": {"value": value, "unit": "neutrons/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "wall_s": total,
    }
    print(json.dumps(line), flush=True)
    return 0


# ---- our arm --------------------------------------------------------------------------------
def _timed(fn, reps):
    """Device time of reps calls of fn on the current stream (ms per call)."""
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def batch_extras(ctx, args):
    """The batched forms against one simulation per launch on the same GPU:
    the 64-simulation incident-energy sweep (sample in an aluminium can, 1e5..1e8 neutrons
    per simulation, one full histogram each) and the single crystal at 181 orientations x 2e6
    neutrons (one full histogram each, 170 GB).  Histograms accumulate (cleared once)."""
    import torch

    import mcv_inputs as mi
    from paper_1504_02776_gb300 import binding as B
    out = {}

    tables = {}

    def per_launch(sims, hists, fp):
        def f():
            for wl, (c, t) in zip(sims, hists):
                table = tables.get(id(wl.sqe.table)) if wl.sqe is not None else None
                ctx.trace(wl, fp_mode=fp, table=table, counts=c, tallies=t, sync=False)
        return f

    # incident-energy sweep
    sims = mi.config5()
    n_tot = sum(w.n for w in sims)
    hists = [ctx.new_hist(w.detector) for w in sims]
    tables[id(sims[0].sqe.table)] = ctx.table(sims[0])
    b = ctx.batch(sims, fp_mode=B.FP32, hists=hists)
    shape = b.tune()
    b.run()
    ms_b = _timed(b.run, args.batch_reps)
    ctx.sync()
    det = sum(float(t[B.T_NDET].item()) for _, t in hists) / (args.batch_reps + 1)
    ms_l32 = _timed(per_launch(sims, hists, B.FP32), 1)
    ms_l64 = _timed(per_launch(sims, hists, B.FP64), 1)
    ctx.sync()
    b.close()
    out["ei_sweep"] = {
        "workload": "64 simulations, Ei log-spaced 10-500 meV, counts log-uniform 1e5-1e8 "
                    "(seed 7; %d neutrons in total), powder S(Q,E) in a 1.5 mm Al can, up to "
                    "5 orders, one 117,760 x 1000 FP64 histogram per simulation, time window "
                    "scaled with 1/v" % n_tot,
        "neutrons": n_tot,
        "batched_fp32": {"value": n_tot / (ms_b / 1e3), "unit": "neutrons/s", "ms": ms_b,
                         "shape": shape, "detected_events_per_s": det / (ms_b / 1e3)},
        "per_launch_fp32": {"value": n_tot / (ms_l32 / 1e3), "unit": "neutrons/s",
                            "ms": ms_l32, "launches": len(sims)},
        "per_launch_fp64": {"value": n_tot / (ms_l64 / 1e3), "unit": "neutrons/s",
                            "ms": ms_l64, "launches": len(sims)},
        "speedup_batched_fp32_over_per_launch_fp64": ms_l64 / ms_b,
    }
    del hists, b
    torch.cuda.empty_cache()

    # single crystal, 181 orientations
    sims = mi.config3_batch()
    n_tot = sum(w.n for w in sims)
    nb = sims[0].detector.n_bins
    free, _ = torch.cuda.mem_get_info()
    if free < (len(sims) + 4) * nb * 8:
        out["crystal_181"] = {"skipped": "needs %.0f GB free" % ((len(sims) + 4) * nb * 8 / 1e9)}
        return out
    hists = [(torch.zeros(nb, dtype=torch.float64, device="cuda"),
              torch.zeros(B.MCV_NTALLY, dtype=torch.float64, device="cuda")) for _ in sims]
    b = ctx.batch(sims, fp_mode=B.FP32, hists=hists)
    shape = b.tune()
    b.run()
    ms_b = _timed(b.run, max(1, args.batch_reps - 1))
    ctx.sync()
    b.close()
    sample = sims[::args.crystal_fp64_stride]
    ms_l64 = _timed(per_launch(sample, hists[::args.crystal_fp64_stride], B.FP64), 1)
    ms_l32 = _timed(per_launch(sims, hists, B.FP32), 1)
    ctx.sync()
    n_s = sum(w.n for w in sample)
    out["crystal_181"] = {
        "workload": "fcc Born-von Karman single crystal, 2 cm cube, Ei=50 meV, 181 "
                    "orientations (0-180 deg) x 2e6 neutrons, one 117,760 x 1000 FP64 "
                    "histogram per orientation (%.0f GB)" % (len(sims) * nb * 8 / 1e9),
        "neutrons": n_tot,
        "batched_fp32": {"value": n_tot / (ms_b / 1e3), "unit": "neutrons/s", "ms": ms_b,
                         "shape": shape},
        "per_launch_fp32": {"value": n_tot / (ms_l32 / 1e3), "unit": "neutrons/s",
                            "ms": ms_l32, "launches": len(sims)},
        "per_launch_fp64": {"value": n_s / (ms_l64 / 1e3), "unit": "neutrons/s",
                            "ms_sample": ms_l64, "launches": len(sample),
                            "sample": "every %d-th orientation (%d of %d), rate applied to "
                                      "the whole batch" % (args.crystal_fp64_stride,
                                                           len(sample), len(sims))},
        "speedup_batched_fp32_over_per_launch_fp64": (n_tot / (ms_b / 1e3)) /
                                                     (n_s / (ms_l64 / 1e3)),
    }
    del hists
    torch.cuda.empty_cache()
    return out


def kernel_extras(ctx, args):
    """The other scattering kernels, the paper's recursive estimator and event mode, each on
    its own workload (args.kernel_n neutrons, one launch per step, histogram and tallies
    cleared before every launch, outside its events), FP32 and FP64: incoming neutrons/s,
    detected events/s, and the FP32 launch against the ALU roof (operations per neutron from
    the instrumented oracle run of the same workload)."""
    import torch

    import mcv_inputs as mi
    from paper_1504_02776_gb300 import api, binding as B
    n = args.kernel_n
    evb = api.EventBuffers(max(1, n // 4))
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    sm_mhz = float(load_peaks().get("sm_max_mhz", 2070.0))
    peak_ops = props.multi_processor_count * 128 * sm_mhz * 1e6
    opcount_of = {"phonon_vanadium": "phonon_vanadium", "bragg_aluminium": "bragg_aluminium",
                  "dispersion_crystal": "dispersion_crystal",
                  "paper_estimator_powder": "paper_powder_sqe",
                  "event_mode_powder": "powder_sqe"}
    cases = [
        ("phonon_vanadium", mi.vanadium_powder(n), B.EST_CHAIN, None,
         "vanadium-like hollow cylinder, incoherent phonon expansion from a DOS (elastic, "
         "one-phonon, multi-phonon to n=5), 100 meV, up to 5 orders"),
        ("bragg_aluminium", mi.aluminium_powder(n), B.EST_CHAIN, None,
         "aluminium-like powder hollow cylinder, Debye-Scherrer reflections + weak incoherent "
         "elastic, 100 meV, up to 5 orders"),
        ("dispersion_crystal", mi.dispersion_crystal(n), B.EST_CHAIN, None,
         "1 cm cube crystal, the paper's example dispersion surface (2.5 meV band), 7.5 meV, "
         "up to 5 orders"),
        ("paper_estimator_powder", mi.config2(n=n), B.EST_PAPER, None,
         "the powder S(Q,E) run of the headline through the paper's recursive estimator "
         "(every interaction splits into transmitted and scattered packets)"),
        ("event_mode_powder", mi.config2(n=n), B.EST_CHAIN, evb,
         "the powder S(Q,E) run of the headline with every detected packet also appended to "
         "an event list (pixel, simulation, time of flight, weight)"),
    ]
    out = {"neutrons_per_launch": n}
    for name, wl, est, ev, what in cases:
        table = ctx.table(wl)
        counts, tallies = ctx.new_hist(wl.detector)
        res = {"workload": what}
        for fp, key in ((B.FP32, "fp32"), (B.FP64, "fp64")):
            reps = args.kernel_reps if fp == B.FP32 else 1
            marks = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                     for _ in range(reps + 1)]
            for a, b in marks:  # the first launch warms up; the clears are not timed
                counts.zero_()
                tallies.zero_()
                if ev is not None:
                    ev.count.zero_()
                a.record()
                ctx.trace(wl, fp_mode=fp, table=table, counts=counts, tallies=tallies,
                          sync=False, estimator=est, events=ev)
                b.record()
            torch.cuda.synchronize()
            ms = sum(a.elapsed_time(b) for a, b in marks[1:]) / reps
            ctx.sync()
            t = tallies.cpu().numpy()
            res[key] = {"value": n / (ms / 1e3), "unit": "neutrons/s", "ms": ms,
                        "detected_events_per_s": float(t[B.T_NDET]) / (ms / 1e3)}
            if ev is not None:
                res[key]["events_listed"] = min(ev.n(), ev.capacity)
        opc = load_opcount(opcount_of[name])
        if opc is not None:
            per_n, per_n_cons = ops_per_neutron(opc, wl)
            ms = res["fp32"]["ms"]
            res["roofline_fp32"] = {
                "bound": "alu", "achieved": per_n * n / (ms / 1e3) / 1e12,
                "peak": peak_ops / 1e12, "unit": "Tops/s",
                "frac": per_n * n / (ms / 1e3) / peak_ops,
                "frac_conservative": per_n_cons * n / (ms / 1e3) / peak_ops,
                "ops_per_neutron": per_n,
                "ops_source": "oracle/opcount.py --workload %s" % opcount_of[name],
                "timing": "CUDA events around each launch (histogram clears outside)"}
        out[name] = res
        del counts, tallies
    del evb
    torch.cuda.empty_cache()
    return out


def grad_extras(ctx, value64):
    """The differentiable form (config 4): chi-squared loss of the 1e7-neutron powder run
    against a seeded target and its adjoint gradient w.r.t. the 200 x 400 S(Q,E) table and
    the cross sections -- one mcv_grad call (forward trace, loss, adjoint trace; FP32 trace,
    FP64 accumulation) -- against the plain FP64 forward of the same neutrons."""
    import torch

    import mcv_inputs as mi
    from paper_1504_02776_gb300 import api, binding as B
    wl = mi.config4()
    table = ctx.table(wl)
    # target: the run with omega scaled by 1.05 (seed 1), Poisson noise, c = n / sum(I)
    tw = mi.config2(n=wl.n, omega_scale=1.05).replace(seed=1)
    counts, _ = ctx.trace(tw, fp_mode=B.FP32, table=ctx.table(tw))
    scale_c = wl.n / float(counts.sum().item())
    gen = torch.Generator(device="cuda")
    gen.manual_seed(2)
    target = torch.poisson(scale_c * counts, generator=gen)
    hist = torch.empty_like(counts)

    def step():
        api._grad_call(ctx, wl, target, scale_c, B.FP32, wl.n, 0, table, None, None, 0, hist)

    for _ in range(2):
        step()
    ms = _timed(step, 3)
    ctx.sync()
    ms64 = wl.n / value64 * 1e3
    return {"workload": "config 4: chi2 of the 1e7-neutron powder run vs a seeded target "
                        "(omega x 1.05, Poisson), gradient w.r.t. 200 x 400 S(Q,E) entries and "
                        "sigma_abs, sigma_s; forward + loss + adjoint in one mcv_grad call",
            "value": wl.n / (ms / 1e3), "unit": "neutrons/s", "ms": ms,
            "plain_fp64_forward_ms_same_neutrons": ms64,
            "speedup_over_plain_fp64_forward": ms64 / ms}


def run_ours(args):
    import torch
    import torch.distributed as dist

    import mcv_inputs as mi
    from paper_1504_02776_gb300 import api, binding as B

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    cpu_base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # before the first GPU call: spawned processes only
        workers = os.cpu_count() or 1
        v, n_cpu, wall = oracle_throughput(args.cpu_per_worker, workers)
        v1, n1, wall1 = oracle_throughput(args.cpu_per_worker, 1)
        cpu_base = {"value": v, "unit": "neutrons/s", "cores": workers, "kind": "oracle",
                    "sample": "%d neutrons of the same workload (%d per process, ids from 0), "
                              "%.1f s wall" % (n_cpu, args.cpu_per_worker, wall),
                    "single_core": {"value": v1, "unit": "neutrons/s", "neutrons": n1,
                                    "s": wall1, "s_scaled_to_1e8": 1e8 / v1}}
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    N = args.n
    ctx = api.Context(local)
    wl = mi.config2(n=N)
    table = ctx.table(wl)
    counts, tallies = ctx.new_hist(wl.detector)
    stream = torch.cuda.current_stream()
    from paper_1504_02776_gb300.shards import shard
    first, _ = shard(rank, world, N)
    sample32 = api.sample_struct(wl, B.FP32, table)
    det = api.detector_struct(wl.detector)
    beam = api.beam_struct(wl.beam)
    hist = B.Hist(counts.data_ptr(), tallies.data_ptr())
    sptr = __import__("ctypes").c_void_p(stream.cuda_stream)

    def step(sample, ev=None):
        B.mcv_zero(ctx.handle, counts.data_ptr(), counts.numel(), sptr)
        B.mcv_zero(ctx.handle, tallies.data_ptr(), tallies.numel(), sptr)
        if ev is not None:
            ev[0].record(stream)
        B.mcv_trace_sample(ctx.handle, sample, beam, None, wl.seed, wl.sim_id, first, N, det,
                           hist, None, sptr)
        if ev is not None:
            ev[1].record(stream)

    # ---- FP32 fast mode (the product path)
    for _ in range(args.warmup):
        step(sample32)
    ctx.sync()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    e0.record(stream)
    for k in range(args.steps):
        step(sample32, evs[k])
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ctx.sync()
    ms = e0.elapsed_time(e1)
    trace_ms = sum(a.elapsed_time(b) for a, b in evs) / args.steps
    tm = torch.tensor([ms], dtype=torch.float64, device="cuda")
    collective = None
    t_local = tallies.cpu().numpy()  # this rank's tallies of the last step
    if world > 1:
        dist.all_reduce(tm, op=dist.ReduceOp.MAX)
        # the run's result: the ranks' histograms and tallies summed (the path's one exchange
        # step), after the timed region and timed on its own
        from paper_1504_02776_gb300.shards import reduce_sum
        r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        r0.record(stream)
        reduce_sum([counts, tallies])
        r1.record(stream)
        torch.cuda.synchronize()
        collective = {"op": "all_reduce(SUM) over NCCL of the FP64 histogram and tallies",
                      "bytes": int((counts.numel() + tallies.numel()) * 8),
                      "ms": r0.elapsed_time(r1), "in_timed_region": False}
    t = tallies.cpu().numpy()  # the whole run's tallies of the last step
    ms = float(tm.item())
    value = world * N * args.steps / (ms / 1e3)
    det_per_s = t[B.T_NDET] * args.steps / (ms / 1e3)

    # ---- end to end through the public API with host buffers, right after the device-timed
    # region and before anything else runs: every step copies the
    # table in from pinned host memory and its histogram and tallies out to pinned host
    # memory; two histogram buffers and a copy stream let step k's read-back overlap step
    # k+1's trace (the timed region ends when the last read-back has landed)
    e2e = None
    if not args.no_e2e:
        host_table = torch.from_numpy(wl.sqe.table).pin_memory()
        dev_bufs = [(counts, tallies), ctx.new_hist(wl.detector)]
        host_bufs = [(torch.empty(counts.numel(), dtype=torch.float64).pin_memory(),
                      torch.empty(tallies.numel(), dtype=torch.float64).pin_memory())
                     for _ in range(2)]
        hists = [B.Hist(c.data_ptr(), tl.data_ptr()) for c, tl in dev_bufs]
        # the read-back is split over several copy streams (one copy engine each)
        n_copy = 8
        copy_streams = [torch.cuda.Stream() for _ in range(n_copy)]
        ready = [torch.cuda.Event() for _ in range(2)]
        copied = [[torch.cuda.Event() for _ in range(n_copy)] for _ in range(2)]
        for evs_j in copied:
            for ev, cs in zip(evs_j, copy_streams):
                ev.record(cs)
        cuts = [counts.numel() * q // n_copy for q in range(n_copy + 1)]

        # a buffer is cleared on its own stream once its read-back has landed, so that the
        # clear overlaps the other buffer's trace (the trace leaves room for it on each SM)
        zero_stream = torch.cuda.Stream()
        zptr = __import__("ctypes").c_void_p(zero_stream.cuda_stream)
        zeroed = [torch.cuda.Event() for _ in range(2)]

        def clear(j):
            c_j, t_j = dev_bufs[j]
            for ev in copied[j]:
                zero_stream.wait_event(ev)
            B.mcv_zero(ctx.handle, c_j.data_ptr(), c_j.numel(), zptr)
            B.mcv_zero(ctx.handle, t_j.data_ptr(), t_j.numel(), zptr)
            zeroed[j].record(zero_stream)

        for j in range(2):
            clear(j)

        def e2e_step(k):
            j = k % 2
            c_j, t_j = dev_bufs[j]
            stream.wait_event(zeroed[j])  # cleared after its previous read-back
            table.copy_(host_table.view(-1).view_as(table), non_blocking=True)
            B.mcv_trace_sample(ctx.handle, sample32, beam, None, wl.seed, wl.sim_id, first, N,
                               det, hists[j], None, sptr)
            ready[j].record(stream)
            for q, cs in enumerate(copy_streams):
                cs.wait_event(ready[j])
                with torch.cuda.stream(cs):
                    a, b = cuts[q], cuts[q + 1]
                    host_bufs[j][0][a:b].copy_(c_j[a:b], non_blocking=True)
                    if q == 0:
                        host_bufs[j][1].copy_(t_j, non_blocking=True)
                copied[j][q].record(cs)
            clear(j)

        for k in range(2):
            e2e_step(k)
        torch.cuda.synchronize()
        # no nvidia-smi sampling here: its driver queries stalled the host-device copies
        # (20-step runs: 6.15 ms per step without it, 6.15 to 8.1 ms with it); the clocks are
        # those sampled over the device-timed region just before.  The timed loop runs
        # args.e2e_reps times (each K steps, the last read-back included) and the median
        # is reported: occasional host-side stalls (up to 9 %) remained without the sampler.
        runs = []
        for _ in range(args.e2e_reps):
            g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            barrier()
            g0.record(stream)
            for k in range(args.e2e_steps):
                e2e_step(k)
            for j in range(2):  # every read-back landed and every buffer cleared again
                stream.wait_event(zeroed[j])
            g1.record(stream)
            torch.cuda.synchronize()
            gm = torch.tensor([g0.elapsed_time(g1)], dtype=torch.float64, device="cuda")
            if world > 1:
                dist.all_reduce(gm, op=dist.ReduceOp.MAX)
            runs.append(float(gm.item()))
        gms = sorted(runs)[len(runs) // 2]
        e2e = {"value": world * N * args.e2e_steps / (gms / 1e3), "unit": "neutrons/s",
               "h2d_bytes_per_step": int(host_table.numel() * 4),
               "d2h_bytes_per_step": int((counts.numel() + tallies.numel()) * 8),
               "ms_per_step": gms / args.e2e_steps, "steps": args.e2e_steps,
               "repetitions": args.e2e_reps,
               "ms_per_step_of_each": [r / args.e2e_steps for r in runs],
               "statistic": "median of the repetitions",
               "pipelining": "two histogram buffers; step k's read-back (split over %d copy "
                             "streams) and then the clear of its buffer (a side stream) "
                             "overlap step k+1's trace" % n_copy,
               "clocks": "not sampled: nvidia-smi's queries stall host-device copies; see "
                         "the device-timed region's clocks"}
        del dev_bufs, host_bufs
        ctx.sync()

    # ---- plain FP64 forward, one simulation per launch, same workload and histogram
    sample64 = api.sample_struct(wl, B.FP64, table)
    step(sample64)
    ctx.sync()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    f0.record(stream)
    for _ in range(args.fp64_steps):
        step(sample64)
    f1.record(stream)
    torch.cuda.synchronize()
    ms64 = f0.elapsed_time(f1)
    fm = torch.tensor([ms64], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(fm, op=dist.ReduceOp.MAX)
    ms64 = float(fm.item())
    value64 = world * N * args.fp64_steps / (ms64 / 1e3)
    ctx.sync()

    # ---- batched forms (rank 0 of a single-GPU run; they hold up to 170 GB of histograms)
    # and the differentiable form
    batched = None
    differentiable = None
    extras = "none" if args.no_batch else args.extras
    if world == 1 and extras in ("all", "batch"):
        batched = batch_extras(ctx, args)
    if world == 1 and extras in ("all", "grad"):
        differentiable = grad_extras(ctx, value64)
    kernels = None
    if world == 1 and extras in ("all", "kernels"):
        kernels = kernel_extras(ctx, args)

    # ---- roofline of the fused trace kernel (ALU bound): operations per neutron counted on an
    # instrumented oracle run, against the FP32/INT32 lane rate
    props = torch.cuda.get_device_properties(local)
    peaks = load_peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak_ops = props.multi_processor_count * 128 * sm_mhz * 1e6   # FP32/INT32 lanes x clock
    opc = load_opcount()
    roof = None
    if opc is not None:
        per_n, per_n_cons = ops_per_neutron(opc, wl)
        ops = per_n * N
        achieved = ops / (trace_ms / 1e3)
        traffic_per_n = load_traffic()
        executed = load_executed()
        roof = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12,
                "unit": "Tops/s", "frac": achieved / peak_ops,
                "traffic": None if traffic_per_n is None else traffic_per_n * N,
                "kernel": "wave_kernel<float,1,TUBES,powder>", "kernel_ms": trace_ms,
                "ops_per_launch": ops,
                "ops_per_neutron": per_n,
                "ops_source": ("instrumented oracle run, oracle/opcount.py (GCC profile counts "
                               "of the oracle's GIMPLE, condition estimate compiled out): "
                               "fp %.1f + int %.1f + %g x xu %.2f per neutron" % (
                                   opc["per_neutron"]["fp"], opc["per_neutron"]["int"],
                                   XU_WEIGHT, opc["per_neutron"]["xu"])),
                "frac_conservative": per_n_cons * N / (trace_ms / 1e3) / peak_ops,
                "ops_per_neutron_conservative": per_n_cons,
                "conservative_note": "without the source draws the oracle makes for the "
                                     "footprints the kernel proves to miss the sample",
                "executed_lane_inst_per_neutron": executed,
                "frac_issue": None if executed is None else
                executed * N / (trace_ms / 1e3) / peak_ops,
                "peak_basis": "%d SMs x 128 FP32/INT32 lanes x %.0f MHz (max SM clock, "
                              "MEASURED_PEAKS.json); a transcendental counts %g lane-ops "
                              "(16 SFU results per clock per SM)" % (
                                  props.multi_processor_count, sm_mhz, XU_WEIGHT),
                # histogram read-modify-writes, one 8-byte word per detected event (read + write)
                "hbm_gbs_algorithmic": t_local[B.T_NDET] * 16 / (trace_ms / 1e3) / 1e9,
                "hbm_peak_gbs_measured": peaks.get("hbm_gbs")}
    # the histogram stage's roof: random FP64 atomic adds into the same 942 MB histogram
    n_at = 50_000_000
    for _ in range(2):
        B.mcv_bench_atomics(ctx.handle, counts.data_ptr(), counts.numel(), n_at, 1, sptr)
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for k in range(5):
        B.mcv_bench_atomics(ctx.handle, counts.data_ptr(), counts.numel(), n_at, 2 + k, sptr)
    a1.record(stream)
    torch.cuda.synchronize()
    at_rate = 5 * n_at / (a0.elapsed_time(a1) / 1e3)
    det_rate_kernel = t_local[B.T_NDET] / (trace_ms / 1e3)
    atomics = {"random_fp64_atomics_per_s": at_rate,
               "histogram_adds_per_s_in_trace": det_rate_kernel,
               "frac": det_rate_kernel / at_rate,
               "how": "mcv_bench_atomics: 5 x 5e7 adds of 1.0 at hashed uniform bins of the "
                      "942 MB histogram, CUDA events"}

    line = {
        "metric": METRIC, "value": value, "unit": "neutrons/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "neutrons_per_gpu_per_step": N,
                   "precision": "FP32 geometry and kernel sampling (division and square "
                                "root to 2 ulp, hardware exp and log, subnormals kept); FP64 "
                                "time of flight, tallies and histogram",
                   "l2": "inputs larger than L2: the 942 MB histogram is cleared and "
                         "rewritten every step",
                   "parallelism": "neutron-id shards per GPU" if world > 1 else "1 GPU"},
        "detected_events_per_s": det_per_s,
        "fp64_forward": {"value": value64, "unit": "neutrons/s",
                         "ms_per_step": ms64 / args.fp64_steps, "steps": args.fp64_steps,
                         "speedup_fp32_over_fp64": value / value64},
        "roofline": roof,
        "atomics": atomics,
        "batched": batched,
        "differentiable": differentiable,
        "kernels": kernels,
        "cpu_baseline": cpu_base,
        "e2e": e2e,
        "collective": collective,
        "gpu_launches": 3 * args.steps,
        "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--fp64-steps", type=int, default=3)
    # default: as many steps as the device-timed region (the last read-back, which nothing
    # overlaps, is spread over the same number of steps)
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--e2e-reps", type=int, default=5)
    ap.add_argument("--cpu-per-worker", type=int, default=1_000_000)
    ap.add_argument("--ref-per-worker", type=int, default=400_000)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batched, differentiable and per-kernel forms (same as "
                         "--extras none)")
    ap.add_argument("--extras", default="all",
                    choices=["all", "batch", "grad", "kernels", "none"],
                    help="which of the batched, differentiable and per-kernel forms to run")
    ap.add_argument("--kernel-n", type=int, default=10_000_000)
    ap.add_argument("--kernel-reps", type=int, default=3)
    ap.add_argument("--batch-reps", type=int, default=3)
    ap.add_argument("--crystal-fp64-stride", type=int, default=18)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.e2e_steps is None:
        args.e2e_steps = args.steps
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
