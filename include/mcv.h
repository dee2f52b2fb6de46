/*
 * mcv.h -- C ABI of the GB300 neutron ray-tracing library (libmcv.so).
 *
 * The library implements the data-parallel hot path of MCViNE's method (Lin et al.,
 * "MCViNE -- An object oriented Monte Carlo neutron ray tracing simulation package"):
 * Monte Carlo ray tracing of neutron packets through a sample assembly and a pixelated
 * 3He detector system into a time-of-flight histogram.  The calls follow the paper's
 * component chain (section 2.2 and section 3's workflow): a source (mcv_beam), the sample
 * assembly (mcv_trace_sample, section 2.4.3 "Ray Tracing" and "Multiple Scattering"), the
 * detector system (mcv_detect, section 2.4.3 "Ray tracing in a detector system").  The
 * adjoint (mcv_grad) and the batched launch (mcv_trace_batch) have no counterpart in the
 * paper.
 *
 * Conventions for every call
 *   - Frame: beam along +z, y up, the sample centred at the origin.  Lengths in m (sample
 *     and detector), velocities in m/s, times in s, energies in meV, momenta in 1/A,
 *     number densities in 1/A^3, cross sections in barn (absorption quoted at 2200 m/s and
 *     scaled as 1/v).
 *   - All array arguments are DEVICE pointers owned by the caller, on the device the
 *     context was created for.  The library allocates device memory only for its own
 *     bookkeeping (the context, a batch's parameter block, the autotuner's scratch; each
 *     call that does says so) and never frees caller memory.
 *   - Calls are asynchronous on the caller's CUDA stream (`stream`, a cudaStream_t; NULL is
 *     the legacy default stream).  Argument errors are reported before anything is
 *     launched (MCV_EINVAL, nothing written).  Launch failures return MCV_ECUDA.  Errors
 *     found by the kernels themselves (an index out of range, invalid data in a caller's
 *     device buffer) set a flag in the context that mcv_sync reports as MCV_EDEVICE.
 *   - Histograms and tallies are ACCUMULATED into; callers zero them (cudaMemset or
 *     mcv_zero) before the first call, and split runs over neutron-id ranges add up.
 *   - Random numbers: Philox4x32-10 with key (seed, sim_id) and counter (neutron id low
 *     32 bits, high 32 bits, 4*(event+1)+block, 0); event -1 is beam generation, event o
 *     the o-th scattering order.  A neutron's history depends only on (seed, sim_id, id),
 *     never on launch shape, so results are reproducible and resumable by id range.
 *   - Nothing throws across the ABI; the message of the last error of the calling thread
 *     is returned by mcv_last_error().
 */
#ifndef MCV_H
#define MCV_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MCV_OK = 0,
  MCV_EINVAL = 1,    /* invalid argument: nothing was launched */
  MCV_ENOMEM = 2,    /* the library could not allocate its own device memory (a context's
                        block, a batch's parameter block, the tuner's scratch histogram);
                        nothing was launched and the context stays usable */
  MCV_ECUDA = 3,     /* a CUDA call failed (message in mcv_last_error) */
  MCV_ETIMEOUT = 4,  /* reserved for a bounded device wait that ran out; no kernel of this
                        library waits on another thread, block or device, so no call
                        returns it */
  MCV_EDEVICE = 5    /* a kernel found invalid device data: an out-of-range index, a packet
                        order above 7, a target bin that is negative or not finite
                        (reported by mcv_sync) */
} mcv_status;

enum { MCV_MAX_SCATTERERS = 4, MCV_MAX_TUBES_PER_ROW = 512, MCV_NTALLY = 8 };
enum { MCV_SHAPE_SOLID_CYL = 0, MCV_SHAPE_HOLLOW_CYL = 1, MCV_SHAPE_BLOCK = 2 };
enum { MCV_KERNEL_ISO = 0, MCV_KERNEL_SQE = 1, MCV_KERNEL_BVK = 2, MCV_KERNEL_PHONON = 3,
       MCV_KERNEL_BRAGG = 4, MCV_KERNEL_DISP = 5 };
enum { MCV_DET_NONE = 0, MCV_DET_SURFACE = 1, MCV_DET_TUBES = 2 };
enum { MCV_FP64 = 0, MCV_FP32 = 1 };
/* estimators of the sample assembly: the bounded chain (the scattering point drawn over all
 * the material ahead) or the paper's own recursion (supplement S3: scatterM, interactM_path1,
 * interactM1; the point drawn on the first segment only, every interaction splitting the
 * packet in a transmitted and a scattered one) */
enum { MCV_EST_CHAIN = 0, MCV_EST_PAPER = 1 };

/* tally slots (FP64 accumulators) */
enum {
  MCV_T_BEAMSTOP = 0, /* summed weight of the unscattered (order-0) packets */
  MCV_T_WDET = 1,     /* summed detected weight inside the tof range */
  MCV_T_WOVER = 2,    /* summed detected weight outside the tof range */
  MCV_T_NDET = 3,     /* detected packets inside the tof range */
  MCV_T_NOVER = 4,    /* detected packets outside the tof range */
  MCV_T_NMISS = 5,    /* scattered packets that missed every tube / the surface */
  MCV_T_NHIT = 6,     /* incident neutrons whose path crosses the sample */
  MCV_T_NEMIT = 7     /* scattered packets emitted (orders >= 1) */
};

typedef struct mcv_ctx mcv_ctx;

/* Synthetic source at the sample position (stands in for the beam simulation, section 3's
 * first step): energy ~ N(ei, (ei_rel_sigma*ei)^2); start point uniform on a width x
 * height rectangle in the plane z = -z0_m; horizontal and vertical divergence angles
 * ~ N(0, div_sigma_rad^2); time of flight from a source l1_m upstream of the origin. */
typedef struct {
  double ei_mev, ei_rel_sigma, div_sigma_rad, width_m, height_m, z0_m, l1_m;
} mcv_beam_params;

/* One homogeneous scatterer (section 2.4.1-2.4.2: one shape, one or two kernels).
 * shape SOLID_CYL dims = (r, h); HOLLOW_CYL dims = (r_in, r_out, h); BLOCK dims =
 * (wx, wy, wz) rotated by rot_y_rad about +y.  Cylinders have their axis along y. */
typedef struct {
  int shape;
  double dims[3];
  double rot_y_rad;
  double n_per_A3;
  double sig_abs_b;        /* at 2200 m/s */
  int n_kernels;           /* 1 or 2; kernel k is picked with probability sig_k / sum */
  int kernel[2];           /* MCV_KERNEL_* */
  double kernel_sig_b[2];  /* scattering cross section of each kernel */
} mcv_scatterer;

/* Tabulated isotropic S(Q,E) (supplement "Multi-phonon scattering" form
 * d2sigma/dOmega dEf = sigma/4pi kf/ki N S(Q,E)); FP32, row-major [iq][ie], nearest bin,
 * Q bins [0, q_max), E bins [e_min, e_max) where E = Ei - Ef. */
typedef struct {
  const float* table;      /* device, nq*ne */
  int nq, ne;
  double q_max, e_min, e_max;
} mcv_sqe;

/* Single-crystal fcc Born-von Karman kernel parameters (coherent one-phonon) */
typedef struct {
  double phi_Nm, mass_u, a_A, msd_A2, temperature_K;
} mcv_bvk;

/* Incoherent scattering from a phonon density of states (supplement "Scattering kernels used
 * in the examples": incoherent elastic with the Debye-Waller factor, incoherent inelastic
 * single-phonon, multi-phonon), as the phonon expansion
 *   S(Q,E) = e^{-2W} [delta(E) + sum_{n=1}^{n_max} (2W)^n/n! A_n(E)],  2W = c_w Q^2,
 *   A_1(E) = Z(|E|)/(|E| gamma_0) (n_B(|E|) + 1 for E > 0, n_B(|E|) for E < 0),
 *   A_n = A_1 * A_{n-1},  gamma_0 = sum coth(E/2kT) Z(E)/E,  c_w = hbar^2 gamma_0 / 2M,
 * E = Ei - Ef.  The density of states is a histogram of mode energies: Z at j*de_mev,
 * j = 1..n_modes, normalised by the library; each A_n is a set of masses on the grid
 * E = i*de_mev, and a sampled energy is spread uniformly over its grid bin.  The kernel picks
 * the elastic, one-phonon or multi-phonon channel with probabilities p[0..2] (summing to 1).
 * tables: device memory of mcv_phonon_table_bytes(n_modes, n_max) bytes filled by
 * mcv_phonon_build, which also writes gamma0 (1/meV) and c_w (A^2). */
typedef struct {
  const void* tables;
  int n_modes, n_max;
  double de_mev, mass_u, temperature_K;
  double p[3];
  double gamma0, c_w;
} mcv_phonon;

/* Coherent elastic scattering from a powder (supplement "Scattering kernels used in the
 * examples", the Debye-Scherrer cone): per atom, reflection tau scatters
 *   sigma_tau = lambda^3 / (4 sin theta_B) w_tau,  w_tau = m |F_tau|^2 / (v0 atoms per cell)
 * for lambda < 2 d_tau (theta_B: lambda = 2 d sin theta_B).  Reflections are taken in order
 * of decreasing d; one is picked with probability sigma_tau / sum sigma, the packet leaves on
 * its cone with an azimuth uniform about its direction, its speed unchanged, and its weight
 * multiplied by sum sigma / sigma_k, sigma_k the kernel's nominal cross section
 * (mcv_scatterer::kernel_sig_b, which sets its share of the attenuation and of the kernel
 * choice).  No allowed reflection (lambda beyond twice the largest d): no scattering.
 * tables: device memory of mcv_bragg_table_bytes(n) bytes filled by mcv_bragg_build. */
typedef struct {
  const void* tables;
  int n;
} mcv_bragg;

/* Scattering from a dispersion surface (supplement "Scattering kernels used in the examples":
 * d2sigma/dOmega dEf = sigma/4pi (kf/ki) S(Q) delta(E - E(Q))), with the paper's example
 * surface E(Q) = amp_mev sqrt(1 - (cos(c_A Qx) cos(c_A Qz))^2) and S(Q) = s0, Q in the
 * crystal frame of the scatterer's rotation ([100] along the beam and [001] vertical at zero
 * rotation, as the single-crystal kernel).  The outgoing direction is drawn uniformly; the
 * roots of Ei - Ef - E(Q(Ef)) are bracketed on 32 sub-intervals of [max(0, Ei - amp), Ei],
 * one is picked uniformly and bisected (50 steps in FP64, 24 in FP32); the weight is
 * n_roots (kf/ki) s0 / |d(Ei - Ef - E)/dEf|.  No root: no scattering. */
typedef struct {
  double amp_mev, c_A, s0;
} mcv_dispersion;

/* The sample assembly: a flat list of scatterers (the composite of section 2.4.1, one level
 * deep).  max_orders = maximum number of scatterings of a packet; packets whose weight
 * drops below min_prob are discarded (section 2.4.3); fp_mode MCV_FP64 traces in FP64,
 * MCV_FP32 traces geometry and kernels in FP32 with FP64 time of flight. */
typedef struct {
  int n_scatterers;
  mcv_scatterer scat[MCV_MAX_SCATTERERS];
  int max_orders;          /* 0..7 */
  double min_prob;
  int fp_mode;
  mcv_sqe sqe;
  mcv_bvk bvk;
  mcv_phonon phonon;
  mcv_bragg bragg;
  mcv_dispersion dispersion;
  int estimator;           /* MCV_EST_CHAIN (0) or MCV_EST_PAPER */
} mcv_sample;

/* Detector system.  SURFACE: ideal cylinder of radius_m, height_m, efficiency 1, n_phi x
 * n_y pixels, pixel = i_phi*n_y + i_y with phi = atan2(x, z) in [-pi, pi).  TUBES: n_rows
 * rows of packs of tubes_per_pack vertical 3He tubes (radius tube_r_m, active length
 * tube_len_m, centred on the circle radius_m, row centre heights row_y_m), tube pitch and
 * pack gap along the circle, first pack edge at phi0_rad; pixel = ((pack)*tubes_per_pack +
 * tube)*pixels_per_tube + i along y, packs numbered row by row.  tof bins: n_tof equal
 * bins on [tof_min_s, tof_max_s). */
typedef struct {
  int kind;
  double radius_m;
  double height_m;
  int n_phi, n_y;
  int n_rows;
  int packs[3];
  double row_y_m[3];
  int tubes_per_pack, pixels_per_tube;
  double tube_r_m, tube_len_m, tube_pitch_m, pack_gap_m, phi0_rad;
  double he3_n_per_A3, he3_sig_abs_b;
  double tof_min_s, tof_max_s;
  int n_tof;
  int multi_tube;          /* TUBES with MCV_EST_PAPER: the weight a tube leaves goes on to the
                              next tubes the packet crosses (1), or first tube only (0) */
} mcv_detector;

/* Structure-of-arrays neutron packets (device).  x..vz and w are float arrays in
 * MCV_FP32 and double arrays in MCV_FP64; t is always double.  id and order may be NULL
 * where a call says so.  n = number of slots. */
typedef struct {
  void *x, *y, *z, *vx, *vy, *vz;
  double* t;
  void* w;
  int64_t* id;
  int32_t* order;          /* -1 marks an empty slot */
  int64_t n;
} mcv_neutrons;

/* Event-mode output (section 3: the detector system records every neutron event, the
 * alternative to a dense histogram): every detected packet, inside the time window or not,
 * is appended as one record (pixel, sim tag = the simulation's sim_id, time of flight in s,
 * detected weight).  Device arrays of `capacity` entries owned by the caller; `count` is a
 * device counter the caller zeroes before the first call; each record takes the next index
 * (atomically, in no particular order) and is written when the index is below capacity, so
 * after a run min(*count, capacity) records are valid and *count > capacity means records
 * were dropped. */
typedef struct {
  int32_t* pixel;
  uint32_t* sim;
  double* tof;
  double* w;
  int64_t capacity;
  unsigned long long* count;
} mcv_event_list;

/* Histogram I[pixel][tof bin] (FP64, n_pixels*n_tof) and MCV_NTALLY FP64 tallies, and an
 * optional event list (host struct pointing at device arrays); any pointer may be NULL. */
typedef struct {
  double* counts;
  double* tallies;
  mcv_event_list* events;
} mcv_hist;

/* Per-packet detector results (device, one entry per packet slot); any pointer may be
 * NULL.  bin = pixel*n_tof + tof bin, -1 missed, -2 tof out of range. */
typedef struct {
  int32_t* pixel;
  double* tof;
  double* w_det;
  int64_t* bin;
} mcv_events;

/* ---- context ------------------------------------------------------------------------- */
/* Creates a context on `device` (allocates a 256-byte device block for the error flag).
 * Returns MCV_EINVAL for a bad device or out pointer, MCV_ECUDA/MCV_ENOMEM on failure. */
mcv_status mcv_create(int device, mcv_ctx** out);
/* Frees the context and its device memory; NULL is ignored. */
mcv_status mcv_destroy(mcv_ctx* ctx);
/* Message of the last error returned to the calling thread ("" if none). */
const char* mcv_last_error(void);
/* Waits for `stream`, then reports and clears the device error flag (MCV_EDEVICE).  With
 * ctx == NULL it reads the error word of mcv_grad_noalloc on the current device instead. */
mcv_status mcv_sync(mcv_ctx* ctx, void* stream);
/* Number of pixels of a detector description (0 if invalid). */
int64_t mcv_detector_pixels(const mcv_detector* det);
/* Sets n doubles at dst (device) to zero on `stream` with the library's own fill kernel. */
mcv_status mcv_zero(mcv_ctx* ctx, double* dst, int64_t n, void* stream);

/* Bytes of the device tables of the Bragg kernel (mcv_bragg) for n reflections (0 if n is not
 * 1..65536). */
int64_t mcv_bragg_table_bytes(int n);
/* Builds the Bragg kernel's tables from n reflections (host arrays: d_A spacings > 0 in A,
 * w >= 0 per-atom strengths in barn/A^3, see mcv_bragg), sorted by decreasing d (ties kept in
 * input order), into `tables` (device, `bytes` >= mcv_bragg_table_bytes(n)) on `stream`; sets
 * out->tables and out->n.  Errors: MCV_EINVAL, MCV_ECUDA. */
mcv_status mcv_bragg_build(const double* d_A, const double* w, int n, mcv_bragg* out,
                           void* tables, int64_t bytes, void* stream);

/* Bytes of the device tables of the phonon kernel (mcv_phonon), 0 for invalid sizes. */
int64_t mcv_phonon_table_bytes(int n_modes, int n_max);
/* Builds the tables of the phonon kernel from the density of states dos_z (host, n_modes
 * values Z(j*de_mev), j = 1..n_modes, >= 0, not all 0) and ph's n_modes, n_max (2..16),
 * de_mev, mass_u, temperature_K and p; writes ph->gamma0 and ph->c_w, copies the tables to
 * `tables` (device, `bytes` >= mcv_phonon_table_bytes) on `stream` and sets ph->tables.
 * The host data may be freed when the call returns.  Errors: MCV_EINVAL, MCV_ECUDA. */
mcv_status mcv_phonon_build(const double* dos_z, mcv_phonon* ph, void* tables, int64_t bytes,
                            void* stream);

/* Measurement of the histogram stage's roof (no counterpart in the paper): n_adds FP64
 * atomic adds of 1.0 into hist (n_bins doubles, device) at bins spread uniformly at random by
 * an integer hash of (seed, add index), the access pattern of the detector's histogram adds
 * without the tracing work.  Time it with events on `stream`. */
mcv_status mcv_bench_atomics(mcv_ctx* ctx, double* hist, int64_t n_bins, int64_t n_adds,
                             uint64_t seed, void* stream);

/* ---- the component chain ------------------------------------------------------------- */
/* Source: writes n packets with ids first_id..first_id+n-1 into out (slots 0..n-1; out->id
 * and out->order, if given, receive the id and 0).  fp_mode selects the array types. */
mcv_status mcv_beam(mcv_ctx* ctx, const mcv_beam_params* beam, int fp_mode, uint32_t seed,
                    uint32_t sim_id, int64_t first_id, int64_t n, mcv_neutrons* out,
                    void* stream);

/* Sample assembly (section 2.4.3, multiple scattering as a bounded chain of at most
 * max_orders scatterings per neutron; the paper's recursion samples the scattering point
 * on the first path segment and handles later segments in later rounds, this chain samples
 * it on all segments ahead at once, with the same expectation).
 * Incident neutrons: `in` (slots 0..n-1, id taken from in->id or first_id + slot) or, if
 * `in` is NULL, generated in registers from `beam` with ids first_id.. (fused source).
 * Outputs (at least one):
 *   det + hist : each scattered packet is traced through the detector and histogrammed in
 *                the same kernel (fused path); order-0 packets go to MCV_T_BEAMSTOP;
 *   packets    : n*(max_orders+1) slots, slot i*(max_orders+1)+o holds the packet of
 *                order o of the i-th neutron (order -1 if none) with its id.
 * With sample->estimator == MCV_EST_PAPER the sample assembly is traced by the paper's own
 * recursion (one neutron per GPU thread walking its tree of packets; random numbers keyed
 * by the packet's place in the tree: key (seed, sim_id ^ 0x80000000), counter (id lo, id hi,
 * 4 (node mod 2^30) + block, node / 2^30), the incident packet node 1 and the transmitted and
 * scattered packets of node x nodes 2x and 2x + 1); it needs det and hist (hist->events,
 * if given, receives every detected packet as with the chain) and takes no `in` or
 * `packets`.  A tree that outgrows the thread's stack of 48 waiting packets loses them and
 * sets the device error flag (MCV_EDEVICE at mcv_sync).
 * Errors: MCV_EINVAL for NULL/ill-formed descriptions, n < 0, unsupported combinations. */
mcv_status mcv_trace_sample(mcv_ctx* ctx, const mcv_sample* sample,
                            const mcv_beam_params* beam, const mcv_neutrons* in,
                            uint32_t seed, uint32_t sim_id, int64_t first_id, int64_t n,
                            const mcv_detector* det, mcv_hist* hist, mcv_neutrons* packets,
                            void* stream);

/* Detector system (section 2.4.3, "Ray tracing in a detector system"): every packet slot
 * with order >= 1 is traced to the first tube (or the surface) it meets; the absorption
 * point is drawn from the truncated exponential of the 3He path, the weight is multiplied
 * by the absorption probability, and (pixel, tof) is histogrammed.  Slots with order 0
 * add their weight to MCV_T_BEAMSTOP; order -1 slots are skipped; a slot with an order
 * above 7 (no packet of the library has one) is skipped and sets the device error flag
 * (MCV_EDEVICE at mcv_sync).  packets->id and packets->order are required (the detector
 * draw uses them).  fp_mode as the packets. */
mcv_status mcv_detect(mcv_ctx* ctx, const mcv_detector* det, int fp_mode,
                      const mcv_neutrons* packets, uint32_t seed, uint32_t sim_id,
                      mcv_hist* hist, mcv_events* events, void* stream);

/* Adjoint (no counterpart in the paper): chi2 = sum_b (c I_b - T_b)^2 / max(T_b, 1) of the
 * histogram of neutrons first_id..first_id+n-1, and its gradient with respect to the S(Q,E)
 * table entries and the absorption and scattering cross sections of scatterer
 * grad_scatterer, differentiating packet weights along the fixed random paths.
 * hist->counts (n_bins) receives I (cleared first); loss (1), dsqe (nq*ne) and dsig (2:
 * d/dsig_abs, d/dsig_s) are FP64 device outputs and are overwritten.  g_work (n_bins, may
 * be NULL) receives dchi2/dI of every bin; without it the adjoint evaluates dchi2/dI only
 * for the bins its packets reach (no per-bin buffer is written: the faster form).  target
 * bins must be finite and >= 0; others set the device error flag (MCV_EDEVICE at mcv_sync). */
mcv_status mcv_grad(mcv_ctx* ctx, const mcv_sample* sample, const mcv_beam_params* beam,
                    const mcv_detector* det, uint32_t seed, uint32_t sim_id,
                    int64_t first_id, int64_t n, const double* target, double scale_c,
                    int grad_scatterer, mcv_hist* hist, double* g_work, double* loss,
                    double* dsqe, double* dsig, void* stream);

/* The loss and the adjoint without the forward step, for a run whose neutrons are split
 * over several calls or devices (no counterpart in the paper): hist (n_bins, device, read
 * only) is the histogram of the WHOLE run -- the sum of every part's forward histogram --
 * and this call adds the gradient of the neutrons first_id..first_id+n-1 only.  loss
 * receives chi2 of hist (the same on every part), dsqe and dsig this part's share (all
 * overwritten; summed over the parts they give mcv_grad's gradient of the whole run).
 * g_work as mcv_grad.  Errors as mcv_grad. */
mcv_status mcv_adjoint(mcv_ctx* ctx, const mcv_sample* sample, const mcv_beam_params* beam,
                       const mcv_detector* det, uint32_t seed, uint32_t sim_id,
                       int64_t first_id, int64_t n, const double* hist, const double* target,
                       double scale_c, int grad_scatterer, double* g_work, double* loss,
                       double* dsqe, double* dsig, void* stream);

/* ---- batched launches ------------------------------------------------------------------- */
/* The paper has no counterpart to these calls.  A batch is many independent simulations
 * (sample orientations, incident energies, neutron counts of any mix) traced in ONE
 * persistent launch of the fused path (source -> sample -> detector -> histogram).  Each
 * simulation's neutron ids are cut into work items handed out by its own device queue; every
 * warp starts at a simulation of its own (warps spread in proportion to the neutron counts),
 * takes that simulation's items until its queue is empty, then helps with the others, so
 * uneven simulations keep every SM busy to the end.  Each neutron's history
 * and arithmetic are those of mcv_trace_sample with the same simulation's arguments; only
 * the order of the FP64 histogram additions differs.
 *
 * One simulation of a batch.  sample, beam: as mcv_trace_sample (sample->fp_mode must be
 * the batch's fp_mode); ids first_id..first_id+n-1 of the stream (seed, sim_id);
 * [tof_min_s, tof_max_s): this simulation's time window (n_tof bins of the batch detector;
 * both 0 keeps the detector's own window); hist: its histogram (n_pixels*n_tof FP64, may be
 * shared with other simulations) and/or tallies, accumulated into. */
typedef struct {
  const mcv_sample* sample;
  const mcv_beam_params* beam;
  uint32_t seed, sim_id;
  int64_t first_id, n;
  double tof_min_s, tof_max_s;
  mcv_hist hist;
} mcv_sim;

typedef struct mcv_batch mcv_batch;

/* Builds the parameter blocks of nsims >= 1 simulations sharing the detector `det` and
 * uploads them to device memory owned by the batch (this call allocates and synchronises;
 * the sims array and what it points to may be freed afterwards, the histograms may not).
 * The launch shape (neutrons per work item, blocks per SM) is the one mcv_batch_tune last
 * chose on this context for the same kind of batch, else a default.
 * Errors: MCV_EINVAL for any invalid simulation (the message names it), MCV_ENOMEM. */
mcv_status mcv_batch_create(mcv_ctx* ctx, const mcv_sim* sims, int nsims,
                            const mcv_detector* det, int fp_mode, mcv_batch** out);
/* Runs the batch on `stream`: clears the queue counter and launches the persistent kernel.
 * Allocates nothing and does not synchronise, so it can be captured in a CUDA graph and
 * replayed; runs of one batch must not overlap on the GPU (they share the queue). */
mcv_status mcv_batch_run(mcv_batch* b, void* stream);
/* Autotuner: times the batch kernel on a proportional sample of about trial_neutrons
 * neutrons (<= 0: 2e7) of this batch for each candidate launch shape -- work-item sizes of
 * 512..8192 neutrons (scaled by the sample's fraction of the batch in the trial, which keeps
 * the number of items per warp) and blocks per SM at and below the occupancy limit -- with
 * histograms in scratch memory (the simulations' own histograms are not touched), keeps the
 * fastest for this batch and records it on the context for later batches of the same kind
 * (real type, number of scatterers, detector kind, kernel set).  Synchronises `stream`;
 * allocates. */
mcv_status mcv_batch_tune(mcv_batch* b, int64_t trial_neutrons, void* stream);
/* The batch's launch shape: neutrons per work item, blocks per SM, grid size, work items. */
mcv_status mcv_batch_shape(const mcv_batch* b, int64_t* chunk, int* blocks_per_sm,
                           int* grid, int64_t* n_items);
/* Frees the batch after waiting for the device (cudaDeviceSynchronize); NULL is ignored. */
mcv_status mcv_batch_destroy(mcv_batch* b);
/* One-shot form: create, run and free in stream order (the parameter blocks live in
 * memory from the stream-ordered allocator, freed on `stream` after the launch; no host
 * synchronisation).  Not for graph capture: use mcv_batch_create + mcv_batch_run there. */
mcv_status mcv_trace_batch(mcv_ctx* ctx, const mcv_sim* sims, int nsims,
                           const mcv_detector* det, int fp_mode, void* stream);

/* ---- without allocation --------------------------------------------------------------- */
/* The paper has no counterpart to this entry point.  It is mcv_grad for callers that cannot
 * allocate device memory: code running inside CUDA graph capture or under someone else's
 * memory pool, processes whose allocator is locked down, or runtimes that only hand out
 * buffers they manage themselves.  It takes no context: the device error word and the
 * per-bin work buffer g (dchi2/dI) that mcv_grad gets from its context and its caller live
 * in one fixed device array inside the library, MCV_NOALLOC_MAX_BINS doubles (8 MiB) plus a
 * header, which every GPU that loads the library holds until the process exits.
 *   - Arguments and outputs are those of mcv_grad (no ctx, no g_work); histograms with more
 *     than MCV_NOALLOC_MAX_BINS bins are rejected with MCV_EINVAL and a message.
 *   - It runs on the current CUDA device.  The first call on a device looks up the array's
 *     device address (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.  Later calls made outside capture look it up again (the
 *     address of a context created anew, e.g. after cudaDeviceReset); calls made during
 *     capture use the address of the last lookup.  No call allocates or frees memory.
 *   - Every call shares the array: the work buffer is overwritten by each call, so
 *     consecutive calls on one stream are independent, but calls that overlap on the GPU
 *     (other streams, other host threads) race on it.
 *   - Errors: argument and launch errors as mcv_grad, returned at once.  Errors the kernels
 *     find on the device (as mcv_grad: an index out of range, a target bin that is negative
 *     or not finite) set the array's error word, which keeps them across calls until
 *     mcv_sync(NULL, stream) waits for `stream` and reports them (MCV_EDEVICE, word cleared).
 *     The message is returned by mcv_last_error(). */
#define MCV_NOALLOC_MAX_BINS (1 << 20)
mcv_status mcv_grad_noalloc(const mcv_sample* sample, const mcv_beam_params* beam,
                            const mcv_detector* det, uint32_t seed, uint32_t sim_id,
                            int64_t first_id, int64_t n, const double* target, double scale_c,
                            int grad_scatterer, mcv_hist* hist, double* loss, double* dsqe,
                            double* dsig, void* stream);

#ifdef __cplusplus
}
#endif
#endif
