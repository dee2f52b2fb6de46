/*
 * Oracle for the neutron ray-tracing hot path of MCViNE (Lin et al., "MCViNE -- An
 * object oriented Monte Carlo neutron ray tracing simulation package").
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, single-threaded FP64 CPU restatement
 * of what the hot path computes.  It exists so that the CUDA path can be checked against
 * something written straight from the paper.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it; the product path never does.  It shares
 * no code, header or constant table with the CUDA library.
 *
 * Every function cites the passage of the paper it follows.  Where the paper is silent
 * the reading taken is stated next to the code.
 *
 * Parity unpinned: the absolute normalisation of the kernels against measured data
 * (no experimental data is available); everything else is pinned by the CPU tests.
 */
#ifndef MCV_ORACLE_H
#define MCV_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* shape kinds (all centred at the origin, axis or rotation axis along +y) */
enum { ORC_SOLID_CYL = 0, ORC_HOLLOW_CYL = 1, ORC_BLOCK = 2 };
/* kernel kinds */
enum { ORC_K_ISO = 0, ORC_K_SQE = 1, ORC_K_BVK = 2, ORC_K_PHONON = 3, ORC_K_BRAGG = 4,
       ORC_K_DISP = 5 };
/* detector kinds */
enum { ORC_DET_NONE = 0, ORC_DET_SURFACE = 1, ORC_DET_TUBES = 2 };

typedef struct {
  int kind;
  double dims[3];      /* SOLID: r,h   HOLLOW: r_in,r_out,h   BLOCK: wx,wy,wz  (m) */
  double rot_y;        /* rotation of the body about +y (rad) */
  double n_per_A3;     /* number density (1/A^3) */
  double sig_abs_b;    /* absorption cross section at 2200 m/s (barn), 1/v law */
  int nk;              /* number of kernels (1 or 2) */
  int ktype[2];        /* ORC_K_* */
  double ksig_b[2];    /* scattering cross section of each kernel (barn) */
} orc_scatterer;

typedef struct {
  /* beam (source -> sample) */
  double ei_mev, ei_rel_sigma, div_sigma_rad, width_m, height_m, z0_m, l1_m;
  /* sample assembly */
  int n_scat;
  orc_scatterer scat[4];
  int max_orders;      /* N_max: maximum number of scatterings of one packet */
  double min_prob;     /* packets with weight below this are dropped */
  /* tabulated S(Q,E), FP32, row-major [iq][ie], bin centred grid */
  const float* sqe;
  int nq, ne;
  double q_max, e_min, e_max;
  /* single-crystal Born-von Karman kernel (fcc, nearest-neighbour central force) */
  double bvk_phi_Nm, bvk_mass_u, bvk_a_A, bvk_msd_A2, temperature_K;
  /* incoherent scattering from a phonon density of states (temperature_K as above):
     dos_z[j-1] = Z(j dos_de), j = 1..dos_n, the modes of the energy bin j dos_de (meV);
     phonon_nmax >= 2 the largest order of the multi-phonon channel; phonon_p the
     probabilities of the elastic, one-phonon and multi-phonon channels */
  const double* dos_z;
  int dos_n;
  double dos_de, phonon_mass_u;
  int phonon_nmax;
  double phonon_p[3];
  /* coherent elastic powder diffraction: n_refl reflections, spacing refl_d (A) and
     per-atom strength refl_w = multiplicity |F|^2 / (v0 atoms per cell) (barn / A^3) */
  const double* refl_d;
  const double* refl_w;
  int n_refl;
  /* detector: the packet's weight left after a tube goes on to the next tubes it crosses
     (the detector system as a composite of absorbing tubes); 0: first tube only */
  int det_multi_tube;
  /* scattering from a dispersion surface E(Q) = disp_amp sqrt(1 - (cos(c Qx) cos(c Qz))^2),
     c = disp_c (A), with S(Q) = disp_s0, Q in the crystal frame of scatterer 0's rotation */
  double disp_amp, disp_c, disp_s0;
  /* detector */
  int det_kind;
  double det_radius_m, det_height_m; /* SURFACE */
  int n_phi, n_y;                    /* SURFACE */
  int n_rows, packs[3];              /* TUBES */
  double row_y_m[3];
  int tubes_per_pack, pixels_per_tube;
  double tube_r_m, tube_len_m, tube_pitch_m, pack_gap_m, phi0_rad;
  double he3_n_per_A3, he3_sig_abs_b;
  double tof_min_s, tof_max_s;
  int n_tof;
  /* random streams */
  uint32_t seed, sim_id;
} orc_config;

/* one emitted packet (the transmitted neutron of one order) and what the detector made of it */
typedef struct {
  int64_t nid;
  int32_t order;       /* -1: slot unused */
  int32_t pixel;       /* -1: missed the detector */
  double x, y, z, vx, vy, vz, t, w;
  double tof, w_det;
  int64_t bin;         /* pixel*n_tof + tof bin; -1 missed, -2 tof out of range */
  double kappa;        /* condition estimate of w: relative change of w per relative
                          rounding of the inputs, summed over the packet's history */
  double kappa_det;    /* the same for w_det (adds the tube chord) */
} orc_packet;

/* per-scatter record (debug / pins) */
typedef struct {
  int64_t nid;
  int32_t order;       /* the order of the packet created by this scatter (1..N_max) */
  int32_t kernel;      /* ORC_K_* */
  int32_t scatterer;
  int32_t entry;       /* S(Q,E) table entry, -1 if none */
  double q, e, ki, kf, factor;
  double w;            /* packet weight right after this scatter */
  int32_t nroots;      /* single-crystal kernel: roots found for the drawn mode */
  int32_t mode;        /* single-crystal kernel: branch + 3 * (annihilation) */
  double qvec[3];      /* ki_vec - kf_vec */
} orc_event;

enum { ORC_T_BEAMSTOP = 0, ORC_T_WDET, ORC_T_WOVER, ORC_T_NDET, ORC_T_NOVER, ORC_T_NMISS,
       ORC_T_NHIT, ORC_T_NPACK0, ORC_NTALLY = ORC_T_NPACK0 + 8 };

/* counter-based generator (Philox4x32-10, Salmon et al. SC'11) */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* the two uniforms in (0,1) drawn for (neutron id, event, block); event -1 = beam */
void orc_uniforms(uint32_t seed, uint32_t sim_id, int64_t nid, int event, int block,
                  double u[2]);

/* geometry: segments [s_a, s_b] of the ray r + s d (s >= 0) inside scatterer sc.
   returns the count (<= 2). */
int orc_shape_segments(const orc_scatterer* sc, const double r[3], const double d[3],
                       double sa[2], double sb[2]);

/* one kernel scatter: in = speed and unit direction; writes the new speed, direction,
   weight factor; returns 0 if the kernel kills the packet.  The single-crystal kernel takes
   the orientation of scatterer 0. */
int orc_kernel_scatter(const orc_config* cfg, int ktype, double speed, const double d[3],
                       const double u[4], double* speed_out, double d_out[3],
                       double* factor, orc_event* ev);

/* the multi-tube detector (tube system): the packet is absorbed in every tube it crosses
   among the three candidates, in order of entry, each taking its absorption probability of
   the weight the earlier ones left; u[i] draws the absorption depth in the i-th tube.  Writes
   up to 3 detections (bin >= 0, -2 out of the time window); returns their number */
int orc_detect_multi(const orc_config* cfg, const double r[3], const double v[3], double t,
                     double w, const double u[3], int32_t pixel[3], double tof[3],
                     double w_det[3], int64_t bin[3]);

/* detect one packet: returns bin (>= 0), -1 miss, -2 tof overflow */
int64_t orc_detect(const orc_config* cfg, const double r[3], const double v[3], double t,
                   double w, double u_det, int32_t* pixel, double* tof, double* w_det);

/* chain-mode tracer.  packets: n*(max_orders+1) slots or NULL; events: n*max_orders slots
   or NULL; hist: n_pixels*n_tof, accumulated into, or NULL; tallies: ORC_NTALLY doubles,
   accumulated into, or NULL. */
int orc_trace(const orc_config* cfg, int64_t first_id, int64_t n, orc_packet* packets,
              orc_event* events, double* hist, double* tallies);

/* paper-literal recursive estimator (scatterM / interactM_path1 / interactM1);
   histogram and tallies only.  Random numbers: key (seed, sim_id ^ 0x80000000), counter
   (nid lo, nid hi, 4 (node mod 2^30) + block, node / 2^30) where node is the packet's place
   in the tree of interactions (the incident packet 1; an interaction of node x gives its
   transmitted packet 2x and its scattered packet 2x + 1), so that any order of visiting the
   tree draws the same numbers; blocks 0-2 of a node serve its interaction, blocks 3 and 0 of
   an emitted packet's node its detector draws */
int orc_trace_paper(const orc_config* cfg, int64_t first_id, int64_t n, double* hist,
                    double* tallies);

int64_t orc_n_pixels(const orc_config* cfg);

/* chi-squared loss on the histogram and its adjoint gradient with respect to the S(Q,E)
   table entries (dsqe, nq*ne) and the absorption and scattering cross sections of
   scatterer `gs` (dsig[0] = d/d sig_abs, dsig[1] = d/d sig_s).  hist_out (n_pixels*n_tof)
   receives the forward histogram. */
int orc_grad(const orc_config* cfg, int64_t first_id, int64_t n, const double* target,
             double scale_c, int gs, double* hist_out, double* loss, double* dsqe,
             double* dsig);

/* the loss of `hist` (the whole run's histogram, n_pixels*n_tof) and the adjoint gradient of
   the neutrons first_id..first_id+n-1 only (dsqe, dsig overwritten): the parts of a split run
   add up to orc_grad of the whole run */
int orc_adjoint(const orc_config* cfg, int64_t first_id, int64_t n, const double* hist,
                const double* target, double scale_c, int gs, double* loss, double* dsqe,
                double* dsig);

/* loss only (for finite differences) */
int orc_loss(const orc_config* cfg, int64_t first_id, int64_t n, const double* target,
             double scale_c, double* hist_work, double* loss);

/* Born-von Karman fcc dispersion: q in 1/A (crystal frame); energies (meV, ascending) and
   eigenvectors (columns, e[3*i+b] = component i of branch b) */
void orc_bvk_modes(const orc_config* cfg, const double q[3], double hw[3], double evec[9]);

/* single-crystal one-phonon kernel with the crystal rotated by rot_y about +y */
int orc_kernel_bvk(const orc_config* cfg, double rot_y, double speed, const double d[3],
                   const double u[4], double* speed_out, double d_out[3], double* factor,
                   orc_event* ev);

/* the tables of the phonon kernel (for the pins): gamma_0 (1/meV), c_w (2W = c_w Q^2, A^2)
   and the masses of A_n on the grid E = i dos_de, i = -n_max*dos_n..n_max*dos_n
   (a[(n-1)*M + i + n_max*dos_n], n = 1..n_max, M = 2*n_max*dos_n + 1); returns M, or 0 */
int orc_phonon_tables(const orc_config* cfg, double* gamma0, double* c_w, double* a, int64_t cap);

#ifdef __cplusplus
}
#endif
#endif
