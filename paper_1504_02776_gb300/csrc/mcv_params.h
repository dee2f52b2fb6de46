// Launch-time parameter blocks of the ray-tracing kernels.  The host (mcv_api.cu) fills
// them from the public descriptions in mcv.h, precomputing the derived constants once, in
// both real types: the FP32 kernels read only float fields (no conversion of parameters at
// run time), the FP64 kernels only double fields.  Kernels receive them by value (kernel
// parameter space).
#pragma once

#include <cstdint>

#include "../../include/mcv.h"

namespace mcv {

// physical constants (CODATA 2018)
constexpr double kNeutronMass = 1.67492749804e-27;  // kg
constexpr double kHbar = 1.054571817e-34;           // J s
constexpr double kElemCharge = 1.602176634e-19;     // C
constexpr double kPi = 3.14159265358979323846;
// E[meV] = kMeVPerV2 v^2 with v in m/s;  k[1/A] = kKPerV v
constexpr double kMeVPerV2 = 0.5 * kNeutronMass / (kElemCharge * 1e-3);
constexpr double kKPerV = kNeutronMass / kHbar * 1e-10;

template <typename R>
struct BeamP {
  R ei, rel, div, width, height, z0, l1;
  R speed0;            // sqrt(ei / kMeVPerV2)
  double t0;           // (l1 - z0) / speed0
  float t0_hi, t0_lo;  // t0 as a float pair
  // every energy draw is positive: rel z > -1 for every Box-Muller z the uniforms can give
  // (|z| <= sqrt(-2 ln 2^-54) = 8.65 for uniforms >= 2^-54), checked as rel * 8.7 < 1
  int energy_positive;
  // footprints with |x| > x_safe or |y| > y_safe miss the sample for every divergence the
  // uniforms can give (+inf: no such shortcut); set from the sample's bounding cylinder
  R x_safe, y_safe;
};

template <typename R>
struct ScatP {
  int shape;
  int nk;
  int ktype0, ktype1;
  R dim0, dim1, dim2, half_h;  // half_h: half height of cylinders
  R cos_rot, sin_rot;
  R n100;       // 100 n   (mu[1/m] = 100 n[1/A^3] sigma[barn])
  R sig_s;      // scattering cross section (sum of the kernels')
  R sab2200;    // sigma_abs 2200: mu_tot(v) = 100 n (sigma_s + sab2200 / v)
  R mu_s;       // 100 n sigma_s
  R ksig0, ksig1, ksig_sum;  // the kernels' nominal cross sections and their sum
};

template <typename R>
struct SampleP {
  int ns;
  int max_orders;
  int nq, ne;
  int has_sqe;
  R min_prob;
  ScatP<R> s[MCV_MAX_SCATTERERS];
  const float* sqe;
  R q_max, e_min, e_max, dq, de;
  // single-crystal Born-von Karman kernel
  int has_bvk;
  R bvk_coef;      // phi / M (1/s^2)
  R bvk_ah;        // a / 2 (A)
  R bvk_hb2m;      // hbar^2 / 2M (meV A^2)
  R bvk_kT;        // k_B T (meV)
  R bvk_msd;       // <u^2> (A^2)
  R bvk_wmax;      // upper bound of hbar omega (meV)
  R bvk_hwu;       // hbar sqrt(phi/M) in meV: hbar omega = bvk_hwu sqrt(lambda')
  // incoherent phonon kernel (mcv_phonon): cumulative masses of A_1 (2J + 1) and of the
  // multi-phonon mixture B (M = 2NJ + 1), the masses of B and A_2..A_N (rows of M), in R
  int has_phonon;
  int ph_J, ph_N, ph_M;
  const R* ph_cdf1;
  const R* ph_cdfb;
  const R* ph_b;
  const R* ph_an;
  R ph_de, ph_cw, ph_p0, ph_p1, ph_p2, ph_p01;
  // coherent elastic powder kernel (mcv_bragg): n_refl reflections by decreasing spacing,
  // their spacings and the prefix sums of strength x spacing
  int has_bragg;
  int n_refl;
  const R* refl_d;
  const R* refl_c;
  // dispersion-surface kernel (mcv_dispersion)
  int has_disp;
  R disp_amp, disp_c, disp_s0;
  // the launch needs the full kernel set (any kernel besides isotropic and S(Q,E))
  int wide;
};

// Event-mode output: records appended at atomically taken indexes (mcv_event_list); tag =
// the simulation's sim_id.  count == nullptr: no event list.
struct EvSink {
  int32_t* pixel;
  uint32_t* sim;
  double* tof;
  double* w;
  int64_t cap;
  unsigned long long* count;
  uint32_t tag;
};

// Round keys of a Philox4x32-10 stream keyed by (seed, sim): round r uses
// (seed + r 0x9E3779B9, sim + r 0xBB67AE85).  They depend on the key only, so the host
// computes them once per launch and the kernels read them as constants.
struct PhiloxKeys {
  uint32_t k0[10], k1[10];
};

// time-of-flight window of the histogram: n_tof bins of width dt from tof_min
struct TofWin {
  double tof_min, dt;
  float tmin_hi, tmin_lo, inv_dt;  // FP32 binning: tof_min as a float pair, 1 / dt
  int n_tof;
};

template <typename R>
struct DetP {
  int kind;
  int n_phi, n_y;
  int n_rows;
  int packs[3];
  int row_off[3];
  int tubes_per_pack, pixels_per_tube;
  int max_tubes_row;
  int64_t n_bins;
  R radius, height, half_h;
  R row_y[3];
  R tube_r, half_len, pitch, period, phi0, pix_len;
  R mu_he_v;        // 100 n sigma 2200: mu(v) = mu_he_v / v (1/m)
  TofWin win;
  // packets that surely miss every tube (tube system; set when the packets start inside a
  // known sample, else off): a packet whose horizontal path to the tube ring is at least
  // miss_r_in - (|x| + |z|) and whose height there lies above miss_y_top or below
  // miss_y_bot, or (miss_phi) whose horizontal direction lies outside the arc from
  // (miss_a_x, miss_a_z) to (miss_b_x, miss_b_z) that holds every tube seen from the sample
  R miss_r_in, miss_y_top, miss_y_bot;
  int miss_phi;
  R miss_a_x, miss_a_z, miss_b_x, miss_b_z;
  int multi_tube;   // the paper estimator's detector: the remainder goes on to the next tubes
  R tube_u[2 * MCV_MAX_TUBES_PER_ROW];  // sin, cos of every tube centre angle of a row
};

struct TraceArgs {
  SampleP<float> Sf;
  SampleP<double> Sd;
  DetP<float> Df;
  DetP<double> Dd;
  BeamP<float> Bf;
  BeamP<double> Bd;
  uint32_t seed, sim_id;
  PhiloxKeys keys;  // round keys of (seed, sim_id)
  PhiloxKeys pkeys; // round keys of (seed, sim_id ^ 0x80000000): the paper estimator's streams
  int64_t first_id, n;
  // fused outputs
  double* hist;
  double* tallies;
  EvSink ev;
  // stored input (null: generate from the beam)
  const void *in_x, *in_y, *in_z, *in_vx, *in_vy, *in_vz, *in_w;
  const double* in_t;
  const int64_t* in_id;
  const int32_t* in_order;
  // packet slots (null: not written)
  void *pk_x, *pk_y, *pk_z, *pk_vx, *pk_vy, *pk_vz, *pk_w;
  double* pk_t;
  int64_t* pk_id;
  int32_t* pk_order;
  int* err;
  int stop_on_zero;
  // adjoint: the scatterer whose cross sections are differentiated, dchi2/dI per bin (g;
  // when null, g_b is evaluated from the forward histogram hist_in, the target and scale_c
  // for the bins the packets reach), and the FP64 gradient outputs
  int gs;
  const double* g;
  const double* hist_in;
  const double* target;
  double scale_c;
  double* dsqe;
  double* dsig;
};

// One simulation of a batched launch: its own sample, beam, random stream, neutron range,
// time window and histogram; the detector geometry is the batch's.
template <typename R>
struct SimP {
  SampleP<R> S;
  BeamP<R> B;
  TofWin win;
  uint32_t seed, sim_id;
  int64_t first_id, n;
  double* hist;
  double* tallies;
  EvSink ev;
};

// The work queues of a batched launch: simulation s is cut into items of `chunk` neutron
// ids, handed out in order by its own counter next[s].  A warp starts at its home
// simulation -- the one holding neutron (total * warp / warps) of the batch in the order of
// the nstart prefix sums -- and, when that queue is empty, moves on to the following
// simulations (cyclically) until every queue is empty.
struct BatchArgs {
  const void* sims;          // SimP<R>[nsims], device
  const int64_t* nstart;     // nsims + 1 prefix sums of the neutron counts, device
  unsigned long long* next;  // nsims item counters, zero at launch, device
  int nsims;
  int64_t chunk;             // neutrons per work item
  int64_t total;             // nstart[nsims]
};

}  // namespace mcv
