// Launch-time parameter blocks of the ray-tracing kernels.  The host (mcv_api.cu) fills
// them from the public descriptions in mcv.h, precomputing the derived constants once;
// kernels receive them by value (kernel parameter space).
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

struct DBeam {
  double ei, rel, div, width, height, z0, l1;
  double speed0;   // sqrt(ei / kMeVPerV2)
  double t0;       // (l1 - z0) / speed0
};

struct DScat {
  int shape;
  int nk;
  int ktype0, ktype1;
  double dim0, dim1, dim2, half_h;  // half_h: half height of cylinders
  double cos_rot, sin_rot;
  double mu_s;       // 100 n sigma_s            (1/m)
  double mu_a_v;     // 100 n sigma_abs 2200     (1/m * m/s): mu_abs(v) = mu_a_v / v
  double ksig0, ksig_sum;
  double n100;       // 100 n (for the adjoint)
  double sig_s;
};

struct DSample {
  int ns;
  int max_orders;
  double min_prob;
  DScat s[MCV_MAX_SCATTERERS];
  const float* sqe;
  int nq, ne;
  double q_max, e_min, e_max, dq, de;
  int has_sqe;
};

struct DDet {
  int kind;
  double radius;
  double height, half_h;
  int n_phi, n_y;
  int n_rows;
  int packs[3];
  int row_off[3];
  double row_y[3];
  int tubes_per_pack, pixels_per_tube;
  int max_tubes_row;
  double tube_r, half_len, pitch, period, phi0, pix_len;
  double mu_he_v;    // 100 n sigma 2200: mu(v) = mu_he_v / v (1/m)
  double tof_min, dt, inv_dt;
  int n_tof;
  int64_t n_bins;
  double tube_u[2 * MCV_MAX_TUBES_PER_ROW];  // sin, cos of every tube centre angle of a row
};

struct TraceArgs {
  DSample S;
  DDet D;
  DBeam B;
  uint32_t seed, sim_id;
  int64_t first_id, n;
  // fused outputs
  double* hist;
  double* tallies;
  // stored input (null: generate from B)
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
  // adjoint: the scatterer whose cross sections are differentiated, dchi2/dI per bin,
  // and the FP64 gradient outputs
  int gs;
  const double* g;
  double* dsqe;
  double* dsig;
};

}  // namespace mcv
