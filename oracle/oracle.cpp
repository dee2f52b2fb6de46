// Oracle for the MCViNE neutron ray-tracing hot path.
//
// TEST INFRASTRUCTURE ONLY: a plain, slow, single-threaded FP64 CPU restatement of the
// method, written from the paper, used to check the CUDA library.  The product path never
// loads it.  It shares no code, header or constant with the CUDA library.
// Built with -ffp-contract=off so every product and sum is rounded separately.
//
// Parity unpinned: absolute kernel normalisation against measured data (none available).
#include "oracle.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <vector>

namespace {

// ---- physical constants (CODATA 2018) -------------------------------------------------
const double kNeutronMass = 1.67492749804e-27;   // kg
const double kHbar = 1.054571817e-34;            // J s
const double kElemCharge = 1.602176634e-19;      // C
const double kBoltzmann = 1.380649e-23;          // J/K
const double kAtomicMass = 1.66053906660e-27;    // kg
const double kPi = 3.14159265358979323846;
// E[meV] = kMeVPerV2 * v^2 (v in m/s);  k[1/A] = kKPerV * v
const double kMeVPerV2 = 0.5 * kNeutronMass / (kElemCharge * 1e-3);
const double kKPerV = kNeutronMass / kHbar * 1e-10;
const double kInf = std::numeric_limits<double>::infinity();

struct Vec3 {
  double x, y, z;
};
Vec3 add(Vec3 a, Vec3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
Vec3 scale(Vec3 a, double s) { return {a.x * s, a.y * s, a.z * s}; }
double dot(Vec3 a, Vec3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
Vec3 cross(Vec3 a, Vec3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

// ---- random numbers -------------------------------------------------------------------
// Counter slot of (event, block): four blocks per event, event -1 is beam generation.
uint32_t slot_of(int event, int block) { return (uint32_t)(4 * (event + 1) + block); }

double u01_from(uint32_t hi, uint32_t lo) {
  // 53 random bits -> (k + 1/2) 2^-53, strictly inside (0,1)
  uint64_t k = ((uint64_t)hi << 21) | (uint64_t)(lo >> 11);
  return (double)k * 0x1p-53 + 0x1p-54;
}

// ---- conditioning ---------------------------------------------------------------------
// The condition estimate below is test infrastructure of its own: it sets the tolerances the
// tests compare rounding-sensitive results with and takes no part in the method.  Every
// statement of it is guarded by ORC_CONDITION, so a build with ORC_CONDITION=0 (the
// operation count of the method, oracle/opcount.py) compiles it out.
#ifndef ORC_CONDITION
#define ORC_CONDITION 1
#endif
// Condition estimate of the current packet's weight: each chord or range width that
// subtracts nearly equal numbers adds its amplification factor (|value| / |difference|).
// It only sets the tolerances the tests compare rounding-sensitive results with.
thread_local double g_kappa = 0.0;
// relative-error budget of the current speed (units of the FP64 epsilon), carried from
// kernel to kernel for the condition estimate
thread_local double g_kappa_v = 0.0;
// error scales (units of the FP64 epsilon) of the current point and direction, for the
// chords computed from them: g_err_r (metres) from the roundings of the point's own
// coordinates, taken in any direction; g_err_a (metres) from the error of the distance
// along the previous ray (g_dprev) that placed the point, which moves a later surface
// crossing only by its component along that surface's normal; g_err_d (dimensionless) of
// the direction, carried while directions are built on each other.  An older error of the
// start point moves the surfaces the ray met with the point, so it is not carried on.
thread_local double g_err_r = 0.0;
thread_local double g_err_a = 0.0;
thread_local Vec3 g_dprev = {0.0, 0.0, 0.0};
thread_local double g_err_d = 0.0;

// ---- geometry -------------------------------------------------------------------------
// One end of a ray interval: its distance s and two absolute error scales (units of the
// FP64 epsilon, metres): er from the roundings of its own computation, ep from the errors
// of the start point and direction (g_err_r, g_err_d).
struct End {
  double s, er, ep;
};

// Interval of s in which the line r + s d lies inside the infinite cylinder x^2+z^2 < R^2
// (axis along y through the origin).  Written with the point of closest approach: its
// squared distance to the axis is (r x d)^2 / a in the xz-plane, which stays accurate when
// the start point is far from the axis compared with R.  e (optional) receives both ends
// with their error scales: the roundings of tc +- half (and of g, R^2 / (half a) after the
// square root), and the shift of a root under a change of the start point or direction,
// whose derivative is R / (half a) (the surface point p obeys p.d = half a, |p| = R).
bool cylinder_interval(double R, Vec3 r, Vec3 d, double* s1, double* s2, End* e = nullptr) {
  double a = d.x * d.x + d.z * d.z;
  if (a == 0.0) {
    if (r.x * r.x + r.z * r.z < R * R) {
      *s1 = -kInf;
      *s2 = kInf;
      if (e) e[0] = {-kInf, 0.0, 0.0}, e[1] = {kInf, 0.0, 0.0};
      return true;
    }
    return false;
  }
  double tc = -(r.x * d.x + r.z * d.z) / a;
  double cr = r.x * d.z - r.z * d.x;
  double g = R * R - cr * cr / a;
  if (!(g > 0.0)) return false;
  if (ORC_CONDITION) g_kappa += R * R / g;
  double half = std::sqrt(g / a);
  *s1 = tc - half;
  *s2 = tc + half;
  if (e && !ORC_CONDITION) e[0] = {*s1, 0.0, 0.0}, e[1] = {*s2, 0.0, 0.0};
  if (e && ORC_CONDITION) {
    double lever = R / (half * a);
    double er = std::fabs(tc) + half + lever * R;
    double ss[2] = {*s1, *s2};
    for (int i = 0; i < 2; ++i) {
      // the crossing point p (|p| = R); a shift of the start along g_dprev moves the root
      // by its component along p over p.d = half a
      double px = r.x + ss[i] * d.x, pz = r.z + ss[i] * d.z;
      double along = std::fabs(px * g_dprev.x + pz * g_dprev.z) / (half * a);
      e[i] = {ss[i], er,
              lever * (g_err_r + std::fabs(ss[i]) * g_err_d) + along * g_err_a};
    }
  }
  return true;
}

// The same for a vertical tube of radius rt whose axis crosses the xz-plane at R (ux, uz),
// (ux, uz) a unit vector: coordinates are taken along and across that direction, so that
// the large distance R cancels exactly once.
bool tube_interval(double R, double ux, double uz, double rt, Vec3 r, Vec3 d, double* s1,
                   double* s2) {
  double a = d.x * d.x + d.z * d.z;
  if (a == 0.0) return false;
  double o_rad = r.x * ux + r.z * uz - R;
  double o_tan = r.x * uz - r.z * ux;
  double d_rad = d.x * ux + d.z * uz;
  double d_tan = d.x * uz - d.z * ux;
  double tc = -(o_rad * d_rad + o_tan * d_tan) / a;
  double cr = o_rad * d_tan - o_tan * d_rad;
  double g = rt * rt - cr * cr / a;
  if (!(g > 0.0)) return false;
  // the chord is sensitive to the tube radius (rt^2/g) and, through the lever arm, to the
  // direction of the ray (closest-approach distance h, distance |tc| sqrt(a))
  // and to the error of the start point (|cr| |dr| / (sqrt(a) g))
  if (ORC_CONDITION)
    g_kappa += rt * rt / g + std::fabs(tc) * std::fabs(cr) / g +
               std::fabs(cr) * (g_err_r + g_err_a) / (std::sqrt(a) * g);
  double half = std::sqrt(g / a);
  *s1 = tc - half;
  *s2 = tc + half;
  return true;
}

// Interval of s in which |p + s dp| < half.  e (optional): both ends with their error
// scales, (|p| + half) / |dp| from the roundings (p_rounding: roundings already in p and dp,
// as multiples of |p| and 1) and (p_err + |s| d_err) / |dp| from the start point and
// direction (dprev_p: the slab-normal component of the previous ray, along which the start
// point's distance error lies).
bool slab_interval(double half, double p, double dp, double* s1, double* s2, End* e = nullptr,
                   double p_rounding = 0.0, double dprev_p = 1.0) {
  if (dp == 0.0) {
    if (std::fabs(p) < half) {
      *s1 = -kInf;
      *s2 = kInf;
      if (e) e[0] = {-kInf, 0.0, 0.0}, e[1] = {kInf, 0.0, 0.0};
      return true;
    }
    return false;
  }
  double a = (-half - p) / dp;
  double b = (half - p) / dp;
  *s1 = std::min(a, b);
  *s2 = std::max(a, b);
  if (e && !ORC_CONDITION) e[0] = {*s1, 0.0, 0.0}, e[1] = {*s2, 0.0, 0.0};
  if (e && ORC_CONDITION) {
    double ad = std::fabs(dp);
    double er = ((1.0 + p_rounding) * std::fabs(p) + half) / ad;
    double ea = g_err_r + std::fabs(dprev_p) * g_err_a;
    e[0] = {*s1, er + p_rounding * std::fabs(*s1) / ad, (ea + std::fabs(*s1) * g_err_d) / ad};
    e[1] = {*s2, er + p_rounding * std::fabs(*s2) / ad, (ea + std::fabs(*s2) * g_err_d) / ad};
  }
  return true;
}

// Keep [a,b] clipped to s >= s0 (s0 = 0 but for the paper mode's transmitted packets, which
// keep their line's origin and the distance s0 travelled along it) if it has positive length.  Its length b - lo loses the
// relative precision |a| + |b| over b - lo (a point close to the exit surface), and the
// error scales of the ends over b - lo (a clipped start, lo = 0, is exact).  ra, rb
// (optional) receive the error scales of the kept ends, ra0 the start's rounding scale
// alone (an error of the start point or direction moves the point placed beyond the start
// surface with that surface).
int push_segment(End a, End b, double* sa, double* sb, double* ra, double* rb, double* ra0,
                 int n, double s0) {
  double lo = std::max(a.s, s0);
  if (b.s > lo) {
    double e_lo = a.s > s0 ? a.er + a.ep : 0.0;
    if (ORC_CONDITION)
      g_kappa += (std::fabs(a.s) + std::fabs(b.s) + e_lo + b.er + b.ep) / (b.s - lo);
    sa[n] = lo;
    sb[n] = b.s;
    if (ORC_CONDITION && ra) {
      ra[n] = e_lo;
      rb[n] = b.er + b.ep;
      ra0[n] = a.s > s0 ? a.er : 0.0;
    }
    return n + 1;
  }
  return n;
}

// the later of two interval starts, and the earlier of two ends
End later(End u, End v) { return v.s > u.s ? v : u; }
End earlier(End u, End v) { return v.s < u.s ? v : u; }

int shape_segments(const orc_scatterer& sc, Vec3 r, Vec3 d, double sa[2], double sb[2],
                   double ra[2] = nullptr, double rb[2] = nullptr, double ra0[2] = nullptr,
                   double s0 = 0.0) {
  // Shapes and their combination (the hollow cylinder is a difference of two cylinders),
  // paper section 2.4.2 ("Shapes" and constructive solid geometry).  ra, rb (optional)
  // receive the error scales of the segment ends, ra0 the starts' rounding scales.
  double y1, y2, c1, c2;
  End ec[2], ey[2];
  if (sc.kind == ORC_SOLID_CYL) {
    if (!cylinder_interval(sc.dims[0], r, d, &c1, &c2, ec)) return 0;
    if (!slab_interval(0.5 * sc.dims[1], r.y, d.y, &y1, &y2, ey, 0.0, g_dprev.y)) return 0;
    return push_segment(later(ec[0], ey[0]), earlier(ec[1], ey[1]), sa, sb, ra, rb, ra0, 0, s0);
  }
  if (sc.kind == ORC_HOLLOW_CYL) {
    if (!cylinder_interval(sc.dims[1], r, d, &c1, &c2, ec)) return 0;
    if (!slab_interval(0.5 * sc.dims[2], r.y, d.y, &y1, &y2, ey, 0.0, g_dprev.y)) return 0;
    End lo = later(ec[0], ey[0]), hi = earlier(ec[1], ey[1]);
    if (!(hi.s > lo.s)) return 0;
    double i1, i2;
    End ei[2];
    if (!cylinder_interval(sc.dims[0], r, d, &i1, &i2, ei))
      return push_segment(lo, hi, sa, sb, ra, rb, ra0, 0, s0);
    int n = 0;
    n = push_segment(lo, earlier(hi, ei[0]), sa, sb, ra, rb, ra0, n, s0);
    n = push_segment(later(lo, ei[1]), hi, sa, sb, ra, rb, ra0, n, s0);
    return n;
  }
  if (sc.kind == ORC_BLOCK) {
    // body frame: the block is rotated by rot_y about +y, so body = R^T lab
    double c = std::cos(sc.rot_y), s = std::sin(sc.rot_y);
    Vec3 rb_ = {c * r.x - s * r.z, r.y, s * r.x + c * r.z};
    Vec3 db = {c * d.x - s * d.z, d.y, s * d.x + c * d.z};
    End lo = {-kInf, 0.0, 0.0}, hi = {kInf, 0.0, 0.0}, e[2];
    double a, b;
    // the rotated coordinates carry a few more roundings of |r| and |d|
    double px = c * g_dprev.x - s * g_dprev.z, pz = s * g_dprev.x + c * g_dprev.z;
    if (!slab_interval(0.5 * sc.dims[0], rb_.x, db.x, &a, &b, e, 3.0, px)) return 0;
    lo = later(lo, e[0]);
    hi = earlier(hi, e[1]);
    if (!slab_interval(0.5 * sc.dims[1], rb_.y, db.y, &a, &b, e, 0.0, g_dprev.y)) return 0;
    lo = later(lo, e[0]);
    hi = earlier(hi, e[1]);
    if (!slab_interval(0.5 * sc.dims[2], rb_.z, db.z, &a, &b, e, 3.0, pz)) return 0;
    lo = later(lo, e[0]);
    hi = earlier(hi, e[1]);
    return push_segment(lo, hi, sa, sb, ra, rb, ra0, 0, s0);
  }
  return 0;
}

struct Segment {
  double sa, sb;
  int j;         // scatterer index
  double ra, rb;  // error scales of the ends (units of the FP64 epsilon, metres)
  double ra0;     // rounding scale of the start alone
};

// All material segments ahead of the ray, sorted by entry distance (ray tracing in a
// composite scatterer, section 2.4.3 "Ray Tracing").
int assembly_segments(const orc_config& cfg, Vec3 r, Vec3 d, Segment* out, double s0 = 0.0) {
  int n = 0;
  for (int j = 0; j < cfg.n_scat; ++j) {
    double sa[2], sb[2], ra[2], rb[2], ra0[2];
    int m = shape_segments(cfg.scat[j], r, d, sa, sb, ra, rb, ra0, s0);
    for (int i = 0; i < m; ++i) out[n++] = {sa[i], sb[i], j, ra[i], rb[i], ra0[i]};
  }
  for (int i = 1; i < n; ++i) {  // insertion sort by entry
    Segment key = out[i];
    int k = i - 1;
    while (k >= 0 && out[k].sa > key.sa) {
      out[k + 1] = out[k];
      --k;
    }
    out[k + 1] = key;
  }
  return n;
}

double sigma_scatt(const orc_scatterer& sc) {
  double s = 0.0;
  for (int k = 0; k < sc.nk; ++k) s += sc.ksig_b[k];
  return s;
}

// attenuation coefficients in 1/m: mu[1/cm] = n[1/A^3] sigma[barn]; absorption ~ 1/v
double mu_total(const orc_scatterer& sc, double speed) {
  return 100.0 * sc.n_per_A3 * (sigma_scatt(sc) + sc.sig_abs_b * 2200.0 / speed);
}
double mu_scatt(const orc_scatterer& sc) { return 100.0 * sc.n_per_A3 * sigma_scatt(sc); }

// unit vector at polar angle (cos c, sin s) and azimuth phi about unit vector d
Vec3 rotate_about(Vec3 d, double c, double s, double phi) {
  Vec3 a = (std::fabs(d.z) < 0.9) ? Vec3{0.0, 0.0, 1.0} : Vec3{1.0, 0.0, 0.0};
  Vec3 e1 = cross(a, d);
  e1 = scale(e1, 1.0 / std::sqrt(dot(e1, e1)));
  Vec3 e2 = cross(d, e1);
  double cp = std::cos(phi), sp = std::sin(phi);
  return add(scale(d, c), scale(add(scale(e1, cp), scale(e2, sp)), s));
}

// ---- state of one neutron packet ------------------------------------------------------
struct Neutron {
  Vec3 r;        // m
  Vec3 d;        // unit direction
  double speed;  // m/s
  double t;      // s
  double w;      // probability weight
};

// Synthetic source at the sample: Gaussian energy spread, uniform rectangular footprint,
// Gaussian divergence (it replaces the McStas beam simulation of section 3's first step).
bool make_beam(const orc_config& cfg, int64_t nid, Neutron* n) {
  double u[2];
  orc_uniforms(cfg.seed, cfg.sim_id, nid, -1, 0, u);
  double zE = std::sqrt(-2.0 * std::log(u[0])) * std::cos(2.0 * kPi * u[1]);
  double E = cfg.ei_mev * (1.0 + cfg.ei_rel_sigma * zE);
  orc_uniforms(cfg.seed, cfg.sim_id, nid, -1, 1, u);
  double x = (u[0] - 0.5) * cfg.width_m;
  double y = (u[1] - 0.5) * cfg.height_m;
  orc_uniforms(cfg.seed, cfg.sim_id, nid, -1, 2, u);
  double rr = std::sqrt(-2.0 * std::log(u[0]));
  double ax = cfg.div_sigma_rad * (rr * std::cos(2.0 * kPi * u[1]));
  double ay = cfg.div_sigma_rad * (rr * std::sin(2.0 * kPi * u[1]));
  if (!(E > 0.0)) return false;
  double tx = std::tan(ax), ty = std::tan(ay);
  double norm = std::sqrt(tx * tx + ty * ty + 1.0);
  n->d = {tx / norm, ty / norm, 1.0 / norm};
  n->speed = std::sqrt(E / kMeVPerV2);
  n->r = {x, y, -cfg.z0_m};
  n->t = (cfg.l1_m - cfg.z0_m) / (n->speed * n->d.z);
  n->w = 1.0;
  return true;
}

int64_t n_pixels(const orc_config& cfg) {
  if (cfg.det_kind == ORC_DET_SURFACE) return (int64_t)cfg.n_phi * cfg.n_y;
  if (cfg.det_kind == ORC_DET_TUBES) {
    int64_t packs = 0;
    for (int i = 0; i < cfg.n_rows; ++i) packs += cfg.packs[i];
    return packs * cfg.tubes_per_pack * cfg.pixels_per_tube;
  }
  return 0;
}

// larger root of the ray with the cylinder of radius R (the ray starts inside it)
bool exit_cylinder(double R, Vec3 r, Vec3 d, double* s) {
  double s1, s2;
  if (!cylinder_interval(R, r, d, &s1, &s2)) return false;
  if (!(s2 > 0.0) || s2 == kInf) return false;
  *s = s2;
  return true;
}

// Detector system ray tracing (section 2.4.3 "Ray tracing in a detector system").
int64_t detect(const orc_config& cfg, Vec3 r, Vec3 d, double speed, double t, double w,
               double u_det, int32_t* pixel, double* tof, double* w_det) {
  *pixel = -1;
  *tof = 0.0;
  *w_det = 0.0;
  if (cfg.det_kind == ORC_DET_SURFACE) {
    // ideal cylindrical surface of efficiency 1
    double s;
    if (!exit_cylinder(cfg.det_radius_m, r, d, &s)) return -1;
    double yh = r.y + s * d.y;
    double half = 0.5 * cfg.det_height_m;
    if (yh < -half || yh >= half) return -1;
    double xh = r.x + s * d.x, zh = r.z + s * d.z;
    double phi = std::atan2(xh, zh);
    int64_t ip = (int64_t)std::floor((phi + kPi) / (2.0 * kPi) * cfg.n_phi);
    ip = std::min<int64_t>(std::max<int64_t>(ip, 0), cfg.n_phi - 1);
    int64_t iy = (int64_t)std::floor((yh + half) / cfg.det_height_m * cfg.n_y);
    iy = std::min<int64_t>(std::max<int64_t>(iy, 0), cfg.n_y - 1);
    *pixel = (int32_t)(ip * cfg.n_y + iy);
    *tof = t + s / speed;
    *w_det = w;
  } else if (cfg.det_kind == ORC_DET_TUBES) {
    // coarse test: crossing of the circle through the tube centres
    double R = cfg.det_radius_m;
    double sR;
    if (!exit_cylinder(R, r, d, &sR)) return -1;
    Vec3 P = add(r, scale(d, sR));
    int row = -1, row_off = 0;
    for (int i = 0, off = 0; i < cfg.n_rows; off += cfg.packs[i], ++i) {
      if (std::fabs(P.y - cfg.row_y_m[i]) <= 0.5 * cfg.tube_len_m) {
        row = i;
        row_off = off;
        break;
      }
    }
    if (row < 0) return -1;
    // the pack and tube nearest to the crossing, then the exact chord of the candidates
    const int tpp = cfg.tubes_per_pack;
    double period = tpp * cfg.tube_pitch_m + cfg.pack_gap_m;
    double arc = (std::atan2(P.x, P.z) - cfg.phi0_rad) * R;
    double p = std::floor(arc / period);
    double within = arc - p * period;
    double k = std::floor(within / cfg.tube_pitch_m);
    if (k > tpp - 1) k = tpp - 1;
    int64_t g = (int64_t)p * tpp + (int64_t)k;
    int64_t n_tubes_row = (int64_t)cfg.packs[row] * tpp;
    double y_lo = cfg.row_y_m[row] - 0.5 * cfg.tube_len_m;
    double y_hi = cfg.row_y_m[row] + 0.5 * cfg.tube_len_m;
    int64_t best = -1;
    double best_in = kInf, best_out = 0.0;
    for (int64_t c = g - 1; c <= g + 1; ++c) {
      if (c < 0 || c >= n_tubes_row) continue;
      int64_t pc = c / tpp, tc = c % tpp;
      double phic = cfg.phi0_rad + (pc * period + (tc + 0.5) * cfg.tube_pitch_m) / R;
      double s1, s2;
      if (!tube_interval(R, std::sin(phic), std::cos(phic), cfg.tube_r_m, r, d, &s1, &s2))
        continue;
      double ys1, ys2;
      if (d.y == 0.0) {
        if (!(r.y >= y_lo && r.y <= y_hi)) continue;
        ys1 = -kInf;
        ys2 = kInf;
      } else {
        double a = (y_lo - r.y) / d.y, b = (y_hi - r.y) / d.y;
        ys1 = std::min(a, b);
        ys2 = std::max(a, b);
      }
      double s_in = std::max(std::max(s1, ys1), 0.0);
      double s_out = std::min(s2, ys2);
      if (!(s_out > s_in)) continue;
      if (s_in < best_in) {
        best = c;
        best_in = s_in;
        best_out = s_out;
      }
    }
    if (best < 0) return -1;
    // 3He gas absorption with a 1/v cross section; absorption depth from the truncated
    // exponential; weight multiplied by the absorption probability
    double L = best_out - best_in;
    double mu = 100.0 * cfg.he3_n_per_A3 * cfg.he3_sig_abs_b * 2200.0 / speed;
    double pabs = -std::expm1(-mu * L);
    double x = -std::log1p(-u_det * pabs) / mu;
    double s_abs = best_in + x;
    double y_abs = r.y + s_abs * d.y;
    double pix_len = cfg.tube_len_m / cfg.pixels_per_tube;
    int64_t j = (int64_t)std::floor((y_abs - y_lo) / pix_len);
    j = std::min<int64_t>(std::max<int64_t>(j, 0), cfg.pixels_per_tube - 1);
    int64_t pc = best / tpp, tc = best % tpp;
    *pixel = (int32_t)(((row_off + pc) * tpp + tc) * cfg.pixels_per_tube + j);
    *tof = t + s_abs / speed;
    *w_det = w * pabs;
  } else {
    return -1;
  }
  double dt = (cfg.tof_max_s - cfg.tof_min_s) / cfg.n_tof;
  double fb = std::floor((*tof - cfg.tof_min_s) / dt);
  if (!(fb >= 0.0 && fb < (double)cfg.n_tof)) return -2;
  return (int64_t)(*pixel) * cfg.n_tof + (int64_t)fb;
}

// ---- scattering kernels (supplement "Scattering kernels used in the examples") --------
struct KernelOut {
  double speed;
  Vec3 d;
  double factor;     // weight multiplier = s_value * rest
  double rest;       // the factor without the table value
  double s_value;    // table value (SQE) or 1
  int entry;         // table entry or -1
  double q, e, ki, kf;
  Vec3 qvec;
  int nroots = 0, mode = 0;
};

// incoherent elastic: isotropic, speed unchanged (d sigma/d Omega = sigma_inc/4pi N e^-2W,
// with the Debye-Waller factor taken as 1)
void kernel_iso(double speed, Vec3 d, const double u[4], KernelOut* o) {
  double ct = 2.0 * u[0] - 1.0;
  double phi = 2.0 * kPi * u[1];
  double st = 2.0 * std::sqrt(u[0] * (1.0 - u[0]));  // sqrt(1 - ct^2) without cancellation
  o->d = {st * std::cos(phi), st * std::sin(phi), ct};
  o->speed = speed;
  o->factor = 1.0;
  o->rest = 1.0;
  o->s_value = 1.0;
  o->entry = -1;
  double k = kKPerV * speed;
  o->ki = k;
  o->kf = k;
  o->e = 0.0;
  o->qvec = add(scale(d, k), scale(o->d, -k));
  o->q = std::sqrt(dot(o->qvec, o->qvec));
}

// tabulated isotropic S(Q,E): d2 sigma/dOmega dEf = sigma/4pi (kf/ki) N S(Q,E).
// E uniform on [e_min, min(e_max, Ei)], Q uniform on [|ki-kf|, min(ki+kf, q_max)], azimuth
// uniform; the weight factor is the cross section over the sampling density,
// S Q dE dQ / (2 ki^2).  Nearest-bin lookup (histogram form of S(Q,E)).
bool kernel_sqe(const orc_config& cfg, double speed, Vec3 d, const double u[4], KernelOut* o) {
  double Ei = kMeVPerV2 * speed * speed;
  double ki = kKPerV * speed;
  double e_lo = cfg.e_min, e_hi = std::min(cfg.e_max, Ei);
  if (!(e_hi > e_lo)) return false;
  double dE = e_hi - e_lo;
  double E = e_lo + u[0] * dE;
  // Ef = Ei - E; when the range ends at Ei it is the sampled offset from that end, which
  // keeps slow final neutrons accurate
  double Ef = (e_hi == Ei) ? (1.0 - u[0]) * dE : Ei - E;
  if (!(Ef > 0.0)) return false;
  double speed_f = std::sqrt(Ef / kMeVPerV2);
  double kf = kKPerV * speed_f;
  double q_lo = std::fabs(ki - kf);
  double q_hi = std::min(ki + kf, cfg.q_max);
  if (!(q_hi > q_lo)) return false;
  double dQ = q_hi - q_lo;
  if (ORC_CONDITION) {
    g_kappa += (ki + kf) / dQ + 2.0 * g_kappa_v * (1.0 + (ki + kf) / dQ);
    g_kappa_v = 1.0 + 0.5 * ((Ei + std::fabs(E) + std::fabs(e_lo)) / Ef + 2.0 * (Ei / Ef) * g_kappa_v);
  }
  double Q = q_lo + u[1] * dQ;
  // scattering angle from Q^2 = ki^2 + kf^2 - 2 ki kf cos(2theta), written through
  // 1 - cos = (Q - q_lo)(Q + q_lo) / (2 ki kf) and 1 + cos = (ki + kf - Q)(ki + kf + Q) /
  // (2 ki kf), whose small factors are the sampled offsets from the ends of the Q range
  double den = 2.0 * ki * kf;
  double one_m = (u[1] * dQ) * (Q + q_lo) / den;
  double top = (q_hi == ki + kf) ? (1.0 - u[1]) * dQ : (ki + kf) - Q;
  double one_p = top * (ki + kf + Q) / den;
  double c2t = (one_m <= one_p) ? 1.0 - one_m : one_p - 1.0;
  c2t = std::min(1.0, std::max(-1.0, c2t));
  double s2t = std::sqrt(std::max(0.0, one_m * one_p));
  double phi = 2.0 * kPi * u[2];
  double bq = cfg.q_max / cfg.nq, be = (cfg.e_max - cfg.e_min) / cfg.ne;
  double fq = std::floor(Q / bq), fe = std::floor((E - cfg.e_min) / be);
  if (!(fq >= 0.0 && fq < cfg.nq && fe >= 0.0 && fe < cfg.ne)) return false;
  int entry = (int)fq * cfg.ne + (int)fe;
  double S = (double)cfg.sqe[entry];
  o->d = rotate_about(d, c2t, s2t, phi);
  o->speed = speed_f;
  o->s_value = S;
  o->entry = entry;
  o->rest = Q * dE * dQ / (2.0 * ki * ki);
  o->factor = S * o->rest;
  o->q = Q;
  o->e = E;
  o->ki = ki;
  o->kf = kf;
  o->qvec = add(scale(d, ki), scale(o->d, -kf));
  return true;
}

// ---- single-crystal coherent one-phonon kernel (Born-von Karman fcc) -------------------
// Supplement S4 gives the coherent one-phonon cross section of a powder and the cross
// section of one mode at Q.  For a single crystal of a Bravais lattice the sum over q and
// tau with delta(Q - q - tau) picks q = Q (periodic dispersion), leaving per atom
//   d2sigma/dOmega dEf = sigma/4pi (kf/ki) e^{-2W} sum_{b,s} hbar^2 (Q.e_b)^2/(2M hw_b)
//                        N_s(hw_b) delta(Ei - Ef - s hw_b(Q)),
// N_+ = n + 1 (creation), N_- = n (annihilation), n the Bose factor.  Sampling: direction
// uniform, mode (b, s) uniform over 6, a root of g(Ef) = Ei - Ef - s hw_b(Q(Ef)) uniform
// over the roots bracketed on 32 equal sub-intervals; weight 6 n_roots (kf/ki) e^{-2W}
// R_b N_s / |g'(Ef)|.
const double kMeVPerJ = 1.0 / (kElemCharge * 1e-3);

struct BvkModel {
  double coef;      // phi / M (1/s^2)
  double a;         // lattice constant (A)
  double hb2m;      // hbar^2 / (2 M) in meV A^2
  double kT;        // meV
  double msd;       // <u^2> (A^2)
  double w_max;     // upper bound of hbar omega (meV): trace bound sqrt(24 phi/M)
};

BvkModel bvk_model(const orc_config& cfg) {
  BvkModel m;
  const double M = cfg.bvk_mass_u * kAtomicMass;
  m.coef = cfg.bvk_phi_Nm / M;
  m.a = cfg.bvk_a_A;
  m.hb2m = kHbar * kHbar / (2.0 * M) * 1e20 * kMeVPerJ;
  m.kT = kBoltzmann * cfg.temperature_K * kMeVPerJ;
  m.msd = cfg.bvk_msd_A2;
  m.w_max = kHbar * std::sqrt(24.0 * m.coef) * kMeVPerJ;
  return m;
}

// the six nearest-neighbour bond directions of fcc (the other six are their negatives)
const double kBond[6][3] = {{1, 1, 0}, {1, -1, 0}, {1, 0, 1}, {1, 0, -1}, {0, 1, 1}, {0, 1, -1}};

// dynamical matrix D(q) = (phi/M) sum over the 12 neighbours of (1 - cos q.delta) dd^T,
// delta = (a/2) n, d = n/sqrt(2); stored xx, yy, zz, xy, xz, yz (1/s^2).  1 - cos x is
// evaluated as 2 sin^2(x/2), which keeps its relative accuracy near the zone centres.
void bvk_dynmat(const BvkModel& m, const double q[3], double D[6]) {
  for (int i = 0; i < 6; ++i) D[i] = 0.0;
  for (int k = 0; k < 6; ++k) {
    const double* n = kBond[k];
    const double qd = 0.5 * m.a * (q[0] * n[0] + q[1] * n[1] + q[2] * n[2]);
    const double sh = std::sin(0.5 * qd);
    const double c = 2.0 * m.coef * (2.0 * sh * sh) * 0.5;  // two neighbours, dd^T = nn^T/2
    D[0] += c * n[0] * n[0];
    D[1] += c * n[1] * n[1];
    D[2] += c * n[2] * n[2];
    D[3] += c * n[0] * n[1];
    D[4] += c * n[0] * n[2];
    D[5] += c * n[1] * n[2];
  }
}

// D v for the packed symmetric matrix
Vec3 sym_mul(const double D[6], Vec3 v) {
  return {D[0] * v.x + D[3] * v.y + D[4] * v.z, D[3] * v.x + D[1] * v.y + D[5] * v.z,
          D[4] * v.x + D[5] * v.y + D[2] * v.z};
}

// Eigenvalues (ascending) and unit eigenvectors of a symmetric 3x3 matrix.
// The trigonometric form of Cardano's solution gives estimates; its accuracy degrades where
// two eigenvalues nearly coincide (the cubic's discriminant is formed with cancellation), so
// it is used only to tell which eigenvalue stands apart from the other two.  That one's
// eigenvector is the largest cross product of two rows of D - lambda I and its eigenvalue
// the Rayleigh quotient; the other two come from the 2x2 matrix D restricted to the plane
// orthogonal to it, solved in closed form.  Eigenvalues are then accurate to a few ulps of
// the largest, and eigenvectors to that over the distance to the nearest other eigenvalue.
void eig_sym3(const double D[6], double lam[3], double vec[9]) {
  const double a00 = D[0], a11 = D[1], a22 = D[2], a01 = D[3], a02 = D[4], a12 = D[5];
  const double p1 = a01 * a01 + a02 * a02 + a12 * a12;
  if (p1 == 0.0) {
    int idx[3] = {0, 1, 2};
    const double d[3] = {a00, a11, a22};
    std::stable_sort(idx, idx + 3, [&](int i, int j) { return d[i] < d[j]; });
    for (int b = 0; b < 3; ++b) {
      lam[b] = d[idx[b]];
      for (int i = 0; i < 3; ++i) vec[i * 3 + b] = (i == idx[b]) ? 1.0 : 0.0;
    }
    return;
  }
  // Cardano estimates
  const double q = (a00 + a11 + a22) / 3.0;
  const double p2 = (a00 - q) * (a00 - q) + (a11 - q) * (a11 - q) + (a22 - q) * (a22 - q) +
                    2.0 * p1;
  const double p = std::sqrt(p2 / 6.0);
  const double b00 = (a00 - q) / p, b11 = (a11 - q) / p, b22 = (a22 - q) / p;
  const double b01 = a01 / p, b02 = a02 / p, b12 = a12 / p;
  double r = 0.5 * (b00 * (b11 * b22 - b12 * b12) - b01 * (b01 * b22 - b12 * b02) +
                    b02 * (b01 * b12 - b11 * b02));
  r = std::min(1.0, std::max(-1.0, r));
  const double phi = std::acos(r) / 3.0;
  const double l2 = q + 2.0 * p * std::cos(phi);
  const double l0 = q + 2.0 * p * std::cos(phi + 2.0 * kPi / 3.0);
  const double l1 = 3.0 * q - l0 - l2;
  // the eigenvalue farther from the other two
  const double li = (l1 - l0 >= l2 - l1) ? l0 : l2;
  const Vec3 r0 = {a00 - li, a01, a02}, r1 = {a01, a11 - li, a12}, r2 = {a02, a12, a22 - li};
  const Vec3 c[3] = {cross(r0, r1), cross(r0, r2), cross(r1, r2)};
  int best = 0;
  double nb = dot(c[0], c[0]);
  for (int i = 1; i < 3; ++i) {
    const double ni = dot(c[i], c[i]);
    if (ni > nb) {
      nb = ni;
      best = i;
    }
  }
  const Vec3 e = nb > 0.0 ? scale(c[best], 1.0 / std::sqrt(nb)) : Vec3{1.0, 0.0, 0.0};
  const double lam_e = dot(e, sym_mul(D, e));
  // orthonormal basis (u, w) of the plane orthogonal to e: u = e x (the axis least along e)
  const double ax = std::fabs(e.x), ay = std::fabs(e.y), az = std::fabs(e.z);
  const Vec3 axis = (ax <= ay && ax <= az) ? Vec3{1, 0, 0} : (ay <= az ? Vec3{0, 1, 0} : Vec3{0, 0, 1});
  Vec3 u = cross(e, axis);
  u = scale(u, 1.0 / std::sqrt(dot(u, u)));
  const Vec3 w = cross(e, u);
  const Vec3 Du = sym_mul(D, u), Dw = sym_mul(D, w);
  const double A = dot(u, Du), B = dot(u, Dw), C = dot(w, Dw);
  const double mid = 0.5 * (A + C), h = 0.5 * (A - C);
  const double rr = std::hypot(h, B);
  const double mu_hi = mid + rr, mu_lo = mid - rr;
  // eigenvector of mu_hi in the (u, w) plane: (rr + h, B) or (B, rr - h), the longer one
  double cu, cw;
  if (h >= 0.0) {
    cu = rr + h;
    cw = B;
  } else {
    cu = B;
    cw = rr - h;
  }
  const double cn = std::hypot(cu, cw);
  if (cn > 0.0) {
    cu /= cn;
    cw /= cn;
  } else {
    cu = 1.0;
    cw = 0.0;
  }
  const Vec3 v_hi = add(scale(u, cu), scale(w, cw));
  const Vec3 v_lo = add(scale(u, -cw), scale(w, cu));
  // ascending order
  double L[3] = {lam_e, mu_lo, mu_hi};
  Vec3 V[3] = {e, v_lo, v_hi};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j + 1 < 3 - i; ++j)
      if (L[j] > L[j + 1]) {
        std::swap(L[j], L[j + 1]);
        std::swap(V[j], V[j + 1]);
      }
  for (int b = 0; b < 3; ++b) {
    lam[b] = L[b];
    vec[0 * 3 + b] = V[b].x;
    vec[1 * 3 + b] = V[b].y;
    vec[2 * 3 + b] = V[b].z;
  }
}

double hbar_omega(double lam) { return kHbar * std::sqrt(std::max(lam, 0.0)) * kMeVPerJ; }

// lab vector -> crystal frame: body = R^T lab for a rotation rot_y about +y; the crystal
// axes are x_c = z_body ([100] along the beam at zero rotation), y_c = x_body, z_c = y_body
Vec3 to_crystal(Vec3 v, double c, double s) {
  const Vec3 b = {c * v.x - s * v.z, v.y, s * v.x + c * v.z};
  return {b.z, b.x, b.y};
}

struct BvkEval {
  double g;       // Ei - Ef - s hw_b
  double hw;      // hbar omega_b (meV)
  Vec3 Qc;        // Q in the crystal frame (1/A)
  double lam[3], vec[9];
};

BvkEval bvk_g(const BvkModel& m, double Ei, double ki, Vec3 di, Vec3 df, double Ef, int b,
              int s, double c, double sn) {
  BvkEval r;
  const double kf = kKPerV * std::sqrt(Ef / kMeVPerV2);
  const Vec3 Q = add(scale(di, ki), scale(df, -kf));
  r.Qc = to_crystal(Q, c, sn);
  double D[6];
  const double q[3] = {r.Qc.x, r.Qc.y, r.Qc.z};
  bvk_dynmat(m, q, D);
  eig_sym3(D, r.lam, r.vec);
  r.hw = hbar_omega(r.lam[b]);
  r.g = Ei - Ef - s * r.hw;
  return r;
}

// The root of one event: outgoing direction and mode (b, s) from u, the roots of
// g(Ef) = Ei - Ef - s hw_b(Q(Ef)) bracketed on 32 sub-intervals of the allowed Ef range, one
// picked uniformly and refined by 50 bisections.
struct BvkRoot {
  bool ok = false;
  int nroots = 0, mode = 0, b = 0, s = 1;
  double Ei = 0.0, ki = 0.0, Ef = 0.0;
  Vec3 df;
};

BvkRoot bvk_root(const BvkModel& m, double c, double sn, double speed, Vec3 d,
                 const double u[4]) {
  BvkRoot R;
  // outgoing direction, uniform
  const double ct = 2.0 * u[0] - 1.0;
  const double st = 2.0 * std::sqrt(u[0] * (1.0 - u[0]));
  const double ph = 2.0 * kPi * u[1];
  R.df = {st * std::cos(ph), st * std::sin(ph), ct};
  // mode: branch b, creation (s = +1) or annihilation (s = -1)
  int mode = (int)std::floor(6.0 * u[2]);
  mode = std::min(std::max(mode, 0), 5);
  R.mode = mode;
  R.b = mode % 3;
  R.s = mode < 3 ? 1 : -1;
  const int b = R.b, s = R.s;
  const Vec3 df = R.df;
  const double Ei = kMeVPerV2 * speed * speed;
  const double ki = kKPerV * speed;
  R.Ei = Ei;
  R.ki = ki;
  const double lo = s > 0 ? 0.0 : Ei;
  const double hi = s > 0 ? Ei : Ei + m.w_max;
  const int M = 32;
  const double step = (hi - lo) / M;
  double gk[M + 1];
  for (int k = 0; k <= M; ++k) gk[k] = bvk_g(m, Ei, ki, d, df, lo + k * step, b, s, c, sn).g;
  int nroots = 0;
  for (int k = 0; k < M; ++k)
    if ((gk[k] > 0.0) != (gk[k + 1] > 0.0)) ++nroots;
  R.nroots = nroots;
  if (nroots == 0) return R;
  int pick = (int)std::floor(u[3] * nroots);
  pick = std::min(std::max(pick, 0), nroots - 1);
  int kb = -1;
  for (int k = 0, seen = 0; k < M; ++k) {
    if ((gk[k] > 0.0) != (gk[k + 1] > 0.0)) {
      if (seen == pick) {
        kb = k;
        break;
      }
      ++seen;
    }
  }
  // bisection on the bracket
  double ea = lo + kb * step, eb = lo + (kb + 1) * step;
  const bool ga_pos = gk[kb] > 0.0;
  for (int it = 0; it < 50; ++it) {
    const double mid = 0.5 * (ea + eb);
    if ((bvk_g(m, Ei, ki, d, df, mid, b, s, c, sn).g > 0.0) == ga_pos)
      ea = mid;
    else
      eb = mid;
  }
  R.Ef = 0.5 * (ea + eb);
  R.ok = R.Ef > 0.0;
  return R;
}

// The weight factor of an event at final energy Ef (at the root: the kernel's factor)
//   6 n_roots (kf/ki) e^{-2W} R_b N_s / |g'(Ef)|
// with g' from the Hellmann-Feynman derivative of the eigenvalue along Q(Ef).
struct BvkWeight {
  double F = 0.0, kf = 0.0, gp = 0.0, dhw = 0.0, qe = 0.0, Q2 = 0.0, grad = 0.0;
  BvkEval r;
  Vec3 e;
};

BvkWeight bvk_weight(const BvkModel& m, double c, double sn, const BvkRoot& R, Vec3 d,
                     double Ef) {
  BvkWeight W;
  const int b = R.b, s = R.s;
  const BvkEval r = bvk_g(m, R.Ei, R.ki, d, R.df, Ef, b, s, c, sn);
  W.r = r;
  const Vec3 e = {r.vec[0 * 3 + b], r.vec[1 * 3 + b], r.vec[2 * 3 + b]};
  W.e = e;
  // d hw / d Ef through Q(Ef) (Hellmann-Feynman: d lambda = e^T dD e)
  const double kf = kKPerV * std::sqrt(Ef / kMeVPerV2);
  const double dkf = kf / (2.0 * Ef);
  const Vec3 dQ = scale(to_crystal(R.df, c, sn), -dkf);  // dQc/dEf
  double dlam = 0.0;
  Vec3 grad = {0.0, 0.0, 0.0};  // d lambda / dQc
  for (int k = 0; k < 6; ++k) {
    const double* n = kBond[k];
    const double qd = 0.5 * m.a * (r.Qc.x * n[0] + r.Qc.y * n[1] + r.Qc.z * n[2]);
    const double ed = (e.x * n[0] + e.y * n[1] + e.z * n[2]);
    const double dqd = 0.5 * m.a * (dQ.x * n[0] + dQ.y * n[1] + dQ.z * n[2]);
    dlam += 2.0 * m.coef * std::sin(qd) * dqd * ed * ed * 0.5;
    const double gk = 2.0 * m.coef * std::sin(qd) * 0.5 * m.a * ed * ed * 0.5;
    grad = add(grad, Vec3{gk * n[0], gk * n[1], gk * n[2]});
  }
  W.grad = std::sqrt(dot(grad, grad));
  const double dhw = kHbar * kMeVPerJ * dlam / (2.0 * std::sqrt(r.lam[b]));
  const double gp = -1.0 - s * dhw;
  const double nB = 1.0 / std::expm1(r.hw / m.kT);
  const double Ns = s > 0 ? nB + 1.0 : nB;
  const double qe = r.Qc.x * e.x + r.Qc.y * e.y + r.Qc.z * e.z;
  const double Q2 = dot(r.Qc, r.Qc);
  const double dw = std::exp(-Q2 * m.msd / 3.0);
  const double Rb = m.hb2m * qe * qe / r.hw;
  W.F = 6.0 * R.nroots * (kf / R.ki) * dw * Rb * Ns / std::fabs(gp);
  W.kf = kf;
  W.gp = gp;
  W.dhw = dhw;
  W.qe = qe;
  W.Q2 = Q2;
  return W;
}

bool kernel_bvk(const orc_config& cfg, double rot_y, double speed, Vec3 d, const double u[4],
                KernelOut* o) {
  const BvkModel m = bvk_model(cfg);
  const double c = std::cos(rot_y), sn = std::sin(rot_y);
  const BvkRoot R = bvk_root(m, c, sn, speed, d, u);
  o->nroots = R.nroots;
  o->mode = R.mode;
  if (R.nroots == 0 || !R.ok) return false;
  const double Ef = R.Ef;
  const BvkWeight W = bvk_weight(m, c, sn, R, d, Ef);
  if (!(W.r.hw >= 1e-3)) return false;
  const double Ei = R.Ei, ki = R.ki, kf = W.kf;
  o->rest = W.F;
  o->factor = o->rest;
  o->s_value = 1.0;
  o->entry = -1;
  o->d = R.df;
  o->speed = std::sqrt(Ef / kMeVPerV2);
  o->q = std::sqrt(W.Q2);
  o->e = Ei - Ef;
  o->ki = ki;
  o->kf = kf;
  o->qvec = add(scale(d, ki), scale(R.df, -kf));

  if (!ORC_CONDITION) return true;
  // Condition estimate (units of the FP64 epsilon): how far rounding at the scale of the
  // epsilon can move this factor.  Sources: the computed eigenvalue (relative error kl:
  // a few ulps of the largest eigenvalue, plus Q's rounding through the dispersion
  // gradient), g rounded near the root, the incoming speed's own error, and the eigenvector
  // (error over the distance to the nearest other eigenvalue).  Their effect on the factor
  // is measured by central differences: against a common scale of the eigenvalues (the force
  // constant), against the incoming speed (both re-solving the root), and against Ef itself.
  const double lam_b = W.r.lam[R.b];
  const double lmax = W.r.lam[2];
  const double gap = std::min(R.b > 0 ? lam_b - W.r.lam[R.b - 1] : 1e300,
                              R.b < 2 ? W.r.lam[R.b + 1] - lam_b : 1e300);
  const double kl = 4.0 * lmax / lam_b + W.grad * (ki + kf) / lam_b;
  const double ag = std::fabs(W.gp);
  const double qq = std::sqrt(W.Q2) / std::max(std::fabs(W.qe), 1e-300);
  const double eig = gap > 0.0 ? lmax / gap : 1e16;
  const double h = 1e-7;
  auto factor_at = [&](const BvkModel& mm, double sp, double* ef) -> double {
    const BvkRoot Rp = bvk_root(mm, c, sn, sp, d, u);
    if (!Rp.ok || Rp.nroots != R.nroots) return -1.0;
    *ef = Rp.Ef;
    return bvk_weight(mm, c, sn, Rp, d, Rp.Ef).F;
  };
  auto dlog = [&](double fp, double fm, double ref) -> double {
    if (!(fp > 0.0) || !(fm > 0.0)) return 1e16;
    (void)ref;
    return std::fabs(std::log(fp / fm)) / (2.0 * h);
  };
  BvkModel mp = m, mm = m;
  mp.coef = m.coef * (1.0 + h);
  mm.coef = m.coef * (1.0 - h);
  double ef_cp = Ef, ef_cm = Ef, ef_vp = Ef, ef_vm = Ef;
  const double s_c = dlog(factor_at(mp, speed, &ef_cp), factor_at(mm, speed, &ef_cm), W.F);
  const double s_v = dlog(factor_at(m, speed * (1.0 + h), &ef_vp),
                          factor_at(m, speed * (1.0 - h), &ef_vm), W.F);
  const double s_ce = std::fabs(ef_cp - ef_cm) / (2.0 * h * Ef);
  const double s_ve = std::fabs(ef_vp - ef_vm) / (2.0 * h * Ef);
  const double s_e = dlog(bvk_weight(m, c, sn, R, d, Ef * (1.0 + h)).F,
                          bvk_weight(m, c, sn, R, d, Ef * (1.0 - h)).F, W.F);
  const double root = (Ei + Ef) / (ag * Ef);  // relative error of the root from g's rounding
  const double kv_in = g_kappa_v;
  g_kappa += 10.0 + 2.0 * qq * (1.0 + eig) + (1.0 + std::fabs(W.dhw) * (1.0 + eig)) / ag +
             s_c * kl + s_v * kv_in + s_e * root;
  g_kappa_v = 1.0 + 0.5 * (s_ce * kl + root + s_ve * kv_in);
  return true;
}

// ---- incoherent scattering from a phonon density of states (supplement S4) ------------
// The incoherent scattering function of a harmonic cubic crystal as a phonon expansion:
//   S(Q,E) = e^{-2W} [ delta(E) + sum_{n=1}^{N} (2W)^n / n! A_n(E) ],
//   A_1(E) = Z(|E|) / (|E| gamma_0) [n(|E|) + 1 if E > 0 (phonon created), n(|E|) if E < 0],
//   A_n = A_1 * A_{n-1} (convolution),  gamma_0 = int coth(E / 2kT) Z(E) / E dE,
//   2W = hbar^2 Q^2 gamma_0 / (2M),  n the Bose factor,  E = Ei - Ef.
// Its n = 0 term is the incoherent elastic kernel with the Debye-Waller factor, its n = 1
// term the incoherent inelastic single-phonon form (hbar^2 Q^2/2M e^{-2W} Z(E)/E
// {coth(E/2kT) +- 1}/2), its n >= 2 terms the multi-phonon form S_n(Q) A_n(E).  The density
// of states is a histogram of mode energies: dos_z[j-1] holds the modes of the bin at
// E_j = j de, normalised here to weights w_j summing to 1, so A_1 is a set of masses on the
// grid E = i de and every A_n is an exact discrete convolution on that grid.  A sampled
// energy is spread uniformly over its bin (E = i de + (u - 1/2) de).
// Sampling: channel c = elastic / one-phonon / multi-phonon with probabilities phonon_p; the
// elastic channel draws an isotropic direction (weight e^{-2W} / p_0); the others draw the
// grid point from A_1 (one-phonon) or from B = (A_2 + ... + A_N) / (N - 1) (multi-phonon),
// then Q uniform over [|ki - kf|, ki + kf] and the azimuth uniform, weight
//   (term of S at (Q, E)) / (sampling mass of E) * Q dQ / (2 ki^2) / p_c
// (the same change of variables as the tabulated S(Q,E) kernel, with the mass of the energy
// bin in place of dE / (e_max - e_min)).
struct PhononModel {
  const double* z = nullptr;
  int J = 0, N = 0, M = 0;
  double de = 0.0, kT = 0.0, mass = 0.0;
  double gamma0 = 0.0, cw = 0.0;
  double p[3] = {0.0, 0.0, 0.0};
  std::vector<double> a1;             // A_1 masses on i = -J..J (index i + J)
  std::vector<double> cdf1;           // cumulative sums of a1
  std::vector<std::vector<double>> an;  // A_n masses on i = -N J..N J (index i + N J), n = 1..N
  std::vector<double> b, cdfb;        // B and its cumulative sums on the same grid
};

double bose(double e, double kT) { return 1.0 / std::expm1(e / kT); }

const PhononModel& phonon_model(const orc_config& cfg) {
  thread_local PhononModel m;
  const double kT = kBoltzmann * cfg.temperature_K * kMeVPerJ;
  if (m.z == cfg.dos_z && m.J == cfg.dos_n && m.de == cfg.dos_de && m.kT == kT &&
      m.mass == cfg.phonon_mass_u && m.N == cfg.phonon_nmax && m.p[0] == cfg.phonon_p[0] &&
      m.p[1] == cfg.phonon_p[1] && m.p[2] == cfg.phonon_p[2])
    return m;
  m = PhononModel();
  m.z = cfg.dos_z;
  m.J = cfg.dos_n;
  m.N = cfg.phonon_nmax;
  m.de = cfg.dos_de;
  m.kT = kT;
  m.mass = cfg.phonon_mass_u;
  for (int c = 0; c < 3; ++c) m.p[c] = cfg.phonon_p[c];
  const int J = m.J, N = m.N;
  m.M = 2 * N * J + 1;
  // mode weights, gamma_0 and the Debye-Waller coefficient
  double zsum = 0.0;
  for (int j = 1; j <= J; ++j) zsum += cfg.dos_z[j - 1];
  m.gamma0 = 0.0;
  for (int j = 1; j <= J; ++j) {
    const double e = j * m.de;
    m.gamma0 += (cfg.dos_z[j - 1] / zsum) / (e * std::tanh(e / (2.0 * kT)));
  }
  // hbar^2 / 2M in meV A^2
  const double hb2m = kHbar * kHbar / (2.0 * m.mass * kAtomicMass) * 1e20 * kMeVPerJ;
  m.cw = hb2m * m.gamma0;
  // A_1 masses
  m.a1.assign(2 * J + 1, 0.0);
  for (int j = 1; j <= J; ++j) {
    const double e = j * m.de, w = cfg.dos_z[j - 1] / zsum;
    const double nb = bose(e, kT);
    m.a1[J + j] = w * (nb + 1.0) / (e * m.gamma0);
    m.a1[J - j] = w * nb / (e * m.gamma0);
  }
  m.cdf1.assign(2 * J + 1, 0.0);
  double acc = 0.0;
  for (int i = 0; i < 2 * J + 1; ++i) m.cdf1[i] = (acc += m.a1[i]);
  // A_n = A_1 * A_{n-1} on the grid i = -N J..N J
  m.an.assign(N + 1, std::vector<double>(m.M, 0.0));
  for (int i = -J; i <= J; ++i) m.an[1][i + N * J] = m.a1[i + J];
  for (int n = 2; n <= N; ++n) {
    for (int i = -n * J; i <= n * J; ++i) {
      double v = 0.0;
      for (int k = -J; k <= J; ++k) {
        const int r = i - k;
        if (r < -(n - 1) * J || r > (n - 1) * J) continue;
        v += m.a1[k + J] * m.an[n - 1][r + N * J];
      }
      m.an[n][i + N * J] = v;
    }
  }
  m.b.assign(m.M, 0.0);
  m.cdfb.assign(m.M, 0.0);
  acc = 0.0;
  for (int i = 0; i < m.M; ++i) {
    for (int n = 2; n <= N; ++n) m.b[i] += m.an[n][i] / (N - 1);
    m.cdfb[i] = (acc += m.b[i]);
  }
  return m;
}

// index of the first cumulative sum above u * total (a draw from the masses)
int draw_index(const std::vector<double>& cdf, double u) {
  const double x = u * cdf.back();
  int i = (int)(std::upper_bound(cdf.begin(), cdf.end(), x) - cdf.begin());
  return std::min(i, (int)cdf.size() - 1);
}

bool kernel_phonon(const orc_config& cfg, double speed, Vec3 d, const double u[4], KernelOut* o) {
  const PhononModel& m = phonon_model(cfg);
  const double Ei = kMeVPerV2 * speed * speed;
  const double ki = kKPerV * speed;
  o->entry = -1;
  o->s_value = 1.0;
  o->ki = ki;
  // channel, and the rescaled uniform of the energy draw
  int ch = 2;
  double lo = m.p[0] + m.p[1];
  if (u[0] < m.p[0]) {
    ch = 0;
    lo = 0.0;
  } else if (u[0] < m.p[0] + m.p[1]) {
    ch = 1;
    lo = m.p[0];
  }
  o->mode = ch;
  if (ch == 0) {
    // elastic: isotropic, weight e^{-2W}
    const double ct = 2.0 * u[2] - 1.0;
    const double st = 2.0 * std::sqrt(u[2] * (1.0 - u[2]));
    const double phi = 2.0 * kPi * u[3];
    o->d = {st * std::cos(phi), st * std::sin(phi), ct};
    o->speed = speed;
    o->kf = ki;
    o->e = 0.0;
    o->qvec = add(scale(d, ki), scale(o->d, -ki));
    o->q = std::sqrt(dot(o->qvec, o->qvec));
    o->rest = std::exp(-m.cw * o->q * o->q) / m.p[0];
    o->factor = o->rest;
    return true;
  }
  const double ue = (u[0] - lo) / m.p[ch];
  int i;
  double mass;
  if (ch == 1) {
    const int k = draw_index(m.cdf1, ue);
    i = k - m.J;
    mass = m.a1[k];
  } else {
    const int k = draw_index(m.cdfb, ue);
    i = k - m.N * m.J;
    mass = m.b[k];
  }
  const double E = (i + (u[1] - 0.5)) * m.de;
  const double Ef = Ei - E;
  if (!(Ef > 0.0)) return false;
  const double speed_f = std::sqrt(Ef / kMeVPerV2);
  const double kf = kKPerV * speed_f;
  const double q_lo = std::fabs(ki - kf), q_hi = ki + kf;
  const double dQ = q_hi - q_lo;
  // condition estimate: the width of the Q range and the final speed, as for S(Q,E)
  if (ORC_CONDITION) {
    g_kappa += (ki + kf) / dQ + 2.0 * g_kappa_v * (1.0 + (ki + kf) / dQ);
    g_kappa_v = 1.0 + 0.5 * ((Ei + std::fabs(E)) / Ef + 2.0 * (Ei / Ef) * g_kappa_v);
  }
  const double Q = q_lo + u[2] * dQ;
  // scattering angle from 1 -/+ cos as products of the offsets from the ends of the range
  const double den = 2.0 * ki * kf;
  const double one_m = (u[2] * dQ) * (Q + q_lo) / den;
  const double one_p = ((1.0 - u[2]) * dQ) * (ki + kf + Q) / den;
  double c2t = (one_m <= one_p) ? 1.0 - one_m : one_p - 1.0;
  c2t = std::min(1.0, std::max(-1.0, c2t));
  const double s2t = std::sqrt(std::max(0.0, one_m * one_p));
  const double phi = 2.0 * kPi * u[3];
  // the term of S at (Q, E) over the sampling mass of E
  const double w2 = m.cw * Q * Q;
  double ratio;
  if (ch == 1) {
    ratio = w2 * std::exp(-w2);  // 2W e^{-2W} A_1 / A_1
  } else {
    const int g = i + m.N * m.J;
    double sum = 0.0, pw = w2;
    double fact = 1.0;
    for (int n = 2; n <= m.N; ++n) {
      pw *= w2;
      fact *= n;
      sum += pw / fact * m.an[n][g];
    }
    ratio = std::exp(-w2) * sum / mass;
  }
  o->d = rotate_about(d, c2t, s2t, phi);
  o->speed = speed_f;
  o->kf = kf;
  o->q = Q;
  o->e = E;
  o->rest = ratio * Q * dQ / (2.0 * ki * ki) / m.p[ch];
  o->factor = o->rest;
  o->qvec = add(scale(d, ki), scale(o->d, -kf));
  return true;
}

// ---- coherent elastic scattering from a powder (supplement S4) ------------------------
// The cross section for scattering into the Debye-Scherrer cone of reflection tau is, per
// atom, sigma_tau = lambda^3 / (4 sin theta_B) m |F_tau|^2 / (v0 n_cell) (the paper's form,
// with theta_B half the scattering angle and lambda = 2 pi / ki), for every reflection with
// lambda < 2 d_tau.  The reflections are taken in order of decreasing d; one is picked with
// probability sigma_tau / sum sigma, the outgoing direction lies on its cone (sin theta_B =
// lambda / 2d, azimuth uniform) with the speed unchanged, and the weight is
// sum sigma / sigma_kernel: the Bragg cross section at this wavelength over the kernel's
// nominal cross section, which sets its share of the attenuation and of the kernel choice.
struct BraggList {
  const double* d = nullptr;
  const double* w = nullptr;
  int n = -1;
  std::vector<int> order;  // by decreasing d, ties in input order
};

const BraggList& bragg_list(const orc_config& cfg) {
  thread_local BraggList L;
  if (L.d == cfg.refl_d && L.w == cfg.refl_w && L.n == cfg.n_refl) return L;
  L = BraggList();
  L.d = cfg.refl_d;
  L.w = cfg.refl_w;
  L.n = cfg.n_refl;
  L.order.resize(cfg.n_refl);
  for (int i = 0; i < cfg.n_refl; ++i) L.order[i] = i;
  std::stable_sort(L.order.begin(), L.order.end(),
                   [&](int a, int b) { return cfg.refl_d[a] > cfg.refl_d[b]; });
  return L;
}

bool kernel_bragg(const orc_config& cfg, double sig_kernel, double speed, Vec3 d,
                  const double u[4], KernelOut* o) {
  const BraggList& L = bragg_list(cfg);
  const double ki = kKPerV * speed;
  const double lam = 2.0 * kPi / ki;
  double total = 0.0;
  int allowed = 0;
  for (int r = 0; r < L.n; ++r) {
    const int t = L.order[r];
    if (!(lam < 2.0 * cfg.refl_d[t])) break;
    const double s = lam / (2.0 * cfg.refl_d[t]);
    total += lam * lam * lam * cfg.refl_w[t] / (4.0 * s);
    ++allowed;
  }
  if (allowed == 0 || !(total > 0.0)) return false;
  const double x = u[0] * total;
  double acc = 0.0;
  int pick = L.order[allowed - 1];
  for (int r = 0; r < allowed; ++r) {
    const int t = L.order[r];
    const double s = lam / (2.0 * cfg.refl_d[t]);
    acc += lam * lam * lam * cfg.refl_w[t] / (4.0 * s);
    if (x < acc) {
      pick = t;
      break;
    }
  }
  const double s = lam / (2.0 * cfg.refl_d[pick]);
  const double c2t = 1.0 - 2.0 * s * s;
  const double s2t = 2.0 * s * std::sqrt((1.0 - s) * (1.0 + s));
  o->d = rotate_about(d, c2t, s2t, 2.0 * kPi * u[1]);
  o->speed = speed;
  o->rest = total / sig_kernel;
  o->factor = o->rest;
  o->s_value = 1.0;
  o->entry = -1;
  o->mode = pick;
  o->ki = ki;
  o->kf = ki;
  o->e = 0.0;
  o->qvec = add(scale(d, ki), scale(o->d, -ki));
  o->q = std::sqrt(dot(o->qvec, o->qvec));
  return true;
}

// ---- scattering from a dispersion surface (supplement S4) ------------------------------
// d2sigma/dOmega dEf = sigma/4pi (kf/ki) S(Q) delta(E - E(Q)), E = Ei - Ef, with the paper's
// example surface E(Q) = A sqrt(1 - (cos(c Qx) cos(c Qz))^2) and a constant S(Q) = S0, Q in
// the crystal frame (the frame of the single-crystal kernel).  1 - cos^2 a cos^2 b is
// evaluated as sin^2 a + cos^2 a sin^2 b (no cancellation near the zeros of E).
// Sampling: the outgoing direction uniform; the roots of g(Ef) = Ei - Ef - E(Q(Ef)) bracketed
// on 32 equal sub-intervals of [max(0, Ei - A), Ei] (E(Q) lies in [0, A]); one picked
// uniformly and refined by 50 bisections; weight n_roots (kf/ki) S0 / |g'(Ef)| with
// g' = -1 - grad E . dQ/dEf, dQ/dEf = -df kf / (2 Ef) (the delta function integrated over Ef
// at the root, over the uniform choice among the roots and the uniform direction).
struct DispEval {
  double E, g;
  Vec3 Qc, grad;
};

DispEval disp_eval(const orc_config& cfg, double Ei, double ki, Vec3 di, Vec3 df, double Ef,
                   double c, double sn) {
  DispEval r;
  const double kf = kKPerV * std::sqrt(Ef / kMeVPerV2);
  r.Qc = to_crystal(add(scale(di, ki), scale(df, -kf)), c, sn);
  const double a = cfg.disp_c * r.Qc.x, b = cfg.disp_c * r.Qc.z;
  const double sa = std::sin(a), ca = std::cos(a), sb = std::sin(b), cb = std::cos(b);
  const double root = std::sqrt(sa * sa + ca * ca * sb * sb);
  r.E = cfg.disp_amp * root;
  r.g = Ei - Ef - r.E;
  if (root > 0.0) {
    r.grad = {cfg.disp_amp * cfg.disp_c * sa * ca * cb * cb / root, 0.0,
              cfg.disp_amp * cfg.disp_c * ca * ca * sb * cb / root};
  } else {
    r.grad = {0.0, 0.0, 0.0};
  }
  return r;
}

bool kernel_disp(const orc_config& cfg, double rot_y, double speed, Vec3 d, const double u[4],
                 KernelOut* o) {
  const double c = std::cos(rot_y), sn = std::sin(rot_y);
  const double ct = 2.0 * u[0] - 1.0;
  const double st = 2.0 * std::sqrt(u[0] * (1.0 - u[0]));
  const double ph = 2.0 * kPi * u[1];
  const Vec3 df = {st * std::cos(ph), st * std::sin(ph), ct};
  const double Ei = kMeVPerV2 * speed * speed;
  const double ki = kKPerV * speed;
  const double lo = std::max(0.0, Ei - cfg.disp_amp), hi = Ei;
  const int M = 32;
  const double step = (hi - lo) / M;
  double gk[M + 1];
  for (int k = 0; k <= M; ++k) gk[k] = disp_eval(cfg, Ei, ki, d, df, lo + k * step, c, sn).g;
  int nroots = 0;
  for (int k = 0; k < M; ++k)
    if ((gk[k] > 0.0) != (gk[k + 1] > 0.0)) ++nroots;
  o->nroots = nroots;
  if (nroots == 0) return false;
  int pick = (int)std::floor(u[2] * nroots);
  pick = std::min(std::max(pick, 0), nroots - 1);
  int kb = -1;
  for (int k = 0, seen = 0; k < M; ++k) {
    if ((gk[k] > 0.0) != (gk[k + 1] > 0.0)) {
      if (seen == pick) {
        kb = k;
        break;
      }
      ++seen;
    }
  }
  double ea = lo + kb * step, eb = lo + (kb + 1) * step;
  const bool ga_pos = gk[kb] > 0.0;
  for (int it = 0; it < 50; ++it) {
    const double mid = 0.5 * (ea + eb);
    if ((disp_eval(cfg, Ei, ki, d, df, mid, c, sn).g > 0.0) == ga_pos)
      ea = mid;
    else
      eb = mid;
  }
  const double Ef = 0.5 * (ea + eb);
  if (!(Ef > 0.0)) return false;
  const DispEval r = disp_eval(cfg, Ei, ki, d, df, Ef, c, sn);
  if (!(r.E > 0.0)) return false;
  const double kf = kKPerV * std::sqrt(Ef / kMeVPerV2);
  const Vec3 dQ = scale(to_crystal(df, c, sn), -kf / (2.0 * Ef));
  const double gp = -1.0 - dot(r.grad, dQ);
  o->rest = nroots * (kf / ki) * cfg.disp_s0 / std::fabs(gp);
  o->factor = o->rest;
  o->s_value = 1.0;
  o->entry = -1;
  o->d = df;
  o->speed = std::sqrt(Ef / kMeVPerV2);
  o->ki = ki;
  o->kf = kf;
  o->e = Ei - Ef;
  o->qvec = add(scale(d, ki), scale(df, -kf));
  o->q = std::sqrt(dot(o->qvec, o->qvec));
  return true;
}

bool kernel_scatter(const orc_config& cfg, int ktype, double speed, Vec3 d, const double u[4],
                    KernelOut* o, double rot_y = 0.0, double sig_kernel = 1.0) {
  if (ktype == ORC_K_BRAGG) return kernel_bragg(cfg, sig_kernel, speed, d, u, o);
  if (ktype == ORC_K_DISP) return kernel_disp(cfg, rot_y, speed, d, u, o);
  if (ktype == ORC_K_ISO) {
    kernel_iso(speed, d, u, o);
    return true;
  }
  if (ktype == ORC_K_SQE) return kernel_sqe(cfg, speed, d, u, o);
  if (ktype == ORC_K_BVK) return kernel_bvk(cfg, rot_y, speed, d, u, o);
  if (ktype == ORC_K_PHONON) return kernel_phonon(cfg, speed, d, u, o);
  return false;
}

void draw_kernel_uniforms(const orc_config& cfg, int64_t nid, int order, double u[4]) {
  double a[2], b[2];
  orc_uniforms(cfg.seed, cfg.sim_id, nid, order, 1, a);
  orc_uniforms(cfg.seed, cfg.sim_id, nid, order, 2, b);
  u[0] = a[0];
  u[1] = a[1];
  u[2] = b[0];
  u[3] = b[1];
}

// ---- chain-mode tracer ----------------------------------------------------------------
// Per-scatter record kept for the adjoint.
struct ScatterRecord {
  double a_factor;   // weight factor of the scatter without the table value
  double s_value;    // table value or 1
  int entry;         // table entry or -1
  double dlog_abs;   // d ln(a_factor) / d sigma_abs of the differentiated scatterer
  double dlog_s;     // d ln(a_factor) / d sigma_s of the differentiated scatterer
};
struct EmitRecord {
  int order;
  Neutron n;
  double w;          // emitted weight
  double atten;      // exp(-tau_tot) of this emission
  double dlog_abs, dlog_s;
  double kappa;      // condition estimate of w
};

// One neutron through the sample assembly, as a chain of at most N_max scatterings.
// Each scattering splits the packet (section 2.4.3 "Multiple Scattering"): the transmitted
// part leaves with weight w e^{-tau}; the scattered part continues from a point picked
// uniformly along the forward path, with the kernel picked at random.  The paper's
// recursion (supplement, scatterM / interactM_path1 / interactM1) samples the point on
// the first segment only and handles later segments in further rounds; here the point is
// picked on all segments ahead at once, which gives the same expectation.
// stop_on_zero: stop when the weight is exactly zero (it cannot contribute); the adjoint
// keeps tracing such paths because their derivative need not be zero.
template <class Emit, class Scat>
void chain_one(const orc_config& cfg, int64_t nid, bool stop_on_zero, int gs, Emit emit,
               Scat on_scatter, double* tallies) {
  Neutron n;
  if (ORC_CONDITION) {
    g_kappa = 1.0;
    g_kappa_v = 2.0;
  }
  if (!make_beam(cfg, nid, &n)) return;
  // the start point's transverse coordinates are rounded once; the direction a few times
  if (ORC_CONDITION) {
    g_err_r = std::fabs(n.r.x) + std::fabs(n.r.y);
    g_err_a = 0.0;
    g_dprev = n.d;
    g_err_d = 4.0;
  }
  for (int o = 0;; ++o) {
    if (n.w < cfg.min_prob) break;
    if (stop_on_zero && n.w == 0.0) break;
    Segment seg[8];
    int ns = assembly_segments(cfg, n.r, n.d, seg);
    double tau = 0.0, L = 0.0, Lg = 0.0;
    for (int i = 0; i < ns; ++i) {
      double len = seg[i].sb - seg[i].sa;
      tau += mu_total(cfg.scat[seg[i].j], n.speed) * len;
      L += len;
      if (seg[i].j == gs) Lg += len;
    }
    if (o == 0 && L > 0.0 && tallies) tallies[ORC_T_NHIT] += 1.0;
    EmitRecord em;
    em.order = o;
    em.n = n;
    em.kappa = g_kappa;
    em.atten = std::exp(-tau);
    em.w = n.w * em.atten;
    em.dlog_abs = 0.0;
    em.dlog_s = 0.0;
    if (gs >= 0) {
      const orc_scatterer& g = cfg.scat[gs];
      em.dlog_abs = -100.0 * g.n_per_A3 * (2200.0 / n.speed) * Lg;
      em.dlog_s = -100.0 * g.n_per_A3 * Lg;
    }
    emit(em);
    if (o == cfg.max_orders || !(L > 0.0)) break;
    double u[2];
    orc_uniforms(cfg.seed, cfg.sim_id, nid, o, 0, u);
    // scattering point, uniform over the material length ahead
    double ell = u[0] * L;
    double acc = 0.0, tau_pt = 0.0, s_pt = 0.0, lg_pt = 0.0;
    // error scale of the scattering distance: the rounding of the chosen segment's start,
    // the lengths summed into acc and (times u) into L, and the roundings of ell and s_pt
    double e_pt = std::fabs(ell);
    for (int i = 0; i < ns; ++i) e_pt += u[0] * (seg[i].ra + seg[i].rb);
    int j = seg[ns - 1].j;
    for (int i = 0; i < ns; ++i) {
      double len = seg[i].sb - seg[i].sa;
      double mu = mu_total(cfg.scat[seg[i].j], n.speed);
      if (ell < acc + len || i == ns - 1) {
        double part = ell - acc;
        s_pt = seg[i].sa + part;
        e_pt += seg[i].ra0 + std::fabs(s_pt);
        for (int m = 0; m < i; ++m) e_pt += seg[m].ra + seg[m].rb;
        tau_pt += mu * part;
        if (seg[i].j == gs) lg_pt += part;
        j = seg[i].j;
        break;
      }
      acc += len;
      tau_pt += mu * len;
      if (seg[i].j == gs) lg_pt += len;
    }
    const orc_scatterer& sc = cfg.scat[j];
    ScatterRecord rec;
    rec.a_factor = mu_scatt(sc) * L * std::exp(-tau_pt);
    rec.dlog_abs = 0.0;
    rec.dlog_s = 0.0;
    if (gs >= 0) {
      const orc_scatterer& g = cfg.scat[gs];
      rec.dlog_abs = -100.0 * g.n_per_A3 * (2200.0 / n.speed) * lg_pt;
      rec.dlog_s = -100.0 * g.n_per_A3 * lg_pt + (j == gs ? 1.0 / sigma_scatt(g) : 0.0);
    }
    n.r = add(n.r, scale(n.d, s_pt));
    n.t = n.t + s_pt / n.speed;
    // the new point: the error of s_pt along the ray, and the roundings of its coordinates
    if (ORC_CONDITION) {
      g_err_a = e_pt;
      g_dprev = n.d;
      g_err_r = std::sqrt(dot(n.r, n.r)) + std::fabs(s_pt);
    }
    // kernel choice with probability sigma_k / sigma_s (weight unchanged)
    int k = 0;
    if (sc.nk == 2 && !(u[1] * (sc.ksig_b[0] + sc.ksig_b[1]) < sc.ksig_b[0])) k = 1;
    double uk[4];
    draw_kernel_uniforms(cfg, nid, o, uk);
    KernelOut ko;
    if (!kernel_scatter(cfg, sc.ktype[k], n.speed, n.d, uk, &ko, sc.rot_y, sc.ksig_b[k])) break;
    rec.s_value = ko.s_value;
    rec.entry = ko.entry;
    n.w = n.w * rec.a_factor * ko.factor;
    rec.a_factor = rec.a_factor * ko.rest;
    n.d = ko.d;
    n.speed = ko.speed;
    // an isotropic direction is drawn afresh; the others are built on the incoming one
    if (ORC_CONDITION) g_err_d = sc.ktype[k] == ORC_K_ISO ? 4.0 : g_err_d + 8.0;
    on_scatter(o + 1, sc.ktype[k], j, ko, rec, n.w);
  }
}

void add_tally(double* tallies, int i, double v) {
  if (tallies) tallies[i] += v;
}

void record_detection(const orc_config& cfg, int64_t nid, const EmitRecord& em, orc_packet* pk,
                      double* hist, double* tallies) {
  if (em.order == 0) {
    add_tally(tallies, ORC_T_BEAMSTOP, em.w);
    if (pk) {
      pk->pixel = -1;
      pk->tof = 0.0;
      pk->w_det = 0.0;
      pk->bin = -1;
    }
    return;
  }
  double u[2];
  orc_uniforms(cfg.seed, cfg.sim_id, nid, em.order, 3, u);
  int32_t pixel;
  double tof, w_det;
  const double k_before = g_kappa;
  if (ORC_CONDITION) g_kappa = 0.0;
  int64_t bin = detect(cfg, em.n.r, em.n.d, em.n.speed, em.n.t, em.w, u[0], &pixel, &tof, &w_det);
  const double k_det = g_kappa;
  if (ORC_CONDITION) g_kappa = k_before;
  if (pk) pk->kappa_det = em.kappa + k_det;
  if (bin >= 0) {
    if (hist) hist[bin] += w_det;
    add_tally(tallies, ORC_T_WDET, w_det);
    add_tally(tallies, ORC_T_NDET, 1.0);
  } else if (bin == -2) {
    add_tally(tallies, ORC_T_WOVER, w_det);
    add_tally(tallies, ORC_T_NOVER, 1.0);
  } else {
    add_tally(tallies, ORC_T_NMISS, 1.0);
  }
  if (pk) {
    pk->pixel = pixel;
    pk->tof = tof;
    pk->w_det = w_det;
    pk->bin = bin;
  }
}

void fill_packet(int64_t nid, const EmitRecord& em, orc_packet* pk) {
  pk->nid = nid;
  pk->order = em.order;
  pk->x = em.n.r.x;
  pk->y = em.n.r.y;
  pk->z = em.n.r.z;
  pk->vx = em.n.speed * em.n.d.x;
  pk->vy = em.n.speed * em.n.d.y;
  pk->vz = em.n.speed * em.n.d.z;
  pk->t = em.n.t;
  pk->w = em.w;
  pk->kappa = em.kappa;
  pk->kappa_det = em.kappa;
}

bool config_ok(const orc_config* cfg) {
  if (!cfg || cfg->n_scat < 0 || cfg->n_scat > 4 || cfg->max_orders < 0) return false;
  for (int j = 0; j < cfg->n_scat; ++j) {
    const orc_scatterer& s = cfg->scat[j];
    if (s.nk < 1 || s.nk > 2) return false;
    for (int k = 0; k < s.nk; ++k) {
      if (s.ktype[k] == ORC_K_SQE && (!cfg->sqe || cfg->nq <= 0 || cfg->ne <= 0)) return false;
      if (s.ktype[k] == ORC_K_BVK && !(cfg->bvk_phi_Nm > 0 && cfg->bvk_mass_u > 0 &&
                                      cfg->bvk_a_A > 0 && cfg->temperature_K > 0))
        return false;
      if (s.ktype[k] == ORC_K_DISP &&
          !(cfg->disp_amp > 0 && cfg->disp_c > 0 && cfg->disp_s0 >= 0))
        return false;
      if (s.ktype[k] == ORC_K_BRAGG) {
        if (!cfg->refl_d || !cfg->refl_w || cfg->n_refl < 1 || !(s.ksig_b[k] > 0)) return false;
        for (int r = 0; r < cfg->n_refl; ++r)
          if (!(cfg->refl_d[r] > 0) || !(cfg->refl_w[r] >= 0)) return false;
      }
      if (s.ktype[k] == ORC_K_PHONON) {
        if (!cfg->dos_z || cfg->dos_n < 1 || !(cfg->dos_de > 0) || !(cfg->phonon_mass_u > 0) ||
            cfg->phonon_nmax < 2 || !(cfg->temperature_K > 0))
          return false;
        double zs = 0.0, ps = 0.0;
        for (int j = 0; j < cfg->dos_n; ++j) {
          if (!(cfg->dos_z[j] >= 0)) return false;
          zs += cfg->dos_z[j];
        }
        for (int c = 0; c < 3; ++c) {
          if (!(cfg->phonon_p[c] > 0)) return false;
          ps += cfg->phonon_p[c];
        }
        if (!(zs > 0) || std::fabs(ps - 1.0) > 1e-12) return false;
      }
    }
  }
  if (cfg->det_kind != ORC_DET_NONE && cfg->n_tof <= 0) return false;
  return true;
}

// ---- paper-literal recursive estimator ------------------------------------------------
// The packet's place in the tree of interactions (supplement S3: every interactM1 splits a
// packet into a transmitted and a scattered one): the incident packet is node 1, the
// transmitted and scattered packets of an interaction of node x are 2x and 2x + 1.  A node
// keys its own random numbers, so that the tree may be visited in any order; a tree deeper
// than 61 interactions is cut (its packet leaves with the attenuation of the material ahead).
// A transmitted packet goes on along its parent's line: it keeps the line's origin (n.r, and
// n.t there) and the distance s0 travelled along it, and the material ahead is what lies
// beyond s0 on that line.  (Re-tracing from the exit point instead, rounded onto or just
// inside the surface it left, would meet a sliver of the material behind it again and again.)
struct PaperPacket {
  Neutron n;
  int m;          // number of scatterings so far
  uint64_t node;  // place in the tree
  double s0;      // distance travelled along the line from n.r
};

const uint64_t kPaperMaxNode = (uint64_t)1 << 61;

// the two uniforms of block `block` of node `node` of neutron nid (the paper mode's stream)
void paper_uniforms(const orc_config& cfg, int64_t nid, uint64_t node, int block, double u[2]) {
  const uint32_t ctr[4] = {(uint32_t)((uint64_t)nid & 0xffffffffu), (uint32_t)((uint64_t)nid >> 32),
                           (uint32_t)(((node & 0x3fffffffu) << 2) | (uint32_t)block),
                           (uint32_t)(node >> 30)};
  const uint32_t key[2] = {cfg.seed, cfg.sim_id ^ 0x80000000u};
  uint32_t out[4];
  orc_philox4x32_10(ctr, key, out);
  u[0] = u01_from(out[0], out[1]);
  u[1] = u01_from(out[2], out[3]);
}

struct PaperRun {
  const orc_config& cfg;
  int64_t nid;
  double* hist;
  double* tallies;
};

void paper_record(PaperRun& pr, int64_t bin, double w_det) {
  if (bin >= 0) {
    if (pr.hist) pr.hist[bin] += w_det;
    add_tally(pr.tallies, ORC_T_WDET, w_det);
    add_tally(pr.tallies, ORC_T_NDET, 1.0);
  } else if (bin == -2) {
    add_tally(pr.tallies, ORC_T_WOVER, w_det);
    add_tally(pr.tallies, ORC_T_NOVER, 1.0);
  }
}

// A packet leaving the sample assembly: order 0 to the beam stop, the others to the
// detector system (every tube crossed, with det_multi_tube), met along the packet's line from
// its origin (the tubes lie metres beyond the sample, far past s0).  Detector draws: blocks 3
// and 0 of the packet's node.
void paper_emit(PaperRun& pr, const PaperPacket& p) {
  if (p.m == 0) {
    add_tally(pr.tallies, ORC_T_BEAMSTOP, p.n.w);
    return;
  }
  double u3[2], u0[2];
  paper_uniforms(pr.cfg, pr.nid, p.node, 3, u3);
  if (pr.cfg.det_multi_tube && pr.cfg.det_kind == ORC_DET_TUBES) {
    paper_uniforms(pr.cfg, pr.nid, p.node, 0, u0);
    const double u[3] = {u3[0], u3[1], u0[0]};
    const double v[3] = {p.n.d.x * p.n.speed, p.n.d.y * p.n.speed, p.n.d.z * p.n.speed};
    const double r[3] = {p.n.r.x, p.n.r.y, p.n.r.z};
    int32_t pix[3];
    double tof[3], wd[3];
    int64_t bins[3];
    const int k = orc_detect_multi(&pr.cfg, r, v, p.n.t, p.n.w, u, pix, tof, wd, bins);
    if (k == 0) add_tally(pr.tallies, ORC_T_NMISS, 1.0);
    for (int i = 0; i < k; ++i) paper_record(pr, bins[i], wd[i]);
    return;
  }
  int32_t pixel;
  double tof, w_det;
  int64_t bin = detect(pr.cfg, p.n.r, p.n.d, p.n.speed, p.n.t, p.n.w, u3[0], &pixel, &tof, &w_det);
  if (bin == -1) add_tally(pr.tallies, ORC_T_NMISS, 1.0);
  paper_record(pr, bin, w_det);
}

// interactM1 of homogeneous scatterer j on its first segment [sa, sb] ahead of the packet:
// the transmitted packet leaves the segment attenuated; the scattered one is taken at a
// uniform point of it (scattered->m stays negative when the kernel cannot scatter).
void paper_interact1(PaperRun& pr, int j, double sa, double sb, const PaperPacket& in,
                     PaperPacket* transmitted, PaperPacket* scattered) {
  const orc_config& cfg = pr.cfg;
  const orc_scatterer& sc = cfg.scat[j];
  double len = sb - sa;
  double mu = mu_total(sc, in.n.speed);
  *transmitted = in;
  transmitted->s0 = sb;
  transmitted->n.w = in.n.w * std::exp(-mu * len);
  transmitted->node = 2 * in.node;
  double u[2];
  paper_uniforms(cfg, pr.nid, in.node, 0, u);
  double ell = u[0] * len;
  double s = sa + ell;
  PaperPacket p = in;
  p.n.r = add(in.n.r, scale(in.n.d, s));
  p.n.t = in.n.t + s / in.n.speed;
  p.n.w = in.n.w * mu_scatt(sc) * len * std::exp(-mu * ell);
  p.s0 = 0.0;
  int k = 0;
  if (sc.nk == 2 && !(u[1] * (sc.ksig_b[0] + sc.ksig_b[1]) < sc.ksig_b[0])) k = 1;
  double a[2], b[2];
  paper_uniforms(cfg, pr.nid, in.node, 1, a);
  paper_uniforms(cfg, pr.nid, in.node, 2, b);
  double uk[4] = {a[0], a[1], b[0], b[1]};
  KernelOut ko;
  if (!kernel_scatter(cfg, sc.ktype[k], p.n.speed, p.n.d, uk, &ko, sc.rot_y, sc.ksig_b[k]))
    return;
  p.n.w = p.n.w * ko.factor;
  p.n.d = ko.d;
  p.n.speed = ko.speed;
  p.m = in.m + 1;
  p.node = 2 * in.node + 1;
  *scattered = p;
}

// the packet still inside a scatterer after its last allowed scattering leaves with the
// attenuation of all material ahead
PaperPacket paper_propagate_out(const orc_config& cfg, PaperPacket p) {
  Segment seg[8];
  int ns = assembly_segments(cfg, p.n.r, p.n.d, seg, p.s0);
  double tau = 0.0;
  for (int i = 0; i < ns; ++i) tau += mu_total(cfg.scat[seg[i].j], p.n.speed) * (seg[i].sb - seg[i].sa);
  p.n.w = p.n.w * std::exp(-tau);
  return p;
}

void paper_one(const orc_config& cfg, int64_t nid, double* hist, double* tallies) {
  PaperRun pr{cfg, nid, hist, tallies};
  Neutron n0;
  if (!make_beam(cfg, nid, &n0)) return;
  {
    Segment seg[8];
    if (assembly_segments(cfg, n0.r, n0.d, seg) > 0) add_tally(tallies, ORC_T_NHIT, 1.0);
  }
  std::vector<PaperPacket> toscatter{PaperPacket{n0, 0, 1, 0.0}};
  while (!toscatter.empty()) {
    std::vector<PaperPacket> scattered;
    for (const PaperPacket& p : toscatter) {
      if (p.n.w < cfg.min_prob) continue;
      Segment seg[8];
      int ns = assembly_segments(cfg, p.n.r, p.n.d, seg, p.s0);
      if (ns == 0) {  // exiting: nothing ahead
        paper_emit(pr, p);
        continue;
      }
      if (p.m >= cfg.max_orders || p.node >= kPaperMaxNode) {  // leave with attenuation
        paper_emit(pr, paper_propagate_out(cfg, p));
        continue;
      }
      // interactM_path1 of the composite: the first constituent met delegates
      int j = seg[0].j;
      double sa = seg[0].sa, sb = seg[0].sb;
      PaperPacket cur = p;
      bool alive = true;
      // interactM_path1 of the homogeneous scatterer: interactM1 on the segment met, then
      // again on the scatterer's first segment ahead while the scattered packet may scatter;
      // what is left is handed back to the next round
      while (true) {
        if (cur.n.w < cfg.min_prob) {
          alive = false;
          break;
        }
        PaperPacket tr, sc;
        sc.m = -1;
        paper_interact1(pr, j, sa, sb, cur, &tr, &sc);
        scattered.push_back(tr);
        if (sc.m < 0) {
          alive = false;
          break;
        }
        cur = sc;
        if (!(cur.m < cfg.max_orders && cur.node < kPaperMaxNode)) break;
        double a2[2], b2[2];
        if (shape_segments(cfg.scat[j], cur.n.r, cur.n.d, a2, b2) == 0) break;
        sa = a2[0];
        sb = b2[0];
      }
      if (alive) scattered.push_back(cur);
    }
    toscatter.swap(scattered);
  }
}

}  // namespace

// ---- C entry points -------------------------------------------------------------------
extern "C" {

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  // Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11): each round multiplies
  // two words by fixed odd constants, swaps and xors the high halves with the other words
  // and the key; the key is bumped by the Weyl constants between rounds.
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c0 = n0;
    c1 = n1;
    c2 = n2;
    c3 = n3;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

void orc_uniforms(uint32_t seed, uint32_t sim_id, int64_t nid, int event, int block, double u[2]) {
  uint32_t ctr[4] = {(uint32_t)((uint64_t)nid & 0xffffffffu), (uint32_t)((uint64_t)nid >> 32),
                     slot_of(event, block), 0u};
  uint32_t key[2] = {seed, sim_id};
  uint32_t o[4];
  orc_philox4x32_10(ctr, key, o);
  u[0] = u01_from(o[0], o[1]);
  u[1] = u01_from(o[2], o[3]);
}

int orc_shape_segments(const orc_scatterer* sc, const double r[3], const double d[3],
                       double sa[2], double sb[2]) {
  return shape_segments(*sc, Vec3{r[0], r[1], r[2]}, Vec3{d[0], d[1], d[2]}, sa, sb);
}

int orc_kernel_scatter(const orc_config* cfg, int ktype, double speed, const double d[3],
                       const double u[4], double* speed_out, double d_out[3], double* factor,
                       orc_event* ev) {
  KernelOut ko;
  const double rot = cfg->n_scat > 0 ? cfg->scat[0].rot_y : 0.0;
  // the nominal cross section of that kernel in scatterer 0 (the Bragg kernel's weight)
  double sig = 1.0;
  if (cfg->n_scat > 0)
    for (int k = 0; k < cfg->scat[0].nk; ++k)
      if (cfg->scat[0].ktype[k] == ktype) sig = cfg->scat[0].ksig_b[k];
  if (!kernel_scatter(*cfg, ktype, speed, Vec3{d[0], d[1], d[2]}, u, &ko, rot, sig)) return 0;
  *speed_out = ko.speed;
  d_out[0] = ko.d.x;
  d_out[1] = ko.d.y;
  d_out[2] = ko.d.z;
  *factor = ko.factor;
  if (ev) {
    ev->kernel = ktype;
    ev->entry = ko.entry;
    ev->mode = ko.mode;
    ev->nroots = ko.nroots;
    ev->q = ko.q;
    ev->e = ko.e;
    ev->ki = ko.ki;
    ev->kf = ko.kf;
    ev->factor = ko.factor;
    ev->qvec[0] = ko.qvec.x;
    ev->qvec[1] = ko.qvec.y;
    ev->qvec[2] = ko.qvec.z;
  }
  return 1;
}

int64_t orc_detect(const orc_config* cfg, const double r[3], const double v[3], double t,
                   double w, double u_det, int32_t* pixel, double* tof, double* w_det) {
  double speed = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  Vec3 d = {v[0] / speed, v[1] / speed, v[2] / speed};
  return detect(*cfg, Vec3{r[0], r[1], r[2]}, d, speed, t, w, u_det, pixel, tof, w_det);
}

int orc_detect_multi(const orc_config* cfg, const double r_[3], const double v[3], double t,
                     double w, const double u[3], int32_t pixel[3], double tof[3],
                     double w_det[3], int64_t bin[3]) {
  // Ray tracing in the detector system as a composite of absorbing tubes (section 2.4.3):
  // the candidate tubes as in the single-tube detector, every one the ray enters absorbing
  // its share of the weight the earlier tubes left.
  if (cfg->det_kind != ORC_DET_TUBES) return 0;
  const double speed = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  const Vec3 d = {v[0] / speed, v[1] / speed, v[2] / speed};
  const Vec3 r = {r_[0], r_[1], r_[2]};
  const double R = cfg->det_radius_m;
  double sR;
  if (!exit_cylinder(R, r, d, &sR)) return 0;
  const Vec3 P = add(r, scale(d, sR));
  int row = -1, row_off = 0;
  for (int i = 0, off = 0; i < cfg->n_rows; off += cfg->packs[i], ++i) {
    if (std::fabs(P.y - cfg->row_y_m[i]) <= 0.5 * cfg->tube_len_m) {
      row = i;
      row_off = off;
      break;
    }
  }
  if (row < 0) return 0;
  const int tpp = cfg->tubes_per_pack;
  const double period = tpp * cfg->tube_pitch_m + cfg->pack_gap_m;
  const double arc = (std::atan2(P.x, P.z) - cfg->phi0_rad) * R;
  const double pk = std::floor(arc / period);
  double k = std::floor((arc - pk * period) / cfg->tube_pitch_m);
  if (k > tpp - 1) k = tpp - 1;
  const int64_t g = (int64_t)pk * tpp + (int64_t)k;
  const int64_t n_tubes_row = (int64_t)cfg->packs[row] * tpp;
  const double y_lo = cfg->row_y_m[row] - 0.5 * cfg->tube_len_m;
  const double y_hi = cfg->row_y_m[row] + 0.5 * cfg->tube_len_m;
  // the candidates the ray enters, by entry distance
  int64_t tube[3];
  double s_in[3], s_out[3];
  int m = 0;
  for (int64_t c = g - 1; c <= g + 1; ++c) {
    if (c < 0 || c >= n_tubes_row) continue;
    const int64_t pc = c / tpp, tc = c % tpp;
    const double phic = cfg->phi0_rad + (pc * period + (tc + 0.5) * cfg->tube_pitch_m) / R;
    double s1, s2;
    if (!tube_interval(R, std::sin(phic), std::cos(phic), cfg->tube_r_m, r, d, &s1, &s2)) continue;
    double ys1, ys2;
    if (d.y == 0.0) {
      if (!(r.y >= y_lo && r.y <= y_hi)) continue;
      ys1 = -kInf;
      ys2 = kInf;
    } else {
      const double a = (y_lo - r.y) / d.y, b = (y_hi - r.y) / d.y;
      ys1 = std::min(a, b);
      ys2 = std::max(a, b);
    }
    const double a_in = std::max(std::max(s1, ys1), 0.0), a_out = std::min(s2, ys2);
    if (!(a_out > a_in)) continue;
    int at = m++;
    while (at > 0 && s_in[at - 1] > a_in) {  // insertion by entry distance
      tube[at] = tube[at - 1];
      s_in[at] = s_in[at - 1];
      s_out[at] = s_out[at - 1];
      --at;
    }
    tube[at] = c;
    s_in[at] = a_in;
    s_out[at] = a_out;
  }
  const double mu = 100.0 * cfg->he3_n_per_A3 * cfg->he3_sig_abs_b * 2200.0 / speed;
  const double pix_len = cfg->tube_len_m / cfg->pixels_per_tube;
  const double dt = (cfg->tof_max_s - cfg->tof_min_s) / cfg->n_tof;
  double left = w;
  for (int i = 0; i < m; ++i) {
    const double L = s_out[i] - s_in[i];
    const double pabs = -std::expm1(-mu * L);
    const double x = -std::log1p(-u[i] * pabs) / mu;
    const double s_abs = s_in[i] + x;
    const double y_abs = r.y + s_abs * d.y;
    int64_t j = (int64_t)std::floor((y_abs - y_lo) / pix_len);
    j = std::min<int64_t>(std::max<int64_t>(j, 0), cfg->pixels_per_tube - 1);
    const int64_t pc = tube[i] / tpp, tc = tube[i] % tpp;
    pixel[i] = (int32_t)(((row_off + pc) * tpp + tc) * cfg->pixels_per_tube + j);
    tof[i] = t + s_abs / speed;
    w_det[i] = left * pabs;
    left = left * (1.0 - pabs);
    const double fb = std::floor((tof[i] - cfg->tof_min_s) / dt);
    bin[i] = (fb >= 0.0 && fb < (double)cfg->n_tof) ? (int64_t)pixel[i] * cfg->n_tof + (int64_t)fb : -2;
  }
  return m;
}

int64_t orc_n_pixels(const orc_config* cfg) { return n_pixels(*cfg); }

void orc_bvk_modes(const orc_config* cfg, const double q[3], double hw[3], double evec[9]) {
  const BvkModel m = bvk_model(*cfg);
  double D[6], lam[3];
  bvk_dynmat(m, q, D);
  eig_sym3(D, lam, evec);
  for (int b = 0; b < 3; ++b) hw[b] = hbar_omega(lam[b]);
}

int orc_kernel_bvk(const orc_config* cfg, double rot_y, double speed, const double d[3],
                   const double u[4], double* speed_out, double d_out[3], double* factor,
                   orc_event* ev) {
  KernelOut ko;
  const bool ok = kernel_bvk(*cfg, rot_y, speed, Vec3{d[0], d[1], d[2]}, u, &ko);
  if (ev) {
    ev->nroots = ko.nroots;
    ev->mode = ko.mode;
  }
  if (!ok) return 0;
  *speed_out = ko.speed;
  d_out[0] = ko.d.x;
  d_out[1] = ko.d.y;
  d_out[2] = ko.d.z;
  *factor = ko.factor;
  if (ev) {
    ev->kernel = ORC_K_BVK;
    ev->entry = -1;
    ev->q = ko.q;
    ev->e = ko.e;
    ev->ki = ko.ki;
    ev->kf = ko.kf;
    ev->factor = ko.factor;
    ev->qvec[0] = ko.qvec.x;
    ev->qvec[1] = ko.qvec.y;
    ev->qvec[2] = ko.qvec.z;
  }
  return 1;
}

int orc_phonon_tables(const orc_config* cfg, double* gamma0, double* c_w, double* a, int64_t cap) {
  if (!cfg || !cfg->dos_z || cfg->dos_n < 1 || cfg->phonon_nmax < 2 || !(cfg->dos_de > 0) ||
      !(cfg->temperature_K > 0) || !(cfg->phonon_mass_u > 0))
    return 0;
  const PhononModel& m = phonon_model(*cfg);
  *gamma0 = m.gamma0;
  *c_w = m.cw;
  if (a && cap >= (int64_t)m.N * m.M)
    for (int n = 1; n <= m.N; ++n)
      for (int i = 0; i < m.M; ++i) a[(int64_t)(n - 1) * m.M + i] = m.an[n][i];
  return m.M;
}

int orc_trace(const orc_config* cfg, int64_t first_id, int64_t n, orc_packet* packets,
              orc_event* events, double* hist, double* tallies) {
  if (!config_ok(cfg) || n < 0) return 1;
  const int slots = cfg->max_orders + 1;
  for (int64_t i = 0; i < n; ++i) {
    int64_t nid = first_id + i;
    orc_packet* base = packets ? packets + i * slots : nullptr;
    if (base)
      for (int s = 0; s < slots; ++s) {
        std::memset(&base[s], 0, sizeof(orc_packet));
        base[s].nid = nid;
        base[s].order = -1;
        base[s].pixel = -1;
        base[s].bin = -1;
      }
    orc_event* ev = events ? events + i * cfg->max_orders : nullptr;
    if (ev)
      for (int s = 0; s < cfg->max_orders; ++s) {
        std::memset(&ev[s], 0, sizeof(orc_event));
        ev[s].nid = nid;
        ev[s].order = -1;
        ev[s].entry = -1;
      }
    auto emit = [&](const EmitRecord& em) {
      if (em.order < 8) add_tally(tallies, ORC_T_NPACK0 + em.order, 1.0);
      orc_packet* pk = base ? &base[em.order] : nullptr;
      if (pk) fill_packet(nid, em, pk);
      if (cfg->det_kind != ORC_DET_NONE || em.order == 0)
        record_detection(*cfg, nid, em, pk, hist, tallies);
    };
    auto on_scatter = [&](int order, int ktype, int j, const KernelOut& ko,
                          const ScatterRecord&, double w_after) {
      if (!ev) return;
      orc_event& e = ev[order - 1];
      e.order = order;
      e.kernel = ktype;
      e.scatterer = j;
      e.entry = ko.entry;
      e.q = ko.q;
      e.e = ko.e;
      e.ki = ko.ki;
      e.kf = ko.kf;
      e.factor = ko.factor;
      e.w = w_after;
      e.nroots = ko.nroots;
      e.mode = ko.mode;
      e.qvec[0] = ko.qvec.x;
      e.qvec[1] = ko.qvec.y;
      e.qvec[2] = ko.qvec.z;
    };
    chain_one(*cfg, nid, true, -1, emit, on_scatter, tallies);
  }
  return 0;
}

int orc_trace_paper(const orc_config* cfg, int64_t first_id, int64_t n, double* hist,
                    double* tallies) {
  if (!config_ok(cfg) || n < 0) return 1;
  for (int64_t i = 0; i < n; ++i) paper_one(*cfg, first_id + i, hist, tallies);
  return 0;
}

static double chi2_and_grad(const orc_config& cfg, const double* hist, const double* target,
                            double c, double* g) {
  int64_t nb = n_pixels(cfg) * cfg.n_tof;
  double loss = 0.0;
  for (int64_t b = 0; b < nb; ++b) {
    double den = std::max(target[b], 1.0);
    double r = c * hist[b] - target[b];
    loss += r * r / den;
    if (g) g[b] = 2.0 * c * r / den;
  }
  return loss;
}

int orc_loss(const orc_config* cfg, int64_t first_id, int64_t n, const double* target,
             double scale_c, double* hist_work, double* loss) {
  if (!config_ok(cfg) || n < 0 || cfg->det_kind == ORC_DET_NONE) return 1;
  int64_t nb = n_pixels(*cfg) * cfg->n_tof;
  std::fill(hist_work, hist_work + nb, 0.0);
  orc_trace(cfg, first_id, n, nullptr, nullptr, hist_work, nullptr);
  *loss = chi2_and_grad(*cfg, hist_work, target, scale_c, nullptr);
  return 0;
}

// Adjoint of the chi-squared loss along fixed random paths: every packet weight is a
// product of factors, so d w / d theta follows from the factors' derivatives.  The loss and
// dchi2/dI are those of `hist` (the whole run's histogram); the gradient sums over the
// neutrons first_id..first_id+n-1 only, so the gradients of the parts of a split run add up
// to that of the whole run.
int orc_adjoint(const orc_config* cfg, int64_t first_id, int64_t n, const double* hist,
                const double* target, double scale_c, int gs, double* loss, double* dsqe,
                double* dsig) {
  if (!config_ok(cfg) || n < 0 || cfg->det_kind == ORC_DET_NONE) return 1;
  if (gs < 0 || gs >= cfg->n_scat) return 1;
  int64_t nb = n_pixels(*cfg) * cfg->n_tof;
  std::vector<double> g(nb);
  *loss = chi2_and_grad(*cfg, hist, target, scale_c, g.data());
  if (cfg->sqe) std::fill(dsqe, dsqe + (int64_t)cfg->nq * cfg->ne, 0.0);
  dsig[0] = 0.0;
  dsig[1] = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    int64_t nid = first_id + i;
    std::vector<ScatterRecord> recs;
    auto on_scatter = [&](int, int, int, const KernelOut&, const ScatterRecord& r, double) {
      recs.push_back(r);
    };
    auto emit = [&](const EmitRecord& em) {
      if (em.order == 0) return;
      double u[2];
      orc_uniforms(cfg->seed, cfg->sim_id, nid, em.order, 3, u);
      int32_t pixel;
      double tof, w_det;
      int64_t bin = detect(*cfg, em.n.r, em.n.d, em.n.speed, em.n.t, em.w, u[0], &pixel, &tof,
                           &w_det);
      if (bin < 0) return;
      // detector factor (independent of the sample parameters)
      double pabs;
      detect(*cfg, em.n.r, em.n.d, em.n.speed, em.n.t, 1.0, u[0], &pixel, &tof, &pabs);
      double gb = g[bin];
      // sigma: d w_det / d sigma = w_det * sum of log-derivatives
      double la = em.dlog_abs, ls = em.dlog_s;
      for (int k = 0; k < em.order; ++k) {
        la += recs[k].dlog_abs;
        ls += recs[k].dlog_s;
      }
      dsig[0] += gb * w_det * la;
      dsig[1] += gb * w_det * ls;
      // table: product of every other factor
      for (int k = 0; k < em.order; ++k) {
        if (recs[k].entry < 0) continue;
        double prod = em.atten * pabs;
        for (int m = 0; m < em.order; ++m) {
          prod *= recs[m].a_factor;
          if (m != k) prod *= recs[m].s_value;
        }
        dsqe[recs[k].entry] += gb * prod;
      }
    };
    chain_one(*cfg, nid, false, gs, emit, on_scatter, nullptr);
  }
  return 0;
}

// The forward histogram of the neutrons first_id..first_id+n-1, then the adjoint of the
// same neutrons.
int orc_grad(const orc_config* cfg, int64_t first_id, int64_t n, const double* target,
             double scale_c, int gs, double* hist_out, double* loss, double* dsqe,
             double* dsig) {
  if (!config_ok(cfg) || n < 0 || cfg->det_kind == ORC_DET_NONE) return 1;
  if (gs < 0 || gs >= cfg->n_scat) return 1;
  int64_t nb = n_pixels(*cfg) * cfg->n_tof;
  std::fill(hist_out, hist_out + nb, 0.0);
  orc_trace(cfg, first_id, n, nullptr, nullptr, hist_out, nullptr);
  return orc_adjoint(cfg, first_id, n, hist_out, target, scale_c, gs, loss, dsqe, dsig);
}

}  // extern "C"
