// C ABI of libmcv.so (declared in include/mcv.h): argument checking, derived constants,
// launch shapes.  No call here allocates device memory except mcv_create.  The batched
// launches are in mcv_batch.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include <cuda_runtime.h>

#include "mcv_host.h"

namespace mcv {
namespace host {

thread_local std::string g_last_error;

mcv_status fail(mcv_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

mcv_status cuda_fail(cudaError_t e, const char* where) {
  return fail(MCV_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

mcv_status alloc_fail(const std::string& msg) {
  (void)cudaGetLastError();
  return fail(MCV_ENOMEM, msg);
}

bool is_finite(double v) { return std::isfinite(v); }

// ---- descriptions -> device parameter blocks -------------------------------------------
mcv_status build_beam(const mcv_beam_params* b, mcv::BeamP<double>* B) {
  if (!b) return fail(MCV_EINVAL, "beam parameters are NULL");
  const double v[] = {b->ei_mev, b->ei_rel_sigma, b->div_sigma_rad, b->width_m, b->height_m,
                      b->z0_m, b->l1_m};
  for (double x : v)
    if (!is_finite(x)) return fail(MCV_EINVAL, "beam parameter is not finite");
  if (!(b->ei_mev > 0.0)) return fail(MCV_EINVAL, "beam energy must be positive");
  if (b->ei_rel_sigma < 0 || b->div_sigma_rad < 0 || b->width_m < 0 || b->height_m < 0)
    return fail(MCV_EINVAL, "beam spreads must be non-negative");
  if (!(b->l1_m >= b->z0_m)) return fail(MCV_EINVAL, "beam needs l1_m >= z0_m");
  B->ei = b->ei_mev;
  B->rel = b->ei_rel_sigma;
  B->div = b->div_sigma_rad;
  B->width = b->width_m;
  B->height = b->height_m;
  B->z0 = b->z0_m;
  B->l1 = b->l1_m;
  B->speed0 = std::sqrt(b->ei_mev / mcv::kMeVPerV2);
  B->t0 = (b->l1_m - b->z0_m) / B->speed0;
  B->t0_hi = (float)B->t0;
  B->t0_lo = (float)(B->t0 - (double)B->t0_hi);
  B->energy_positive = b->ei_rel_sigma * 8.7 < 1.0 ? 1 : 0;
  B->x_safe = INFINITY;
  B->y_safe = INFINITY;
  return MCV_OK;
}

mcv_status build_sample(const mcv_sample* s, mcv::SampleP<double>* S) {
  if (!s) return fail(MCV_EINVAL, "sample is NULL");
  std::memset(S, 0, sizeof(*S));
  if (s->n_scatterers < 1 || s->n_scatterers > MCV_MAX_SCATTERERS)
    return fail(MCV_EINVAL, "n_scatterers must be 1..4");
  if (s->max_orders < 0 || s->max_orders > 7) return fail(MCV_EINVAL, "max_orders must be 0..7");
  if (s->fp_mode != MCV_FP64 && s->fp_mode != MCV_FP32) return fail(MCV_EINVAL, "bad fp_mode");
  if (std::isnan(s->min_prob)) return fail(MCV_EINVAL, "min_prob is NaN");
  S->ns = s->n_scatterers;
  S->max_orders = s->max_orders;
  S->min_prob = s->min_prob;
  bool need_sqe = false, need_bvk = false, need_phonon = false, need_bragg = false;
  bool need_disp = false;
  for (int j = 0; j < s->n_scatterers; ++j) {
    const mcv_scatterer& a = s->scat[j];
    mcv::ScatP<double>& d = S->s[j];
    for (double x : {a.dims[0], a.dims[1], a.dims[2], a.rot_y_rad, a.n_per_A3, a.sig_abs_b,
                     a.kernel_sig_b[0], a.kernel_sig_b[1]})
      if (!is_finite(x)) return fail(MCV_EINVAL, "scatterer parameter is not finite");
    if (a.n_per_A3 < 0 || a.sig_abs_b < 0) return fail(MCV_EINVAL, "negative density or cross section");
    if (a.n_kernels < 1 || a.n_kernels > 2) return fail(MCV_EINVAL, "n_kernels must be 1 or 2");
    double sig = 0.0;
    for (int k = 0; k < a.n_kernels; ++k) {
      if (a.kernel[k] != MCV_KERNEL_ISO && a.kernel[k] != MCV_KERNEL_SQE &&
          a.kernel[k] != MCV_KERNEL_BVK && a.kernel[k] != MCV_KERNEL_PHONON &&
          a.kernel[k] != MCV_KERNEL_BRAGG && a.kernel[k] != MCV_KERNEL_DISP)
        return fail(MCV_EINVAL, "unknown kernel kind");
      if (a.kernel[k] == MCV_KERNEL_DISP) need_disp = true;
      if (a.kernel[k] == MCV_KERNEL_BRAGG) {
        need_bragg = true;
        if (!(a.kernel_sig_b[k] > 0))
          return fail(MCV_EINVAL, "the Bragg kernel needs a positive nominal cross section");
      }
      if (a.kernel[k] == MCV_KERNEL_BVK) need_bvk = true;
      if (a.kernel[k] == MCV_KERNEL_PHONON) need_phonon = true;
      if (a.kernel_sig_b[k] < 0) return fail(MCV_EINVAL, "negative kernel cross section");
      if (a.kernel[k] == MCV_KERNEL_SQE) need_sqe = true;
      sig += a.kernel_sig_b[k];
    }
    d.shape = a.shape;
    d.dim0 = a.dims[0];
    d.dim1 = a.dims[1];
    d.dim2 = a.dims[2];
    if (a.shape == MCV_SHAPE_SOLID_CYL) {
      if (!(a.dims[0] > 0 && a.dims[1] > 0)) return fail(MCV_EINVAL, "cylinder needs r, h > 0");
      d.half_h = 0.5 * a.dims[1];
    } else if (a.shape == MCV_SHAPE_HOLLOW_CYL) {
      if (!(a.dims[0] >= 0 && a.dims[1] > a.dims[0] && a.dims[2] > 0))
        return fail(MCV_EINVAL, "hollow cylinder needs 0 <= r_in < r_out, h > 0");
      d.half_h = 0.5 * a.dims[2];
    } else if (a.shape == MCV_SHAPE_BLOCK) {
      if (!(a.dims[0] > 0 && a.dims[1] > 0 && a.dims[2] > 0))
        return fail(MCV_EINVAL, "block needs positive sides");
    } else {
      return fail(MCV_EINVAL, "unknown shape");
    }
    d.cos_rot = std::cos(a.rot_y_rad);
    d.sin_rot = std::sin(a.rot_y_rad);
    d.nk = a.n_kernels;
    d.ktype0 = a.kernel[0];
    d.ktype1 = a.n_kernels == 2 ? a.kernel[1] : a.kernel[0];
    d.ksig0 = a.kernel_sig_b[0];
    d.ksig1 = a.n_kernels == 2 ? a.kernel_sig_b[1] : a.kernel_sig_b[0];
    d.ksig_sum = a.n_kernels == 2 ? a.kernel_sig_b[0] + a.kernel_sig_b[1] : a.kernel_sig_b[0];
    d.sig_s = sig;
    d.n100 = 100.0 * a.n_per_A3;
    d.mu_s = 100.0 * a.n_per_A3 * sig;
    d.sab2200 = a.sig_abs_b * 2200.0;
  }
  if (need_sqe) {
    const mcv_sqe& q = s->sqe;
    if (!q.table || q.nq <= 0 || q.ne <= 0) return fail(MCV_EINVAL, "S(Q,E) table missing");
    if ((int64_t)q.nq * q.ne > (int64_t)1 << 30) return fail(MCV_EINVAL, "S(Q,E) table too large");
    if (!(q.q_max > 0 && q.e_max > q.e_min && is_finite(q.q_max) && is_finite(q.e_min) && is_finite(q.e_max)))
      return fail(MCV_EINVAL, "bad S(Q,E) grid");
    S->sqe = q.table;
    S->nq = q.nq;
    S->ne = q.ne;
    S->q_max = q.q_max;
    S->e_min = q.e_min;
    S->e_max = q.e_max;
    S->dq = q.q_max / q.nq;
    S->de = (q.e_max - q.e_min) / q.ne;
    S->has_sqe = 1;
  }
  if (need_bvk) {
    const mcv_bvk& b = s->bvk;
    for (double x : {b.phi_Nm, b.mass_u, b.a_A, b.msd_A2, b.temperature_K})
      if (!is_finite(x)) return fail(MCV_EINVAL, "Born-von Karman parameter is not finite");
    if (!(b.phi_Nm > 0 && b.mass_u > 0 && b.a_A > 0 && b.temperature_K > 0 && b.msd_A2 >= 0))
      return fail(MCV_EINVAL, "bad Born-von Karman parameters");
    const double kAtomicMass = 1.66053906660e-27, kBoltzmann = 1.380649e-23;
    const double mev_per_j = 1.0 / (mcv::kElemCharge * 1e-3);
    const double M = b.mass_u * kAtomicMass;
    S->has_bvk = 1;
    S->bvk_coef = b.phi_Nm / M;
    S->bvk_ah = 0.5 * b.a_A;
    S->bvk_hb2m = mcv::kHbar * mcv::kHbar / (2.0 * M) * 1e20 * mev_per_j;
    S->bvk_kT = kBoltzmann * b.temperature_K * mev_per_j;
    S->bvk_msd = b.msd_A2;
    S->bvk_wmax = mcv::kHbar * std::sqrt(24.0 * S->bvk_coef) * mev_per_j;
    S->bvk_hwu = mcv::kHbar * std::sqrt(S->bvk_coef) * mev_per_j;
  }
  if (need_phonon) {
    const mcv_phonon& p = s->phonon;
    const int64_t bytes = mcv_phonon_table_bytes(p.n_modes, p.n_max);
    if (!p.tables || bytes == 0) return fail(MCV_EINVAL, "phonon tables missing (mcv_phonon_build)");
    if (!(p.de_mev > 0 && is_finite(p.de_mev) && p.gamma0 > 0 && is_finite(p.gamma0) &&
          p.c_w > 0 && is_finite(p.c_w)))
      return fail(MCV_EINVAL, "bad phonon description (build it with mcv_phonon_build)");
    double ps = 0.0;
    for (int c = 0; c < 3; ++c) {
      if (!(p.p[c] > 0) || !is_finite(p.p[c])) return fail(MCV_EINVAL, "bad phonon channel probabilities");
      ps += p.p[c];
    }
    if (std::fabs(ps - 1.0) > 1e-12) return fail(MCV_EINVAL, "phonon channel probabilities must sum to 1");
    const int J = p.n_modes, N = p.n_max, M = 2 * N * J + 1;
    const double* base = static_cast<const double*>(p.tables);
    S->has_phonon = 1;
    S->ph_J = J;
    S->ph_N = N;
    S->ph_M = M;
    S->ph_cdf1 = base;
    S->ph_cdfb = base + (2 * J + 1);
    S->ph_b = S->ph_cdfb + M;
    S->ph_an = S->ph_b + M;
    S->ph_de = p.de_mev;
    S->ph_cw = p.c_w;
    S->ph_p0 = p.p[0];
    S->ph_p1 = p.p[1];
    S->ph_p2 = p.p[2];
    S->ph_p01 = p.p[0] + p.p[1];
  }
  if (need_bragg) {
    const mcv_bragg& b = s->bragg;
    if (!b.tables || mcv_bragg_table_bytes(b.n) == 0)
      return fail(MCV_EINVAL, "Bragg tables missing (mcv_bragg_build)");
    S->has_bragg = 1;
    S->n_refl = b.n;
    S->refl_d = static_cast<const double*>(b.tables);
    S->refl_c = S->refl_d + b.n;
  }
  if (need_disp) {
    const mcv_dispersion& q = s->dispersion;
    if (!(q.amp_mev > 0 && is_finite(q.amp_mev) && q.c_A > 0 && is_finite(q.c_A) &&
          q.s0 >= 0 && is_finite(q.s0)))
      return fail(MCV_EINVAL, "bad dispersion surface (amp_mev > 0, c_A > 0, s0 >= 0)");
    S->has_disp = 1;
    S->disp_amp = q.amp_mev;
    S->disp_c = q.c_A;
    S->disp_s0 = q.s0;
  }
  S->wide = (need_bvk || need_phonon || need_bragg || need_disp) ? 1 : 0;
  return MCV_OK;
}

mcv_status build_detector(const mcv_detector* d, mcv::DetP<double>* D) {
  if (!d) return fail(MCV_EINVAL, "detector is NULL");
  std::memset(D, 0, sizeof(*D));
  if (d->kind != MCV_DET_SURFACE && d->kind != MCV_DET_TUBES)
    return fail(MCV_EINVAL, "unknown detector kind");
  if (d->n_tof < 1 || !(d->tof_max_s > d->tof_min_s) || !is_finite(d->tof_min_s) || !is_finite(d->tof_max_s))
    return fail(MCV_EINVAL, "bad tof binning");
  if (!(d->radius_m > 0) || !is_finite(d->radius_m)) return fail(MCV_EINVAL, "bad detector radius");
  D->kind = d->kind;
  D->radius = d->radius_m;
  if (d->multi_tube != 0 && d->multi_tube != 1) return fail(MCV_EINVAL, "multi_tube must be 0 or 1");
  D->multi_tube = d->kind == MCV_DET_TUBES ? d->multi_tube : 0;
  D->win = tof_window(d->tof_min_s, d->tof_max_s, d->n_tof);
  int64_t npix = 0;
  if (d->kind == MCV_DET_SURFACE) {
    if (d->n_phi < 1 || d->n_y < 1 || !(d->height_m > 0) || !is_finite(d->height_m))
      return fail(MCV_EINVAL, "bad surface detector");
    D->height = d->height_m;
    D->half_h = 0.5 * d->height_m;
    D->n_phi = d->n_phi;
    D->n_y = d->n_y;
    npix = (int64_t)d->n_phi * d->n_y;
  } else {
    if (d->n_rows < 1 || d->n_rows > 3 || d->tubes_per_pack < 1 || d->pixels_per_tube < 1)
      return fail(MCV_EINVAL, "bad tube detector layout");
    for (double x : {d->tube_r_m, d->tube_len_m, d->tube_pitch_m, d->pack_gap_m, d->phi0_rad,
                     d->he3_n_per_A3, d->he3_sig_abs_b})
      if (!is_finite(x)) return fail(MCV_EINVAL, "tube parameter is not finite");
    if (!(d->tube_r_m > 0 && d->tube_len_m > 0 && d->tube_pitch_m > 0 && d->pack_gap_m >= 0 &&
          d->he3_n_per_A3 > 0 && d->he3_sig_abs_b > 0))
      return fail(MCV_EINVAL, "bad tube dimensions or gas");
    int max_packs = 0, off = 0;
    for (int i = 0; i < d->n_rows; ++i) {
      if (d->packs[i] < 1) return fail(MCV_EINVAL, "a row needs at least one pack");
      if (!is_finite(d->row_y_m[i])) return fail(MCV_EINVAL, "row height is not finite");
      D->packs[i] = d->packs[i];
      D->row_y[i] = d->row_y_m[i];
      D->row_off[i] = off;
      off += d->packs[i];
      if (d->packs[i] > max_packs) max_packs = d->packs[i];
    }
    if ((int64_t)max_packs * d->tubes_per_pack > MCV_MAX_TUBES_PER_ROW)
      return fail(MCV_EINVAL, "more than 512 tubes in a row");
    D->n_rows = d->n_rows;
    D->tubes_per_pack = d->tubes_per_pack;
    D->pixels_per_tube = d->pixels_per_tube;
    D->max_tubes_row = max_packs * d->tubes_per_pack;
    D->tube_r = d->tube_r_m;
    D->half_len = 0.5 * d->tube_len_m;
    D->pitch = d->tube_pitch_m;
    D->period = d->tubes_per_pack * d->tube_pitch_m + d->pack_gap_m;
    D->phi0 = d->phi0_rad;
    D->pix_len = d->tube_len_m / d->pixels_per_tube;
    D->mu_he_v = 100.0 * d->he3_n_per_A3 * d->he3_sig_abs_b * 2200.0;
    for (int c = 0; c < D->max_tubes_row; ++c) {
      const int pc = c / d->tubes_per_pack, tc = c % d->tubes_per_pack;
      const double phic =
          d->phi0_rad + (pc * D->period + (tc + 0.5) * d->tube_pitch_m) / d->radius_m;
      D->tube_u[2 * c] = std::sin(phic);
      D->tube_u[2 * c + 1] = std::cos(phic);
    }
    npix = (int64_t)off * d->tubes_per_pack * d->pixels_per_tube;
  }
  if (npix > ((int64_t)1 << 31) - 1) return fail(MCV_EINVAL, "too many pixels");
  D->n_bins = npix * d->n_tof;
  set_det_miss_bounds(-1.0, D);  // off until the packets are known to start in a sample
  return MCV_OK;
}

// Footprint bounds beyond which a neutron misses the sample for every divergence the
// uniforms can give: the sample lies within radius r of the vertical axis and |y| <= hh; a
// ray from the start plane z = -z0 with divergence angles |a| <= 8.66 div (Box-Muller
// normals of uniforms >= 2^-54 stay within 8.65) moves sideways by at most
// (z0 + r) tan(8.66 div) before it has passed the sample.  With a 1 % and 1 um margin.
void set_miss_bounds(const mcv::SampleP<double>& S, mcv::BeamP<double>* B) {
  B->x_safe = INFINITY;
  B->y_safe = INFINITY;
  // only for a start plane upstream of the sample centre and energies that are all positive
  if (!B->energy_positive || !(B->z0 >= 0.0)) return;
  double r = 0.0, hh = 0.0;
  for (int j = 0; j < S.ns; ++j) {
    const mcv::ScatP<double>& c = S.s[j];
    double rj = 0.0, hj = 0.0;
    if (c.shape == MCV_SHAPE_SOLID_CYL) {
      rj = c.dim0;
      hj = 0.5 * c.dim1;
    } else if (c.shape == MCV_SHAPE_HOLLOW_CYL) {
      rj = c.dim1;
      hj = 0.5 * c.dim2;
    } else {
      rj = 0.5 * std::hypot(c.dim0, c.dim2);
      hj = 0.5 * c.dim1;
    }
    r = std::max(r, rj);
    hh = std::max(hh, hj);
  }
  const double a = 8.66 * B->div;
  if (!(a < 1.0)) return;
  const double shift = (B->z0 + r) * std::tan(a) * 1.01 + 1e-6;
  B->x_safe = r + shift;
  B->y_safe = hh + shift;
}

// radius of a cylinder about the y axis that holds every scatterer of the sample
double sample_radius(const mcv::SampleP<double>& S) {
  double r = 0.0;
  for (int j = 0; j < S.ns; ++j) {
    const mcv::ScatP<double>& c = S.s[j];
    if (c.shape == MCV_SHAPE_SOLID_CYL)
      r = std::max(r, c.dim0);
    else if (c.shape == MCV_SHAPE_HOLLOW_CYL)
      r = std::max(r, c.dim1);
    else
      r = std::max(r, 0.5 * std::hypot(c.dim0, c.dim2));
  }
  return r;
}

// Sure-miss bounds of the tube system for packets that start inside a sample of radius
// r_s (every scattered packet does).  Height: the tubes' vertical extent, 1 mm margin; the
// horizontal path to the tube ring is at least R - r_t - 1 mm minus the start's |x| + |z|.
// Direction: the arc of tube centres widened by the tube radius, by the angle the sample's
// extent subtends at the ring (asin(r_s / (R - r_t))) and by 1 mrad; off when it comes
// within 10 mrad of half a turn.  The bounds only skip packets the detector trace would find missing.
void set_det_miss_bounds(double r_s, mcv::DetP<double>* D) {
  D->miss_r_in = 0.0;
  D->miss_y_top = INFINITY;
  D->miss_y_bot = -INFINITY;
  D->miss_phi = 0;
  if (D->kind != MCV_DET_TUBES || !(r_s >= 0.0)) return;
  const double r_in = D->radius - D->tube_r - 1e-3;
  if (!(r_in > 2.0 * r_s)) return;
  double top = -INFINITY, bot = INFINITY;
  int packs = 0;
  for (int i = 0; i < D->n_rows; ++i) {
    top = std::max(top, D->row_y[i] + D->half_len);
    bot = std::min(bot, D->row_y[i] - D->half_len);
    packs = std::max(packs, D->packs[i]);
  }
  D->miss_r_in = r_in;
  D->miss_y_top = top + 1e-3;
  D->miss_y_bot = bot - 1e-3;
  const double widen = std::asin(std::min(1.0, r_s / r_in)) +
                       std::asin(std::min(1.0, D->tube_r / r_in)) + 1e-3;
  const double lo = D->phi0 - widen;
  const double hi = D->phi0 + packs * D->period / D->radius + widen;
  if (!(hi - lo < mcv::kPi - 0.01)) return;  // the two-sided test holds for arcs under a half turn
  D->miss_phi = 1;
  D->miss_a_x = std::sin(lo);
  D->miss_a_z = std::cos(lo);
  D->miss_b_x = std::sin(hi);
  D->miss_b_z = std::cos(hi);
}

// float copies of the parameter blocks for the FP32 kernels
void cast_beam(const mcv::BeamP<double>& d, mcv::BeamP<float>* f) {
  f->ei = (float)d.ei;
  f->rel = (float)d.rel;
  f->div = (float)d.div;
  f->width = (float)d.width;
  f->height = (float)d.height;
  f->z0 = (float)d.z0;
  f->l1 = (float)d.l1;
  f->speed0 = (float)d.speed0;
  f->t0 = d.t0;
  f->t0_hi = d.t0_hi;
  f->t0_lo = d.t0_lo;
  f->energy_positive = d.energy_positive;
  // rounded up: the float bounds stay on the safe side
  f->x_safe = (float)d.x_safe;
  if ((double)f->x_safe < d.x_safe) f->x_safe = std::nextafter(f->x_safe, INFINITY);
  f->y_safe = (float)d.y_safe;
  if ((double)f->y_safe < d.y_safe) f->y_safe = std::nextafter(f->y_safe, INFINITY);
}

void cast_sample(const mcv::SampleP<double>& d, mcv::SampleP<float>* f) {
  f->ns = d.ns;
  f->max_orders = d.max_orders;
  f->nq = d.nq;
  f->ne = d.ne;
  f->has_sqe = d.has_sqe;
  f->min_prob = (float)d.min_prob;
  for (int j = 0; j < MCV_MAX_SCATTERERS; ++j) {
    const mcv::ScatP<double>& a = d.s[j];
    mcv::ScatP<float>& b = f->s[j];
    b.shape = a.shape;
    b.nk = a.nk;
    b.ktype0 = a.ktype0;
    b.ktype1 = a.ktype1;
    b.dim0 = (float)a.dim0;
    b.dim1 = (float)a.dim1;
    b.dim2 = (float)a.dim2;
    b.half_h = (float)a.half_h;
    b.cos_rot = (float)a.cos_rot;
    b.sin_rot = (float)a.sin_rot;
    b.n100 = (float)a.n100;
    b.sig_s = (float)a.sig_s;
    b.sab2200 = (float)a.sab2200;
    b.mu_s = (float)a.mu_s;
    b.ksig0 = (float)a.ksig0;
    b.ksig1 = (float)a.ksig1;
    b.ksig_sum = (float)a.ksig_sum;
  }
  f->sqe = d.sqe;
  f->q_max = (float)d.q_max;
  f->e_min = (float)d.e_min;
  f->e_max = (float)d.e_max;
  f->dq = (float)d.dq;
  f->de = (float)d.de;
  f->has_bvk = d.has_bvk;
  f->bvk_coef = (float)d.bvk_coef;
  f->bvk_ah = (float)d.bvk_ah;
  f->bvk_hb2m = (float)d.bvk_hb2m;
  f->bvk_kT = (float)d.bvk_kT;
  f->bvk_msd = (float)d.bvk_msd;
  f->bvk_wmax = (float)d.bvk_wmax;
  f->bvk_hwu = (float)d.bvk_hwu;
  f->has_phonon = d.has_phonon;
  f->ph_J = d.ph_J;
  f->ph_N = d.ph_N;
  f->ph_M = d.ph_M;
  if (d.has_phonon) {
    // the float copy of the tables follows the double one (mcv_phonon_build)
    const int64_t T = (2 * (int64_t)d.ph_J + 1) + 2 * (int64_t)d.ph_M + (int64_t)(d.ph_N - 1) * d.ph_M;
    const float* fb = reinterpret_cast<const float*>(d.ph_cdf1 + T);
    f->ph_cdf1 = fb;
    f->ph_cdfb = fb + (d.ph_cdfb - d.ph_cdf1);
    f->ph_b = fb + (d.ph_b - d.ph_cdf1);
    f->ph_an = fb + (d.ph_an - d.ph_cdf1);
  }
  f->ph_de = (float)d.ph_de;
  f->ph_cw = (float)d.ph_cw;
  f->ph_p0 = (float)d.ph_p0;
  f->ph_p1 = (float)d.ph_p1;
  f->ph_p2 = (float)d.ph_p2;
  f->ph_p01 = (float)d.ph_p01;
  f->has_disp = d.has_disp;
  f->disp_amp = (float)d.disp_amp;
  f->disp_c = (float)d.disp_c;
  f->disp_s0 = (float)d.disp_s0;
  f->has_bragg = d.has_bragg;
  f->n_refl = d.n_refl;
  if (d.has_bragg) {
    // the float copies follow the doubles (mcv_bragg_build)
    const float* fb = reinterpret_cast<const float*>(d.refl_d + 2 * (int64_t)d.n_refl);
    f->refl_d = fb;
    f->refl_c = fb + d.n_refl;
  }
  f->wide = d.wide;
}

void cast_detector(const mcv::DetP<double>& d, mcv::DetP<float>* f) {
  f->kind = d.kind;
  f->multi_tube = d.multi_tube;
  f->n_phi = d.n_phi;
  f->n_y = d.n_y;
  f->n_rows = d.n_rows;
  for (int i = 0; i < 3; ++i) {
    f->packs[i] = d.packs[i];
    f->row_off[i] = d.row_off[i];
    f->row_y[i] = (float)d.row_y[i];
  }
  f->tubes_per_pack = d.tubes_per_pack;
  f->pixels_per_tube = d.pixels_per_tube;
  f->max_tubes_row = d.max_tubes_row;
  f->n_bins = d.n_bins;
  f->radius = (float)d.radius;
  f->height = (float)d.height;
  f->half_h = (float)d.half_h;
  f->tube_r = (float)d.tube_r;
  f->half_len = (float)d.half_len;
  f->pitch = (float)d.pitch;
  f->period = (float)d.period;
  f->phi0 = (float)d.phi0;
  f->pix_len = (float)d.pix_len;
  f->mu_he_v = (float)d.mu_he_v;
  f->win = d.win;
  f->miss_r_in = (float)d.miss_r_in;
  f->miss_y_top = (float)d.miss_y_top;
  f->miss_y_bot = (float)d.miss_y_bot;
  f->miss_phi = d.miss_phi;
  f->miss_a_x = (float)d.miss_a_x;
  f->miss_a_z = (float)d.miss_a_z;
  f->miss_b_x = (float)d.miss_b_x;
  f->miss_b_z = (float)d.miss_b_z;
  for (int i = 0; i < 2 * MCV_MAX_TUBES_PER_ROW; ++i) f->tube_u[i] = (float)d.tube_u[i];
}

void cast_all(mcv::TraceArgs* A) {
  cast_beam(A->Bd, &A->Bf);
  cast_sample(A->Sd, &A->Sf);
  cast_detector(A->Dd, &A->Df);
}

bool neutrons_ok(const mcv_neutrons* a, bool need_ids) {
  if (!a) return false;
  if (!a->x || !a->y || !a->z || !a->vx || !a->vy || !a->vz || !a->t || !a->w) return false;
  if (need_ids && (!a->id || !a->order)) return false;
  return a->n >= 0;
}

int ns_index(int ns) { return ns <= 1 ? 0 : (ns == 2 ? 1 : 2); }

mcv_status check_ctx(mcv_ctx* ctx) {
  if (!ctx) return fail(MCV_EINVAL, "context is NULL");
  int cur = -1;
  cudaError_t e = cudaGetDevice(&cur);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (cur != ctx->device) {
    e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  }
  return MCV_OK;
}

mcv_status event_sink(const mcv_event_list* l, uint32_t tag, mcv::EvSink* out) {
  if (!l->count || !l->pixel || !l->sim || !l->tof || !l->w || l->capacity < 0)
    return fail(MCV_EINVAL, "an event list needs its four arrays, a counter and capacity >= 0");
  *out = mcv::EvSink{l->pixel, l->sim, l->tof, l->w, l->capacity, l->count, tag};
  return MCV_OK;
}

int grid_for(mcv_ctx* ctx, int64_t items, int per_sm) {
  const int64_t full = (int64_t)ctx->sm_count * per_sm;
  const int64_t need = (items + mcv::trace_threads() - 1) / mcv::trace_threads();
  int64_t g = need < full ? need : full;
  return (int)(g < 1 ? 1 : g);
}

PhiloxKeys philox_keys(uint32_t seed, uint32_t sim_id) {
  PhiloxKeys K;
  uint32_t k0 = seed, k1 = sim_id;
  for (int r = 0; r < 10; ++r) {
    K.k0[r] = k0;
    K.k1[r] = k1;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return K;
}

TofWin tof_window(double tof_min_s, double tof_max_s, int n_tof) {
  TofWin w;
  w.n_tof = n_tof;
  w.tof_min = tof_min_s;
  w.dt = (tof_max_s - tof_min_s) / n_tof;
  w.inv_dt = (float)(1.0 / w.dt);
  w.tmin_hi = (float)tof_min_s;
  w.tmin_lo = (float)(tof_min_s - (double)w.tmin_hi);
  return w;
}

}  // namespace host
}  // namespace mcv

using namespace mcv::host;

namespace mcv {
void set_last_error(const std::string& msg) { g_last_error = msg; }

// the parameter blocks of a gradient call (sample, beam, detector), in both real types
mcv_status build_trace_args_for_grad(const mcv_sample* sample, const mcv_beam_params* beam,
                                     const mcv_detector* det, TraceArgs* A) {
  mcv_status st = build_sample(sample, &A->Sd);
  if (st != MCV_OK) return st;
  st = build_beam(beam, &A->Bd);
  if (st != MCV_OK) return st;
  set_miss_bounds(A->Sd, &A->Bd);
  st = build_detector(det, &A->Dd);
  if (st != MCV_OK) return st;
  set_det_miss_bounds(sample_radius(A->Sd), &A->Dd);
  cast_all(A);
  return MCV_OK;
}
}  // namespace mcv

extern "C" {

const char* mcv_last_error(void) { return g_last_error.c_str(); }

mcv_status mcv_create(int device, mcv_ctx** out) {
  if (!out) return fail(MCV_EINVAL, "out is NULL");
  *out = nullptr;
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
  if (device < 0 || device >= count) return fail(MCV_EINVAL, "no such device");
  e = cudaSetDevice(device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  mcv_ctx* c = new mcv_ctx();
  c->device = device;
  e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) {
    delete c;
    return cuda_fail(e, "cudaDeviceGetAttribute");
  }
  e = cudaMalloc(&c->d_err, 256);
  if (e != cudaSuccess) {
    delete c;
    return alloc_fail("cannot allocate the context's device block");
  }
  e = cudaMemset(c->d_err, 0, 256);
  if (e != cudaSuccess) {
    cudaFree(c->d_err);
    delete c;
    return cuda_fail(e, "cudaMemset");
  }
  std::memset(c->occ, 0, sizeof(c->occ));
  std::memset(c->occ_adj, 0, sizeof(c->occ_adj));
  std::memset(c->tuned, 0, sizeof(c->tuned));
  *out = c;
  return MCV_OK;
}

mcv_status mcv_destroy(mcv_ctx* ctx) {
  if (!ctx) return MCV_OK;
  cudaSetDevice(ctx->device);
  cudaFree(ctx->d_err);
  delete ctx;
  return MCV_OK;
}

mcv_status mcv_sync(mcv_ctx* ctx, void* stream) {
  if (!ctx) return mcv::noalloc_sync(static_cast<cudaStream_t>(stream));
  mcv_status st = check_ctx(ctx);
  if (st != MCV_OK) return st;
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  int flag = 0;
  e = cudaMemcpy(&flag, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy");
  if (flag) {
    cudaMemset(ctx->d_err, 0, sizeof(int));
    return fail(MCV_EDEVICE,
                "a kernel found an out-of-range index, a packet order above 7 or a target bin "
                "that is negative or not finite");
  }
  return MCV_OK;
}

int64_t mcv_detector_pixels(const mcv_detector* det) {
  mcv::DetP<double> D;
  if (build_detector(det, &D) != MCV_OK) return 0;
  return D.n_bins / D.win.n_tof;
}

mcv_status mcv_bench_atomics(mcv_ctx* ctx, double* hist, int64_t n_bins, int64_t n_adds,
                             uint64_t seed, void* stream) {
  mcv::host::CallRange range_("mcv_bench_atomics");
  mcv_status st = check_ctx(ctx);
  if (st != MCV_OK) return st;
  if (n_bins < 1 || n_adds < 0 || !hist) return fail(MCV_EINVAL, "bad histogram or count");
  cudaError_t e = mcv::launch_atomics(hist, n_bins, n_adds, seed, ctx->sm_count * 16,
                                      static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "atomics kernel launch");
  return MCV_OK;
}

mcv_status mcv_zero(mcv_ctx* ctx, double* dst, int64_t n, void* stream) {
  mcv_status st = check_ctx(ctx);
  if (st != MCV_OK) return st;
  if (n < 0 || (n > 0 && !dst)) return fail(MCV_EINVAL, "bad buffer");
  cudaError_t e = mcv::launch_zero(dst, n, ctx->sm_count * 8, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "zero kernel launch");
  return MCV_OK;
}

mcv_status mcv_beam(mcv_ctx* ctx, const mcv_beam_params* beam, int fp_mode, uint32_t seed,
                    uint32_t sim_id, int64_t first_id, int64_t n, mcv_neutrons* out,
                    void* stream) {
  mcv::host::CallRange range_("mcv_beam");
  mcv_status st = check_ctx(ctx);
  if (st != MCV_OK) return st;
  if (fp_mode != MCV_FP64 && fp_mode != MCV_FP32) return fail(MCV_EINVAL, "bad fp_mode");
  if (n < 0 || n > kMaxNeutrons || first_id < 0 || first_id > (((int64_t)1 << 62) - n))
    return fail(MCV_EINVAL, "bad neutron range");
  if (!neutrons_ok(out, false) || out->n < n) return fail(MCV_EINVAL, "bad output arrays");
  mcv::TraceArgs A;
  std::memset(&A, 0, sizeof(A));
  st = build_beam(beam, &A.Bd);
  if (st != MCV_OK) return st;
  if (n == 0) return MCV_OK;
  A.seed = seed;
  A.sim_id = sim_id;
  A.keys = philox_keys(seed, sim_id);
  A.first_id = first_id;
  A.n = n;
  A.pk_x = out->x;
  A.pk_y = out->y;
  A.pk_z = out->z;
  A.pk_vx = out->vx;
  A.pk_vy = out->vy;
  A.pk_vz = out->vz;
  A.pk_w = out->w;
  A.pk_t = out->t;
  A.pk_id = out->id;
  A.pk_order = out->order;
  cast_all(&A);
  cudaError_t e = mcv::launch_beam(A, fp_mode, grid_for(ctx, n, 16), static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "beam kernel launch");
  return MCV_OK;
}

mcv_status mcv_trace_sample(mcv_ctx* ctx, const mcv_sample* sample, const mcv_beam_params* beam,
                            const mcv_neutrons* in, uint32_t seed, uint32_t sim_id,
                            int64_t first_id, int64_t n, const mcv_detector* det, mcv_hist* hist,
                            mcv_neutrons* packets, void* stream) {
  mcv::host::CallRange range_("mcv_trace_sample");
  mcv_status st = check_ctx(ctx);
  if (st != MCV_OK) return st;
  mcv::TraceArgs A;
  std::memset(&A, 0, sizeof(A));
  st = build_sample(sample, &A.Sd);
  if (st != MCV_OK) return st;
  if (n < 0 || n > kMaxNeutrons || first_id < 0 || first_id > (((int64_t)1 << 62) - n))
    return fail(MCV_EINVAL, "bad neutron range");
  if (in) {
    if (!neutrons_ok(in, false) || in->n < n) return fail(MCV_EINVAL, "bad input arrays");
  } else {
    st = build_beam(beam, &A.Bd);
    if (st != MCV_OK) return st;
    set_miss_bounds(A.Sd, &A.Bd);
  }
  const bool fused = det != nullptr;
  if (fused) {
    st = build_detector(det, &A.Dd);
    if (st != MCV_OK) return st;
    // generated neutrons: every detected packet starts at a scattering point in the sample
    if (!in) set_det_miss_bounds(sample_radius(A.Sd), &A.Dd);
    if (!hist || (!hist->counts && !hist->tallies))
      return fail(MCV_EINVAL, "a detector needs a histogram or tallies");
  }
  if (packets) {
    if (!neutrons_ok(packets, true)) return fail(MCV_EINVAL, "bad packet arrays");
    if (packets->n / (A.Sd.max_orders + 1) < n) return fail(MCV_EINVAL, "too few packet slots");
  }
  if (!fused && !packets && !(hist && hist->tallies))
    return fail(MCV_EINVAL, "no output requested");
  if (hist && hist->events) {
    if (!fused) return fail(MCV_EINVAL, "an event list needs a detector");
    st = event_sink(hist->events, sim_id, &A.ev);
    if (st != MCV_OK) return st;
  }
  const bool paper = sample->estimator == MCV_EST_PAPER;
  if (sample->estimator != MCV_EST_CHAIN && !paper) return fail(MCV_EINVAL, "unknown estimator");
  if (paper && (!fused || in || packets))
    return fail(MCV_EINVAL, "the paper estimator needs a detector and a histogram, and takes no "
                            "stored beam or packet slots");
  if (n == 0) return MCV_OK;
  A.seed = seed;
  A.sim_id = sim_id;
  A.keys = philox_keys(seed, sim_id);
  A.pkeys = philox_keys(seed, sim_id ^ 0x80000000u);
  A.first_id = first_id;
  A.n = n;
  A.stop_on_zero = 1;
  if (hist) {
    A.hist = fused ? hist->counts : nullptr;
    A.tallies = hist->tallies;
  }
  if (in) {
    A.in_x = in->x;
    A.in_y = in->y;
    A.in_z = in->z;
    A.in_vx = in->vx;
    A.in_vy = in->vy;
    A.in_vz = in->vz;
    A.in_w = in->w;
    A.in_t = in->t;
    A.in_id = in->id;
  }
  if (packets) {
    A.pk_x = packets->x;
    A.pk_y = packets->y;
    A.pk_z = packets->z;
    A.pk_vx = packets->vx;
    A.pk_vy = packets->vy;
    A.pk_vz = packets->vz;
    A.pk_w = packets->w;
    A.pk_t = packets->t;
    A.pk_id = packets->id;
    A.pk_order = packets->order;
  }
  A.err = ctx->d_err;
  const int detk = fused ? A.Dd.kind : MCV_DET_NONE;
  const int fp = sample->fp_mode;
  if (paper) {
    cast_all(&A);
    // one neutron per thread; the thread's stack of packets lives in local memory
    cudaError_t e = mcv::launch_paper(A, fp, detk, ctx->sm_count * 16,
                                      static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "paper kernel launch");
    return MCV_OK;
  }
  int& occ = ctx->occ[fp][ns_index(A.Sd.ns)][detk][A.Sd.wide ? 1 : 0];
  if (occ == 0) {
    cudaError_t e = mcv::trace_blocks_per_sm(fp, A.Sd.ns, detk, A.Sd.wide, &occ);
    if (e != cudaSuccess || occ < 1) occ = 1;
  }
  const int grid = grid_for(ctx, n, occ);
  cast_all(&A);
  cudaError_t e = mcv::launch_trace(A, fp, detk, grid, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "trace kernel launch");
  return MCV_OK;
}

mcv_status mcv_detect(mcv_ctx* ctx, const mcv_detector* det, int fp_mode,
                      const mcv_neutrons* packets, uint32_t seed, uint32_t sim_id, mcv_hist* hist,
                      mcv_events* events, void* stream) {
  mcv::host::CallRange range_("mcv_detect");
  mcv_status st = check_ctx(ctx);
  if (st != MCV_OK) return st;
  if (fp_mode != MCV_FP64 && fp_mode != MCV_FP32) return fail(MCV_EINVAL, "bad fp_mode");
  mcv::TraceArgs A;
  std::memset(&A, 0, sizeof(A));
  st = build_detector(det, &A.Dd);
  if (st != MCV_OK) return st;
  if (!neutrons_ok(packets, true)) return fail(MCV_EINVAL, "bad packet arrays (id and order required)");
  if (!hist && !events) return fail(MCV_EINVAL, "no output requested");
  if (hist && hist->events) {
    st = event_sink(hist->events, sim_id, &A.ev);
    if (st != MCV_OK) return st;
  }
  if (packets->n == 0) return MCV_OK;
  A.seed = seed;
  A.sim_id = sim_id;
  A.keys = philox_keys(seed, sim_id);
  A.n = packets->n;
  A.in_x = packets->x;
  A.in_y = packets->y;
  A.in_z = packets->z;
  A.in_vx = packets->vx;
  A.in_vy = packets->vy;
  A.in_vz = packets->vz;
  A.in_w = packets->w;
  A.in_t = packets->t;
  A.in_id = packets->id;
  A.in_order = packets->order;
  if (hist) {
    A.hist = hist->counts;
    A.tallies = hist->tallies;
  }
  A.err = ctx->d_err;
  mcv::EventsArgs E{nullptr, nullptr, nullptr, nullptr};
  if (events) E = mcv::EventsArgs{events->pixel, events->tof, events->w_det, events->bin};
  cast_all(&A);
  cudaError_t e = mcv::launch_detect(A, E, fp_mode, A.Dd.kind, grid_for(ctx, packets->n, 16),
                                     static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "detect kernel launch");
  return MCV_OK;
}

}  // extern "C"

namespace {

// What mcv_grad and mcv_adjoint share: the parameter blocks and the checks of the gradient
// outputs.
mcv_status grad_args(mcv_ctx* ctx, const mcv_sample* sample, const mcv_beam_params* beam,
                     const mcv_detector* det, uint32_t seed, uint32_t sim_id, int64_t first_id,
                     int64_t n, const double* target, double scale_c, int grad_scatterer,
                     const double* hist, double* loss, double* dsqe, double* dsig,
                     mcv::TraceArgs* A) {
  mcv_status st = check_ctx(ctx);
  if (st != MCV_OK) return st;
  std::memset(A, 0, sizeof(*A));
  st = build_sample(sample, &A->Sd);
  if (st != MCV_OK) return st;
  st = build_beam(beam, &A->Bd);
  if (st != MCV_OK) return st;
  set_miss_bounds(A->Sd, &A->Bd);
  st = build_detector(det, &A->Dd);
  if (st != MCV_OK) return st;
  set_det_miss_bounds(sample_radius(A->Sd), &A->Dd);
  if (n < 0 || n > kMaxNeutrons || first_id < 0 || first_id > (((int64_t)1 << 62) - n))
    return fail(MCV_EINVAL, "bad neutron range");
  if (!target || !loss || !dsig || !hist)
    return fail(MCV_EINVAL, "the gradient needs target, the histogram, loss and dsig");
  if (A->Sd.has_sqe && !dsqe) return fail(MCV_EINVAL, "the gradient needs dsqe for an S(Q,E) sample");
  if (grad_scatterer < 0 || grad_scatterer >= A->Sd.ns)
    return fail(MCV_EINVAL, "grad_scatterer out of range");
  if (!(A->Sd.s[grad_scatterer].sig_s > 0.0))
    return fail(MCV_EINVAL, "the differentiated scatterer needs a positive cross section");
  if (!is_finite(scale_c)) return fail(MCV_EINVAL, "scale_c is not finite");
  A->seed = seed;
  A->sim_id = sim_id;
  A->keys = philox_keys(seed, sim_id);
  A->first_id = first_id;
  A->n = n;
  A->err = ctx->d_err;
  A->gs = grad_scatterer;
  cast_all(A);
  return MCV_OK;
}

// The loss of the histogram `hist` and the adjoint of the neutron range of A: clears loss,
// dsig and dsqe, then the chi-squared kernel and the adjoint kernel.
mcv_status loss_and_adjoint(mcv_ctx* ctx, mcv::TraceArgs& A, int fp, const double* hist,
                            const double* target, double scale_c, double* g_work, double* loss,
                            double* dsqe, double* dsig, cudaStream_t s) {
  const int zgrid = ctx->sm_count * 8;
  cudaError_t e = mcv::launch_zero(loss, 1, 1, s);
  if (e == cudaSuccess) e = mcv::launch_zero(dsig, 2, 1, s);
  if (e == cudaSuccess && A.Sd.has_sqe) e = mcv::launch_zero(dsqe, (int64_t)A.Sd.nq * A.Sd.ne, zgrid, s);
  if (e != cudaSuccess) return cuda_fail(e, "zero kernel launch");
  e = mcv::launch_chi2(hist, target, scale_c, A.Dd.n_bins, g_work, loss, ctx->d_err, zgrid, s);
  if (e != cudaSuccess) return cuda_fail(e, "chi2 kernel launch");
  if (A.n > 0) {
    // adjoint: the same paths, traced through zero weights
    A.hist = nullptr;
    A.tallies = nullptr;
    A.stop_on_zero = 0;
    A.g = g_work;
    A.hist_in = hist;
    A.target = target;
    A.scale_c = scale_c;
    A.dsqe = A.Sd.has_sqe ? dsqe : nullptr;
    A.dsig = dsig;
    int& occ_a = ctx->occ_adj[fp][ns_index(A.Sd.ns)][A.Dd.kind][A.Sd.wide ? 1 : 0];
    if (occ_a == 0) {
      e = mcv::adjoint_blocks_per_sm(fp, A.Sd.ns, A.Dd.kind, A.Sd.wide, &occ_a);
      if (e != cudaSuccess || occ_a < 1) occ_a = 1;
    }
    e = mcv::launch_adjoint(A, fp, A.Dd.kind, grid_for(ctx, A.n, occ_a), s);
    if (e != cudaSuccess) return cuda_fail(e, "adjoint kernel launch");
  }
  return MCV_OK;
}

}  // namespace

extern "C" {

mcv_status mcv_grad(mcv_ctx* ctx, const mcv_sample* sample, const mcv_beam_params* beam,
                    const mcv_detector* det, uint32_t seed, uint32_t sim_id, int64_t first_id,
                    int64_t n, const double* target, double scale_c, int grad_scatterer,
                    mcv_hist* hist, double* g_work, double* loss, double* dsqe, double* dsig,
                    void* stream) {
  mcv::host::CallRange range_("mcv_grad");
  mcv::TraceArgs A;
  mcv_status st = grad_args(ctx, sample, beam, det, seed, sim_id, first_id, n, target, scale_c,
                            grad_scatterer, hist ? hist->counts : nullptr, loss, dsqe, dsig, &A);
  if (st != MCV_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int zgrid = ctx->sm_count * 8;
  cudaError_t e = mcv::launch_zero(hist->counts, A.Dd.n_bins, zgrid, s);
  if (e == cudaSuccess && hist->tallies) e = mcv::launch_zero(hist->tallies, MCV_NTALLY, 1, s);
  if (e != cudaSuccess) return cuda_fail(e, "zero kernel launch");
  const int fp = sample->fp_mode;
  if (n > 0) {
    // forward: the histogram of this neutron range
    A.hist = hist->counts;
    A.tallies = hist->tallies;
    A.stop_on_zero = 1;
    int& occ = ctx->occ[fp][ns_index(A.Sd.ns)][A.Dd.kind][A.Sd.wide ? 1 : 0];
    if (occ == 0) {
      e = mcv::trace_blocks_per_sm(fp, A.Sd.ns, A.Dd.kind, A.Sd.wide, &occ);
      if (e != cudaSuccess || occ < 1) occ = 1;
    }
    e = mcv::launch_trace(A, fp, A.Dd.kind, grid_for(ctx, n, occ), s);
    if (e != cudaSuccess) return cuda_fail(e, "trace kernel launch");
  }
  return loss_and_adjoint(ctx, A, fp, hist->counts, target, scale_c, g_work, loss, dsqe, dsig, s);
}

mcv_status mcv_adjoint(mcv_ctx* ctx, const mcv_sample* sample, const mcv_beam_params* beam,
                       const mcv_detector* det, uint32_t seed, uint32_t sim_id,
                       int64_t first_id, int64_t n, const double* hist, const double* target,
                       double scale_c, int grad_scatterer, double* g_work, double* loss,
                       double* dsqe, double* dsig, void* stream) {
  mcv::host::CallRange range_("mcv_adjoint");
  mcv::TraceArgs A;
  mcv_status st = grad_args(ctx, sample, beam, det, seed, sim_id, first_id, n, target, scale_c,
                            grad_scatterer, hist, loss, dsqe, dsig, &A);
  if (st != MCV_OK) return st;
  return loss_and_adjoint(ctx, A, sample->fp_mode, hist, target, scale_c, g_work, loss, dsqe,
                          dsig, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
