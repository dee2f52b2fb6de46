// Device-side building blocks of the neutron ray-tracing hot path (MCViNE, Lin et al.):
// counter-based random numbers, ray/shape intersection, the scattering kernels, the
// detector system and the per-neutron chain of scatterings.  Everything is templated on
// the real type R (float: the FP32 fast mode, double: the FP64 mode); time of flight is
// always carried in double.
#pragma once

#include <cstdint>
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <math_constants.h>

#include "mcv_params.h"

namespace mcv {

// ---- math by real type ----------------------------------------------------------------
template <typename R>
struct Mth;

template <>
struct Mth<float> {
  static __device__ __forceinline__ float sqrt(float x) { return sqrtf(x); }
  // exp and log from the hardware approximations (a few ulp; subnormals kept, so a tiny
  // table value or weight is not flushed to zero)
  static __device__ __forceinline__ float exp(float x) { return __expf(x); }
  static __device__ __forceinline__ float log(float x) { return __logf(x); }
  static __device__ __forceinline__ float log1p(float x) { return log1pf(x); }
  static __device__ __forceinline__ float expm1(float x) { return expm1f(x); }
  // tan, sin and cos through sincospif: its argument reduction is exact and it has no long
  // slow path, and these keep their relative accuracy for small arguments
  static __device__ __forceinline__ float tan(float x) {
    float s, c;
    sincospif(x * 0.318309886f, &s, &c);
    return s / c;
  }
  static __device__ __forceinline__ float atan2(float y, float x) { return atan2f(y, x); }
  static __device__ __forceinline__ float floor(float x) { return floorf(x); }
  static __device__ __forceinline__ float fabs(float x) { return fabsf(x); }
  static __device__ __forceinline__ float fmin(float a, float b) { return fminf(a, b); }
  static __device__ __forceinline__ float fmax(float a, float b) { return fmaxf(a, b); }
  static __device__ __forceinline__ float hypot(float a, float b) { return hypotf(a, b); }
  // sin and cos of 2 pi u
  static __device__ __forceinline__ void sincos2pi(float u, float* s, float* c) {
    sincospif(2.0f * u, s, c);
  }
  static __device__ __forceinline__ float inf() { return CUDART_INF_F; }
  static __device__ __forceinline__ float cos_(float x) { return cospif(x * 0.318309886f); }
  static __device__ __forceinline__ float sin_(float x) { return sinpif(x * 0.318309886f); }
  static __device__ __forceinline__ float acos_(float x) { return acosf(x); }
};

template <>
struct Mth<double> {
  static __device__ __forceinline__ double sqrt(double x) { return ::sqrt(x); }
  static __device__ __forceinline__ double exp(double x) { return ::exp(x); }
  static __device__ __forceinline__ double log(double x) { return ::log(x); }
  static __device__ __forceinline__ double log1p(double x) { return ::log1p(x); }
  static __device__ __forceinline__ double expm1(double x) { return ::expm1(x); }
  static __device__ __forceinline__ double tan(double x) { return ::tan(x); }
  static __device__ __forceinline__ double atan2(double y, double x) { return ::atan2(y, x); }
  static __device__ __forceinline__ double floor(double x) { return ::floor(x); }
  static __device__ __forceinline__ double fabs(double x) { return ::fabs(x); }
  static __device__ __forceinline__ double fmin(double a, double b) { return ::fmin(a, b); }
  static __device__ __forceinline__ double fmax(double a, double b) { return ::fmax(a, b); }
  static __device__ __forceinline__ double hypot(double a, double b) { return ::hypot(a, b); }
  // the FP64 mode evaluates sin and cos of (2 pi) u as written
  static __device__ __forceinline__ void sincos2pi(double u, double* s, double* c) {
    ::sincos(2.0 * kPi * u, s, c);
  }
  static __device__ __forceinline__ double inf() { return CUDART_INF; }
  static __device__ __forceinline__ double cos_(double x) { return ::cos(x); }
  static __device__ __forceinline__ double sin_(double x) { return ::sin(x); }
  static __device__ __forceinline__ double acos_(double x) { return ::acos(x); }
};

// ---- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) ----------------------------------
struct Words {
  uint32_t a, b, c, d;
};

// Round keys of the ten rounds: from a table computed on the host (PhiloxKeys, kept in
// kernel parameter space, where the kernel reads them as constants), or computed from the
// key (seed, sim) as they are used (one add per round, for keys that vary between warps).
struct KeysTable {
  const PhiloxKeys* p;
  __device__ __forceinline__ KeysTable(const PhiloxKeys& k) : p(&k) {}
  __device__ __forceinline__ uint32_t key0(int r) const { return p->k0[r]; }
  __device__ __forceinline__ uint32_t key1(int r) const { return p->k1[r]; }
};

struct KeysOnTheFly {
  uint32_t s0, s1;
  __device__ __forceinline__ uint32_t key0(int r) const { return s0 + (uint32_t)r * 0x9E3779B9u; }
  __device__ __forceinline__ uint32_t key1(int r) const { return s1 + (uint32_t)r * 0xBB67AE85u; }
};

template <class KS>
__device__ __forceinline__ Words philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                          const KS& ks) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ ks.key0(round);
    const uint32_t n2 = hi0 ^ c3 ^ ks.key1(round);
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  return Words{c0, c1, c2, c3};
}

// 53 random bits -> (k + 1/2) 2^-53 in (0,1); the FP32 mode rounds the same number to float
template <typename R>
__device__ __forceinline__ R to_unit(uint32_t hi, uint32_t lo);

template <>
__device__ __forceinline__ double to_unit<double>(uint32_t hi, uint32_t lo) {
  const uint64_t k = ((uint64_t)hi << 21) | (uint64_t)(lo >> 11);
  return __fma_rn((double)k, 0x1p-53, 0x1p-54);
}

// FP32: the same 53-bit number rounded to float, built on the integer and FP32 pipes only
// (exact small-integer to float through the 2^23 bias; one rounding in the final FMA).
__device__ __forceinline__ float small_int_to_float(uint32_t v) {  // v < 2^23, exact
  return __int_as_float(0x4b000000u | v) - 8388608.0f;
}
template <>
__device__ __forceinline__ float to_unit<float>(uint32_t hi, uint32_t lo) {
  // u = (hi 2^21 + (lo >> 11) + 1/2) 2^-53 = hi 2^-32 + c,  c = (2 (lo >> 11) + 1) 2^-54
  const float h = __fmaf_rn(small_int_to_float(hi >> 16), 65536.0f, small_int_to_float(hi & 0xffffu));
  const float c = small_int_to_float(((lo >> 11) << 1) | 1u) * 0x1p-54f;
  return fminf(__fmaf_rn(h, 0x1p-32f, c), 0x1.fffffep-1f);
}

// The stream of one neutron: key (seed, sim) given by its round keys, counter
// (id lo, id hi, 4*(event+1)+block, 0).
template <class KS>
struct NeutronRngT {
  KS ks;
  uint32_t n0, n1;
  __device__ __forceinline__ NeutronRngT(KS keys, int64_t nid)
      : ks(keys), n0((uint32_t)((uint64_t)nid & 0xffffffffu)),
        n1((uint32_t)((uint64_t)nid >> 32)) {}
  template <typename R>
  __device__ __forceinline__ void pair(int event, int block, R* u0, R* u1) const {
    const Words w = philox10(n0, n1, (uint32_t)(4 * (event + 1) + block), 0u, ks);
    *u0 = to_unit<R>(w.a, w.b);
    *u1 = to_unit<R>(w.c, w.d);
  }
  template <typename R>
  __device__ __forceinline__ R first(int event, int block) const {
    const Words w = philox10(n0, n1, (uint32_t)(4 * (event + 1) + block), 0u, ks);
    return to_unit<R>(w.a, w.b);
  }
};
using NeutronRng = NeutronRngT<KeysTable>;

// ---- time of flight ---------------------------------------------------------------------
// FP64 mode: a double.  FP32 mode: an unevaluated sum of two floats (48 significant bits,
// ~1e-17 s over millisecond flights) accumulated with the FP32 pipes only.
template <typename R>
struct Tof;

template <>
struct Tof<double> {
  double v;
  __device__ __forceinline__ void set(double t) { v = t; }
  __device__ __forceinline__ void add(double dt) { v = v + dt; }
  __device__ __forceinline__ double value() const { return v; }
};

template <>
struct Tof<float> {
  float hi, lo;
  __device__ __forceinline__ void set(double t) {
    hi = (float)t;
    lo = (float)(t - (double)hi);
  }
  __device__ __forceinline__ void set2(float h, float l) {
    const float s = h + l;
    lo = l - (s - h);
    hi = s;
  }
  // |dt| <= |hi| for flight increments after the start: fast two-sum
  __device__ __forceinline__ void add(float dt) {
    const float s = hi + dt;
    const float e = dt - (s - hi);
    hi = s;
    lo = lo + e;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// ---- packet state ---------------------------------------------------------------------
template <typename R>
struct Ray {
  R x, y, z;        // m
  R dx, dy, dz;     // unit direction
  R speed;          // m/s
  Tof<R> t;         // s
  R w;              // probability weight
};

// ---- parameter blocks of one real type ---------------------------------------------------
template <typename R>
__device__ __forceinline__ const SampleP<R>& Sof(const TraceArgs& A);
template <>
__device__ __forceinline__ const SampleP<float>& Sof<float>(const TraceArgs& A) { return A.Sf; }
template <>
__device__ __forceinline__ const SampleP<double>& Sof<double>(const TraceArgs& A) { return A.Sd; }
template <typename R>
__device__ __forceinline__ const DetP<R>& Dof(const TraceArgs& A);
template <>
__device__ __forceinline__ const DetP<float>& Dof<float>(const TraceArgs& A) { return A.Df; }
template <>
__device__ __forceinline__ const DetP<double>& Dof<double>(const TraceArgs& A) { return A.Dd; }
template <typename R>
__device__ __forceinline__ const BeamP<R>& Bof(const TraceArgs& A);
template <>
__device__ __forceinline__ const BeamP<float>& Bof<float>(const TraceArgs& A) { return A.Bf; }
template <>
__device__ __forceinline__ const BeamP<double>& Bof<double>(const TraceArgs& A) { return A.Bd; }

// ---- source -----------------------------------------------------------------------------
// Synthetic beam at the sample: Gaussian energy (random block 0), uniform footprint
// (block 1), Gaussian divergence (block 2).  The position and direction come first: they
// alone decide whether the neutron meets the sample, and a neutron that misses it needs no
// energy when every energy draw is positive (BeamP::energy_positive).
// aux: what the energy part needs from the direction part (FP32: tan^2 ax + tan^2 ay).
// The footprint alone already settles most misses: a neutron whose footprint lies outside
// (x_safe, y_safe) cannot reach the sample whatever its divergence (BeamP::x_safe).
template <class Rng>
__device__ __forceinline__ void beam_footprint(const BeamP<double>& B,
                                                       const Rng& rng, Ray<double>* n) {
  double u0, u1;
  rng.template pair<double>(-1, 1, &u0, &u1);
  n->x = (u0 - 0.5) * B.width;
  n->y = (u1 - 0.5) * B.height;
  n->z = -B.z0;
  n->w = 1.0;
}

template <class Rng>
__device__ __forceinline__ void beam_divergence(const BeamP<double>& B,
                                                        const Rng& rng, Ray<double>* n,
                                                        double* aux) {
  using M = Mth<double>;
  double u0, u1, s, c;
  rng.template pair<double>(-1, 2, &u0, &u1);
  M::sincos2pi(u1, &s, &c);
  const double rr = M::sqrt(-2.0 * M::log(u0));
  const double ax = B.div * (rr * c), ay = B.div * (rr * s);
  const double tx = M::tan(ax), ty = M::tan(ay);
  const double norm = M::sqrt(tx * tx + ty * ty + 1.0);
  n->dx = tx / norm;
  n->dy = ty / norm;
  n->dz = 1.0 / norm;
  *aux = 0.0;
}

template <class Rng>
__device__ __forceinline__ bool beam_energy(const BeamP<double>& B,
                                                    const Rng& rng, double,
                                                    Ray<double>* n) {
  using M = Mth<double>;
  double u0, u1, s, c;
  rng.template pair<double>(-1, 0, &u0, &u1);
  M::sincos2pi(u1, &s, &c);
  const double zE = M::sqrt(-2.0 * M::log(u0)) * c;
  const double E = B.ei * (1.0 + B.rel * zE);
  if (!(E > 0.0)) return false;
  n->speed = M::sqrt(E / kMeVPerV2);
  n->t.set((B.l1 - B.z0) / (n->speed * n->dz));
  return true;
}

// FP32: speed and the flight time to the start plane are written as the nominal values
// (computed once in FP64 on the host) times small FP32 corrections, so that the FP64 time
// keeps ~1e-12 s accuracy: speed = v0 (1 + eta), eta = d/(1 + sqrt(1 + d)), d = rel z;
// path/speed = t0 (1 + xi)/(1 + eta), xi = e/(1 + sqrt(1 + e)), e = tan^2 ax + tan^2 ay.
template <class Rng>
__device__ __forceinline__ void beam_footprint(const BeamP<float>& B,
                                                      const Rng& rng, Ray<float>* n) {
  float u0, u1;
  rng.template pair<float>(-1, 1, &u0, &u1);
  n->x = (u0 - 0.5f) * B.width;
  n->y = (u1 - 0.5f) * B.height;
  n->z = -B.z0;
  n->w = 1.0f;
}

template <class Rng>
__device__ __forceinline__ void beam_divergence(const BeamP<float>& B,
                                                       const Rng& rng, Ray<float>* n,
                                                       float* aux) {
  using M = Mth<float>;
  float u0, u1, s, c;
  rng.template pair<float>(-1, 2, &u0, &u1);
  M::sincos2pi(u1, &s, &c);
  const float rr = M::sqrt(-2.0f * M::log(u0));
  const float ax = B.div * (rr * c), ay = B.div * (rr * s);
  const float tx = M::tan(ax), ty = M::tan(ay);
  const float e = tx * tx + ty * ty;
  const float sq = M::sqrt(1.0f + e);
  n->dx = tx / sq;
  n->dy = ty / sq;
  n->dz = 1.0f / sq;
  *aux = e;
}

template <class Rng>
__device__ __forceinline__ bool beam_energy(const BeamP<float>& B,
                                                   const Rng& rng, float e,
                                                   Ray<float>* n) {
  using M = Mth<float>;
  float u0, u1, s, c;
  rng.template pair<float>(-1, 0, &u0, &u1);
  M::sincos2pi(u1, &s, &c);
  const float zE = M::sqrt(-2.0f * M::log(u0)) * c;
  const float dE = B.rel * zE;
  if (!(1.0f + dE > 0.0f)) return false;
  const float sq = M::sqrt(1.0f + e);
  const float eta = dE / (1.0f + M::sqrt(1.0f + dE));
  const float xi = e / (1.0f + sq);
  n->speed = B.speed0 * (1.0f + eta);
  n->t.set2(B.t0_hi, B.t0_lo);
  n->t.add(B.t0_hi * ((xi - eta) / (1.0f + eta)));
  return true;
}

// The whole source draw; returns false when the drawn energy is not positive (no packet).
template <typename R, class Rng>
__device__ __forceinline__ bool make_beam(const BeamP<R>& B, const Rng& rng, Ray<R>* n) {
  R aux;
  beam_footprint(B, rng, n);
  beam_divergence(B, rng, n, &aux);
  return beam_energy(B, rng, aux, n);
}

// the footprint is far enough from the sample that the neutron misses it for any divergence
template <typename R>
__device__ __forceinline__ bool surely_misses(const BeamP<R>& B, const Ray<R>& n) {
  return Mth<R>::fabs(n.x) > B.x_safe || Mth<R>::fabs(n.y) > B.y_safe;
}

// ---- geometry ----------------------------------------------------------------------------
// Line r + s d inside the infinite cylinder x^2 + z^2 < rad^2 (axis y): closest-approach
// form, squared axis distance (r x d)^2 / a with a = dx^2 + dz^2.
template <typename R>
__device__ __forceinline__ bool cyl_span(R rad, R x, R z, R dx, R dz, R* s1, R* s2) {
  using M = Mth<R>;
  const R a = dx * dx + dz * dz;
  if (a == R(0)) {
    if (x * x + z * z < rad * rad) {
      *s1 = -M::inf();
      *s2 = M::inf();
      return true;
    }
    return false;
  }
  const R tc = -(x * dx + z * dz) / a;
  const R cr = x * dz - z * dx;
  const R g = rad * rad - cr * cr / a;
  if (!(g > R(0))) return false;
  const R half = M::sqrt(g / a);
  *s1 = tc - half;
  *s2 = tc + half;
  return true;
}

// |p + s dp| < half
template <typename R>
__device__ __forceinline__ bool slab_span(R half, R p, R dp, R* s1, R* s2) {
  using M = Mth<R>;
  if (dp == R(0)) {
    if (M::fabs(p) < half) {
      *s1 = -M::inf();
      *s2 = M::inf();
      return true;
    }
    return false;
  }
  const R a = (-half - p) / dp, b = (half - p) / dp;
  *s1 = M::fmin(a, b);
  *s2 = M::fmax(a, b);
  return true;
}

template <typename R>
struct Seg {
  R a, b;
  int j;
};

// [a, b] clipped to s >= s0 (s0 = 0 but for the paper estimator's transmitted packets, which
// keep their line's origin and the distance s0 travelled along it), kept if not empty
template <typename R>
__device__ __forceinline__ void put_seg(R a, R b, int j, R s0, Seg<R>* out, int* cnt) {
  const R lo = Mth<R>::fmax(a, s0);
  if (b > lo) {
    out[*cnt].a = lo;
    out[*cnt].b = b;
    out[*cnt].j = j;
    *cnt += 1;
  }
}

// Segments of one scatterer's shape (section 2.4.2, shapes combined by CSG: the hollow
// cylinder is a difference).  Writes up to two segments at out[0..1].
template <typename R>
__device__ __forceinline__ int shape_segs(const ScatP<R>& S, int j, const Ray<R>& n, Seg<R>* out,
                                          R s0 = R(0)) {
  using M = Mth<R>;
  int cnt = 0;
  R c1, c2, y1, y2;
  if (S.shape == MCV_SHAPE_SOLID_CYL) {
    if (cyl_span<R>((R)S.dim0, n.x, n.z, n.dx, n.dz, &c1, &c2) &&
        slab_span<R>((R)S.half_h, n.y, n.dy, &y1, &y2))
      put_seg<R>(M::fmax(c1, y1), M::fmin(c2, y2), j, s0, out, &cnt);
  } else if (S.shape == MCV_SHAPE_HOLLOW_CYL) {
    if (cyl_span<R>((R)S.dim1, n.x, n.z, n.dx, n.dz, &c1, &c2) &&
        slab_span<R>((R)S.half_h, n.y, n.dy, &y1, &y2)) {
      const R lo = M::fmax(c1, y1), hi = M::fmin(c2, y2);
      if (hi > lo) {
        R i1, i2;
        if (!cyl_span<R>((R)S.dim0, n.x, n.z, n.dx, n.dz, &i1, &i2)) {
          put_seg<R>(lo, hi, j, s0, out, &cnt);
        } else {
          put_seg<R>(lo, M::fmin(hi, i1), j, s0, out, &cnt);
          put_seg<R>(M::fmax(lo, i2), hi, j, s0, out, &cnt);
        }
      }
    }
  } else if (S.shape == MCV_SHAPE_BLOCK) {
    const R c = (R)S.cos_rot, s = (R)S.sin_rot;
    const R xb = c * n.x - s * n.z, zb = s * n.x + c * n.z;
    const R dxb = c * n.dx - s * n.dz, dzb = s * n.dx + c * n.dz;
    R lo = -M::inf(), hi = M::inf(), a, b;
    bool ok = slab_span<R>(R(0.5) * S.dim0, xb, dxb, &a, &b);
    lo = M::fmax(lo, a);
    hi = M::fmin(hi, b);
    ok = ok && slab_span<R>(R(0.5) * S.dim1, n.y, n.dy, &a, &b);
    lo = M::fmax(lo, a);
    hi = M::fmin(hi, b);
    ok = ok && slab_span<R>(R(0.5) * S.dim2, zb, dzb, &a, &b);
    lo = M::fmax(lo, a);
    hi = M::fmin(hi, b);
    if (ok) put_seg<R>(lo, hi, j, s0, out, &cnt);
  }
  return cnt;
}

// All segments ahead in the sample assembly, sorted by entry (ray tracing in a composite,
// section 2.4.3).  NS = number of scatterers (compile time); unused entries get a = +inf.
template <typename R, int NS>
__device__ __forceinline__ int assembly_segs(const SampleP<R>& S, const Ray<R>& n, Seg<R> (&seg)[2 * NS],
                                             R s0 = R(0)) {
  using M = Mth<R>;
  int total = 0;
#pragma unroll
  for (int j = 0; j < NS; ++j) {
    Seg<R> two[2];
    two[0].a = M::inf();
    two[1].a = M::inf();
    two[0].b = two[1].b = R(0);
    two[0].j = two[1].j = j;
    const int c = (j < S.ns) ? shape_segs<R>(S.s[j], j, n, two, s0) : 0;
    seg[2 * j] = two[0];
    seg[2 * j + 1] = two[1];
    total += c;
  }
  // stable odd-even transposition sort on the entry distance
#pragma unroll
  for (int pass = 0; pass < 2 * NS; ++pass) {
#pragma unroll
    for (int i = (pass & 1); i + 1 < 2 * NS; i += 2) {
      if (seg[i].a > seg[i + 1].a) {
        const Seg<R> t = seg[i];
        seg[i] = seg[i + 1];
        seg[i + 1] = t;
      }
    }
  }
  return total;
}

template <typename R, int NS>
__device__ __forceinline__ R pick_mu(const R (&mu)[NS], int j) {
  R m = mu[0];
#pragma unroll
  for (int k = 1; k < NS; ++k)
    if (j == k) m = mu[k];
  return m;
}

// ---- scattering kernels (supplement: "Scattering kernels used in the examples") -----------
template <typename R>
struct Scatter {
  R factor;   // weight multiplier
  R rest;     // the multiplier without the table value
  R s_value;  // table value or 1
  int entry;  // table entry or -1
  R q, e;
};

// unit vector at polar angle (c, s) and azimuth 2 pi u about the unit vector d
template <typename R>
__device__ __forceinline__ void turn(R c, R s, R u, R* dx, R* dy, R* dz) {
  using M = Mth<R>;
  const R x = *dx, y = *dy, z = *dz;
  R e1x, e1y, e1z;
  if (M::fabs(z) < R(0.9)) {  // (0,0,1) x d
    e1x = -y;
    e1y = x;
    e1z = R(0);
  } else {                    // (1,0,0) x d
    e1x = R(0);
    e1y = -z;
    e1z = y;
  }
  const R inv = R(1) / M::sqrt(e1x * e1x + e1y * e1y + e1z * e1z);
  e1x *= inv;
  e1y *= inv;
  e1z *= inv;
  const R e2x = y * e1z - z * e1y, e2y = z * e1x - x * e1z, e2z = x * e1y - y * e1x;
  R sp, cp;
  M::sincos2pi(u, &sp, &cp);
  *dx = x * c + (e1x * cp + e2x * sp) * s;
  *dy = y * c + (e1y * cp + e2y * sp) * s;
  *dz = z * c + (e1z * cp + e2z * sp) * s;
}

// incoherent elastic: isotropic, speed unchanged (Debye-Waller factor taken as 1)
template <typename R, class Rng>
__device__ __forceinline__ void kernel_iso(const Rng& rng, int o, Ray<R>* n, Scatter<R>* sc) {
  using M = Mth<R>;
  R u0, u1, sp, cp;
  rng.template pair<R>(o, 1, &u0, &u1);
  const R ct = R(2) * u0 - R(1);
  const R st = R(2) * M::sqrt(u0 * (R(1) - u0));
  M::sincos2pi(u1, &sp, &cp);
  n->dx = st * cp;
  n->dy = st * sp;
  n->dz = ct;
  sc->factor = R(1);
  sc->rest = R(1);
  sc->s_value = R(1);
  sc->entry = -1;
  sc->q = R(0);
  sc->e = R(0);
}

// tabulated isotropic S(Q,E): E uniform on [e_min, min(e_max, Ei)], Q uniform on
// [|ki - kf|, min(ki + kf, q_max)], azimuth uniform; weight S Q dE dQ / (2 ki^2); nearest bin.
// Returns false when the kernel cannot scatter (empty range or outside the table).
template <typename R, class Rng>
__device__ __forceinline__ bool kernel_sqe(const SampleP<R>& S, const Rng& rng, int o,
                                           Ray<R>* n, Scatter<R>* sc, int* err) {
  using M = Mth<R>;
  const R Ei = (R)kMeVPerV2 * n->speed * n->speed;
  const R ki = (R)kKPerV * n->speed;
  const R e_lo = (R)S.e_min, e_hi = M::fmin((R)S.e_max, Ei);
  if (!(e_hi > e_lo)) return false;
  const R dE = e_hi - e_lo;
  R u0, u1;
  rng.template pair<R>(o, 1, &u0, &u1);
  const R E = e_lo + u0 * dE;
  // Ef = Ei - E; when the range ends at Ei it is the sampled offset from that end
  const R Ef = (e_hi == Ei) ? (R(1) - u0) * dE : Ei - E;
  if (!(Ef > R(0))) return false;
  const R speed_f = M::sqrt(Ef / (R)kMeVPerV2);
  const R kf = (R)kKPerV * speed_f;
  const R q_lo = M::fabs(ki - kf);
  const R q_hi = M::fmin(ki + kf, (R)S.q_max);
  if (!(q_hi > q_lo)) return false;
  const R dQ = q_hi - q_lo;
  const R Q = q_lo + u1 * dQ;
  // cos and sin of the scattering angle from 1 -/+ cos, each a product whose small factor
  // is the sampled offset from an end of the Q range (no cancellation near 0 or pi)
  const R den = R(2) * ki * kf;
  const R one_m = (u1 * dQ) * (Q + q_lo) / den;
  const R top = (q_hi == ki + kf) ? (R(1) - u1) * dQ : (ki + kf) - Q;
  const R one_p = top * (ki + kf + Q) / den;
  R c2t = (one_m <= one_p) ? R(1) - one_m : one_p - R(1);
  c2t = M::fmin(R(1), M::fmax(R(-1), c2t));
  const R s2t = M::sqrt(M::fmax(R(0), one_m * one_p));
  const R fq = M::floor(Q / (R)S.dq), fe = M::floor((E - (R)S.e_min) / (R)S.de);
  if (!(fq >= R(0) && fq < (R)S.nq && fe >= R(0) && fe < (R)S.ne)) return false;
  const int entry = (int)fq * S.ne + (int)fe;
  if (entry < 0 || entry >= S.nq * S.ne) {
    *err = 1;
    return false;
  }
  const R Sv = (R)__ldg(S.sqe + entry);
  const R u2 = rng.template first<R>(o, 2);
  turn<R>(c2t, s2t, u2, &n->dx, &n->dy, &n->dz);
  n->speed = speed_f;
  sc->rest = Q * dE * dQ / (R(2) * ki * ki);
  sc->factor = Sv * sc->rest;
  sc->s_value = Sv;
  sc->entry = entry;
  sc->q = Q;
  sc->e = E;
  return true;
}

// ---- incoherent scattering from a phonon density of states (supplement S4) -------------
// The phonon expansion S(Q,E) = e^{-2W} [delta(E) + sum_{n>=1} (2W)^n/n! A_n(E)], 2W = c_w Q^2,
// with A_1 and the multi-phonon mixture B = (A_2 + ... + A_N)/(N - 1) as masses on the grid
// E = i de (tables of mcv_phonon_build).  Channel: elastic (isotropic, weight e^{-2W}),
// one-phonon (grid point from A_1, weight 2W e^{-2W}) or multi-phonon (grid point from B,
// weight e^{-2W} sum_{n>=2} (2W)^n/n! A_n / B) with probabilities p0, p1, p2; the energy is
// spread over its grid bin; Q uniform over [|ki - kf|, ki + kf], azimuth uniform; the
// inelastic weights carry Q dQ / (2 ki^2), and every channel's weight is divided by its
// probability.  Returns false when the drawn energy loss leaves no final energy.

// first index whose cumulative mass exceeds u times the total (a draw from the masses)
template <typename R>
__device__ __forceinline__ int draw_mass(const R* __restrict__ cdf, int size, R u) {
  const R x = u * __ldg(cdf + size - 1);
  int lo = 0, hi = size;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(cdf + mid) > x) hi = mid;
    else lo = mid + 1;
  }
  return lo < size - 1 ? lo : size - 1;
}

template <typename R, class Rng>
__device__ __forceinline__ bool kernel_phonon(const SampleP<R>& S, const Rng& rng, int o,
                                              Ray<R>* n, Scatter<R>* sc) {
  using M = Mth<R>;
  const R Ei = (R)kMeVPerV2 * n->speed * n->speed;
  const R ki = (R)kKPerV * n->speed;
  R u0, u1, u2, u3;
  rng.template pair<R>(o, 1, &u0, &u1);
  rng.template pair<R>(o, 2, &u2, &u3);
  sc->entry = -1;
  sc->s_value = R(1);
  if (u0 < S.ph_p0) {
    // elastic: isotropic direction, speed unchanged
    const R ct = R(2) * u2 - R(1);
    const R st = R(2) * M::sqrt(u2 * (R(1) - u2));
    R sp, cp;
    M::sincos2pi(u3, &sp, &cp);
    const R dx = st * cp, dy = st * sp, dz = ct;
    const R qx = n->dx * ki + dx * (-ki), qy = n->dy * ki + dy * (-ki), qz = n->dz * ki + dz * (-ki);
    const R q = M::sqrt(qx * qx + qy * qy + qz * qz);
    n->dx = dx;
    n->dy = dy;
    n->dz = dz;
    sc->rest = M::exp(-S.ph_cw * q * q) / S.ph_p0;
    sc->factor = sc->rest;
    sc->q = q;
    sc->e = R(0);
    return true;
  }
  const bool one = u0 < S.ph_p01;
  const R p_ch = one ? S.ph_p1 : S.ph_p2;
  const R ue = (u0 - (one ? S.ph_p0 : S.ph_p01)) / p_ch;
  // one search for both channels (the lanes of a warp pick either), from A_1 or from B
  const int k = draw_mass<R>(one ? S.ph_cdf1 : S.ph_cdfb, one ? 2 * S.ph_J + 1 : S.ph_M, ue);
  const int i = k - (one ? S.ph_J : S.ph_N * S.ph_J);
  const R mass = one ? R(1) : __ldg(S.ph_b + k);
  const R E = ((R)i + (u1 - R(0.5))) * S.ph_de;
  const R Ef = Ei - E;
  if (!(Ef > R(0))) return false;
  const R speed_f = M::sqrt(Ef / (R)kMeVPerV2);
  const R kf = (R)kKPerV * speed_f;
  const R q_lo = M::fabs(ki - kf), q_hi = ki + kf;
  const R dQ = q_hi - q_lo;
  const R Q = q_lo + u2 * dQ;
  // scattering angle from 1 -/+ cos as products of the offsets from the ends of the range
  const R den = R(2) * ki * kf;
  const R one_m = (u2 * dQ) * (Q + q_lo) / den;
  const R one_p = ((R(1) - u2) * dQ) * (ki + kf + Q) / den;
  R c2t = (one_m <= one_p) ? R(1) - one_m : one_p - R(1);
  c2t = M::fmin(R(1), M::fmax(R(-1), c2t));
  const R s2t = M::sqrt(M::fmax(R(0), one_m * one_p));
  // the term of S at (Q, E) over the sampling mass of E
  const R w2 = S.ph_cw * Q * Q;
  R ratio;
  if (one) {
    ratio = w2 * M::exp(-w2);
  } else {
    const int g = i + S.ph_N * S.ph_J;
    R sum = R(0), pw = w2, fact = R(1);
    for (int k = 2; k <= S.ph_N; ++k) {
      pw *= w2;
      fact *= (R)k;
      sum += pw / fact * __ldg(S.ph_an + (int64_t)(k - 2) * S.ph_M + g);
    }
    ratio = M::exp(-w2) * sum / mass;
  }
  turn<R>(c2t, s2t, u3, &n->dx, &n->dy, &n->dz);
  n->speed = speed_f;
  sc->rest = ratio * Q * dQ / (R(2) * ki * ki) / p_ch;
  sc->factor = sc->rest;
  sc->q = Q;
  sc->e = E;
  return true;
}

// ---- coherent elastic scattering from a powder (supplement S4) --------------------------
// Per atom, reflection tau scatters sigma_tau = lambda^3 w_tau / (4 sin theta_B) with
// sin theta_B = lambda / 2 d_tau, i.e. lambda^2 w_tau d_tau / 2, for lambda < 2 d_tau (the
// Debye-Scherrer cone).  The reflections come by decreasing d, so the allowed ones form a
// prefix, found by a binary search of d; the table's prefix sums C of w d give their sum,
// lambda^2 C / 2, and the one picked with probability sigma_tau / sum sigma (a binary search
// of u C); the packet leaves on its cone (azimuth uniform, speed unchanged) and its weight
// takes sum sigma / sig_k (sig_k: the kernel's nominal cross section).  Returns false when no
// reflection is allowed.
template <typename R, class Rng>
__device__ __forceinline__ bool kernel_bragg(const SampleP<R>& S, R sig_k, const Rng& rng,
                                             int o, Ray<R>* n, Scatter<R>* sc) {
  using M = Mth<R>;
  const R ki = (R)kKPerV * n->speed;
  const R lam = R(2.0 * kPi) / ki;
  int lo = 0, hi = S.n_refl;  // allowed: the reflections with lam < 2 d
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (lam < R(2) * __ldg(S.refl_d + mid)) lo = mid + 1;
    else hi = mid;
  }
  const int allowed = lo;
  if (allowed == 0) return false;
  const R csum = __ldg(S.refl_c + allowed - 1);
  const R total = R(0.5) * lam * lam * csum;
  if (!(total > R(0))) return false;
  R u0, u1;
  rng.template pair<R>(o, 1, &u0, &u1);
  const R x = u0 * csum;
  lo = 0;
  hi = allowed - 1;  // the first reflection whose prefix sum exceeds x (the last if none)
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (x < __ldg(S.refl_c + mid)) hi = mid;
    else lo = mid + 1;
  }
  const int pick = lo;
  const R s = lam / (R(2) * __ldg(S.refl_d + pick));
  const R c2t = R(1) - R(2) * s * s;
  const R s2t = R(2) * s * M::sqrt((R(1) - s) * (R(1) + s));
  turn<R>(c2t, s2t, u1, &n->dx, &n->dy, &n->dz);
  sc->rest = total / sig_k;
  sc->factor = sc->rest;
  sc->s_value = R(1);
  sc->entry = -1;
  sc->q = R(2) * ki * s;
  sc->e = R(0);
  return true;
}

// ---- single-crystal coherent one-phonon kernel (Born-von Karman fcc) -------------------
// Per atom of a Bravais crystal (supplement S4, coherent one-phonon, with q = Q reduced):
//   d2sigma/dOmega dEf = sigma/4pi (kf/ki) e^{-2W} sum_{b,s} hbar^2 (Q.e_b)^2/(2M hw_b)
//                        N_s delta(Ei - Ef - s hw_b(Q)),  N_+ = n + 1, N_- = n.
// Direction uniform, mode (b, s) uniform over six, root of g(Ef) = Ei - Ef - s hw_b(Q(Ef))
// uniform over those bracketed on 32 sub-intervals and refined by bisection; weight
// 6 n_roots (kf/ki) e^{-2W} R_b N_s / |g'|.  Dynamical matrix of the 12 nearest neighbours
// (a/2)(+-1,+-1,0)... with 1 - cos x evaluated as 2 sin^2(x/2) (accurate near the zone
// centres); eigenpairs as described at eig3_branch.
// The dynamical matrix is kept in units of phi/M (its entries are O(1); in s^-2 their
// squares would overflow FP32): hbar omega = hbar sqrt(phi/M) sqrt(lambda').
template <typename R>
__device__ __forceinline__ void bvk_dynmat(const SampleP<R>& S, R qx, R qy, R qz, R D[6]) {
  // the six bond directions n (the other six are -n): (1,1,0) (1,-1,0) (1,0,1) (1,0,-1)
  // (0,1,1) (0,1,-1); each pair adds 2 (1 - cos q.delta) n n^T / 2
  const R nb[6][3] = {{1, 1, 0}, {1, -1, 0}, {1, 0, 1}, {1, 0, -1}, {0, 1, 1}, {0, 1, -1}};
#pragma unroll
  for (int i = 0; i < 6; ++i) D[i] = R(0);
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const R* n = nb[k];
    const R qd = S.bvk_ah * (qx * n[0] + qy * n[1] + qz * n[2]);
    const R sh = Mth<R>::sin_(R(0.5) * qd);
    const R c = R(2) * (R(2) * sh * sh) * R(0.5);
    D[0] += c * n[0] * n[0];
    D[1] += c * n[1] * n[1];
    D[2] += c * n[2] * n[2];
    D[3] += c * n[0] * n[1];
    D[4] += c * n[0] * n[2];
    D[5] += c * n[1] * n[2];
  }
}

// Eigenpair of branch b (0, 1, 2 in ascending order of the eigenvalue) of the symmetric 3x3
// matrix D (xx yy zz xy xz yz).  Cardano's trigonometric solution of the characteristic
// cubic only estimates the eigenvalues -- its accuracy degrades where two of them nearly
// coincide -- and tells which eigenvalue stands apart from the other two.  That one's
// eigenvector is the largest cross product of two rows of D - lambda I and its eigenvalue
// the Rayleigh quotient; the other two are the eigenpairs of D restricted to the plane
// orthogonal to it (a 2x2 problem in closed form).  Eigenvalues come out accurate to a few
// ulps of the largest, eigenvectors to that over the distance to the nearest other one.
template <typename R>
__device__ __forceinline__ void eig3_branch(const R D[6], int b, R* lam, R* ex, R* ey, R* ez) {
  using M = Mth<R>;
  const R a00 = D[0], a11 = D[1], a22 = D[2], a01 = D[3], a02 = D[4], a12 = D[5];
  const R p1 = a01 * a01 + a02 * a02 + a12 * a12;
  if (p1 == R(0)) {
    // diagonal: a stable sort of the three entries
    R v0 = a00, v1 = a11, v2 = a22, t;
    int i0 = 0, i1 = 1, i2 = 2, ti;
    if (v0 > v1) { t = v0; v0 = v1; v1 = t; ti = i0; i0 = i1; i1 = ti; }
    if (v1 > v2) { t = v1; v1 = v2; v2 = t; ti = i1; i1 = i2; i2 = ti; }
    if (v0 > v1) { t = v0; v0 = v1; v1 = t; ti = i0; i0 = i1; i1 = ti; }
    const int ib = b == 0 ? i0 : (b == 1 ? i1 : i2);
    *lam = b == 0 ? v0 : (b == 1 ? v1 : v2);
    *ex = ib == 0 ? R(1) : R(0);
    *ey = ib == 1 ? R(1) : R(0);
    *ez = ib == 2 ? R(1) : R(0);
    return;
  }
  // Cardano estimates
  const R q = (a00 + a11 + a22) / R(3);
  const R p2 = (a00 - q) * (a00 - q) + (a11 - q) * (a11 - q) + (a22 - q) * (a22 - q) + R(2) * p1;
  const R p = M::sqrt(p2 / R(6));
  const R b00 = (a00 - q) / p, b11 = (a11 - q) / p, b22 = (a22 - q) / p;
  const R b01 = a01 / p, b02 = a02 / p, b12 = a12 / p;
  R r = R(0.5) * (b00 * (b11 * b22 - b12 * b12) - b01 * (b01 * b22 - b12 * b02) +
                  b02 * (b01 * b12 - b11 * b02));
  r = M::fmin(R(1), M::fmax(R(-1), r));
  const R phi = M::acos_(r) / R(3);
  const R l2 = q + R(2) * p * M::cos_(phi);
  const R l0 = q + R(2) * p * M::cos_(phi + R(2) * (R)kPi / R(3));
  const R l1 = R(3) * q - l0 - l2;
  // the isolated eigenvalue's eigenvector: largest cross product of two rows of D - li I
  const R li = (l1 - l0 >= l2 - l1) ? l0 : l2;
  const R r0x = a00 - li, r0y = a01, r0z = a02;
  const R r1x = a01, r1y = a11 - li, r1z = a12;
  const R r2x = a02, r2y = a12, r2z = a22 - li;
  R cx[3], cy[3], cz[3];
  cx[0] = r0y * r1z - r0z * r1y; cy[0] = r0z * r1x - r0x * r1z; cz[0] = r0x * r1y - r0y * r1x;
  cx[1] = r0y * r2z - r0z * r2y; cy[1] = r0z * r2x - r0x * r2z; cz[1] = r0x * r2y - r0y * r2x;
  cx[2] = r1y * r2z - r1z * r2y; cy[2] = r1z * r2x - r1x * r2z; cz[2] = r1x * r2y - r1y * r2x;
  R gx = cx[0], gy = cy[0], gz = cz[0];
  R nb = gx * gx + gy * gy + gz * gz;
#pragma unroll
  for (int i = 1; i < 3; ++i) {
    const R ni = cx[i] * cx[i] + cy[i] * cy[i] + cz[i] * cz[i];
    if (ni > nb) {
      nb = ni;
      gx = cx[i];
      gy = cy[i];
      gz = cz[i];
    }
  }
  if (nb > R(0)) {
    const R inv = R(1) / M::sqrt(nb);
    gx = gx * inv;
    gy = gy * inv;
    gz = gz * inv;
  } else {
    gx = R(1);
    gy = R(0);
    gz = R(0);
  }
  const R dgx = a00 * gx + a01 * gy + a02 * gz;
  const R dgy = a01 * gx + a11 * gy + a12 * gz;
  const R dgz = a02 * gx + a12 * gy + a22 * gz;
  const R lam_e = gx * dgx + gy * dgy + gz * dgz;
  // orthonormal basis (u, w) of the plane orthogonal to it: u = e x (axis least along e)
  const R ax = M::fabs(gx), ay = M::fabs(gy), az = M::fabs(gz);
  const int axis = (ax <= ay && ax <= az) ? 0 : (ay <= az ? 1 : 2);
  R ux, uy, uz;
  if (axis == 0) {
    ux = R(0);
    uy = gz;
    uz = -gy;
  } else if (axis == 1) {
    ux = -gz;
    uy = R(0);
    uz = gx;
  } else {
    ux = gy;
    uy = -gx;
    uz = R(0);
  }
  const R un = R(1) / M::sqrt(ux * ux + uy * uy + uz * uz);
  ux = ux * un;
  uy = uy * un;
  uz = uz * un;
  const R wx = gy * uz - gz * uy, wy = gz * ux - gx * uz, wz = gx * uy - gy * ux;
  const R dux = a00 * ux + a01 * uy + a02 * uz;
  const R duy = a01 * ux + a11 * uy + a12 * uz;
  const R duz = a02 * ux + a12 * uy + a22 * uz;
  const R dwx = a00 * wx + a01 * wy + a02 * wz;
  const R dwy = a01 * wx + a11 * wy + a12 * wz;
  const R dwz = a02 * wx + a12 * wy + a22 * wz;
  const R A = ux * dux + uy * duy + uz * duz;
  const R B = ux * dwx + uy * dwy + uz * dwz;
  const R C = wx * dwx + wy * dwy + wz * dwz;
  const R mid = R(0.5) * (A + C), h = R(0.5) * (A - C);
  const R rr = M::hypot(h, B);
  const R mu_hi = mid + rr, mu_lo = mid - rr;
  // position of lam_e among the three (ties keep it first)
  const int pos_e = !(lam_e > mu_lo) ? 0 : (!(lam_e > mu_hi) ? 1 : 2);
  if (b == pos_e) {
    *lam = lam_e;
    *ex = gx;
    *ey = gy;
    *ez = gz;
    return;
  }
  const bool want_hi = b > pos_e ? (b == 2) : (b == 1);
  *lam = want_hi ? mu_hi : mu_lo;
  // eigenvector of mu_hi in the (u, w) plane: (rr + h, B) or (B, rr - h), the longer one
  R cu, cw;
  if (h >= R(0)) {
    cu = rr + h;
    cw = B;
  } else {
    cu = B;
    cw = rr - h;
  }
  const R cn = M::hypot(cu, cw);
  if (cn > R(0)) {
    cu = cu / cn;
    cw = cw / cn;
  } else {
    cu = R(1);
    cw = R(0);
  }
  if (want_hi) {
    *ex = ux * cu + wx * cw;
    *ey = uy * cu + wy * cw;
    *ez = uz * cu + wz * cw;
  } else {
    *ex = ux * -cw + wx * cu;
    *ey = uy * -cw + wy * cu;
    *ez = uz * -cw + wz * cu;
  }
}

// lab vector -> crystal frame (body = R^T lab, rotation about +y; x_c = z_b, y_c = x_b,
// z_c = y_b: [100] along the beam at zero rotation)
template <typename R>
__device__ __forceinline__ void to_crystal(R c, R s, R vx, R vy, R vz, R* ox, R* oy, R* oz) {
  *ox = s * vx + c * vz;
  *oy = c * vx - s * vz;
  *oz = vy;
}

template <typename R>
struct BvkPoint {
  R g, hw, qx, qy, qz;
  R lam, ex, ey, ez;  // eigenvalue and unit eigenvector of the branch
};

template <typename R>
__device__ __forceinline__ BvkPoint<R> bvk_point(const SampleP<R>& S, R c, R s, R Ei, R ki,
                                                  R dix, R diy, R diz, R dfx, R dfy, R dfz,
                                                  R Ef, int b, int sg) {
  BvkPoint<R> P;
  const R kf = (R)kKPerV * Mth<R>::sqrt(Ef / (R)kMeVPerV2);
  const R Qx = dix * ki - dfx * kf, Qy = diy * ki - dfy * kf, Qz = diz * ki - dfz * kf;
  to_crystal<R>(c, s, Qx, Qy, Qz, &P.qx, &P.qy, &P.qz);
  R D[6];
  bvk_dynmat<R>(S, P.qx, P.qy, P.qz, D);
  eig3_branch<R>(D, b, &P.lam, &P.ex, &P.ey, &P.ez);
  P.hw = S.bvk_hwu * Mth<R>::sqrt(Mth<R>::fmax(P.lam, R(0)));
  P.g = Ei - Ef - (R)sg * P.hw;
  return P;
}

template <typename R, class Rng>
__device__ __forceinline__ bool kernel_bvk(const SampleP<R>& S, R crot, R srot,
                                           const Rng& rng, int o, Ray<R>* n,
                                           Scatter<R>* sc) {
  using M = Mth<R>;
  R u0, u1, u2, u3;
  rng.template pair<R>(o, 1, &u0, &u1);
  rng.template pair<R>(o, 2, &u2, &u3);
  const R ct = R(2) * u0 - R(1);
  const R st = R(2) * M::sqrt(u0 * (R(1) - u0));
  R sp, cp;
  M::sincos2pi(u1, &sp, &cp);
  const R dfx = st * cp, dfy = st * sp, dfz = ct;
  int mode = (int)M::floor(R(6) * u2);
  mode = min(max(mode, 0), 5);
  const int b = mode % 3;
  const int sg = mode < 3 ? 1 : -1;
  const R Ei = (R)kMeVPerV2 * n->speed * n->speed;
  const R ki = (R)kKPerV * n->speed;
  const R lo = sg > 0 ? R(0) : Ei;
  const R hi = sg > 0 ? Ei : Ei + S.bvk_wmax;
  constexpr int kM = 32;
  const R step = (hi - lo) / (R)kM;
  // signs of g on the grid, one bit per node
  uint64_t pos = 0;
  for (int k = 0; k <= kM; ++k) {
    const BvkPoint<R> P = bvk_point<R>(S, crot, srot, Ei, ki, n->dx, n->dy, n->dz, dfx, dfy, dfz,
                                       lo + (R)k * step, b, sg);
    if (P.g > R(0)) pos |= (uint64_t)1 << k;
  }
  const uint64_t change = (pos ^ (pos >> 1)) & ((((uint64_t)1) << kM) - 1);
  const int nroots = __popcll(change);
  if (nroots == 0) return false;
  int pick = (int)M::floor(u3 * (R)nroots);
  pick = min(max(pick, 0), nroots - 1);
  uint64_t ch = change;
  for (int i = 0; i < pick; ++i) ch &= ch - 1;  // drop the lowest set bits
  const int kb = __ffsll((long long)ch) - 1;
  R ea = lo + (R)kb * step, eb = lo + (R)(kb + 1) * step;
  const bool ga_pos = (pos >> kb) & 1;
  const int iters = sizeof(R) == 8 ? 50 : 24;
  for (int it = 0; it < iters; ++it) {
    const R mid = R(0.5) * (ea + eb);
    const BvkPoint<R> P = bvk_point<R>(S, crot, srot, Ei, ki, n->dx, n->dy, n->dz, dfx, dfy, dfz,
                                       mid, b, sg);
    if ((P.g > R(0)) == ga_pos)
      ea = mid;
    else
      eb = mid;
  }
  const R Ef = R(0.5) * (ea + eb);
  if (!(Ef > R(0))) return false;
  const BvkPoint<R> P = bvk_point<R>(S, crot, srot, Ei, ki, n->dx, n->dy, n->dz, dfx, dfy, dfz,
                                     Ef, b, sg);
  if (!(P.hw >= R(1e-3))) return false;
  const R ex = P.ex, ey = P.ey, ez = P.ez;
  // d hw / d Ef through Q(Ef) (Hellmann-Feynman: d lambda = e^T dD e)
  const R kf = (R)kKPerV * M::sqrt(Ef / (R)kMeVPerV2);
  const R dkf = kf / (R(2) * Ef);
  R dqx, dqy, dqz;
  to_crystal<R>(crot, srot, dfx, dfy, dfz, &dqx, &dqy, &dqz);
  dqx *= -dkf;
  dqy *= -dkf;
  dqz *= -dkf;
  const R nb[6][3] = {{1, 1, 0}, {1, -1, 0}, {1, 0, 1}, {1, 0, -1}, {0, 1, 1}, {0, 1, -1}};
  R dlam = R(0);
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const R* v = nb[k];
    const R qd = S.bvk_ah * (P.qx * v[0] + P.qy * v[1] + P.qz * v[2]);
    const R ed = ex * v[0] + ey * v[1] + ez * v[2];
    const R dqd = S.bvk_ah * (dqx * v[0] + dqy * v[1] + dqz * v[2]);
    dlam += R(2) * M::sin_(qd) * dqd * ed * ed * R(0.5);
  }
  const R dhw = S.bvk_hwu * dlam / (R(2) * M::sqrt(P.lam));
  const R gp = R(-1) - (R)sg * dhw;
  const R nB = R(1) / M::expm1(P.hw / S.bvk_kT);
  const R Ns = sg > 0 ? nB + R(1) : nB;
  const R qe = P.qx * ex + P.qy * ey + P.qz * ez;
  const R Q2 = P.qx * P.qx + P.qy * P.qy + P.qz * P.qz;
  const R dw = M::exp(-Q2 * S.bvk_msd / R(3));
  const R Rb = S.bvk_hb2m * qe * qe / P.hw;
  sc->rest = R(6) * (R)nroots * (kf / ki) * dw * Rb * Ns / M::fabs(gp);
  sc->factor = sc->rest;
  sc->s_value = R(1);
  sc->entry = -1;
  sc->q = M::sqrt(Q2);
  sc->e = Ei - Ef;
  n->dx = dfx;
  n->dy = dfy;
  n->dz = dfz;
  n->speed = M::sqrt(Ef / (R)kMeVPerV2);
  return true;
}

// ---- scattering from a dispersion surface (supplement S4) --------------------------------
// S(Q) delta(E - E(Q)) with E(Q) = amp sqrt(1 - (cos(c Qx) cos(c Qz))^2) (the paper's example
// surface, 1 - cos^2 a cos^2 b written as sin^2 a + cos^2 a sin^2 b) and S = s0, Q in the
// crystal frame.  Direction uniform; roots of g(Ef) = Ei - Ef - E(Q(Ef)) bracketed on 32
// sub-intervals of [max(0, Ei - amp), Ei], one picked uniformly and bisected; weight
// n_roots (kf/ki) s0 / |g'|, g' = -1 - grad E . dQ/dEf, dQ/dEf = -df kf / (2 Ef).
template <typename R>
struct DispPoint {
  R g, E, sa, ca, sb, cb, root;
};

template <typename R>
__device__ __forceinline__ DispPoint<R> disp_point(const SampleP<R>& S, R c, R s, R Ei, R ki,
                                                    R dix, R diy, R diz, R dfx, R dfy, R dfz,
                                                    R Ef) {
  using M = Mth<R>;
  DispPoint<R> P;
  const R kf = (R)kKPerV * M::sqrt(Ef / (R)kMeVPerV2);
  const R Qx = dix * ki - dfx * kf, Qy = diy * ki - dfy * kf, Qz = diz * ki - dfz * kf;
  R qx, qy, qz;
  to_crystal<R>(c, s, Qx, Qy, Qz, &qx, &qy, &qz);
  const R a = S.disp_c * qx, b = S.disp_c * qz;
  P.sa = M::sin_(a);
  P.ca = M::cos_(a);
  P.sb = M::sin_(b);
  P.cb = M::cos_(b);
  P.root = M::sqrt(P.sa * P.sa + P.ca * P.ca * P.sb * P.sb);
  P.E = S.disp_amp * P.root;
  P.g = Ei - Ef - P.E;
  return P;
}

template <typename R, class Rng>
__device__ __forceinline__ bool kernel_disp(const SampleP<R>& S, R crot, R srot,
                                            const Rng& rng, int o, Ray<R>* n, Scatter<R>* sc) {
  using M = Mth<R>;
  R u0, u1, u2;
  rng.template pair<R>(o, 1, &u0, &u1);
  u2 = rng.template first<R>(o, 2);
  const R ct = R(2) * u0 - R(1);
  const R st = R(2) * M::sqrt(u0 * (R(1) - u0));
  R sp, cp;
  M::sincos2pi(u1, &sp, &cp);
  const R dfx = st * cp, dfy = st * sp, dfz = ct;
  const R Ei = (R)kMeVPerV2 * n->speed * n->speed;
  const R ki = (R)kKPerV * n->speed;
  const R lo = M::fmax(R(0), Ei - S.disp_amp), hi = Ei;
  constexpr int kM = 32;
  const R step = (hi - lo) / (R)kM;
  uint64_t pos = 0;  // signs of g on the grid, one bit per node
  for (int k = 0; k <= kM; ++k) {
    const DispPoint<R> P = disp_point<R>(S, crot, srot, Ei, ki, n->dx, n->dy, n->dz, dfx, dfy,
                                         dfz, lo + (R)k * step);
    if (P.g > R(0)) pos |= (uint64_t)1 << k;
  }
  const uint64_t change = (pos ^ (pos >> 1)) & ((((uint64_t)1) << kM) - 1);
  const int nroots = __popcll(change);
  if (nroots == 0) return false;
  int pick = (int)M::floor(u2 * (R)nroots);
  pick = min(max(pick, 0), nroots - 1);
  uint64_t ch = change;
  for (int i = 0; i < pick; ++i) ch &= ch - 1;  // drop the lowest set bits
  const int kb = __ffsll((long long)ch) - 1;
  R ea = lo + (R)kb * step, eb = lo + (R)(kb + 1) * step;
  const bool ga_pos = (pos >> kb) & 1;
  const int iters = sizeof(R) == 8 ? 50 : 24;
  for (int it = 0; it < iters; ++it) {
    const R mid = R(0.5) * (ea + eb);
    const DispPoint<R> P = disp_point<R>(S, crot, srot, Ei, ki, n->dx, n->dy, n->dz, dfx, dfy,
                                         dfz, mid);
    if ((P.g > R(0)) == ga_pos)
      ea = mid;
    else
      eb = mid;
  }
  const R Ef = R(0.5) * (ea + eb);
  if (!(Ef > R(0))) return false;
  const DispPoint<R> P = disp_point<R>(S, crot, srot, Ei, ki, n->dx, n->dy, n->dz, dfx, dfy,
                                       dfz, Ef);
  if (!(P.E > R(0))) return false;
  const R kf = (R)kKPerV * M::sqrt(Ef / (R)kMeVPerV2);
  R dqx, dqy, dqz;
  to_crystal<R>(crot, srot, dfx, dfy, dfz, &dqx, &dqy, &dqz);
  const R sc_q = -kf / (R(2) * Ef);
  dqx *= sc_q;
  dqz *= sc_q;
  const R ac = S.disp_amp * S.disp_c;
  const R gx = ac * P.sa * P.ca * P.cb * P.cb / P.root;
  const R gz = ac * P.ca * P.ca * P.sb * P.cb / P.root;
  const R gp = R(-1) - (gx * dqx + gz * dqz);
  sc->rest = (R)nroots * (kf / ki) * S.disp_s0 / M::fabs(gp);
  sc->factor = sc->rest;
  sc->s_value = R(1);
  sc->entry = -1;
  sc->q = R(0);
  sc->e = Ei - Ef;
  n->dx = dfx;
  n->dy = dfy;
  n->dz = dfz;
  n->speed = M::sqrt(Ef / (R)kMeVPerV2);
  return true;
}

// ---- detector system (section 2.4.3, "Ray tracing in a detector system") -----------------
template <typename R>
struct Hit {
  int64_t bin;      // >= 0 in range, -1 miss, -2 tof out of range
  int32_t pixel;
  Tof<R> tof;
  R w_det;
  R pabs;           // detector weight factor (1 for the ideal surface)
};

// larger root of the ray with the origin-centred cylinder (the ray starts inside it)
template <typename R>
__device__ __forceinline__ bool exit_cyl(R rad, const Ray<R>& n, R* s) {
  R s1, s2;
  if (!cyl_span<R>(rad, n.x, n.z, n.dx, n.dz, &s1, &s2)) return false;
  if (!(s2 > R(0)) || s2 == Mth<R>::inf()) return false;
  *s = s2;
  return true;
}

// Chord of a vertical tube (axis through R (ux, uz)) in coordinates along / across the
// tube direction, so the large distance R cancels once.
template <typename R>
__device__ __forceinline__ bool tube_span(R Rad, R ux, R uz, R rt, const Ray<R>& n, R* s1, R* s2) {
  const R a = n.dx * n.dx + n.dz * n.dz;
  if (a == R(0)) return false;
  const R o_rad = n.x * ux + n.z * uz - Rad;
  const R o_tan = n.x * uz - n.z * ux;
  const R d_rad = n.dx * ux + n.dz * uz;
  const R d_tan = n.dx * uz - n.dz * ux;
  const R tc = -(o_rad * d_rad + o_tan * d_tan) / a;
  const R cr = o_rad * d_tan - o_tan * d_rad;
  const R g = rt * rt - cr * cr / a;
  if (!(g > R(0))) return false;
  const R half = Mth<R>::sqrt(g / a);
  *s1 = tc - half;
  *s2 = tc + half;
  return true;
}

// tof bin: FP64 mode as written; FP32 mode takes the offset from tof_min from the float
// pair exactly (the two differences are exact or nearly so) and scales it in float
template <typename R>
__device__ __forceinline__ int64_t tof_bin(const TofWin& W, const Tof<R>& tof);
template <>
__device__ __forceinline__ int64_t tof_bin<double>(const TofWin& W, const Tof<double>& tof) {
  const double fb = ::floor((tof.v - W.tof_min) / W.dt);
  if (!(fb >= 0.0 && fb < (double)W.n_tof)) return -1;
  return (int64_t)fb;
}
template <>
__device__ __forceinline__ int64_t tof_bin<float>(const TofWin& W, const Tof<float>& tof) {
  const float off = (tof.hi - W.tmin_hi) + (tof.lo - W.tmin_lo);
  const float fb = floorf(off * W.inv_dt);
  if (!(fb >= 0.0f && fb < (float)W.n_tof)) return -1;
  return (int64_t)fb;
}

template <typename R>
__device__ __forceinline__ Hit<R> detect_surface(const DetP<R>& D, const TofWin& W,
                                                 const Ray<R>& n) {
  using M = Mth<R>;
  Hit<R> h;
  h.bin = -1;
  h.pixel = -1;
  h.tof = n.t;
  h.w_det = R(0);
  h.pabs = R(0);
  R s;
  if (!exit_cyl<R>((R)D.radius, n, &s)) return h;
  const R yh = n.y + s * n.dy;
  const R half = (R)D.half_h;
  if (yh < -half || yh >= half) return h;
  const R xh = n.x + s * n.dx, zh = n.z + s * n.dz;
  const R phi = M::atan2(xh, zh);
  int ip = (int)M::floor((phi + (R)kPi) / (R)(2.0 * kPi) * (R)D.n_phi);
  ip = min(max(ip, 0), D.n_phi - 1);
  int iy = (int)M::floor((yh + half) / (R)D.height * (R)D.n_y);
  iy = min(max(iy, 0), D.n_y - 1);
  h.pixel = ip * D.n_y + iy;
  h.tof.add(s / n.speed);
  h.w_det = n.w;
  h.pabs = R(1);
  const int64_t tb = tof_bin<R>(W, h.tof);
  h.bin = (tb < 0) ? -2 : (int64_t)h.pixel * W.n_tof + tb;
  return h;
}

// tube centre directions staged in shared memory: tu[2*i] = sin(phi_i), tu[2*i+1] = cos(phi_i)
// A packet that surely misses every tube (DetP::miss_*: set for packets that start inside the
// sample): on its way out to the tube ring its height only moves further beyond the rows,
// or its horizontal direction points away from the arc of tubes.  A few operations, no
// square root; the detector trace would find the same packets missing.
template <typename R>
__device__ __forceinline__ bool det_surely_misses(const DetP<R>& D, const Ray<R>& n) {
  using M = Mth<R>;
  // horizontal path to the ring >= lmin = miss_r_in - (|x| + |z|); along it y moves by
  // |dy| lmin / |d_h| at least: beyond the rows when the room left above (below) the start,
  // a, is below that, a |d_h| < |dy| lmin, compared squared (no square root)
  const R lmin = D.miss_r_in - (M::fabs(n.x) + M::fabs(n.z));
  if (lmin > R(0)) {
    const R a = n.dy >= R(0) ? D.miss_y_top - n.y : n.y - D.miss_y_bot;
    const R h2 = n.dx * n.dx + n.dz * n.dz;
    const R m = n.dy * lmin;
    if (a <= R(0) || a * a * h2 < m * m) return true;
  }
  // sin of the angle from each end of the arc to the direction (phi = atan2(x, z))
  return D.miss_phi && (n.dx * D.miss_a_z - n.dz * D.miss_a_x < R(0) ||
                        n.dz * D.miss_b_x - n.dx * D.miss_b_z < R(0));
}

// Where a packet meets the tube rows: the row at its crossing of the tube-centre circle and
// the tube g nearest to that crossing (candidates g - 1, g, g + 1).  False: it meets no row
// or lies outside the rows' arc (no candidate tube), i.e. it misses the detector.
template <typename R>
__device__ __forceinline__ bool tubes_locate(const DetP<R>& D, const Ray<R>& n, int* row_out,
                                             int* g_out) {
  using M = Mth<R>;
  const R Rad = (R)D.radius;
  R sR;
  if (!exit_cyl<R>(Rad, n, &sR)) return false;
  const R Px = n.x + sR * n.dx, Py = n.y + sR * n.dy, Pz = n.z + sR * n.dz;
  int row = -1;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    if (row < 0 && i < D.n_rows && M::fabs(Py - (R)D.row_y[i]) <= (R)D.half_len) row = i;
  }
  if (row < 0) return false;
  const int tpp = D.tubes_per_pack;
  const R period = (R)D.period, pitch = (R)D.pitch;
  const R arc = (M::atan2(Px, Pz) - (R)D.phi0) * Rad;
  const R p = M::floor(arc / period);
  const R within = arc - p * period;
  R k = M::floor(within / pitch);
  if (k > (R)(tpp - 1)) k = (R)(tpp - 1);
  // more than one tube outside the rows' arc: no candidate (the range check on the float
  // also keeps its conversion to int in range)
  if (!(p >= R(-1) && p <= (R)D.packs[row])) return false;
  const int g = (int)p * tpp + (int)k;
  if (g + 1 < 0 || g - 1 >= D.packs[row] * tpp) return false;
  *row_out = row;
  *g_out = g;
  return true;
}

// The rest of the tube detector for a located packet: the first of the candidate tubes the
// ray enters, the absorption point drawn from the truncated exponential of the 3He path
// (u_det), pixel, time of flight and bin.
template <typename R>
__device__ __forceinline__ Hit<R> tubes_absorb(const DetP<R>& D, const TofWin& W,
                                               const R* __restrict__ tu, const Ray<R>& n,
                                               R u_det, int row, int g) {
  using M = Mth<R>;
  Hit<R> h;
  h.bin = -1;
  h.pixel = -1;
  h.tof = n.t;
  h.w_det = R(0);
  h.pabs = R(0);
  const R Rad = (R)D.radius;
  const int tpp = D.tubes_per_pack;
  const int row_off = D.row_off[row];
  const int n_tubes_row = D.packs[row] * tpp;
  const R y_lo = (R)D.row_y[row] - (R)D.half_len;
  const R y_hi = (R)D.row_y[row] + (R)D.half_len;
  int best = -1;
  R best_in = M::inf(), best_out = R(0);
#pragma unroll
  for (int dc = -1; dc <= 1; ++dc) {
    const int c = g + dc;
    if (c < 0 || c >= n_tubes_row) continue;
    R s1, s2;
    if (!tube_span<R>(Rad, tu[2 * c], tu[2 * c + 1], (R)D.tube_r, n, &s1, &s2)) continue;
    R ys1, ys2;
    if (n.dy == R(0)) {
      if (!(n.y >= y_lo && n.y <= y_hi)) continue;
      ys1 = -M::inf();
      ys2 = M::inf();
    } else {
      const R a = (y_lo - n.y) / n.dy, b = (y_hi - n.y) / n.dy;
      ys1 = M::fmin(a, b);
      ys2 = M::fmax(a, b);
    }
    const R s_in = M::fmax(M::fmax(s1, ys1), R(0));
    const R s_out = M::fmin(s2, ys2);
    if (!(s_out > s_in)) continue;
    if (s_in < best_in) {
      best = c;
      best_in = s_in;
      best_out = s_out;
    }
  }
  if (best < 0) return h;
  const R L = best_out - best_in;
  const R mu = (R)D.mu_he_v / n.speed;
  const R pabs = -M::expm1(-mu * L);
  const R x = -M::log1p(-u_det * pabs) / mu;
  const R s_abs = best_in + x;
  const R y_abs = n.y + s_abs * n.dy;
  int j = (int)M::floor((y_abs - y_lo) / (R)D.pix_len);
  j = min(max(j, 0), D.pixels_per_tube - 1);
  const int pc = best / tpp, tc = best - pc * tpp;
  h.pixel = ((row_off + pc) * tpp + tc) * D.pixels_per_tube + j;
  h.tof.add(s_abs / n.speed);
  h.pabs = pabs;
  h.w_det = n.w * pabs;
  const int64_t tb = tof_bin<R>(W, h.tof);
  h.bin = (tb < 0) ? -2 : (int64_t)h.pixel * W.n_tof + tb;
  return h;
}

// Tube detector system (section 2.4.3, "Ray tracing in a detector system"): the packet's
// crossing of the tube-centre circle picks the row and three candidate tubes; the first
// tube the ray enters absorbs it.
template <typename R>
__device__ __forceinline__ Hit<R> detect_tubes(const DetP<R>& D, const TofWin& W,
                                               const R* __restrict__ tu, const Ray<R>& n,
                                               R u_det) {
  int row = 0, g = 0;
  if (!tubes_locate<R>(D, n, &row, &g)) {
    Hit<R> h;
    h.bin = -1;
    h.pixel = -1;
    h.tof = n.t;
    h.w_det = R(0);
    h.pabs = R(0);
    return h;
  }
  return tubes_absorb<R>(D, W, tu, n, u_det, row, g);
}

template <typename R, int DET, class Rng>
__device__ __forceinline__ Hit<R> detect(const DetP<R>& D, const TofWin& W, const R* tu,
                                         const Rng& rng, int order, const Ray<R>& n) {
  if (DET == MCV_DET_SURFACE) return detect_surface<R>(D, W, n);
  const R u = rng.template first<R>(order, 3);
  return detect_tubes<R>(D, W, tu, n, u);
}

// ---- tallies ---------------------------------------------------------------------------
// FP64 accumulators in FP64 mode; compensated (Kahan) FP32 sums in FP32 mode
template <typename R>
struct Acc;
template <>
struct Acc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double v) { s += v; }
  __device__ __forceinline__ double value() const { return s; }
};
template <>
struct Acc<float> {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float v) {
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

struct Counts {
  uint32_t ndet = 0, nover = 0, nmiss = 0, nhit = 0, nemit = 0;
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}
__device__ __forceinline__ uint32_t warp_sum(uint32_t v) {
  return __reduce_add_sync(0xffffffffu, v);
}

// Appends one detected packet to an event list: the lanes that append together take
// consecutive indexes with one atomic add (warp-aggregated); an index at or beyond the
// capacity is counted but not written.
__device__ __forceinline__ void append_event(const EvSink& ev, int pixel, double tof, double w) {
  cooperative_groups::coalesced_group g = cooperative_groups::coalesced_threads();
  unsigned long long base = 0;
  if (g.thread_rank() == 0) base = atomicAdd(ev.count, (unsigned long long)g.size());
  base = g.shfl(base, 0);
  const unsigned long long k = base + g.thread_rank();
  if (k < (unsigned long long)ev.cap) {
    ev.pixel[k] = pixel;
    ev.sim[k] = ev.tag;
    ev.tof[k] = tof;
    ev.w[k] = w;
  }
}

}  // namespace mcv
