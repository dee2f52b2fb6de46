// The chi-squared loss of a simulated histogram against a measured one, bin by bin:
//   chi2 = sum_b (c I_b - T_b)^2 / max(T_b, 1),   g_b = dchi2/dI_b = 2 c (c I_b - T_b) / max(T_b, 1).
// Used by the loss kernel (every bin) and by the adjoint kernel, which evaluates g_b only for
// the bins its packets reach instead of reading a per-bin work buffer.  Both evaluate g_b with
// the same function, so they agree bit for bit.
#pragma once

#include <cuda_runtime.h>

namespace mcv {

// 1/d for d >= 1 without an FP64 division (GB300's FP64 rate is about 1/64 of its FP32
// rate, and a division is a long FP64 sequence): the FP32 reciprocal as the seed, then two
// Newton-Raphson steps x <- x + x (1 - d x) in FP64, each of which squares the relative
// error (2^-23 -> 2^-46 -> below FP64 rounding).  Very large d take the division.
__device__ __forceinline__ double recip_ge1(double d) {
  if (!(d < 1e30)) return 1.0 / d;
  double x = (double)__frcp_rn((float)d);
  x = fma(x, fma(-d, x, 1.0), x);
  x = fma(x, fma(-d, x, 1.0), x);
  return x;
}

// A measured bin must be a finite count >= 0: from its bits with integer operations (no
// FP64 comparison: the loss kernel tests every bin), a sign bit clear (or -0) and an
// exponent below the all-ones one of infinities and NaNs.
__device__ __forceinline__ bool target_ok(double T) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(T);
  return ((u >> 63) == 0ull || u == 0x8000000000000000ull) && ((u >> 52) & 0x7ffull) != 0x7ffull;
}

// One bin: its gradient entry g_b, its loss term added to *part.  A bin with nothing
// simulated and nothing measured (both values +0: almost all of a large detector's bins) is
// recognised from the bits with integer operations and costs no FP64 work (c is finite:
// the difference would be 0).
__device__ __forceinline__ double chi2_bin(double h, double T, double c, double* part) {
  if ((__double_as_longlong(h) | __double_as_longlong(T)) == 0) return 0.0;
  const double r = c * h - T;
  if (r == 0.0) return 0.0;
  const double ri = r * recip_ge1(fmax(T, 1.0));
  *part += r * ri;
  return 2.0 * c * ri;
}

// g_b alone (the adjoint's per-packet lookup)
__device__ __forceinline__ double chi2_grad_bin(double h, double T, double c) {
  double unused = 0.0;
  return chi2_bin(h, T, c, &unused);
}

// g_b in FP32 (the FP32 adjoint): the difference c h - T is formed in FP64, where it cancels,
// and rounded once; the rest is FP32 (relative error a few FP32 units).
__device__ __forceinline__ float chi2_grad_bin_f32(double h, double T, double c) {
  if ((__double_as_longlong(h) | __double_as_longlong(T)) == 0) return 0.0f;
  const float r = (float)(c * h - T);
  return (2.0f * (float)c) * r / fmaxf((float)T, 1.0f);
}

}  // namespace mcv
