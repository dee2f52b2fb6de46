// Adjoint of the chi-squared loss of the simulated histogram (no counterpart in the paper).
//
// Along a fixed random path every emitted packet's detected weight is a product of factors:
//   w_det = e^{-tau_o} p_abs prod_k (mu_s L_k e^{-tau_k} rest_k) S_k
// (S_k the S(Q,E) table value used by scattering k, rest_k the kernel's other factor).  The
// scattering points, kernel choices and (Q, E) draws do not depend on the table or on the
// cross sections, so dL/dtheta = sum over detected packets of g_b dw_det/dtheta with
// g_b = dL/dI_b:
//   dw/dS_e  = e^{-tau_o} p_abs prod_k a_k prod_{m != k} S_m  for each k with entry e
//   dw/dsig  = w (sum of the log-derivatives of the attenuation and mu_s factors).
// The adjoint kernel recomputes each neutron's path with the forward arithmetic (the shared
// chain step) instead of storing it, keeps the per-scattering records in the thread, and
// scatter-adds into dS (FP64 atomics, the table is L2-resident) and dsig (warp-reduced).
#include <cuda_runtime.h>

#include "mcv_chain.cuh"
#include "mcv_launch.h"

namespace mcv {

namespace {

constexpr int kThreads = 128;
constexpr int kMaxOrders = 7;

template <typename R, int DET>
struct Adjoint {
  static constexpr bool kWantsGs = true;
  R a[kMaxOrders];   // scattering factor without the table value
  R s[kMaxOrders];   // table value (1 for kernels without a table)
  int e[kMaxOrders]; // table entry or -1
  double cum_dabs = 0.0, cum_ds = 0.0;
  double acc_abs = 0.0, acc_s = 0.0;
  int err = 0;

  __device__ __forceinline__ void start(const Lane<R>&) {
    cum_dabs = 0.0;
    cum_ds = 0.0;
  }

  __device__ __forceinline__ void emit(const TraceArgs& A, const R* tu, const NeutronRng& rng,
                                       const Lane<R>& L, R we, R atten, R lg, R) {
    if (L.o == 0) return;
    Ray<R> pe = L.n;
    pe.w = R(1);
    const Hit<R> h = detect<R, DET>(A.D, tu, rng, L.o, pe);
    if (h.bin < 0) return;
    if (h.bin >= A.D.n_bins) {
      err = 1;
      return;
    }
    const double gb = A.g[h.bin];
    if (gb == 0.0) return;
    const DScat& g = A.S.s[A.gs];
    const double w_det = (double)(we * h.pabs);
    const double dabs = cum_dabs - g.n100 * (2200.0 / (double)L.n.speed) * (double)lg;
    const double ds = cum_ds - g.n100 * (double)lg;
    acc_abs += gb * w_det * dabs;
    acc_s += gb * w_det * ds;
    if (!A.dsqe) return;
    R base = atten * h.pabs;
    for (int m = 0; m < L.o; ++m) base *= a[m];
    for (int k = 0; k < L.o; ++k) {
      if (e[k] < 0) continue;
      R prod = base;
      for (int m = 0; m < L.o; ++m)
        if (m != k) prod *= s[m];
      atomicAdd(A.dsqe + e[k], gb * (double)prod);
    }
  }

  __device__ __forceinline__ void scatter(const TraceArgs& A, const Lane<R>& L, int j, R a_fac,
                                          const Scatter<R>& out, R lg_pt, R speed_in) {
    const int k = L.o;
    a[k] = a_fac * out.rest;
    s[k] = out.s_value;
    e[k] = out.entry;
    const DScat& g = A.S.s[A.gs];
    cum_dabs -= g.n100 * (2200.0 / (double)speed_in) * (double)lg_pt;
    cum_ds -= g.n100 * (double)lg_pt;
    if (j == A.gs) cum_ds += 1.0 / g.sig_s;
  }

  __device__ __forceinline__ void clear(const TraceArgs&, int64_t, int) {}

  __device__ __forceinline__ void flush(const TraceArgs& A, int lane) {
    const double s_abs = warp_sum(acc_abs), s_s = warp_sum(acc_s);
    if (lane == 0) {
      atomicAdd(A.dsig + 0, s_abs);
      atomicAdd(A.dsig + 1, s_s);
    }
    if (__any_sync(0xffffffffu, err != 0) && lane == 0 && A.err) atomicOr(A.err, 1);
  }
};

template <typename R, int NS, int DET>
__global__ void __launch_bounds__(kThreads) adjoint_kernel(const __grid_constant__ TraceArgs A) {
  __shared__ R tu[2 * MCV_MAX_TUBES_PER_ROW];
  stage_tubes<R, DET>(A, tu);
  Adjoint<R, DET> pol;
  run_chain<R, NS, DET, Adjoint<R, DET>>(A, tu, pol);
}

// chi2 = sum_b (c I_b - T_b)^2 / max(T_b, 1);  g_b = 2 c (c I_b - T_b) / max(T_b, 1)
__global__ void __launch_bounds__(256) chi2_kernel(const double* __restrict__ hist,
                                                   const double* __restrict__ target, double c,
                                                   int64_t nb, double* __restrict__ g,
                                                   double* __restrict__ loss) {
  double part = 0.0;
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nb;
       b += (int64_t)gridDim.x * blockDim.x) {
    const double T = target[b];
    const double den = fmax(T, 1.0);
    const double r = c * hist[b] - T;
    part += r * r / den;
    g[b] = 2.0 * c * r / den;
  }
  part = warp_sum(part);
  __shared__ double red[8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) red[w] = part;
  __syncthreads();
  if (w == 0) {
    double v = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
    v = warp_sum(v);
    if (lane == 0) atomicAdd(loss, v);
  }
}

template <typename R, int NS>
cudaError_t launch_adjoint_ns(const TraceArgs& A, int det, int grid, cudaStream_t s) {
  if (det == MCV_DET_SURFACE)
    adjoint_kernel<R, NS, MCV_DET_SURFACE><<<grid, kThreads, 0, s>>>(A);
  else
    adjoint_kernel<R, NS, MCV_DET_TUBES><<<grid, kThreads, 0, s>>>(A);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_adjoint_r(const TraceArgs& A, int det, int grid, cudaStream_t s) {
  if (A.S.ns <= 1) return launch_adjoint_ns<R, 1>(A, det, grid, s);
  if (A.S.ns == 2) return launch_adjoint_ns<R, 2>(A, det, grid, s);
  return launch_adjoint_ns<R, 4>(A, det, grid, s);
}

}  // namespace

cudaError_t launch_chi2(const double* hist, const double* target, double c, int64_t nb,
                        double* g, double* loss, int grid, cudaStream_t s) {
  chi2_kernel<<<grid, 256, 0, s>>>(hist, target, c, nb, g, loss);
  return cudaGetLastError();
}

cudaError_t launch_adjoint(const TraceArgs& A, int fp_mode, int det, int grid, cudaStream_t s) {
  if (fp_mode == MCV_FP32) return launch_adjoint_r<float>(A, det, grid, s);
  return launch_adjoint_r<double>(A, det, grid, s);
}

}  // namespace mcv
