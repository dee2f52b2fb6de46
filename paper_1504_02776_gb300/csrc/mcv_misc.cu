// Real-type independent kernels (clearing buffers, the chi-squared loss) and the
// dispatch of the per-type entry points.
#include <cuda_runtime.h>

#include "mcv_chi2.cuh"
#include "mcv_device.cuh"
#include "mcv_launch.h"

namespace mcv {

cudaError_t launch_trace_f32(const TraceArgs& A, int det, int grid, cudaStream_t s);
cudaError_t launch_trace_f64(const TraceArgs& A, int det, int grid, cudaStream_t s);
cudaError_t blocks_per_sm_f32(int ns, int det, int bvk, int* blocks);
cudaError_t blocks_per_sm_f64(int ns, int det, int bvk, int* blocks);
cudaError_t launch_beam_f32(const TraceArgs& A, int grid, cudaStream_t s);
cudaError_t launch_beam_f64(const TraceArgs& A, int grid, cudaStream_t s);
cudaError_t launch_detect_f32(const TraceArgs& A, const EventsArgs& E, int det, int grid,
                              cudaStream_t s);
cudaError_t launch_detect_f64(const TraceArgs& A, const EventsArgs& E, int det, int grid,
                              cudaStream_t s);
cudaError_t launch_adjoint_f32(const TraceArgs& A, int det, int grid, cudaStream_t s);
cudaError_t launch_adjoint_f64(const TraceArgs& A, int det, int grid, cudaStream_t s);
cudaError_t launch_paper_f32(const TraceArgs& A, int det, int grid, cudaStream_t s);
cudaError_t launch_paper_f64(const TraceArgs& A, int det, int grid, cudaStream_t s);
cudaError_t adjoint_blocks_per_sm_f32(int ns, int det, int bvk, int* blocks);
cudaError_t adjoint_blocks_per_sm_f64(int ns, int det, int bvk, int* blocks);
cudaError_t batch_blocks_per_sm_f32(int ns, int det, int bvk, int ss, int* blocks);
cudaError_t batch_blocks_per_sm_f64(int ns, int det, int bvk, int ss, int* blocks);
cudaError_t batch_blocks_per_sm_f32_ev(int ns, int det, int bvk, int ss, int* blocks);
cudaError_t batch_blocks_per_sm_f64_ev(int ns, int det, int bvk, int ss, int* blocks);
cudaError_t launch_batch_f32(const TraceArgs& A, const BatchArgs& Q, int ns, int det, int bvk,
                             int ss, int grid, cudaStream_t s);
cudaError_t launch_batch_f64(const TraceArgs& A, const BatchArgs& Q, int ns, int det, int bvk,
                             int ss, int grid, cudaStream_t s);
cudaError_t launch_batch_f32_ev(const TraceArgs& A, const BatchArgs& Q, int ns, int det, int bvk,
                                int ss, int grid, cudaStream_t s);
cudaError_t launch_batch_f64_ev(const TraceArgs& A, const BatchArgs& Q, int ns, int det, int bvk,
                                int ss, int grid, cudaStream_t s);

namespace {

__global__ void zero_kernel(double* __restrict__ p, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  // 16-byte stores where aligned
  const bool aligned = (reinterpret_cast<uintptr_t>(p) & 15u) == 0;
  if (aligned) {
    double2* q = reinterpret_cast<double2*>(p);
    const int64_t n2 = n / 2;
    for (int64_t k = i; k < n2; k += stride) q[k] = make_double2(0.0, 0.0);
    if (i == 0 && (n & 1)) p[n - 1] = 0.0;
  } else {
    for (int64_t k = i; k < n; k += stride) p[k] = 0.0;
  }
}

// chi2 = sum_b (c I_b - T_b)^2 / max(T_b, 1) into *loss; g (optional) receives
// g_b = dchi2/dI_b for every bin.  Without g the kernel only reads (16 bytes per bin, streamed
// past the caches): the adjoint evaluates g_b itself for the bins its packets reach.  A
// measured bin that is negative or not finite sets the error flag (err, optional).
__global__ void __launch_bounds__(256) chi2_kernel(const double* __restrict__ hist,
                                                   const double* __restrict__ target, double c,
                                                   int64_t nb, double* __restrict__ g,
                                                   double* __restrict__ loss, int* err) {
  double part = 0.0;
  bool bad = false;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool aligned = ((reinterpret_cast<uintptr_t>(hist) | reinterpret_cast<uintptr_t>(target) |
                         reinterpret_cast<uintptr_t>(g)) & 15u) == 0;
  if (aligned) {
    // pairs of bins as 16-byte loads, four pairs of a thread in flight at once
    const double2* h2 = reinterpret_cast<const double2*>(hist);
    const double2* t2 = reinterpret_cast<const double2*>(target);
    double2* g2 = reinterpret_cast<double2*>(g);
    const int64_t np = nb / 2;
    for (; b + 3 * stride < np; b += 4 * stride) {
      double2 h[4], T[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        h[k] = __ldcs(h2 + b + k * stride);
        T[k] = __ldcs(t2 + b + k * stride);
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        bad |= !target_ok(T[k].x) || !target_ok(T[k].y);
        const double gx = chi2_bin(h[k].x, T[k].x, c, &part);
        const double gy = chi2_bin(h[k].y, T[k].y, c, &part);
        if (g) g2[b + k * stride] = make_double2(gx, gy);
      }
    }
    for (; b < np; b += stride) {
      const double2 h = h2[b], T = t2[b];
      bad |= !target_ok(T.x) || !target_ok(T.y);
      const double gx = chi2_bin(h.x, T.x, c, &part);
      const double gy = chi2_bin(h.y, T.y, c, &part);
      if (g) g2[b] = make_double2(gx, gy);
    }
    // the odd last bin
    if ((nb & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
      const double T = target[nb - 1];
      bad |= !target_ok(T);
      const double gb = chi2_bin(hist[nb - 1], T, c, &part);
      if (g) g[nb - 1] = gb;
    }
  } else {
    for (; b < nb; b += stride) {
      const double T = target[b];
      bad |= !target_ok(T);
      const double gb = chi2_bin(hist[b], T, c, &part);
      if (g) g[b] = gb;
    }
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0 && err) atomicOr(err, 1);
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

// Random FP64 atomic adds into a histogram of nb bins: n_adds adds of 1.0 at bins drawn by
// a 64-bit integer hash of (seed, add index) -- the access pattern of the histogram stage
// (scattered single adds) without any of the tracing work.
__global__ void __launch_bounds__(256) atomics_kernel(double* __restrict__ hist, int64_t nb,
                                                      int64_t n_adds, uint64_t seed) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_adds; i += stride) {
    uint64_t h = (uint64_t)i * 0x9E3779B97F4A7C15ull + seed;  // splitmix64 finaliser
    h = (h ^ (h >> 30)) * 0xBF58476D1CE4E5B9ull;
    h = (h ^ (h >> 27)) * 0x94D049BB133111EBull;
    h ^= h >> 31;
    atomicAdd(hist + (int64_t)(h % (uint64_t)nb), 1.0);
  }
}

}  // namespace

cudaError_t launch_atomics(double* hist, int64_t nb, int64_t n_adds, uint64_t seed, int grid,
                           cudaStream_t s) {
  if (n_adds <= 0) return cudaSuccess;
  atomics_kernel<<<grid, 256, 0, s>>>(hist, nb, n_adds, seed);
  return cudaGetLastError();
}

int trace_threads() { return 128; }

cudaError_t trace_blocks_per_sm(int fp_mode, int ns, int det, int bvk, int* blocks) {
  return fp_mode == MCV_FP32 ? blocks_per_sm_f32(ns, det, bvk, blocks)
                             : blocks_per_sm_f64(ns, det, bvk, blocks);
}

cudaError_t launch_trace(const TraceArgs& A, int fp_mode, int det, int grid, cudaStream_t s) {
  return fp_mode == MCV_FP32 ? launch_trace_f32(A, det, grid, s) : launch_trace_f64(A, det, grid, s);
}

cudaError_t launch_beam(const TraceArgs& A, int fp_mode, int grid, cudaStream_t s) {
  return fp_mode == MCV_FP32 ? launch_beam_f32(A, grid, s) : launch_beam_f64(A, grid, s);
}

cudaError_t launch_detect(const TraceArgs& A, const EventsArgs& E, int fp_mode, int det, int grid,
                          cudaStream_t s) {
  return fp_mode == MCV_FP32 ? launch_detect_f32(A, E, det, grid, s)
                             : launch_detect_f64(A, E, det, grid, s);
}

cudaError_t launch_adjoint(const TraceArgs& A, int fp_mode, int det, int grid, cudaStream_t s) {
  return fp_mode == MCV_FP32 ? launch_adjoint_f32(A, det, grid, s) : launch_adjoint_f64(A, det, grid, s);
}

cudaError_t launch_paper(const TraceArgs& A, int fp_mode, int det, int grid, cudaStream_t s) {
  return fp_mode == MCV_FP32 ? launch_paper_f32(A, det, grid, s) : launch_paper_f64(A, det, grid, s);
}

cudaError_t adjoint_blocks_per_sm(int fp_mode, int ns, int det, int bvk, int* blocks) {
  return fp_mode == MCV_FP32 ? adjoint_blocks_per_sm_f32(ns, det, bvk, blocks)
                             : adjoint_blocks_per_sm_f64(ns, det, bvk, blocks);
}

cudaError_t batch_blocks_per_sm(int fp_mode, int ns, int det, int bvk, int ss, int ev,
                                int* blocks) {
  if (ev)
    return fp_mode == MCV_FP32 ? batch_blocks_per_sm_f32_ev(ns, det, bvk, ss, blocks)
                               : batch_blocks_per_sm_f64_ev(ns, det, bvk, ss, blocks);
  return fp_mode == MCV_FP32 ? batch_blocks_per_sm_f32(ns, det, bvk, ss, blocks)
                             : batch_blocks_per_sm_f64(ns, det, bvk, ss, blocks);
}

cudaError_t launch_batch(const TraceArgs& A, const BatchArgs& Q, int fp_mode, int ns, int det,
                         int bvk, int ss, int ev, int grid, cudaStream_t s) {
  if (ev)
    return fp_mode == MCV_FP32 ? launch_batch_f32_ev(A, Q, ns, det, bvk, ss, grid, s)
                               : launch_batch_f64_ev(A, Q, ns, det, bvk, ss, grid, s);
  return fp_mode == MCV_FP32 ? launch_batch_f32(A, Q, ns, det, bvk, ss, grid, s)
                             : launch_batch_f64(A, Q, ns, det, bvk, ss, grid, s);
}

cudaError_t launch_zero(double* p, int64_t n, int grid, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  zero_kernel<<<grid, 256, 0, s>>>(p, n);
  return cudaGetLastError();
}

cudaError_t launch_chi2(const double* hist, const double* target, double c, int64_t nb,
                        double* g, double* loss, int* err, int grid, cudaStream_t s) {
  chi2_kernel<<<grid, 256, 0, s>>>(hist, target, c, nb, g, loss, err);
  return cudaGetLastError();
}

}  // namespace mcv
