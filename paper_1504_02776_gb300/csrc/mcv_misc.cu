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
cudaError_t adjoint_blocks_per_sm_f32(int ns, int det, int bvk, int* blocks);
cudaError_t adjoint_blocks_per_sm_f64(int ns, int det, int bvk, int* blocks);
cudaError_t batch_blocks_per_sm_f32(int ns, int det, int bvk, int ss, int* blocks);
cudaError_t batch_blocks_per_sm_f64(int ns, int det, int bvk, int ss, int* blocks);
cudaError_t launch_batch_f32(const TraceArgs& A, const BatchArgs& Q, int ns, int det, int bvk,
                             int ss, int grid, cudaStream_t s);
cudaError_t launch_batch_f64(const TraceArgs& A, const BatchArgs& Q, int ns, int det, int bvk,
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
// g_b = dchi2/dI_b for every bin.  Without g the kernel only reads (16 bytes per bin): the
// adjoint evaluates g_b itself for the bins its packets reach.  A measured bin that is
// negative or not finite sets the error flag (err, optional).
__global__ void __launch_bounds__(256) chi2_kernel(const double* __restrict__ hist,
                                                   const double* __restrict__ target, double c,
                                                   int64_t nb, double* __restrict__ g,
                                                   double* __restrict__ loss, int* err) {
  double part = 0.0;
  bool bad = false;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  // four grid-strided bins per pass, their loads issued together; the bins of a thread are
  // summed in the same order as one at a time
  for (; b + 3 * stride < nb; b += 4 * stride) {
    double h[4], T[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      h[k] = hist[b + k * stride];
      T[k] = target[b + k * stride];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      bad |= !target_ok(T[k]);
      const double gb = chi2_bin(h[k], T[k], c, &part);
      if (g) g[b + k * stride] = gb;
    }
  }
  for (; b < nb; b += stride) {
    const double T = target[b];
    bad |= !target_ok(T);
    const double gb = chi2_bin(hist[b], T, c, &part);
    if (g) g[b] = gb;
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

}  // namespace

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

cudaError_t adjoint_blocks_per_sm(int fp_mode, int ns, int det, int bvk, int* blocks) {
  return fp_mode == MCV_FP32 ? adjoint_blocks_per_sm_f32(ns, det, bvk, blocks)
                             : adjoint_blocks_per_sm_f64(ns, det, bvk, blocks);
}

cudaError_t batch_blocks_per_sm(int fp_mode, int ns, int det, int bvk, int ss, int* blocks) {
  return fp_mode == MCV_FP32 ? batch_blocks_per_sm_f32(ns, det, bvk, ss, blocks)
                             : batch_blocks_per_sm_f64(ns, det, bvk, ss, blocks);
}

cudaError_t launch_batch(const TraceArgs& A, const BatchArgs& Q, int fp_mode, int ns, int det,
                         int bvk, int ss, int grid, cudaStream_t s) {
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
