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
//
// GB300's FP64 pipe runs a warp instruction at 2 lanes per clock per SM whatever the number of
// lanes it needs, and almost every bin of a large detector is empty (both values +0).  Each
// warp therefore streams its range as integers and queues only the non-empty bins in shared
// memory (value pair and index); the FP64 arithmetic runs on full batches of 32 queued bins
// (and once on the remainder).
constexpr int kChi2Threads = 256;
constexpr int kChi2Warps = kChi2Threads / 32;

struct Chi2Queue {
  double h[64], T[64];
  int64_t bin[64];
};

// one queued bin per lane, lanes [0, n): its loss term into *part, its g_b into g
__device__ __forceinline__ void chi2_drain(const Chi2Queue& q, int first, int n, double c,
                                           double* __restrict__ g, double* part) {
  const int lane = threadIdx.x & 31;
  if (lane < n) {
    const double gb = chi2_bin(q.h[first + lane], q.T[first + lane], c, part);
    if (g) g[q.bin[first + lane]] = gb;
  }
}

__global__ void __launch_bounds__(kChi2Threads) chi2_kernel(const double* __restrict__ hist,
                                                           const double* __restrict__ target,
                                                           double c, int64_t nb,
                                                           double* __restrict__ g,
                                                           double* __restrict__ loss, int* err) {
  __shared__ Chi2Queue queues[kChi2Warps];
  double part = 0.0;
  bool bad = false;
  const unsigned kFull = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  const bool aligned = ((reinterpret_cast<uintptr_t>(hist) | reinterpret_cast<uintptr_t>(target) |
                         reinterpret_cast<uintptr_t>(g)) & 15u) == 0;
  if (aligned) {
    // each warp takes a contiguous range of bin pairs, 32 lanes x 4 pairs (16-byte loads)
    // per step, so that every step and every branch below is the whole warp's
    Chi2Queue& q = queues[threadIdx.x >> 5];
    const double2* h2 = reinterpret_cast<const double2*>(hist);
    const double2* t2 = reinterpret_cast<const double2*>(target);
    const int64_t np = nb / 2;
    const int64_t nwarps = (int64_t)gridDim.x * kChi2Warps;
    const int64_t w = (int64_t)blockIdx.x * kChi2Warps + (threadIdx.x >> 5);
    const int64_t per = ((np + nwarps - 1) / nwarps + 127) / 128 * 128;
    const int64_t lo = min(np, w * per), hi = min(np, lo + per);
    int qn = 0;  // queued bins (the same in every lane)
    for (int64_t p0 = lo; p0 < hi; p0 += 128) {
      double2 h[4], T[4];
      bool valid[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int64_t p = p0 + 32 * k + lane;
        valid[k] = p < hi;  // pairs past hi are the next warp's
        if (valid[k]) {
          h[k] = __ldcs(h2 + p);
          T[k] = __ldcs(t2 + p);
        } else {
          h[k] = make_double2(0.0, 0.0);
          T[k] = make_double2(0.0, 0.0);
        }
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const double hv = (k & 1) ? h[k >> 1].y : h[k >> 1].x;
        const double Tv = (k & 1) ? T[k >> 1].y : T[k >> 1].x;
        const int64_t bin = 2 * (p0 + 32 * (k >> 1) + lane) + (k & 1);
        bad |= !target_ok(Tv);
        const bool nz = (__double_as_longlong(hv) | __double_as_longlong(Tv)) != 0;
        const unsigned m = __ballot_sync(kFull, nz);
        if (nz) {
          const int at = qn + __popc(m & lt_mask);
          q.h[at] = hv;
          q.T[at] = Tv;
          q.bin[at] = bin;
        } else if (g && valid[k >> 1]) {
          g[bin] = 0.0;
        }
        qn += __popc(m);
        if (qn >= 32) {
          __syncwarp();
          chi2_drain(q, qn - 32, 32, c, g, &part);
          __syncwarp();
          qn -= 32;
        }
      }
    }
    __syncwarp();
    chi2_drain(q, 0, qn, c, g, &part);
    // the odd last bin
    if ((nb & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
      const double T = target[nb - 1];
      bad |= !target_ok(T);
      const double gb = chi2_bin(hist[nb - 1], T, c, &part);
      if (g) g[nb - 1] = gb;
    }
  } else {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += stride) {
      const double T = target[b];
      bad |= !target_ok(T);
      const double gb = chi2_bin(hist[b], T, c, &part);
      if (g) g[b] = gb;
    }
  }
  if (__any_sync(kFull, bad) && lane == 0 && err) atomicOr(err, 1);
  part = warp_sum(part);
  __shared__ double red[kChi2Warps];
  const int wi = threadIdx.x >> 5;
  if (lane == 0) red[wi] = part;
  __syncthreads();
  if (wi == 0) {
    double v = lane < kChi2Warps ? red[lane] : 0.0;
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
  chi2_kernel<<<grid, kChi2Threads, 0, s>>>(hist, target, c, nb, g, loss, err);
  return cudaGetLastError();
}

}  // namespace mcv
