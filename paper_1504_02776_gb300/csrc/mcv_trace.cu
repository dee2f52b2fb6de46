// Kernels of the forward path: the source, the sample assembly traced as a bounded chain of
// scatterings per neutron (optionally fused with the detector system and the histogram),
// and the detector system on stored packets.
//
// Work layout of the chain kernel: one neutron per lane, a persistent grid, and each warp
// owning a contiguous range of neutron ids.  A lane whose neutron has finished (missed the
// sample, left it, reached max_orders, or was dropped) takes the next id of its warp's
// range at the top of the next step, so every step of the loop runs the same code on all
// 32 lanes (the warp-level compaction of surviving neutrons between scattering orders).
#include <cuda_runtime.h>

#include "mcv_chain.cuh"
#include "mcv_launch.h"

namespace mcv {

namespace {

constexpr int kThreads = 128;

template <typename R>
__device__ __forceinline__ void store_slot(const TraceArgs& A, int64_t slot, const Ray<R>& n, R w,
                                           int64_t nid, int order) {
  static_cast<R*>(A.pk_x)[slot] = n.x;
  static_cast<R*>(A.pk_y)[slot] = n.y;
  static_cast<R*>(A.pk_z)[slot] = n.z;
  static_cast<R*>(A.pk_vx)[slot] = n.speed * n.dx;
  static_cast<R*>(A.pk_vy)[slot] = n.speed * n.dy;
  static_cast<R*>(A.pk_vz)[slot] = n.speed * n.dz;
  static_cast<R*>(A.pk_w)[slot] = w;
  A.pk_t[slot] = n.t;
  A.pk_id[slot] = nid;
  A.pk_order[slot] = order;
}

// Forward policy: packets go to the packet slots and/or through the detector into the
// histogram; order-0 packets go to the beam stop.
template <typename R, int DET>
struct Forward {
  static constexpr bool kWantsGs = false;
  Acc<R> a_bs, a_det, a_over;
  Counts cnt;
  int err = 0;

  __device__ __forceinline__ void start(const Lane<R>&) {}

  __device__ __forceinline__ void emit(const TraceArgs& A, const R* tu, const NeutronRng& rng,
                                       const Lane<R>& L, R we, R, R, R len_tot) {
    if (L.o == 0 && len_tot > R(0)) cnt.nhit++;
    if (A.pk_order) store_slot<R>(A, L.idx * (A.S.max_orders + 1) + L.o, L.n, we, L.nid, L.o);
    if (L.o == 0) {
      a_bs.add(we);
      return;
    }
    cnt.nemit++;
    if (DET == MCV_DET_NONE) return;
    Ray<R> pe = L.n;
    pe.w = we;
    const Hit<R> h = detect<R, DET>(A.D, tu, rng, L.o, pe);
    if (h.bin >= 0) {
      if (h.bin >= A.D.n_bins) {
        err = 1;
        return;
      }
      if (A.hist) atomicAdd(A.hist + h.bin, (double)h.w_det);
      a_det.add(h.w_det);
      cnt.ndet++;
    } else if (h.bin == -2) {
      a_over.add(h.w_det);
      cnt.nover++;
    } else {
      cnt.nmiss++;
    }
  }

  __device__ __forceinline__ void scatter(const TraceArgs&, const Lane<R>&, int, R,
                                          const Scatter<R>&, R, R) {}

  __device__ __forceinline__ void clear(const TraceArgs& A, int64_t idx, int first) {
    if (!A.pk_order) return;
    const int slots = A.S.max_orders + 1;
    for (int o = first; o < slots; ++o) {
      A.pk_order[idx * slots + o] = -1;
      A.pk_id[idx * slots + o] = -1;
    }
  }

  __device__ __forceinline__ void flush(const TraceArgs& A, int lane) {
    if (A.tallies) {
      const double v_bs = warp_sum(a_bs.value());
      const double v_det = warp_sum(a_det.value());
      const double v_over = warp_sum(a_over.value());
      const uint32_t n_det = warp_sum(cnt.ndet), n_over = warp_sum(cnt.nover);
      const uint32_t n_miss = warp_sum(cnt.nmiss), n_hit = warp_sum(cnt.nhit);
      const uint32_t n_emit = warp_sum(cnt.nemit);
      if (lane == 0) {
        atomicAdd(A.tallies + MCV_T_BEAMSTOP, v_bs);
        atomicAdd(A.tallies + MCV_T_WDET, v_det);
        atomicAdd(A.tallies + MCV_T_WOVER, v_over);
        atomicAdd(A.tallies + MCV_T_NDET, (double)n_det);
        atomicAdd(A.tallies + MCV_T_NOVER, (double)n_over);
        atomicAdd(A.tallies + MCV_T_NMISS, (double)n_miss);
        atomicAdd(A.tallies + MCV_T_NHIT, (double)n_hit);
        atomicAdd(A.tallies + MCV_T_NEMIT, (double)n_emit);
      }
    }
    if (__any_sync(0xffffffffu, err != 0) && lane == 0 && A.err) atomicOr(A.err, 1);
  }
};

template <typename R, int NS, int DET>
__global__ void __launch_bounds__(kThreads) trace_kernel(const __grid_constant__ TraceArgs A) {
  __shared__ R tu[2 * MCV_MAX_TUBES_PER_ROW];
  stage_tubes<R, DET>(A, tu);
  Forward<R, DET> pol;
  run_chain<R, NS, DET, Forward<R, DET>>(A, tu, pol);
}

template <typename R>
__global__ void __launch_bounds__(kThreads) beam_kernel(const __grid_constant__ TraceArgs A) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < A.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t nid = A.first_id + i;
    const NeutronRng rng(A.seed, A.sim_id, nid);
    Ray<R> n;
    const bool ok = make_beam<R>(A.B, rng, &n);
    if (!ok) {
      n.x = n.y = n.z = R(0);
      n.dx = n.dy = n.dz = R(0);
      n.speed = R(0);
      n.t = 0.0;
      n.w = R(0);
    }
    static_cast<R*>(A.pk_x)[i] = n.x;
    static_cast<R*>(A.pk_y)[i] = n.y;
    static_cast<R*>(A.pk_z)[i] = n.z;
    static_cast<R*>(A.pk_vx)[i] = n.speed * n.dx;
    static_cast<R*>(A.pk_vy)[i] = n.speed * n.dy;
    static_cast<R*>(A.pk_vz)[i] = n.speed * n.dz;
    static_cast<R*>(A.pk_w)[i] = n.w;
    A.pk_t[i] = n.t;
    if (A.pk_id) A.pk_id[i] = nid;
    if (A.pk_order) A.pk_order[i] = ok ? 0 : -1;
  }
}

template <typename R, int DET>
__global__ void __launch_bounds__(kThreads) detect_kernel(const __grid_constant__ TraceArgs A,
                                                          EventsArgs E) {
  __shared__ R tu[2 * MCV_MAX_TUBES_PER_ROW];
  stage_tubes<R, DET>(A, tu);
  Acc<R> a_bs, a_det, a_over;
  Counts cnt;
  int err = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < A.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int o = A.in_order[i];
    if (o < 0) continue;
    const R w = static_cast<const R*>(A.in_w)[i];
    if (o == 0) {
      a_bs.add(w);
      if (E.bin) E.bin[i] = -1;
      if (E.pixel) E.pixel[i] = -1;
      if (E.tof) E.tof[i] = 0.0;
      if (E.w_det) E.w_det[i] = 0.0;
      continue;
    }
    Ray<R> n;
    if (!load_input<R>(A, i, &n)) continue;
    cnt.nemit++;
    const NeutronRng rng(A.seed, A.sim_id, A.in_id[i]);
    const Hit<R> h = detect<R, DET>(A.D, tu, rng, o, n);
    if (h.bin >= 0) {
      if (h.bin >= A.D.n_bins) {
        err = 1;
        continue;
      }
      if (A.hist) atomicAdd(A.hist + h.bin, (double)h.w_det);
      a_det.add(h.w_det);
      cnt.ndet++;
    } else if (h.bin == -2) {
      a_over.add(h.w_det);
      cnt.nover++;
    } else {
      cnt.nmiss++;
    }
    if (E.bin) E.bin[i] = h.bin;
    if (E.pixel) E.pixel[i] = h.pixel;
    if (E.tof) E.tof[i] = h.tof;
    if (E.w_det) E.w_det[i] = (double)h.w_det;
  }
  const int lane = threadIdx.x & 31;
  if (A.tallies) {
    const double v_bs = warp_sum(a_bs.value());
    const double v_det = warp_sum(a_det.value());
    const double v_over = warp_sum(a_over.value());
    const uint32_t n_det = warp_sum(cnt.ndet), n_over = warp_sum(cnt.nover);
    const uint32_t n_miss = warp_sum(cnt.nmiss), n_emit = warp_sum(cnt.nemit);
    if (lane == 0) {
      atomicAdd(A.tallies + MCV_T_BEAMSTOP, v_bs);
      atomicAdd(A.tallies + MCV_T_WDET, v_det);
      atomicAdd(A.tallies + MCV_T_WOVER, v_over);
      atomicAdd(A.tallies + MCV_T_NDET, (double)n_det);
      atomicAdd(A.tallies + MCV_T_NOVER, (double)n_over);
      atomicAdd(A.tallies + MCV_T_NMISS, (double)n_miss);
      atomicAdd(A.tallies + MCV_T_NEMIT, (double)n_emit);
    }
  }
  if (__any_sync(0xffffffffu, err != 0) && lane == 0 && A.err) atomicOr(A.err, 1);
}

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

template <typename R, int NS>
cudaError_t launch_trace_ns(const TraceArgs& A, int det, int grid, cudaStream_t s) {
  switch (det) {
    case MCV_DET_SURFACE:
      trace_kernel<R, NS, MCV_DET_SURFACE><<<grid, kThreads, 0, s>>>(A);
      break;
    case MCV_DET_TUBES:
      trace_kernel<R, NS, MCV_DET_TUBES><<<grid, kThreads, 0, s>>>(A);
      break;
    default:
      trace_kernel<R, NS, MCV_DET_NONE><<<grid, kThreads, 0, s>>>(A);
      break;
  }
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_trace_r(const TraceArgs& A, int det, int grid, cudaStream_t s) {
  if (A.S.ns <= 1) return launch_trace_ns<R, 1>(A, det, grid, s);
  if (A.S.ns == 2) return launch_trace_ns<R, 2>(A, det, grid, s);
  return launch_trace_ns<R, 4>(A, det, grid, s);
}

template <typename R>
const void* trace_fn(int ns, int det) {
  if (ns <= 1) {
    if (det == MCV_DET_SURFACE) return (const void*)trace_kernel<R, 1, MCV_DET_SURFACE>;
    if (det == MCV_DET_TUBES) return (const void*)trace_kernel<R, 1, MCV_DET_TUBES>;
    return (const void*)trace_kernel<R, 1, MCV_DET_NONE>;
  }
  if (ns == 2) {
    if (det == MCV_DET_SURFACE) return (const void*)trace_kernel<R, 2, MCV_DET_SURFACE>;
    if (det == MCV_DET_TUBES) return (const void*)trace_kernel<R, 2, MCV_DET_TUBES>;
    return (const void*)trace_kernel<R, 2, MCV_DET_NONE>;
  }
  if (det == MCV_DET_SURFACE) return (const void*)trace_kernel<R, 4, MCV_DET_SURFACE>;
  if (det == MCV_DET_TUBES) return (const void*)trace_kernel<R, 4, MCV_DET_TUBES>;
  return (const void*)trace_kernel<R, 4, MCV_DET_NONE>;
}

}  // namespace

int trace_threads() { return kThreads; }

cudaError_t trace_blocks_per_sm(int fp_mode, int ns, int det, int* blocks) {
  const void* fn = (fp_mode == MCV_FP32) ? trace_fn<float>(ns, det) : trace_fn<double>(ns, det);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, fn, kThreads, 0);
}

cudaError_t launch_trace(const TraceArgs& A, int fp_mode, int det, int grid, cudaStream_t s) {
  if (fp_mode == MCV_FP32) return launch_trace_r<float>(A, det, grid, s);
  return launch_trace_r<double>(A, det, grid, s);
}

cudaError_t launch_beam(const TraceArgs& A, int fp_mode, int grid, cudaStream_t s) {
  if (fp_mode == MCV_FP32)
    beam_kernel<float><<<grid, kThreads, 0, s>>>(A);
  else
    beam_kernel<double><<<grid, kThreads, 0, s>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_detect(const TraceArgs& A, const EventsArgs& E, int fp_mode, int det, int grid,
                          cudaStream_t s) {
  if (fp_mode == MCV_FP32) {
    if (det == MCV_DET_SURFACE)
      detect_kernel<float, MCV_DET_SURFACE><<<grid, kThreads, 0, s>>>(A, E);
    else
      detect_kernel<float, MCV_DET_TUBES><<<grid, kThreads, 0, s>>>(A, E);
  } else {
    if (det == MCV_DET_SURFACE)
      detect_kernel<double, MCV_DET_SURFACE><<<grid, kThreads, 0, s>>>(A, E);
    else
      detect_kernel<double, MCV_DET_TUBES><<<grid, kThreads, 0, s>>>(A, E);
  }
  return cudaGetLastError();
}

cudaError_t launch_zero(double* p, int64_t n, int grid, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  zero_kernel<<<grid, 256, 0, s>>>(p, n);
  return cudaGetLastError();
}

}  // namespace mcv
