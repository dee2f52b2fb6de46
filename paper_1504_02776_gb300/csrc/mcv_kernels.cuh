// Kernel templates of the hot path, instantiated once per real type: mcv_fp32.cu (FP32
// fast mode) and mcv_fp64.cu (FP64 mode, compiled without FMA contraction so that its
// arithmetic rounds like the plain restatement of the method).
//
// The chain kernel: one neutron per lane, a persistent grid, and each warp owning a
// contiguous range of neutron ids.  A lane whose neutron has finished (missed the sample,
// left it, reached max_orders, or was dropped) takes the next id of its warp's range at
// the top of the next step, so every step of the loop runs the same code on all 32 lanes
// (the warp-level compaction of surviving neutrons between scattering orders).
#pragma once

#include <cuda_runtime.h>

#include "mcv_chain.cuh"
#include "mcv_chi2.cuh"
#include "mcv_launch.h"

namespace mcv {

// largest number of scattering orders of a packet (mcv_sample::max_orders <= 7)
constexpr int kMaxOrders = 7;

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
  A.pk_t[slot] = n.t.value();
  A.pk_id[slot] = nid;
  A.pk_order[slot] = order;
}

// Where the forward path's histogram and tallies are: the launch's (kernel parameters).
// EV: the launch may append to an event list (the code for it is compiled in only then).
template <bool EV>
struct LaunchOutT {
  static constexpr bool kEvents = EV;
  static __device__ __forceinline__ double* hist(const TraceArgs& A) { return A.hist; }
  static __device__ __forceinline__ double* tallies(const TraceArgs& A) { return A.tallies; }
  static __device__ __forceinline__ const EvSink& events(const TraceArgs& A) { return A.ev; }
};
using LaunchOut = LaunchOutT<true>;

// one thread's running tallies: beam stop, detected and out-of-window weights, counts
template <typename R>
struct Tally {
  Acc<R> bs, det, over;
  Counts cnt;
};

// the tallies held in registers
template <typename R>
struct RegTally {
  Tally<R> t;
  __device__ __forceinline__ Tally<R>& get() { return t; }
};

// Forward policy: packets go to the packet slots and/or through the detector into the
// histogram; order-0 packets go to the beam stop.  Out: where the histogram and tallies of
// the simulation being traced are (read where used, so they hold no registers).  Store:
// where the thread's running tallies are kept.
template <typename R, int DET, class Out = LaunchOut, class Store = RegTally<R>>
struct Forward {
  static constexpr bool kWantsGs = false;
  static constexpr bool kMeetingOnly = false;
  Store store;
  int err = 0;

  __device__ __forceinline__ void start(const Lane<R>&) {}

  template <class Rng>
  __device__ __forceinline__ void emit(const TraceArgs& A, const R* tu, const Rng& rng,
                                       const Lane<R>& L, R we, R, R, R len_tot) {
    Tally<R>& t = store.get();
    if (L.o == 0 && len_tot > R(0)) t.cnt.nhit++;
    if (A.pk_order) store_slot<R>(A, L.idx * (Sof<R>(A).max_orders + 1) + L.o, L.n, we, L.nid, L.o);
    if (L.o == 0) {
      t.bs.add(we);
      return;
    }
    t.cnt.nemit++;
    if (DET == MCV_DET_NONE) return;
    Ray<R> pe = L.n;
    pe.w = we;
    record(A, detect<R, DET>(Dof<R>(A), Dof<R>(A).win, tu, rng, L.o, pe));
  }

  // a packet's detector result into the histogram and the tallies
  __device__ __forceinline__ void record(const TraceArgs& A, const Hit<R>& h) {
    Tally<R>& t = store.get();
    if constexpr (Out::kEvents) {
      if (h.pixel >= 0 && Out::events(A).count)
        append_event(Out::events(A), h.pixel, h.tof.value(), (double)h.w_det);
    }
    // Equal bins among the lanes recording together (a detector batch) are summed in the
    // group's lowest lane and added with one FP64 atomic: fewer atomics on the bins that
    // collect many events (the elastic line; low incident energies concentrate more).
    const bool valid = h.bin >= 0 && h.bin < Dof<R>(A).n_bins;
    const unsigned act = __activemask();
    const int lane = threadIdx.x & 31;
    const long long key = valid ? (long long)h.bin : -1ll - lane;
    const unsigned peers = __match_any_sync(act, key);
    if (valid) {
      double* hist = Out::hist(A);
      const double v = (double)h.w_det;
      if (peers == (1u << lane)) {
        if (hist) atomicAdd(hist + h.bin, v);
      } else {
        const int leader = __ffs(peers) - 1;
        double sum = 0.0;
        for (unsigned m = peers; m; m &= m - 1) {
          const double x = __shfl_sync(peers, v, __ffs(m) - 1);
          sum += x;
        }
        if (hist && lane == leader) atomicAdd(hist + h.bin, sum);
      }
    }
    if (h.bin >= 0) {
      if (h.bin >= Dof<R>(A).n_bins) {
        err = 1;
        return;
      }
      t.det.add(h.w_det);
      t.cnt.ndet++;
    } else if (h.bin == -2) {
      t.over.add(h.w_det);
      t.cnt.nover++;
    } else {
      t.cnt.nmiss++;
    }
  }

  // the beam stop's share of a packet of order 0, and an incident neutron meeting the sample
  __device__ __forceinline__ void beam_stop(R w) { store.get().bs.add(w); }
  // a packet that misses the detector system
  __device__ __forceinline__ void missed() { store.get().cnt.nmiss++; }
  __device__ __forceinline__ void hit() { store.get().cnt.nhit++; }
  __device__ __forceinline__ void emitted() { store.get().cnt.nemit++; }

  __device__ __forceinline__ void scatter(const TraceArgs&, const Lane<R>&, int, R,
                                          const Scatter<R>&, R, R) {}

  __device__ __forceinline__ void clear(const TraceArgs& A, int64_t idx, int first) {
    if (!A.pk_order) return;
    const int slots = Sof<R>(A).max_orders + 1;
    for (int o = first; o < slots; ++o) {
      A.pk_order[idx * slots + o] = -1;
      A.pk_id[idx * slots + o] = -1;
    }
  }

  // the warp's tallies into `tallies`; the accumulators start again from zero
  __device__ __forceinline__ void flush(const TraceArgs& A, int lane) {
    double* tallies = Out::tallies(A);
    Tally<R>& t = store.get();
    if (tallies) {
      const double v_bs = warp_sum(t.bs.value());
      const double v_det = warp_sum(t.det.value());
      const double v_over = warp_sum(t.over.value());
      const uint32_t n_det = warp_sum(t.cnt.ndet), n_over = warp_sum(t.cnt.nover);
      const uint32_t n_miss = warp_sum(t.cnt.nmiss), n_hit = warp_sum(t.cnt.nhit);
      const uint32_t n_emit = warp_sum(t.cnt.nemit);
      if (lane == 0) {
        atomicAdd(tallies + MCV_T_BEAMSTOP, v_bs);
        atomicAdd(tallies + MCV_T_WDET, v_det);
        atomicAdd(tallies + MCV_T_WOVER, v_over);
        atomicAdd(tallies + MCV_T_NDET, (double)n_det);
        atomicAdd(tallies + MCV_T_NOVER, (double)n_over);
        atomicAdd(tallies + MCV_T_NMISS, (double)n_miss);
        atomicAdd(tallies + MCV_T_NHIT, (double)n_hit);
        atomicAdd(tallies + MCV_T_NEMIT, (double)n_emit);
      }
    }
    if (__any_sync(0xffffffffu, err != 0) && lane == 0 && A.err) atomicOr(A.err, 1);
    t = Tally<R>();
  }
};

// ---- the fused forward path, organised as waves --------------------------------------------
// Three stages per warp, each run by all 32 lanes on their own work items:
//   source:   32 new neutrons at a time; those that miss the sample only add their weight
//             to the beam stop, those that meet it are queued (warp queue in shared memory);
//   sample:   one order step of every lane's neutron (idle lanes take queued neutrons); the
//             transmitted packets of orders >= 1 are queued for the detector;
//   detector: whenever 32 packets are queued, each lane traces one through the detector
//             system and histograms it.
// The per-neutron arithmetic is the chain step's and the detector's: only the order in
// which lanes do the work changes, which keeps the lanes of a warp busy on the same code.
constexpr int kWarps = kThreads / 32;
constexpr int kQueue = 64;  // per-warp queue capacity (at most 63 entries are ever held)

template <typename R>
struct QNeutron {  // an incident neutron that meets the sample
  R x, y, z, dx, dy, dz, speed;
  Tof<R> t;
  int64_t nid;
};

template <typename R>
struct QPacket {  // a transmitted packet of order >= 1 on its way to the detector
  R x, y, z, dx, dy, dz, speed, w;
  Tof<R> t;
  int64_t nid;
  int order;
  int16_t row, g;  // located packets (FP64 tube detector): row, tube nearest to the crossing
};

template <typename R>
struct QFoot {  // a footprint that may lead into the sample
  R x, y;
  int64_t nid;
};

template <typename R>
constexpr size_t wave_smem_bytes() {
  return (size_t)kWarps * kQueue * (sizeof(QNeutron<R>) + sizeof(QPacket<R>) + sizeof(QFoot<R>));
}

extern __shared__ __align__(16) unsigned char g_wave_smem[];

// Sources of neutron-id ranges for the waves: a single range, or further items of the same
// simulation from its work queue (warp-collective: called by all 32 lanes together).
struct NoMoreIds {
  __device__ __forceinline__ bool more(int64_t*, int64_t*) { return false; }
};

// A warp's slot in the batched kernel's shared memory: the simulation it traces and that
// simulation's work queue, and the warp's walk over the simulations.  Warp-uniform values
// that are read where they are used rather than held in registers.
struct QueueSlot {
  unsigned long long* ctr;
  int64_t n, chunk, items;
};

template <typename R>
struct BatchWarp {
  SimP<R> sim;
  QueueSlot q;
  int home, v;
};

// Dynamic shared memory of the wave kernels: the warp queues, [the warps' batch slots,] and
// every thread's running tallies (kept there rather than in registers).
template <typename R>
struct SmemTally {
  size_t off;  // byte offset of the tallies in the dynamic shared memory
  __device__ __forceinline__ Tally<R>& get() {
    return reinterpret_cast<Tally<R>*>(g_wave_smem + off)[threadIdx.x];
  }
};

template <typename R>
constexpr size_t wave_kernel_smem_bytes() {
  return wave_smem_bytes<R>() + (size_t)kThreads * sizeof(Tally<R>);
}

template <typename R>
constexpr size_t batch_tally_offset() {
  return wave_smem_bytes<R>() + (size_t)kWarps * sizeof(BatchWarp<R>);
}

template <typename R>
constexpr size_t batch_smem_bytes() {
  return batch_tally_offset<R>() + (size_t)kThreads * sizeof(Tally<R>);
}

template <typename R>
__device__ __forceinline__ BatchWarp<R>& batch_warp() {
  return reinterpret_cast<BatchWarp<R>*>(g_wave_smem + wave_smem_bytes<R>())[threadIdx.x >> 5];
}

// further items of the simulation in the warp's slot, from its work queue
template <typename R>
struct QueuedIds {
  __device__ __forceinline__ bool more(int64_t* lo, int64_t* hi) {
    const QueueSlot& q = batch_warp<R>().q;
    unsigned long long k = 0;
    if ((threadIdx.x & 31) == 0) k = atomicAdd(q.ctr, 1ull);
    k = __shfl_sync(0xffffffffu, k, 0);
    if (k >= (unsigned long long)q.items) return false;
    *lo = (int64_t)k * q.chunk;
    *hi = min(*lo + q.chunk, q.n);
    return true;
  }
};

// the histogram and tallies of the simulation in the warp's slot
template <typename R, bool EV>
struct SlotOut {
  static constexpr bool kEvents = EV;
  static __device__ __forceinline__ double* hist(const TraceArgs&) { return batch_warp<R>().sim.hist; }
  static __device__ __forceinline__ double* tallies(const TraceArgs&) {
    return batch_warp<R>().sim.tallies;
  }
  static __device__ __forceinline__ const EvSink& events(const TraceArgs&) {
    return batch_warp<R>().sim.ev;
  }
};

// The simulation the waves trace: its parameters from kernel parameter space (single launch)
// or from the warp's slot of shared memory (batched launch), read where they are used.
template <typename R>
struct ParamJob {
  const TraceArgs& A;
  __device__ __forceinline__ const SampleP<R>& S() const { return Sof<R>(A); }
  __device__ __forceinline__ const BeamP<R>& B() const { return Bof<R>(A); }
  __device__ __forceinline__ const TofWin& W() const { return Dof<R>(A).win; }
  __device__ __forceinline__ NeutronRng rng(int64_t nid) const { return NeutronRng(A.keys, nid); }
  __device__ __forceinline__ int64_t first_id() const { return A.first_id; }
};

// The batched launch's simulation: the one in the warp's slot.  SS: every simulation has the
// launch's sample, which then stays in kernel parameter space.
template <typename R, bool SS>
struct SlotJob {
  const TraceArgs& A;
  __device__ __forceinline__ const SampleP<R>& S() const {
    return SS ? Sof<R>(A) : batch_warp<R>().sim.S;
  }
  __device__ __forceinline__ const BeamP<R>& B() const { return batch_warp<R>().sim.B; }
  __device__ __forceinline__ const TofWin& W() const { return batch_warp<R>().sim.win; }
  // keys computed as used: a table in shared memory would cost a load per round
  __device__ __forceinline__ NeutronRngT<KeysOnTheFly> rng(int64_t nid) const {
    const SimP<R>& J = batch_warp<R>().sim;
    return NeutronRngT<KeysOnTheFly>(KeysOnTheFly{J.seed, J.sim_id}, nid);
  }
  __device__ __forceinline__ int64_t first_id() const { return batch_warp<R>().sim.first_id; }
};

// The waves of one warp over neutron ids first_id + [lo, hi) of one simulation, and over
// every further range `src` hands out for it.  Returns with both queues empty.
template <typename R, int NS, int DET, int KS, class Job, class Src, class P>
__device__ __forceinline__ void run_waves(const TraceArgs& A, const Job& job, int64_t lo,
                                          int64_t hi, const R* tu, P& pol, Src& src) {
  const SampleP<R>& S = job.S();
  const DetP<R>& D = Dof<R>(A);
  const unsigned kFull = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const unsigned lt_mask = (1u << lane) - 1u;
  QNeutron<R>* hq = reinterpret_cast<QNeutron<R>*>(g_wave_smem) + wib * kQueue;
  QPacket<R>* dq = reinterpret_cast<QPacket<R>*>(g_wave_smem + (size_t)kWarps * kQueue *
                                                   sizeof(QNeutron<R>)) + wib * kQueue;
  QFoot<R>* fq = reinterpret_cast<QFoot<R>*>(
                     g_wave_smem + (size_t)kWarps * kQueue * (sizeof(QNeutron<R>) + sizeof(QPacket<R>))) +
                 wib * kQueue;
  int64_t next = lo;
  int hq_n = 0, dq_n = 0, fq_n = 0;
  Lane<R> L;
  L.active = false;
  L.o = 0;
  L.idx = 0;
  L.nid = 0;
  for (;;) {
    const unsigned idle = __ballot_sync(kFull, !L.active);
    const int n_idle = __popc(idle);
    // ---- source stage.  Footprints first, 32 new ids at a time: a neutron whose footprint
    // cannot lead into the sample only adds its weight to the beam stop; the others are
    // queued.  Then 32 queued footprints at a time get their divergence and, where they meet
    // the sample, their energy: those are queued for the sample stage, the rest add to the
    // beam stop.  (Misses need no energy: BeamP::x_safe is finite only when every energy
    // draw is positive.)
    while (hq_n < n_idle && (fq_n > 0 || next < hi || src.more(&next, &hi))) {
      if (fq_n < 32 && (next < hi || src.more(&next, &hi))) {
        const int64_t i = next + lane;
        bool maybe = false;
        Ray<R> nr;
        int64_t nid = 0;
        if (i < hi) {
          nid = job.first_id() + i;
          const auto rng = job.rng(nid);
          beam_footprint(job.B(), rng, &nr);
          if (!surely_misses<R>(job.B(), nr))
            maybe = true;
          else if (!(nr.w < S.min_prob) && !(A.stop_on_zero && nr.w == R(0)))
            pol.beam_stop(nr.w * Mth<R>::exp(R(0)));  // order-0 packet, no material ahead
        }
        const unsigned mm = __ballot_sync(kFull, maybe);
        if (maybe) {
          QFoot<R>& f = fq[fq_n + __popc(mm & lt_mask)];
          f.x = nr.x;
          f.y = nr.y;
          f.nid = nid;
        }
        fq_n += __popc(mm);
        next += 32;
        __syncwarp();
        continue;
      }
      const int take_f = fq_n < 32 ? fq_n : 32;
      bool hit = false;
      Ray<R> nr;
      int64_t nid = 0;
      if (lane < take_f) {
        const QFoot<R>& f = fq[fq_n - take_f + lane];
        nid = f.nid;
        nr.x = f.x;
        nr.y = f.y;
        nr.z = -job.B().z0;
        nr.w = R(1);
      }
      fq_n -= take_f;
      __syncwarp();
      if (lane < take_f) {
        const auto rng = job.rng(nid);
        R aux;
        beam_divergence(job.B(), rng, &nr, &aux);
        Seg<R> seg[2 * NS];
        const bool meets = assembly_segs<R, NS>(S, nr, seg) > 0;
        bool ok = (meets || !job.B().energy_positive) ? beam_energy(job.B(), rng, aux, &nr)
                                                      : true;
        ok = ok && !(nr.w < S.min_prob) && !(A.stop_on_zero && nr.w == R(0));
        if (ok) {
          if (meets)
            hit = true;
          else
            pol.beam_stop(nr.w * Mth<R>::exp(R(0)));  // order-0 packet, no material ahead
        }
      }
      const unsigned hm = __ballot_sync(kFull, hit);
      if (hit) {
        QNeutron<R>& q = hq[hq_n + __popc(hm & lt_mask)];
        q.x = nr.x;
        q.y = nr.y;
        q.z = nr.z;
        q.dx = nr.dx;
        q.dy = nr.dy;
        q.dz = nr.dz;
        q.speed = nr.speed;
        q.t = nr.t;
        q.nid = nid;
      }
      hq_n += __popc(hm);
      __syncwarp();
    }
    const int take = min(n_idle, hq_n);
    if (!L.active) {
      const int r = __popc(idle & lt_mask);
      if (r < take) {
        const QNeutron<R>& q = hq[hq_n - take + r];
        L.n.x = q.x;
        L.n.y = q.y;
        L.n.z = q.z;
        L.n.dx = q.dx;
        L.n.dy = q.dy;
        L.n.dz = q.dz;
        L.n.speed = q.speed;
        L.n.t = q.t;
        L.n.w = R(1);
        L.nid = q.nid;
        L.o = 0;
        L.active = true;
      }
    }
    hq_n -= take;
    __syncwarp();
    // ---- sample stage.  FP64: a transmitted packet of order >= 1 is first located on the
    // tube rows (row and candidate tubes) and only packets that can reach a tube are queued
    // for the detector stage (the FP64 detector arithmetic is costly enough that skipping it
    // for the ~3/4 of packets that miss pays for the idle order-0 lanes here); FP32: all of
    // them are queued and the detector stage locates them, with every lane busy.
    constexpr bool kLocateEarly = DET == MCV_DET_TUBES && sizeof(R) == 8;
    StepState<R, NS> st;
    R we = R(0);
    bool to_det = false;
    int row = 0, g = 0;
    if (L.active) {
      we = step_segments<R, NS, false>(A, S, L, st);
      if (L.o == 0) {
        pol.beam_stop(we);
        if (st.len_tot > R(0)) pol.hit();
      } else {
        pol.emitted();
        if (DET == MCV_DET_TUBES && det_surely_misses<R>(D, L.n))
          pol.missed();
        else if (!kLocateEarly || tubes_locate<R>(D, L.n, &row, &g))
          to_det = true;
        else
          pol.missed();
      }
    }
    const unsigned dm = __ballot_sync(kFull, to_det);
    if (to_det) {
      QPacket<R>& p = dq[dq_n + __popc(dm & lt_mask)];
      p.row = (int16_t)row;
      p.g = (int16_t)g;
      p.x = L.n.x;
      p.y = L.n.y;
      p.z = L.n.z;
      p.dx = L.n.dx;
      p.dy = L.n.dy;
      p.dz = L.n.dz;
      p.speed = L.n.speed;
      p.w = we;
      p.t = L.n.t;
      p.nid = L.nid;
      p.order = L.o;
    }
    dq_n += __popc(dm);
    if (L.active) {
      if (L.o == S.max_orders || !(st.len_tot > R(0))) {
        L.active = false;
      } else {
        const auto rng = job.rng(L.nid);
        L.active = step_scatter<R, NS, KS, P>(A, S, rng, L, st, pol);
      }
    }
    __syncwarp();
    // ---- detector stage: full batches now, the remainder once the range is done.  This is
    // the only place packets are detected, so a packet's arithmetic does not depend on the
    // batch it falls in (or on the launch shape).
    bool done = !__any_sync(kFull, L.active) && next >= hi && hq_n == 0 && fq_n == 0;
    if (done) done = !src.more(&next, &hi);
    while (dq_n >= 32 || (done && dq_n > 0)) {
      const int take = dq_n < 32 ? dq_n : 32;
      Ray<R> pe;
      int order = 0, row = 0, g = 0;
      int64_t nid = 0;
      if (lane < take) {
        const QPacket<R>& p = dq[dq_n - take + lane];
        row = p.row;
        g = p.g;
        pe.x = p.x;
        pe.y = p.y;
        pe.z = p.z;
        pe.dx = p.dx;
        pe.dy = p.dy;
        pe.dz = p.dz;
        pe.speed = p.speed;
        pe.t = p.t;
        pe.w = p.w;
        nid = p.nid;
        order = p.order;
      }
      __syncwarp();
      if (lane < take) {
        const auto rng = job.rng(nid);
        if (kLocateEarly) {
          const R u = rng.template first<R>(order, 3);
          pol.record(A, tubes_absorb<R>(D, job.W(), tu, pe, u, row, g));
        } else {
          pol.record(A, detect<R, DET>(D, job.W(), tu, rng, order, pe));
        }
      }
      dq_n -= take;
    }
    if (done) break;
  }
}

template <typename R, int NS, int DET, int KS>
__global__ void __launch_bounds__(kThreads) trace_kernel(const __grid_constant__ TraceArgs A) {
  __shared__ R tu[2 * MCV_MAX_TUBES_PER_ROW];
  stage_tubes<R, DET>(A, tu);
  Forward<R, DET> pol;
  run_chain<R, NS, DET, KS, Forward<R, DET>>(A, tu, pol);
}

// resident blocks per SM the register allocation aims at (FP64 state needs more registers)
#ifndef MCV_WAVE_BLOCKS_F32
#define MCV_WAVE_BLOCKS_F32 5
#endif
#ifndef MCV_WAVE_BLOCKS_F64
#define MCV_WAVE_BLOCKS_F64 3
#endif
template <typename R>
struct WaveBlocks {
  static constexpr int value = sizeof(R) == 4 ? MCV_WAVE_BLOCKS_F32 : MCV_WAVE_BLOCKS_F64;
};

template <typename R, int NS, int DET, int KS, bool EV>
__global__ void __launch_bounds__(kThreads, WaveBlocks<R>::value)
    wave_kernel(const __grid_constant__ TraceArgs A) {
  __shared__ R tu[2 * MCV_MAX_TUBES_PER_ROW];
  stage_tubes<R, DET>(A, tu);
  Forward<R, DET, LaunchOutT<EV>, SmemTally<R>> pol{SmemTally<R>{wave_smem_bytes<R>()}};
  pol.store.get() = Tally<R>();
  // each warp owns one contiguous range of the launch's neutron ids
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t lo = (A.n * wid) / nw, hi = (A.n * (wid + 1)) / nw;
  NoMoreIds src;
  const ParamJob<R> job{A};
  run_waves<R, NS, DET, KS>(A, job, lo, hi, tu, pol, src);
  pol.flush(A, threadIdx.x & 31);
}

// ---- batched launch (no counterpart in the paper) -------------------------------------------
// Many simulations (sample orientations, incident energies, neutron counts) in one persistent
// launch.  Each simulation's neutron ids are cut into work items handed out by its own
// device counter.  A warp starts at its home simulation (warps are spread over the
// simulations in proportion to their neutron counts), copies that simulation's parameter
// block into its slot of shared memory, and keeps taking items of it -- without draining its
// queues between items -- until that queue is empty; then it moves on to the next
// simulation that still has items.  Each neutron's arithmetic is the single-simulation
// kernel's.
// SS: every simulation has the batch's sample (A.Sf / A.Sd), kept in parameter space
template <typename R, int NS, int DET, int KS, bool SS, bool EV>
__global__ void __launch_bounds__(kThreads, WaveBlocks<R>::value)
    batch_wave_kernel(const __grid_constant__ TraceArgs A, const __grid_constant__ BatchArgs Q) {
  __shared__ R tu[2 * MCV_MAX_TUBES_PER_ROW];
  stage_tubes<R, DET>(A, tu);
  const int lane = threadIdx.x & 31;
  {
    // home simulation: the last s with nstart[s] <= total * warp / warps
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t target = (int64_t)(((double)Q.total * (double)wid) / (double)nw);
    int home = 0, h_hi = Q.nsims - 1;
    while (home < h_hi) {
      const int mid = (home + h_hi + 1) >> 1;
      if (Q.nstart[mid] <= target)
        home = mid;
      else
        h_hi = mid - 1;
    }
    if (lane == 0) {
      batch_warp<R>().home = home;
      batch_warp<R>().v = 0;
    }
    __syncwarp();
  }
  Forward<R, DET, SlotOut<R, EV>, SmemTally<R>> pol{SmemTally<R>{batch_tally_offset<R>()}};
  pol.store.get() = Tally<R>();
  const SlotJob<R, SS> job{A};
  QueuedIds<R> src;
  for (;;) {
    BatchWarp<R>& me = batch_warp<R>();
    const int v = me.v;
    if (v >= Q.nsims) break;
    int s = me.home + v;
    if (s >= Q.nsims) s -= Q.nsims;
    const int64_t n = Q.nstart[s + 1] - Q.nstart[s];
    __syncwarp();
    if (lane == 0) {
      me.v = v + 1;
      me.q.ctr = Q.next + s;
      me.q.n = n;
      me.q.chunk = Q.chunk;
      me.q.items = (n + Q.chunk - 1) / Q.chunk;
    }
    __syncwarp();
    int64_t lo = 0, hi = 0;
    if (!src.more(&lo, &hi)) continue;
    const uint32_t* from = reinterpret_cast<const uint32_t*>(static_cast<const SimP<R>*>(Q.sims) + s);
    uint32_t* to = reinterpret_cast<uint32_t*>(&me.sim);
    for (int w = lane; w < (int)(sizeof(SimP<R>) / 4); w += 32) to[w] = from[w];
    __syncwarp();
    run_waves<R, NS, DET, KS>(A, job, lo, hi, tu, pol, src);
    pol.flush(A, lane);
  }
}

// the fused forward runs as waves (dynamic shared memory for the warp queues) unless it
// stores packets or reads a stored beam
inline bool uses_waves(const TraceArgs& A, int det) {
  return det != MCV_DET_NONE && A.pk_order == nullptr && A.in_x == nullptr;
}

template <typename R>
__global__ void __launch_bounds__(kThreads) beam_kernel(const __grid_constant__ TraceArgs A) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < A.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t nid = A.first_id + i;
    const NeutronRng rng(A.keys, nid);
    Ray<R> n;
    const bool ok = make_beam<R>(Bof<R>(A), rng, &n);
    if (!ok) {
      n.x = n.y = n.z = R(0);
      n.dx = n.dy = n.dz = R(0);
      n.speed = R(0);
      n.t.set(0.0);
      n.w = R(0);
    }
    static_cast<R*>(A.pk_x)[i] = n.x;
    static_cast<R*>(A.pk_y)[i] = n.y;
    static_cast<R*>(A.pk_z)[i] = n.z;
    static_cast<R*>(A.pk_vx)[i] = n.speed * n.dx;
    static_cast<R*>(A.pk_vy)[i] = n.speed * n.dy;
    static_cast<R*>(A.pk_vz)[i] = n.speed * n.dz;
    static_cast<R*>(A.pk_w)[i] = n.w;
    A.pk_t[i] = n.t.value();
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
    if (o > kMaxOrders) {  // no packet of the library has such an order: flag it, skip it
      err = 1;
      continue;
    }
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
    const NeutronRng rng(A.keys, A.in_id[i]);
    const Hit<R> h = detect<R, DET>(Dof<R>(A), Dof<R>(A).win, tu, rng, o, n);
    if (h.pixel >= 0 && A.ev.count) append_event(A.ev, h.pixel, h.tof.value(), (double)h.w_det);
    if (h.bin >= 0) {
      if (h.bin >= Dof<R>(A).n_bins) {
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
    if (E.tof) E.tof[i] = h.tof.value();
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

// ---- adjoint (no counterpart in the paper) --------------------------------------------
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

// The path sums (cum_*) and the per-thread accumulators are kept in the real type of the
// trace: FP64 in FP64 mode, compensated FP32 sums in FP32 mode (the FP64 pipe of GB300 runs
// at about 1/64 of the FP32 rate, so FP64 arithmetic per packet would dominate the FP32
// adjoint); the table-gradient atomics are FP64 in both.
template <typename R, int DET>
struct Adjoint {
  static constexpr bool kWantsGs = true;
  // a neutron that does not meet the sample only reaches the beam stop, which carries no
  // gradient: its divergence and energy are not drawn
  static constexpr bool kMeetingOnly = true;
  R a[kMaxOrders];   // scattering factor without the table value
  R s[kMaxOrders];   // table value (1 for kernels without a table)
  int e[kMaxOrders]; // table entry or -1
  R cum_dabs = R(0), cum_ds = R(0);
  Acc<R> acc_abs, acc_s;
  int err = 0;

  __device__ __forceinline__ void start(const Lane<R>&) {
    cum_dabs = R(0);
    cum_ds = R(0);
  }

  template <class Rng>
  __device__ __forceinline__ void emit(const TraceArgs& A, const R* tu, const Rng& rng,
                                       const Lane<R>& L, R we, R atten, R lg, R) {
    if (L.o == 0) return;
    Ray<R> pe = L.n;
    pe.w = R(1);
    const Hit<R> h = detect<R, DET>(Dof<R>(A), Dof<R>(A).win, tu, rng, L.o, pe);
    if (h.bin < 0) return;
    if (h.bin >= Dof<R>(A).n_bins) {
      err = 1;
      return;
    }
    // g_b = dchi2/dI_b of the bin.  FP32 mode: from the FP64 difference c I_b - T_b rounded
    // once to FP32 (a warp instruction on GB300's FP64 pipe costs the same whatever lanes it
    // needs, and only a few lanes of a step detect); FP64 mode: in FP64.
    double g64 = 0.0;
    R gb;
    if constexpr (sizeof(R) == 4) {
      gb = A.g ? (R)A.g[h.bin] : chi2_grad_bin_f32(A.hist_in[h.bin], A.target[h.bin], A.scale_c);
      if (gb == R(0)) return;
    } else {
      g64 = A.g ? A.g[h.bin] : chi2_grad_bin(A.hist_in[h.bin], A.target[h.bin], A.scale_c);
      if (g64 == 0.0) return;
      gb = (R)g64;
    }
    const ScatP<R>& g = Sof<R>(A).s[A.gs];
    const R w_det = we * h.pabs;
    const R dabs = cum_dabs - g.n100 * (R(2200) / L.n.speed) * lg;
    const R ds = cum_ds - g.n100 * lg;
    acc_abs.add(gb * w_det * dabs);
    acc_s.add(gb * w_det * ds);
    if (!A.dsqe) return;
    R base = atten * h.pabs;
    for (int m = 0; m < L.o; ++m) base *= a[m];
    for (int k = 0; k < L.o; ++k) {
      if (e[k] < 0) continue;
      R prod = base;
      for (int m = 0; m < L.o; ++m)
        if (m != k) prod *= s[m];
      if constexpr (sizeof(R) == 4)
        atomicAdd(A.dsqe + e[k], (double)(gb * prod));
      else
        atomicAdd(A.dsqe + e[k], g64 * (double)prod);
    }
  }

  __device__ __forceinline__ void scatter(const TraceArgs& A, const Lane<R>& L, int j, R a_fac,
                                          const Scatter<R>& out, R lg_pt, R speed_in) {
    const int k = L.o;
    a[k] = a_fac * out.rest;
    s[k] = out.s_value;
    e[k] = out.entry;
    const ScatP<R>& g = Sof<R>(A).s[A.gs];
    cum_dabs -= g.n100 * (R(2200) / speed_in) * lg_pt;
    cum_ds -= g.n100 * lg_pt;
    if (j == A.gs) cum_ds += R(1) / g.sig_s;
  }

  __device__ __forceinline__ void clear(const TraceArgs&, int64_t, int) {}

  __device__ __forceinline__ void flush(const TraceArgs& A, int lane) {
    const double s_abs = warp_sum(acc_abs.value()), s_s = warp_sum(acc_s.value());
    if (lane == 0) {
      atomicAdd(A.dsig + 0, s_abs);
      atomicAdd(A.dsig + 1, s_s);
    }
    if (__any_sync(0xffffffffu, err != 0) && lane == 0 && A.err) atomicOr(A.err, 1);
  }
};

// Warp loop of a policy that keeps only the neutrons meeting the sample (the adjoint): the
// source draws are compacted as in the waves -- footprints 32 new ids at a time, those that
// may lead into the sample queued; then 32 queued footprints at a time get their direction
// and, where they meet the sample, their energy, and are queued as neutrons -- and the lanes
// without a neutron take queued ones, so that the chain steps run on full warps.  The
// neutrons and their arithmetic are those of run_chain with make_beam_meeting.
template <typename R, int NS, int DET, int KS, class P>
__device__ __forceinline__ void run_chain_meeting(const TraceArgs& A, const R* tu, P& pol,
                                                  QNeutron<R>* hq, QFoot<R>* fq) {
  const unsigned kFull = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t lo = (A.n * wid) / nw, hi = (A.n * (wid + 1)) / nw;
  const SampleP<R>& S = Sof<R>(A);
  const BeamP<R>& Bm = Bof<R>(A);
  int64_t next = lo;
  int hq_n = 0, fq_n = 0;  // queued neutrons and footprints (each at most 63)
  Lane<R> L;
  L.active = false;
  L.o = 0;
  L.idx = 0;
  L.nid = 0;
  for (;;) {
    const unsigned idle = __ballot_sync(kFull, !L.active);
    const int n_idle = __popc(idle);
    while (hq_n < n_idle && (fq_n > 0 || next < hi)) {
      if (fq_n < 32 && next < hi) {
        const int64_t i = next + lane;
        bool maybe = false;
        Ray<R> nr;
        int64_t nid = 0;
        if (i < hi) {
          nid = A.first_id + i;
          const NeutronRng rng(A.keys, nid);
          beam_footprint(Bm, rng, &nr);
          maybe = !surely_misses<R>(Bm, nr);
        }
        const unsigned mm = __ballot_sync(kFull, maybe);
        if (maybe) {
          QFoot<R>& f = fq[fq_n + __popc(mm & lt_mask)];
          f.x = nr.x;
          f.y = nr.y;
          f.nid = nid;
        }
        fq_n += __popc(mm);
        next += 32;
        __syncwarp();
        continue;
      }
      const int take_f = fq_n < 32 ? fq_n : 32;
      bool hit = false;
      Ray<R> nr;
      int64_t nid = 0;
      if (lane < take_f) {
        const QFoot<R>& f = fq[fq_n - take_f + lane];
        nid = f.nid;
        nr.x = f.x;
        nr.y = f.y;
        nr.z = -Bm.z0;
        nr.w = R(1);
      }
      fq_n -= take_f;
      __syncwarp();
      if (lane < take_f) {
        const NeutronRng rng(A.keys, nid);
        R aux;
        beam_divergence(Bm, rng, &nr, &aux);
        Seg<R> seg[2 * NS];
        if (assembly_segs<R, NS>(S, nr, seg) > 0 && beam_energy(Bm, rng, aux, &nr))
          hit = !(nr.w < S.min_prob) && !(A.stop_on_zero && nr.w == R(0));
      }
      const unsigned hm = __ballot_sync(kFull, hit);
      if (hit) {
        QNeutron<R>& q = hq[hq_n + __popc(hm & lt_mask)];
        q.x = nr.x;
        q.y = nr.y;
        q.z = nr.z;
        q.dx = nr.dx;
        q.dy = nr.dy;
        q.dz = nr.dz;
        q.speed = nr.speed;
        q.t = nr.t;
        q.nid = nid;
      }
      hq_n += __popc(hm);
      __syncwarp();
    }
    const int take = min(n_idle, hq_n);
    if (!L.active) {
      const int r = __popc(idle & lt_mask);
      if (r < take) {
        const QNeutron<R>& q = hq[hq_n - take + r];
        L.n.x = q.x;
        L.n.y = q.y;
        L.n.z = q.z;
        L.n.dx = q.dx;
        L.n.dy = q.dy;
        L.n.dz = q.dz;
        L.n.speed = q.speed;
        L.n.t = q.t;
        L.n.w = R(1);
        L.nid = q.nid;
        L.idx = q.nid - A.first_id;
        L.o = 0;
        L.active = true;
        pol.start(L);
      }
    }
    hq_n -= take;
    __syncwarp();
    // no lane holds a neutron only once the queues are empty and the range is done
    if (!__any_sync(kFull, L.active)) break;
    if (L.active) L.active = chain_step<R, NS, DET, KS, P>(A, tu, L, pol);
  }
  pol.flush(A, lane);
}

template <typename R, int NS, int DET, int KS>
__global__ void __launch_bounds__(kThreads) adjoint_kernel(const __grid_constant__ TraceArgs A) {
  __shared__ R tu[2 * MCV_MAX_TUBES_PER_ROW];
  __shared__ QNeutron<R> hq[kWarps * kQueue];
  __shared__ QFoot<R> fq[kWarps * kQueue];
  stage_tubes<R, DET>(A, tu);
  Adjoint<R, DET> pol;
  const int wib = threadIdx.x >> 5;
  run_chain_meeting<R, NS, DET, KS, Adjoint<R, DET>>(A, tu, pol, hq + wib * kQueue,
                                                       fq + wib * kQueue);
}

}  // namespace mcv

// the paper's recursive estimator (its kernel uses kThreads)
#include "mcv_paper.cuh"

namespace mcv {

// ---- launchers, one set per real type -----------------------------------------------------
// The fused waves with an event list are instantiated in translation units of their own
// (mcv_fp32_ev.cu, mcv_fp64_ev.cu); these declare their entry points.
cudaError_t launch_waves_ev_f32(const TraceArgs& A, int det, int grid, cudaStream_t s);
cudaError_t launch_waves_ev_f64(const TraceArgs& A, int det, int grid, cudaStream_t s);
template <typename R>
cudaError_t launch_waves_ev(const TraceArgs& A, int det, int grid, cudaStream_t s) {
  return sizeof(R) == 4 ? launch_waves_ev_f32(A, det, grid, s) : launch_waves_ev_f64(A, det, grid, s);
}

template <typename R, int NS, int DET, int KS>
cudaError_t launch_trace_k(const TraceArgs& A, int grid, cudaStream_t s) {
  if (DET != MCV_DET_NONE && uses_waves(A, DET)) {
    if (A.ev.count) return launch_waves_ev<R>(A, DET, grid, s);
    const size_t smem = wave_kernel_smem_bytes<R>();
    cudaError_t e = cudaFuncSetAttribute(wave_kernel<R, NS, DET, KS, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    wave_kernel<R, NS, DET, KS, false><<<grid, kThreads, smem, s>>>(A);
  } else {
    trace_kernel<R, NS, DET, KS><<<grid, kThreads, 0, s>>>(A);
  }
  return cudaGetLastError();
}

// the waves with an event list, over the shapes (used by the _ev translation units)
template <typename R, int NS, int KS>
cudaError_t launch_waves_ev_k(const TraceArgs& A, int det, int grid, cudaStream_t s) {
  const size_t smem = wave_kernel_smem_bytes<R>();
  const void* fn = det == MCV_DET_SURFACE ? (const void*)wave_kernel<R, NS, MCV_DET_SURFACE, KS, true>
                                          : (const void*)wave_kernel<R, NS, MCV_DET_TUBES, KS, true>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  void* args[] = {const_cast<TraceArgs*>(&A)};
  return cudaLaunchKernel(fn, dim3(grid), dim3(kThreads), args, smem, s);
}

template <typename R>
cudaError_t launch_waves_ev_t(const TraceArgs& A, int det, int grid, cudaStream_t s) {
  const bool all = A.Sd.wide;
  if (A.Sd.ns <= 1)
    return all ? launch_waves_ev_k<R, 1, kKernelsAll>(A, det, grid, s)
               : launch_waves_ev_k<R, 1, kKernelsPowder>(A, det, grid, s);
  if (A.Sd.ns == 2)
    return all ? launch_waves_ev_k<R, 2, kKernelsAll>(A, det, grid, s)
               : launch_waves_ev_k<R, 2, kKernelsPowder>(A, det, grid, s);
  return all ? launch_waves_ev_k<R, 4, kKernelsAll>(A, det, grid, s)
             : launch_waves_ev_k<R, 4, kKernelsPowder>(A, det, grid, s);
}

template <typename R, int NS, int KS>
cudaError_t launch_trace_nk(const TraceArgs& A, int det, int grid, cudaStream_t s) {
  switch (det) {
    case MCV_DET_SURFACE:
      return launch_trace_k<R, NS, MCV_DET_SURFACE, KS>(A, grid, s);
    case MCV_DET_TUBES:
      return launch_trace_k<R, NS, MCV_DET_TUBES, KS>(A, grid, s);
    default:
      return launch_trace_k<R, NS, MCV_DET_NONE, KS>(A, grid, s);
  }
}

template <typename R, int NS>
cudaError_t launch_trace_ns(const TraceArgs& A, int det, int grid, cudaStream_t s) {
  if (A.Sd.wide) return launch_trace_nk<R, NS, kKernelsAll>(A, det, grid, s);
  return launch_trace_nk<R, NS, kKernelsPowder>(A, det, grid, s);
}

template <typename R>
cudaError_t launch_trace_t(const TraceArgs& A, int det, int grid, cudaStream_t s) {
  if (A.Sd.ns <= 1) return launch_trace_ns<R, 1>(A, det, grid, s);
  if (A.Sd.ns == 2) return launch_trace_ns<R, 2>(A, det, grid, s);
  return launch_trace_ns<R, 4>(A, det, grid, s);
}

// the kernel the fused forward of this shape launches (waves when a detector is fused)
template <typename R, int NS, int KS>
const void* trace_fn_nk(int det) {
  if (det == MCV_DET_SURFACE) return (const void*)wave_kernel<R, NS, MCV_DET_SURFACE, KS, false>;
  if (det == MCV_DET_TUBES) return (const void*)wave_kernel<R, NS, MCV_DET_TUBES, KS, false>;
  return (const void*)trace_kernel<R, NS, MCV_DET_NONE, KS>;
}

template <typename R, int NS>
const void* trace_fn_ns(int det, bool bvk) {
  return bvk ? trace_fn_nk<R, NS, kKernelsAll>(det) : trace_fn_nk<R, NS, kKernelsPowder>(det);
}

template <typename R>
cudaError_t blocks_per_sm_t(int ns, int det, int bvk, int* blocks) {
  const void* fn = ns <= 1 ? trace_fn_ns<R, 1>(det, bvk) : (ns == 2 ? trace_fn_ns<R, 2>(det, bvk)
                                                                    : trace_fn_ns<R, 4>(det, bvk));
  const size_t smem = det != MCV_DET_NONE ? wave_kernel_smem_bytes<R>() : 0;
  if (smem) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, fn, kThreads, smem);
}

// the batched kernel of a shape; its dynamic shared memory limit is set where its occupancy
// is queried (batch_blocks_per_sm_t), once before the first launch, so that a launch is only
// the launch (and can be captured in a CUDA graph)
template <typename R, int NS, int KS, bool SS, bool EV>
const void* batch_fn_nk(int det) {
  if (det == MCV_DET_SURFACE)
    return (const void*)batch_wave_kernel<R, NS, MCV_DET_SURFACE, KS, SS, EV>;
  return (const void*)batch_wave_kernel<R, NS, MCV_DET_TUBES, KS, SS, EV>;
}

template <typename R, bool SS, bool EV>
const void* batch_fn_s(int ns, int det, int bvk) {
  if (ns <= 1)
    return bvk ? batch_fn_nk<R, 1, kKernelsAll, SS, EV>(det)
               : batch_fn_nk<R, 1, kKernelsPowder, SS, EV>(det);
  if (ns == 2)
    return bvk ? batch_fn_nk<R, 2, kKernelsAll, SS, EV>(det)
               : batch_fn_nk<R, 2, kKernelsPowder, SS, EV>(det);
  return bvk ? batch_fn_nk<R, 4, kKernelsAll, SS, EV>(det)
             : batch_fn_nk<R, 4, kKernelsPowder, SS, EV>(det);
}

// EV: the batch appends to event lists (the _ev translation units instantiate those kernels)
template <typename R, bool EV>
const void* batch_fn_t(int ns, int det, int bvk, int ss) {
  return ss ? batch_fn_s<R, true, EV>(ns, det, bvk) : batch_fn_s<R, false, EV>(ns, det, bvk);
}

template <typename R, bool EV>
cudaError_t batch_blocks_per_sm_t(int ns, int det, int bvk, int ss, int* blocks) {
  const void* fn = batch_fn_t<R, EV>(ns, det, bvk, ss);
  const size_t smem = batch_smem_bytes<R>();
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, fn, kThreads, smem);
}

template <typename R, bool EV>
cudaError_t launch_batch_t(const TraceArgs& A, const BatchArgs& Q, int ns, int det, int bvk,
                           int ss, int grid, cudaStream_t s) {
  const void* fn = batch_fn_t<R, EV>(ns, det, bvk, ss);
  void* args[] = {const_cast<TraceArgs*>(&A), const_cast<BatchArgs*>(&Q)};
  return cudaLaunchKernel(fn, dim3(grid), dim3(kThreads), args, batch_smem_bytes<R>(), s);
}

template <typename R>
cudaError_t launch_beam_t(const TraceArgs& A, int grid, cudaStream_t s) {
  beam_kernel<R><<<grid, kThreads, 0, s>>>(A);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_detect_t(const TraceArgs& A, const EventsArgs& E, int det, int grid,
                            cudaStream_t s) {
  if (det == MCV_DET_SURFACE)
    detect_kernel<R, MCV_DET_SURFACE><<<grid, kThreads, 0, s>>>(A, E);
  else
    detect_kernel<R, MCV_DET_TUBES><<<grid, kThreads, 0, s>>>(A, E);
  return cudaGetLastError();
}

template <typename R, int NS, int KS>
cudaError_t launch_adjoint_nk(const TraceArgs& A, int det, int grid, cudaStream_t s) {
  if (det == MCV_DET_SURFACE)
    adjoint_kernel<R, NS, MCV_DET_SURFACE, KS><<<grid, kThreads, 0, s>>>(A);
  else
    adjoint_kernel<R, NS, MCV_DET_TUBES, KS><<<grid, kThreads, 0, s>>>(A);
  return cudaGetLastError();
}

// resident blocks per SM of the adjoint kernel of a shape
template <typename R, int NS, int KS>
const void* adjoint_fn_nk(int det) {
  if (det == MCV_DET_SURFACE) return (const void*)adjoint_kernel<R, NS, MCV_DET_SURFACE, KS>;
  return (const void*)adjoint_kernel<R, NS, MCV_DET_TUBES, KS>;
}

template <typename R>
cudaError_t adjoint_blocks_per_sm_t(int ns, int det, int bvk, int* blocks) {
  const void* fn;
  if (ns <= 1)
    fn = bvk ? adjoint_fn_nk<R, 1, kKernelsAll>(det) : adjoint_fn_nk<R, 1, kKernelsPowder>(det);
  else if (ns == 2)
    fn = bvk ? adjoint_fn_nk<R, 2, kKernelsAll>(det) : adjoint_fn_nk<R, 2, kKernelsPowder>(det);
  else
    fn = bvk ? adjoint_fn_nk<R, 4, kKernelsAll>(det) : adjoint_fn_nk<R, 4, kKernelsPowder>(det);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, fn, kThreads, 0);
}

template <typename R, int NS>
cudaError_t launch_adjoint_ns(const TraceArgs& A, int det, int grid, cudaStream_t s) {
  if (A.Sd.wide) return launch_adjoint_nk<R, NS, kKernelsAll>(A, det, grid, s);
  return launch_adjoint_nk<R, NS, kKernelsPowder>(A, det, grid, s);
}

template <typename R>
cudaError_t launch_adjoint_t(const TraceArgs& A, int det, int grid, cudaStream_t s) {
  if (A.Sd.ns <= 1) return launch_adjoint_ns<R, 1>(A, det, grid, s);
  if (A.Sd.ns == 2) return launch_adjoint_ns<R, 2>(A, det, grid, s);
  return launch_adjoint_ns<R, 4>(A, det, grid, s);
}

// the paper's recursive estimator
template <typename R, int NS, int KS>
cudaError_t launch_paper_nk(const TraceArgs& A, int det, int grid, cudaStream_t s) {
  const size_t smem = paper_smem_bytes<R>();
  const void* fn = det == MCV_DET_SURFACE ? (const void*)paper_kernel<R, NS, MCV_DET_SURFACE, KS>
                                          : (const void*)paper_kernel<R, NS, MCV_DET_TUBES, KS>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  void* args[] = {const_cast<TraceArgs*>(&A)};
  return cudaLaunchKernel(fn, dim3(grid), dim3(kPaperThreads), args, smem, s);
}

template <typename R>
cudaError_t launch_paper_t(const TraceArgs& A, int det, int grid, cudaStream_t s) {
  const bool all = A.Sd.wide;
  if (A.Sd.ns <= 1)
    return all ? launch_paper_nk<R, 1, kKernelsAll>(A, det, grid, s)
               : launch_paper_nk<R, 1, kKernelsPowder>(A, det, grid, s);
  if (A.Sd.ns == 2)
    return all ? launch_paper_nk<R, 2, kKernelsAll>(A, det, grid, s)
               : launch_paper_nk<R, 2, kKernelsPowder>(A, det, grid, s);
  return all ? launch_paper_nk<R, 4, kKernelsAll>(A, det, grid, s)
             : launch_paper_nk<R, 4, kKernelsPowder>(A, det, grid, s);
}

// defines the fused-trace entry points of one real type (mcv_fp32.cu / mcv_fp64.cu)
#define MCV_DEFINE_TRACE_ENTRY_POINTS(R, SUFFIX)                                            \
  cudaError_t launch_trace_##SUFFIX(const TraceArgs& A, int det, int grid, cudaStream_t s) { \
    return launch_trace_t<R>(A, det, grid, s);                                              \
  }                                                                                         \
  cudaError_t blocks_per_sm_##SUFFIX(int ns, int det, int bvk, int* blocks) {               \
    return blocks_per_sm_t<R>(ns, det, bvk, blocks);                                        \
  }

// the fused waves with an event list (mcv_fp32_ev.cu / mcv_fp64_ev.cu)
#define MCV_DEFINE_EVENT_ENTRY_POINTS(R, SUFFIX)                                            \
  cudaError_t launch_waves_ev_##SUFFIX(const TraceArgs& A, int det, int grid, cudaStream_t s) { \
    return launch_waves_ev_t<R>(A, det, grid, s);                                           \
  }

// the source, detector and adjoint entry points (mcv_fp32_aux.cu / mcv_fp64_aux.cu)
#define MCV_DEFINE_AUX_ENTRY_POINTS(R, SUFFIX)                                              \
  cudaError_t launch_beam_##SUFFIX(const TraceArgs& A, int grid, cudaStream_t s) {          \
    return launch_beam_t<R>(A, grid, s);                                                    \
  }                                                                                         \
  cudaError_t launch_detect_##SUFFIX(const TraceArgs& A, const EventsArgs& E, int det,      \
                                     int grid, cudaStream_t s) {                            \
    return launch_detect_t<R>(A, E, det, grid, s);                                          \
  }                                                                                         \
  cudaError_t launch_adjoint_##SUFFIX(const TraceArgs& A, int det, int grid,                \
                                      cudaStream_t s) {                                     \
    return launch_adjoint_t<R>(A, det, grid, s);                                            \
  }                                                                                         \
  cudaError_t adjoint_blocks_per_sm_##SUFFIX(int ns, int det, int bvk, int* blocks) {       \
    return adjoint_blocks_per_sm_t<R>(ns, det, bvk, blocks);                                \
  }                                                                                         \
  cudaError_t launch_paper_##SUFFIX(const TraceArgs& A, int det, int grid, cudaStream_t s) { \
    return launch_paper_t<R>(A, det, grid, s);                                              \
  }

// defines the batched entry points of one real type and event flavour EV (mcv_batch_fp32.cu,
// mcv_batch_fp64.cu; with EV, mcv_batch_fp32_ev.cu and mcv_batch_fp64_ev.cu)
#define MCV_DEFINE_BATCH_ENTRY_POINTS(R, SUFFIX, EV)                                        \
  cudaError_t batch_blocks_per_sm_##SUFFIX(int ns, int det, int bvk, int ss, int* blocks) { \
    return batch_blocks_per_sm_t<R, EV>(ns, det, bvk, ss, blocks);                          \
  }                                                                                         \
  cudaError_t launch_batch_##SUFFIX(const TraceArgs& A, const BatchArgs& Q, int ns, int det, \
                                    int bvk, int ss, int grid, cudaStream_t s) {            \
    return launch_batch_t<R, EV>(A, Q, ns, det, bvk, ss, grid, s);                          \
  }

}  // namespace mcv
