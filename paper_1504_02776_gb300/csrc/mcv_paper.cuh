// The paper's own recursive estimator (supplement S3: scatterM -> interactM_path1 ->
// interactM1) on the GPU, as a fidelity mode next to the bounded chain.  Every interaction
// splits a packet into a transmitted packet (attenuated over the first segment of the
// scatterer it meets) and a scattered one (taken at a uniform point of that segment, then
// scattered by a kernel); the scattered packet keeps interacting with the same scatterer while
// it may scatter again, the transmitted ones start over from the sample assembly; a packet
// with nothing ahead leaves -- order 0 to the beam stop, the others to the detector system,
// where (with multi_tube) the weight a tube leaves goes on to the next tubes it crosses.
//
// A lane walks one neutron's tree of packets depth first with a stack in local memory; the
// warp's source draws are compacted and its packets leaving for the detector are queued and
// detected 32 at a time, as in the chain's waves.  Each packet's random numbers are keyed by its place in the tree (the incident packet is
// node 1, an interaction of node x gives the transmitted packet 2x and the scattered packet
// 2x + 1; counter (id lo, id hi, 4 (node mod 2^30) + block, node / 2^30), key (seed,
// sim_id ^ 0x80000000)), so the walk's order does not change any packet.
#pragma once

#include "mcv_chain.cuh"

namespace mcv {

// threads per block of the paper estimator's kernel (the chain kernels' block size)
constexpr int kPaperThreads = 128;
constexpr int kPaperStack = 48;                          // packets waiting per thread
constexpr uint64_t kPaperMaxNode = (uint64_t)1 << 61;    // deeper trees are cut

// A transmitted packet goes on along its parent's line: it keeps the line's origin (n's
// position, and its time there) and the distance s0 travelled along it; the material ahead is
// what lies beyond s0 on that line.  (Re-tracing from the rounded exit point instead would
// meet a sliver of the material behind it again and again.)
template <typename R>
struct PaperPk {
  Ray<R> n;
  int m;          // scatterings so far
  uint64_t node;  // place in the tree
  R s0;           // distance travelled along the line from n's position
};

// the stream of one node of one neutron's tree (the kernels' interface: the event is ignored)
struct PaperRng {
  KeysTable ks;
  uint32_t n0, n1, c2, c3;
  __device__ __forceinline__ PaperRng(const PhiloxKeys& keys, int64_t nid, uint64_t node)
      : ks{keys}, n0((uint32_t)((uint64_t)nid & 0xffffffffu)),
        n1((uint32_t)((uint64_t)nid >> 32)),
        c2((uint32_t)((node & 0x3fffffffu) << 2)), c3((uint32_t)(node >> 30)) {}
  template <typename R>
  __device__ __forceinline__ void pair(int, int block, R* u0, R* u1) const {
    const Words w = philox10(n0, n1, c2 | (uint32_t)block, c3, ks);
    *u0 = to_unit<R>(w.a, w.b);
    *u1 = to_unit<R>(w.c, w.d);
  }
  template <typename R>
  __device__ __forceinline__ R first(int, int block) const {
    const Words w = philox10(n0, n1, c2 | (uint32_t)block, c3, ks);
    return to_unit<R>(w.a, w.b);
  }
};

// The multi-tube detector: the three candidate tubes around the ring crossing, those the ray
// enters taken by entry distance, each absorbing its share of the weight the earlier ones
// left (u[i]: the i-th absorption depth).  Returns the number of detections written to h.
template <typename R>
__device__ __forceinline__ int tubes_absorb_multi(const DetP<R>& D, const TofWin& W,
                                                  const R* __restrict__ tu, const Ray<R>& n,
                                                  const R (&u)[3], int row, int g, Hit<R> (&h)[3]) {
  using M = Mth<R>;
  const R Rad = (R)D.radius;
  const int tpp = D.tubes_per_pack;
  const int row_off = D.row_off[row];
  const int n_tubes_row = D.packs[row] * tpp;
  const R y_lo = (R)D.row_y[row] - (R)D.half_len;
  const R y_hi = (R)D.row_y[row] + (R)D.half_len;
  int tube[3];
  R s_in[3], s_out[3];
  int m = 0;
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
    const R a_in = M::fmax(M::fmax(s1, ys1), R(0)), a_out = M::fmin(s2, ys2);
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
  const R mu = (R)D.mu_he_v / n.speed;
  R left = n.w;
  for (int i = 0; i < m; ++i) {
    const R L = s_out[i] - s_in[i];
    const R pabs = -M::expm1(-mu * L);
    const R x = -M::log1p(-u[i] * pabs) / mu;
    const R s_abs = s_in[i] + x;
    const R y_abs = n.y + s_abs * n.dy;
    int j = (int)M::floor((y_abs - y_lo) / (R)D.pix_len);
    j = min(max(j, 0), D.pixels_per_tube - 1);
    const int pc = tube[i] / tpp, tc = tube[i] - pc * tpp;
    h[i].pixel = ((row_off + pc) * tpp + tc) * D.pixels_per_tube + j;
    h[i].tof = n.t;
    h[i].tof.add(s_abs / n.speed);
    h[i].pabs = pabs;
    h[i].w_det = left * pabs;
    left = left * (R(1) - pabs);
    const int64_t tb = tof_bin<R>(W, h[i].tof);
    h[i].bin = (tb < 0) ? -2 : (int64_t)h[i].pixel * W.n_tof + tb;
  }
  return m;
}

// event mode of the paper estimator, out of line: runs without an event list keep the
// registers and code of the append out of their detector stage
static __device__ __noinline__ void paper_append_event(const EvSink& ev, int pixel, double tof,
                                                       double w) {
  append_event(ev, pixel, tof, w);
}

// the running tallies of a thread (the chain kernels' slots)
template <typename R>
struct PaperTally {
  Acc<R> bs, det, over;
  Counts cnt;
  int err = 0;
  __device__ __forceinline__ void record(const TraceArgs& A, const Hit<R>& h) {
    // event mode: every detected packet, in or outside the time window
    if (h.pixel >= 0 && A.ev.count)
      paper_append_event(A.ev, h.pixel, h.tof.value(), (double)h.w_det);
    if (h.bin >= 0) {
      if (h.bin >= Dof<R>(A).n_bins) {
        err = 1;
        return;
      }
      if (A.hist) atomicAdd(A.hist + h.bin, (double)h.w_det);
      det.add(h.w_det);
      cnt.ndet++;
    } else if (h.bin == -2) {
      over.add(h.w_det);
      cnt.nover++;
    }
  }
};

// a packet of order >= 1 leaving the sample, queued for the detector stage
template <typename R>
struct PaperDet {
  Ray<R> n;
  uint64_t node;
  int64_t nid;
  int m;
};

// dynamic shared memory of the paper kernel: per warp, the queues of neutrons, footprints and
// packets for the detector
constexpr int kPaperWarps = kPaperThreads / 32;
template <typename R>
constexpr size_t paper_smem_bytes() {
  return (size_t)kPaperWarps * kQueue *
         (sizeof(QNeutron<R>) + sizeof(QFoot<R>) + sizeof(PaperDet<R>));
}

// a packet leaving the sample assembly
template <typename R, int DET>
__device__ __forceinline__ void paper_emit(const TraceArgs& A, const R* tu, int64_t nid,
                                           const PaperPk<R>& p, PaperTally<R>& T) {
  if (p.m == 0) {
    T.bs.add(p.n.w);
    return;
  }
  T.cnt.nemit++;
  const DetP<R>& D = Dof<R>(A);
  const PaperRng rng(A.pkeys, nid, p.node);
  if (DET == MCV_DET_TUBES && D.multi_tube) {
    int row = 0, g = 0;
    if (!tubes_locate<R>(D, p.n, &row, &g)) {
      T.cnt.nmiss++;
      return;
    }
    R u[3];
    rng.template pair<R>(0, 3, &u[0], &u[1]);
    u[2] = rng.template first<R>(0, 0);
    Hit<R> h[3];
    const int k = tubes_absorb_multi<R>(D, D.win, tu, p.n, u, row, g, h);
    if (k == 0) T.cnt.nmiss++;
    for (int i = 0; i < k; ++i) T.record(A, h[i]);
    return;
  }
  const Hit<R> h = detect<R, DET>(D, D.win, tu, rng, 0, p.n);
  if (h.bin == -1) T.cnt.nmiss++;
  T.record(A, h);
}

// The packet leaves with the attenuation of all the material ahead (its ns segments in seg).
template <typename R, int NS>
__device__ __forceinline__ void paper_propagate_out(const SampleP<R>& S, const Seg<R> (&seg)[2 * NS],
                                                    int ns, PaperPk<R>* p) {
  R tau = R(0);
#pragma unroll
  for (int k = 0; k < 2 * NS; ++k) {
    if (k < ns) {
      const ScatP<R>& sc = S.s[seg[k].j];
      tau += sc.n100 * (sc.sig_s + sc.sab2200 / p->n.speed) * (seg[k].b - seg[k].a);
    }
  }
  p->n.w = p->n.w * Mth<R>::exp(-tau);
}

// interactM1 of scatterer j on its first segment [a, b] ahead of the packet: 1 with both
// packets; 2 with the transmitted packet only (the kernel cannot scatter).
template <typename R, int KS>
__device__ __forceinline__ int paper_interact1(const TraceArgs& A, const SampleP<R>& S, int j,
                                               R a, R b, int64_t nid, const PaperPk<R>& in,
                                               PaperPk<R>* tr, PaperPk<R>* sc_out, int* err) {
  using M = Mth<R>;
  const ScatP<R>& sc = S.s[j];
  const R len = b - a;
  const R mu = sc.n100 * (sc.sig_s + sc.sab2200 / in.n.speed);
  *tr = in;
  tr->s0 = b;
  tr->n.w = in.n.w * M::exp(-mu * len);
  tr->node = 2 * in.node;
  const PaperRng rng(A.pkeys, nid, in.node);
  R u_pt, u_k;
  rng.template pair<R>(0, 0, &u_pt, &u_k);
  const R ell = u_pt * len;
  const R s = a + ell;
  PaperPk<R> p = in;
  p.n.x = in.n.x + in.n.dx * s;
  p.n.y = in.n.y + in.n.dy * s;
  p.n.z = in.n.z + in.n.dz * s;
  p.n.t.add(s / in.n.speed);
  p.n.w = in.n.w * sc.mu_s * len * M::exp(-mu * ell);
  p.s0 = R(0);
  const int kk = (sc.nk == 2 && !(u_k * sc.ksig_sum < sc.ksig0)) ? 1 : 0;
  Scatter<R> out;
  if (!scatter_kernel<R, KS>(S, sc, kk, rng, 0, &p.n, &out, err)) return 2;
  p.n.w = p.n.w * out.factor;
  p.m = in.m + 1;
  p.node = 2 * in.node + 1;
  *sc_out = p;
  return 1;
}

// One step of a lane's walk of its tree: the packet in hand (cur, when have) or the next one
// off the stack goes through the assembly; it leaves (*emit: cur is a packet for the
// detector), or interacts once (the transmitted packet onto the stack, the scattered one
// kept in hand while it may scatter again).
// jp: the scatterer of the interactM_path1 under way (its scattered packet is cur), or -1
// for a packet that starts over from the sample assembly.  The segments of every packet come
// from the one assembly trace here, so that the distance a transmitted packet has travelled
// (the end of a segment) and the trace that later clips at it are the same arithmetic in
// FP32 as in FP64.
template <typename R, int NS, int DET, int KS>
__device__ __forceinline__ void paper_step(const TraceArgs& A, int64_t nid, PaperPk<R>& cur,
                                           bool& have, int& jp,
                                           PaperPk<R> (&stack)[kPaperStack], int& sp,
                                           PaperTally<R>& T, bool* emit) {
  const SampleP<R>& S = Sof<R>(A);
  if (!have) {
    cur = stack[--sp];
    jp = -1;
  }
  have = false;
  Seg<R> seg[2 * NS];
  const int ns = assembly_segs<R, NS>(S, cur.n, seg, cur.s0);
  if (cur.node == 1 && ns > 0) T.cnt.nhit++;
  if (cur.n.w < S.min_prob) return;
  int j = -1;
  R a = R(0), b = R(0);
  if (jp >= 0) {  // path1 goes on: the scatterer's first segment ahead, if any
#pragma unroll
    for (int k = 2 * NS - 1; k >= 0; --k) {
      if (k < ns && seg[k].j == jp) {
        j = jp;
        a = seg[k].a;
        b = seg[k].b;
      }
    }
  }
  if (j < 0) {  // from the sample assembly
    if (ns == 0 || cur.m >= S.max_orders || cur.node >= kPaperMaxNode) {
      // it leaves (with the attenuation of what is still ahead): order 0 to the beam stop,
      // the others queued for the detector stage (cur)
      if (ns > 0) paper_propagate_out<R, NS>(S, seg, ns, &cur);
      if (cur.m == 0)
        T.bs.add(cur.n.w);
      else
        *emit = true;
      return;
    }
    j = seg[0].j;  // interactM_path1 of the first scatterer met
    a = seg[0].a;
    b = seg[0].b;
  }
  PaperPk<R> tr, sc;
  const int res = paper_interact1<R, KS>(A, S, j, a, b, nid, cur, &tr, &sc, &T.err);
  if (sp < kPaperStack) stack[sp++] = tr;
  else T.err = 1;  // the tree outgrew the stack: the packet is lost and reported
  if (res == 2) return;
  // the scattered packet goes on with the same scatterer while it may scatter again (every
  // interaction at least doubles the node, so the walk ends)
  cur = sc;
  have = true;
  jp = (cur.m < S.max_orders && cur.node < kPaperMaxNode) ? j : -1;
}

// Each warp takes a contiguous range of neutron ids.  Their source draws are compacted as in
// the waves (footprints 32 new ids at a time; those that may lead into the sample get their
// direction and, where needed, their energy 32 at a time); a neutron that misses the sample
// is one order-0 packet, added to the beam stop there, and those that meet it are queued.
// A lane without a tree to walk takes a queued neutron, so the warps' lanes walk trees
// together instead of drifting apart over the two thirds of the beam that misses; the
// packets that leave for the detector are queued and detected 32 at a time.  Queues in
// dynamic shared memory (paper_smem_bytes).
template <typename R, int NS, int DET, int KS>
__global__ void __launch_bounds__(kPaperThreads) paper_kernel(const __grid_constant__ TraceArgs A) {
  __shared__ R tu[2 * MCV_MAX_TUBES_PER_ROW];
  const int wib = threadIdx.x >> 5;
  QNeutron<R>* hq = reinterpret_cast<QNeutron<R>*>(g_wave_smem) + wib * kQueue;
  QFoot<R>* fq = reinterpret_cast<QFoot<R>*>(
                     g_wave_smem + (size_t)kPaperWarps * kQueue * sizeof(QNeutron<R>)) +
                 wib * kQueue;
  PaperDet<R>* dq = reinterpret_cast<PaperDet<R>*>(
                        g_wave_smem + (size_t)kPaperWarps * kQueue *
                                          (sizeof(QNeutron<R>) + sizeof(QFoot<R>))) +
                    wib * kQueue;
  stage_tubes<R, DET>(A, tu);
  const SampleP<R>& S = Sof<R>(A);
  const BeamP<R>& Bm = Bof<R>(A);
  const unsigned kFull = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t lo = (A.n * wid) / nw, hi = (A.n * (wid + 1)) / nw;
  int64_t next = lo;
  int hq_n = 0, fq_n = 0, dq_n = 0;  // queued neutrons, footprints, packets (each <= 63)
  PaperTally<R> T;
  PaperPk<R> stack[kPaperStack];
  PaperPk<R> cur;
  int64_t nid = 0;
  int sp = 0, jp = -1;
  bool have = false, busy = false;  // busy: the lane has a tree to walk (have || sp > 0)
  for (;;) {
    const unsigned idle = __ballot_sync(kFull, !busy);
    const int n_idle = __popc(idle);
    while (hq_n < n_idle && (fq_n > 0 || next < hi)) {
      if (fq_n < 32 && next < hi) {
        const int64_t i = next + lane;
        bool maybe = false;
        Ray<R> nr;
        int64_t id = 0;
        if (i < hi) {
          id = A.first_id + i;
          const NeutronRng rng(A.keys, id);
          beam_footprint(Bm, rng, &nr);
          if (!surely_misses<R>(Bm, nr))
            maybe = true;
          else if (!(nr.w < S.min_prob))
            T.bs.add(nr.w);  // order-0 packet, no material ahead
        }
        const unsigned mm = __ballot_sync(kFull, maybe);
        if (maybe) {
          QFoot<R>& f = fq[fq_n + __popc(mm & lt_mask)];
          f.x = nr.x;
          f.y = nr.y;
          f.nid = id;
        }
        fq_n += __popc(mm);
        next += 32;
        __syncwarp();
        continue;
      }
      const int take_f = fq_n < 32 ? fq_n : 32;
      bool hit = false;
      Ray<R> nr;
      int64_t id = 0;
      if (lane < take_f) {
        const QFoot<R>& f = fq[fq_n - take_f + lane];
        id = f.nid;
        nr.x = f.x;
        nr.y = f.y;
        nr.z = -Bm.z0;
        nr.w = R(1);
      }
      fq_n -= take_f;
      __syncwarp();
      if (lane < take_f) {
        const NeutronRng rng(A.keys, id);
        R aux;
        beam_divergence(Bm, rng, &nr, &aux);
        Seg<R> seg[2 * NS];
        const bool meets = assembly_segs<R, NS>(S, nr, seg) > 0;
        const bool ok = (meets || !Bm.energy_positive) ? beam_energy(Bm, rng, aux, &nr) : true;
        if (ok) {
          if (meets)
            hit = true;
          else if (!(nr.w < S.min_prob))
            T.bs.add(nr.w);  // order-0 packet, no material ahead
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
        q.nid = id;
      }
      hq_n += __popc(hm);
      __syncwarp();
    }
    const int take = min(n_idle, hq_n);
    if (!busy) {
      const int r = __popc(idle & lt_mask);
      if (r < take) {
        const QNeutron<R>& q = hq[hq_n - take + r];
        cur.n.x = q.x;
        cur.n.y = q.y;
        cur.n.z = q.z;
        cur.n.dx = q.dx;
        cur.n.dy = q.dy;
        cur.n.dz = q.dz;
        cur.n.speed = q.speed;
        cur.n.t = q.t;
        cur.n.w = R(1);
        cur.m = 0;
        cur.node = 1;
        cur.s0 = R(0);
        nid = q.nid;
        sp = 0;
        jp = -1;
        have = true;
        busy = true;
      }
    }
    hq_n -= take;
    __syncwarp();
    // no lane has a tree only once the source queues are empty and the range is done
    if (!__any_sync(kFull, busy) && dq_n == 0) break;
    bool emit = false;
    if (busy) {
      paper_step<R, NS, DET, KS>(A, nid, cur, have, jp, stack, sp, T, &emit);
      busy = have || sp > 0;
    }
    const unsigned em = __ballot_sync(kFull, emit);
    if (emit) {
      PaperDet<R>& d = dq[dq_n + __popc(em & lt_mask)];
      d.n = cur.n;
      d.node = cur.node;
      d.nid = nid;
      d.m = cur.m;
    }
    dq_n += __popc(em);
    __syncwarp();
    // detector stage: full batches of 32 packets, and the remainder at the end
    const bool last = !__any_sync(kFull, busy) && hq_n == 0 && fq_n == 0 && next >= hi;
    while (dq_n >= 32 || (last && dq_n > 0)) {
      const int take_d = dq_n < 32 ? dq_n : 32;
      PaperPk<R> p;
      int64_t id = 0;
      if (lane < take_d) {
        const PaperDet<R>& d = dq[dq_n - take_d + lane];
        p.n = d.n;
        p.node = d.node;
        p.m = d.m;
        id = d.nid;
      }
      dq_n -= take_d;
      __syncwarp();
      if (lane < take_d) paper_emit<R, DET>(A, tu, id, p, T);
    }
  }
  if (A.tallies) {
    const double v_bs = warp_sum(T.bs.value());
    const double v_det = warp_sum(T.det.value());
    const double v_over = warp_sum(T.over.value());
    const uint32_t n_det = warp_sum(T.cnt.ndet), n_over = warp_sum(T.cnt.nover);
    const uint32_t n_miss = warp_sum(T.cnt.nmiss), n_hit = warp_sum(T.cnt.nhit);
    const uint32_t n_emit = warp_sum(T.cnt.nemit);
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
  if (__any_sync(0xffffffffu, T.err != 0) && lane == 0 && A.err) atomicOr(A.err, 1);
}

}  // namespace mcv
