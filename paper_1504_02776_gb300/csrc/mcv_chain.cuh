// The per-neutron chain of scatterings and the warp loop that feeds it, shared by the
// forward kernels (histogram) and the adjoint kernel (gradient).  What happens to each
// emitted packet and each scattering is left to a policy object, so that both kernels
// trace exactly the same paths with exactly the same arithmetic.
//
// Policy interface (device, per lane):
//   kWantsGs                        compile-time: path lengths in scatterer A.gs are needed
//   kMeetingOnly                    compile-time: only neutrons that meet the sample matter
//                                   (their other packets carry nothing the policy uses)
//   start(L)                        a new neutron begins
//   emit(A, tu, rng, L, we, atten, lg)   packet of order L.o with weight we = w e^{-tau}
//   scatter(A, L, j, a_fac, out, lg_pt, speed_in)  after the kernel of order L.o scattered
//   clear(A, idx, first)            slots first..max_orders of neutron idx stay empty
//   flush(A, lane)                  once per thread at the end
#pragma once

#include "mcv_device.cuh"

namespace mcv {

template <typename R>
struct Lane {
  Ray<R> n;
  int64_t idx, nid;
  int o;
  bool active;
};

template <typename R>
__device__ __forceinline__ bool load_input(const TraceArgs& A, int64_t i, Ray<R>* n) {
  const R vx = static_cast<const R*>(A.in_vx)[i];
  const R vy = static_cast<const R*>(A.in_vy)[i];
  const R vz = static_cast<const R*>(A.in_vz)[i];
  const R sp = Mth<R>::sqrt(vx * vx + vy * vy + vz * vz);
  if (!(sp > R(0))) return false;
  n->x = static_cast<const R*>(A.in_x)[i];
  n->y = static_cast<const R*>(A.in_y)[i];
  n->z = static_cast<const R*>(A.in_z)[i];
  n->dx = vx / sp;
  n->dy = vy / sp;
  n->dz = vz / sp;
  n->speed = sp;
  n->t.set(A.in_t[i]);
  n->w = static_cast<const R*>(A.in_w)[i];
  return true;
}

// What the first half of an order step leaves for the second: the material segments
// ahead, their attenuation coefficients and lengths.
template <typename R, int NS>
struct StepState {
  Seg<R> seg[2 * NS];
  R mu[NS];
  int ns;
  R len_tot, atten, lg;
};

// First half of one order: segments ahead of the packet and the weight of the transmitted
// packet we = w e^{-tau} (section 2.4.3: the packet split into a transmitted and a
// scattered part).  lg: path length inside scatterer A.gs (only when WANTS_GS).
template <typename R, int NS, bool WANTS_GS>
__device__ __forceinline__ R step_segments(const TraceArgs& A, const SampleP<R>& S,
                                           const Lane<R>& L, StepState<R, NS>& st) {
  using M = Mth<R>;
  st.ns = assembly_segs<R, NS>(S, L.n, st.seg);
#pragma unroll
  for (int j = 0; j < NS; ++j)
    st.mu[j] = S.s[j].n100 * (S.s[j].sig_s + S.s[j].sab2200 / L.n.speed);
  R tau = R(0), len_tot = R(0), lg = R(0);
#pragma unroll
  for (int k = 0; k < 2 * NS; ++k) {
    if (k < st.ns) {
      const R len = st.seg[k].b - st.seg[k].a;
      tau += pick_mu<R, NS>(st.mu, st.seg[k].j) * len;
      len_tot += len;
      if (WANTS_GS && st.seg[k].j == A.gs) lg += len;
    }
  }
  st.len_tot = len_tot;
  st.lg = lg;
  st.atten = M::exp(-tau);
  return L.n.w * st.atten;
}

// Second half: the scattered packet continues from a point uniform over the material
// ahead, with a kernel picked at random (section 2.4.3 "Multiple Scattering", bounded
// chain).  Call only when the packet has material ahead and L.o < max_orders.  Returns
// whether the neutron is still alive.
// kernel sets compiled into a launch: the single-crystal kernel only where it is used
constexpr int kKernelsPowder = (1 << MCV_KERNEL_ISO) | (1 << MCV_KERNEL_SQE);
constexpr int kKernelsAll = kKernelsPowder | (1 << MCV_KERNEL_BVK) | (1 << MCV_KERNEL_PHONON) |
                            (1 << MCV_KERNEL_BRAGG) | (1 << MCV_KERNEL_DISP);

// One scattering kernel of a scatterer: kernel kk (0 or 1) of sc, draws from rng's blocks 1-2
// of event o.  Returns whether the packet scatters (false: a parameter-independent zero).
template <typename R, int KS, class Rng>
__device__ __forceinline__ bool scatter_kernel(const SampleP<R>& S, const ScatP<R>& sc, int kk,
                                               const Rng& rng, int o, Ray<R>* n,
                                               Scatter<R>* out, int* err) {
  const int ktype = kk ? sc.ktype1 : sc.ktype0;
  if ((KS & (1 << MCV_KERNEL_ISO)) && ktype == MCV_KERNEL_ISO) {
    kernel_iso<R>(rng, o, n, out);
    return true;
  }
  if ((KS & (1 << MCV_KERNEL_SQE)) && ktype == MCV_KERNEL_SQE)
    return kernel_sqe<R>(S, rng, o, n, out, err);
  if ((KS & (1 << MCV_KERNEL_BVK)) && ktype == MCV_KERNEL_BVK)
    return kernel_bvk<R>(S, sc.cos_rot, sc.sin_rot, rng, o, n, out);
  if ((KS & (1 << MCV_KERNEL_PHONON)) && ktype == MCV_KERNEL_PHONON)
    return kernel_phonon<R>(S, rng, o, n, out);
  if ((KS & (1 << MCV_KERNEL_BRAGG)) && ktype == MCV_KERNEL_BRAGG)
    return kernel_bragg<R>(S, kk ? sc.ksig1 : sc.ksig0, rng, o, n, out);
  if ((KS & (1 << MCV_KERNEL_DISP)) && ktype == MCV_KERNEL_DISP)
    return kernel_disp<R>(S, sc.cos_rot, sc.sin_rot, rng, o, n, out);
  return false;
}

template <typename R, int NS, int KS, class P, class Rng>
__device__ __forceinline__ bool step_scatter(const TraceArgs& A, const SampleP<R>& S,
                                             const Rng& rng, Lane<R>& L,
                                             const StepState<R, NS>& st, P& pol) {
  using M = Mth<R>;
  R u_pt, u_k;
  rng.template pair<R>(L.o, 0, &u_pt, &u_k);
  const R ell = u_pt * st.len_tot;
  R acc = R(0), tau_pt = R(0), s_pt = R(0), lg_pt = R(0);
  int j = 0;
  bool found = false;
#pragma unroll
  for (int k = 0; k < 2 * NS; ++k) {
    if (k < st.ns && !found) {
      const R len = st.seg[k].b - st.seg[k].a;
      const R m = pick_mu<R, NS>(st.mu, st.seg[k].j);
      if (ell < acc + len || k == st.ns - 1) {
        const R part = ell - acc;
        s_pt = st.seg[k].a + part;
        tau_pt += m * part;
        if (P::kWantsGs && st.seg[k].j == A.gs) lg_pt += part;
        j = st.seg[k].j;
        found = true;
      } else {
        acc += len;
        tau_pt += m * len;
        if (P::kWantsGs && st.seg[k].j == A.gs) lg_pt += len;
      }
    }
  }
  const ScatP<R>& sc = S.s[j];
  const R a_fac = sc.mu_s * st.len_tot * M::exp(-tau_pt);
  const R speed_in = L.n.speed;
  L.n.x += s_pt * L.n.dx;
  L.n.y += s_pt * L.n.dy;
  L.n.z += s_pt * L.n.dz;
  L.n.t.add(s_pt / L.n.speed);
  const int kk = (sc.nk == 2 && !(u_k * sc.ksig_sum < sc.ksig0)) ? 1 : 0;
  Scatter<R> out;
  const bool ok = scatter_kernel<R, KS>(S, sc, kk, rng, L.o, &L.n, &out, &pol.err);
  if (!ok) {
    pol.clear(A, L.idx, L.o + 1);
    return false;
  }
  L.n.w = L.n.w * a_fac * out.factor;
  pol.scatter(A, L, j, a_fac, out, lg_pt, speed_in);
  L.o += 1;
  if (L.n.w < S.min_prob || (A.stop_on_zero && L.n.w == R(0))) {
    pol.clear(A, L.idx, L.o);
    return false;
  }
  return true;
}

// The source draw of a neutron that matters only if it meets the sample: false as soon as
// the footprint (host-derived sure-miss bounds) or the direction shows that it misses, which
// skips the later draws; otherwise the same packet as make_beam.
template <typename R, int NS, class Rng>
__device__ __forceinline__ bool make_beam_meeting(const BeamP<R>& B, const SampleP<R>& S,
                                                  const Rng& rng, Ray<R>* n) {
  R aux;
  beam_footprint(B, rng, n);
  if (surely_misses<R>(B, *n)) return false;
  beam_divergence(B, rng, n, &aux);
  Seg<R> seg[2 * NS];
  if (assembly_segs<R, NS>(S, *n, seg) == 0) return false;
  return beam_energy(B, rng, aux, n);
}

// One order of one neutron: segments ahead, emission of the transmitted packet, then the
// scattered packet continues.  Returns whether the neutron is still alive.
template <typename R, int NS, int DET, int KS, class P>
__device__ __forceinline__ bool chain_step(const TraceArgs& A, const R* tu, Lane<R>& L, P& pol) {
  const SampleP<R>& S = Sof<R>(A);
  const NeutronRng rng(A.keys, L.nid);
  StepState<R, NS> st;
  const R we = step_segments<R, NS, P::kWantsGs>(A, S, L, st);
  pol.emit(A, tu, rng, L, we, st.atten, st.lg, st.len_tot);
  if (L.o == S.max_orders || !(st.len_tot > R(0))) {
    pol.clear(A, L.idx, L.o + 1);
    return false;
  }
  return step_scatter<R, NS, KS, P>(A, S, rng, L, st, pol);
}

// Warp loop: each warp owns ids [lo, hi) of the launch; lanes whose neutron finished take
// the next ids at the top of each step, again while some lane is still without a live
// neutron (a policy that keeps only the neutrons meeting the sample drops two thirds of its
// draws), so all 32 lanes run chain_step together.
template <typename R, int NS, int DET, int KS, class P>
__device__ __forceinline__ void run_chain(const TraceArgs& A, const R* tu, P& pol) {
  const unsigned kFull = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t lo = (A.n * wid) / nw, hi = (A.n * (wid + 1)) / nw;
  const bool from_input = A.in_x != nullptr;
  int64_t next = lo;
  Lane<R> L;
  L.active = false;
  L.o = 0;
  L.idx = 0;
  L.nid = 0;
  for (;;) {
    for (unsigned idle = __ballot_sync(kFull, !L.active); idle != 0u && next < hi;
         idle = __ballot_sync(kFull, !L.active)) {
      if (!L.active) {
        const int64_t i = next + __popc(idle & lt_mask);
        if (i < hi) {
          L.idx = i;
          L.nid = (from_input && A.in_id) ? A.in_id[i] : A.first_id + i;
          L.o = 0;
          bool ok;
          if (from_input) {
            ok = load_input<R>(A, i, &L.n);
          } else {
            const NeutronRng rng(A.keys, L.nid);
            ok = P::kMeetingOnly ? make_beam_meeting<R, NS>(Bof<R>(A), Sof<R>(A), rng, &L.n)
                                 : make_beam<R>(Bof<R>(A), rng, &L.n);
          }
          ok = ok && !(L.n.w < Sof<R>(A).min_prob) && !(A.stop_on_zero && L.n.w == R(0));
          if (!ok) pol.clear(A, i, 0);
          if (ok) pol.start(L);
          L.active = ok;
        }
      }
      next += __popc(idle);
    }
    if (!__any_sync(kFull, L.active)) break;  // every id of the range taken and done
    if (L.active) L.active = chain_step<R, NS, DET, KS, P>(A, tu, L, pol);
  }
  pol.flush(A, lane);
}

template <typename R, int DET>
__device__ __forceinline__ void stage_tubes(const TraceArgs& A, R* tu) {
  if (DET == MCV_DET_TUBES) {
    const DetP<R>& D = Dof<R>(A);
    for (int i = threadIdx.x; i < 2 * D.max_tubes_row; i += blockDim.x) tu[i] = D.tube_u[i];
    __syncthreads();
  }
}

}  // namespace mcv
