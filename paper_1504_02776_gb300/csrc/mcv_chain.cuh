// The per-neutron chain of scatterings and the warp loop that feeds it, shared by the
// forward kernels (histogram) and the adjoint kernel (gradient).  What happens to each
// emitted packet and each scattering is left to a policy object, so that both kernels
// trace exactly the same paths with exactly the same arithmetic.
//
// Policy interface (device, per lane):
//   kWantsGs                        compile-time: path lengths in scatterer A.gs are needed
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
  n->t = A.in_t[i];
  n->w = static_cast<const R*>(A.in_w)[i];
  return true;
}

// One order of one neutron: segments ahead, emission of the transmitted packet, then the
// scattered packet continues from a point uniform over the material ahead with a kernel
// picked at random (section 2.4.3 "Multiple Scattering", as a bounded chain).  Returns
// whether the neutron is still alive.
template <typename R, int NS, int DET, class P>
__device__ __forceinline__ bool chain_step(const TraceArgs& A, const R* tu, Lane<R>& L, P& pol) {
  using M = Mth<R>;
  const DSample& S = A.S;
  const NeutronRng rng(A.seed, A.sim_id, L.nid);
  Seg<R> seg[2 * NS];
  const int ns = assembly_segs<R, NS>(S, L.n, seg);
  R mu[NS];
#pragma unroll
  for (int j = 0; j < NS; ++j) mu[j] = (R)S.s[j].mu_s + (R)S.s[j].mu_a_v / L.n.speed;
  R tau = R(0), len_tot = R(0), lg = R(0);
#pragma unroll
  for (int k = 0; k < 2 * NS; ++k) {
    if (k < ns) {
      const R len = seg[k].b - seg[k].a;
      tau += pick_mu<R, NS>(mu, seg[k].j) * len;
      len_tot += len;
      if (P::kWantsGs && seg[k].j == A.gs) lg += len;
    }
  }
  const R atten = M::exp(-tau);
  const R we = L.n.w * atten;
  pol.emit(A, tu, rng, L, we, atten, lg, len_tot);
  if (L.o == S.max_orders || !(len_tot > R(0))) {
    pol.clear(A, L.idx, L.o + 1);
    return false;
  }
  R u_pt, u_k;
  rng.pair<R>(L.o, 0, &u_pt, &u_k);
  const R ell = u_pt * len_tot;
  R acc = R(0), tau_pt = R(0), s_pt = R(0), lg_pt = R(0);
  int j = 0;
  bool found = false;
#pragma unroll
  for (int k = 0; k < 2 * NS; ++k) {
    if (k < ns && !found) {
      const R len = seg[k].b - seg[k].a;
      const R m = pick_mu<R, NS>(mu, seg[k].j);
      if (ell < acc + len || k == ns - 1) {
        const R part = ell - acc;
        s_pt = seg[k].a + part;
        tau_pt += m * part;
        if (P::kWantsGs && seg[k].j == A.gs) lg_pt += part;
        j = seg[k].j;
        found = true;
      } else {
        acc += len;
        tau_pt += m * len;
        if (P::kWantsGs && seg[k].j == A.gs) lg_pt += len;
      }
    }
  }
  const DScat& sc = S.s[j];
  const R a_fac = (R)sc.mu_s * len_tot * M::exp(-tau_pt);
  const R speed_in = L.n.speed;
  L.n.x += s_pt * L.n.dx;
  L.n.y += s_pt * L.n.dy;
  L.n.z += s_pt * L.n.dz;
  L.n.t = add_time<R>(L.n.t, s_pt, L.n.speed);
  const int kk = (sc.nk == 2 && !(u_k * (R)sc.ksig_sum < (R)sc.ksig0)) ? 1 : 0;
  const int ktype = kk ? sc.ktype1 : sc.ktype0;
  Scatter<R> out;
  bool ok = false;
  if (ktype == MCV_KERNEL_ISO) {
    kernel_iso<R>(rng, L.o, &L.n, &out);
    ok = true;
  } else if (ktype == MCV_KERNEL_SQE) {
    ok = kernel_sqe<R>(S, rng, L.o, &L.n, &out, &pol.err);
  }
  if (!ok) {
    pol.clear(A, L.idx, L.o + 1);
    return false;
  }
  L.n.w = L.n.w * a_fac * out.factor;
  pol.scatter(A, L, j, a_fac, out, lg_pt, speed_in);
  L.o += 1;
  if (L.n.w < (R)S.min_prob || (A.stop_on_zero && L.n.w == R(0))) {
    pol.clear(A, L.idx, L.o);
    return false;
  }
  return true;
}

// Warp loop: each warp owns ids [lo, hi) of the launch; lanes whose neutron finished take
// the next ids at the top of each step, so all 32 lanes run chain_step together.
template <typename R, int NS, int DET, class P>
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
    const unsigned idle = __ballot_sync(kFull, !L.active);
    if (idle != 0u && next < hi) {
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
            const NeutronRng rng(A.seed, A.sim_id, L.nid);
            ok = make_beam<R>(A.B, rng, &L.n);
          }
          ok = ok && !(L.n.w < (R)A.S.min_prob) && !(A.stop_on_zero && L.n.w == R(0));
          if (!ok) pol.clear(A, i, 0);
          if (ok) pol.start(L);
          L.active = ok;
        }
      }
      next += __popc(idle);
    }
    if (!__any_sync(kFull, L.active)) {
      if (next >= hi) break;
      continue;
    }
    if (L.active) L.active = chain_step<R, NS, DET, P>(A, tu, L, pol);
  }
  pol.flush(A, lane);
}

template <typename R, int DET>
__device__ __forceinline__ void stage_tubes(const TraceArgs& A, R* tu) {
  if (DET == MCV_DET_TUBES) {
    for (int i = threadIdx.x; i < 2 * A.D.max_tubes_row; i += blockDim.x) tu[i] = (R)A.D.tube_u[i];
    __syncthreads();
  }
}

}  // namespace mcv
