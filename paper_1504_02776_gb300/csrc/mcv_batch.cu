// Batched launches of the C ABI (mcv_batch_* and mcv_trace_batch, declared in mcv.h): many
// simulations traced by one persistent kernel fed by a device work queue, and the
// autotuner that picks its launch shape.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "mcv_host.h"

using namespace mcv::host;

namespace {

constexpr int kWarpsPerBlock = 4;  // the kernels' 128 threads
constexpr int64_t kDefaultChunk = 8192;
constexpr int64_t kMinChunk = 256;

// The simulations of a batch as the kernel reads them: host images of the parameter blocks
// in the batch's real type, and the shape of the batch.
struct BatchImage {
  int fp = 0, ns = 1, det = 0, bvk = 0;
  int ss = 1;  // every simulation has the same sample (kept in kernel parameter space)
  int ev = 0;  // some simulation appends to an event list
  int nsims = 0;
  int64_t total_n = 0;
  std::vector<unsigned char> sims;  // SimP<R>[nsims]
  size_t sim_bytes = 0;
  std::vector<int64_t> n;           // neutrons per simulation
};

template <typename R>
void put_sim(BatchImage* im, int k, const mcv::SimP<R>& p) {
  std::memcpy(im->sims.data() + (size_t)k * sizeof(p), &p, sizeof(p));
}

// Checks every simulation and builds the kernel's images.  A->Dd/Df receive the detector.
mcv_status build_image(const mcv_sim* sims, int nsims, const mcv_detector* det, int fp_mode,
                       mcv::TraceArgs* A, BatchImage* im) {
  if (!sims || nsims < 1) return fail(MCV_EINVAL, "a batch needs at least one simulation");
  if (fp_mode != MCV_FP64 && fp_mode != MCV_FP32) return fail(MCV_EINVAL, "bad fp_mode");
  mcv_status st = build_detector(det, &A->Dd);
  if (st != MCV_OK) return st;
  im->fp = fp_mode;
  im->det = A->Dd.kind;
  im->nsims = nsims;
  im->sim_bytes = fp_mode == MCV_FP32 ? sizeof(mcv::SimP<float>) : sizeof(mcv::SimP<double>);
  im->sims.assign((size_t)nsims * im->sim_bytes, 0);
  im->n.assign(nsims, 0);
  int ns = 1, bvk = 0, same = 1;
  int64_t total = 0;
  double r_s = 0.0;  // radius holding every simulation's sample
  mcv::SampleP<double> first;
  for (int k = 0; k < nsims; ++k) {
    const mcv_sim& s = sims[k];
    const std::string who = "simulation " + std::to_string(k) + ": ";
    mcv::SimP<double> d;
    std::memset(&d, 0, sizeof(d));
    st = build_sample(s.sample, &d.S);
    if (st != MCV_OK) return fail(st, who + mcv_last_error());
    if (s.sample->fp_mode != fp_mode)
      return fail(MCV_EINVAL, who + "sample fp_mode differs from the batch's");
    st = build_beam(s.beam, &d.B);
    if (st != MCV_OK) return fail(st, who + mcv_last_error());
    set_miss_bounds(d.S, &d.B);
    r_s = std::max(r_s, sample_radius(d.S));
    if (s.n < 0 || s.n > kMaxNeutrons || s.first_id < 0 ||
        s.first_id > (((int64_t)1 << 62) - s.n))
      return fail(MCV_EINVAL, who + "bad neutron range");
    if (!s.hist.counts && !s.hist.tallies && !s.hist.events)
      return fail(MCV_EINVAL, who + "needs a histogram, tallies or an event list");
    if (s.tof_min_s == 0.0 && s.tof_max_s == 0.0) {
      d.win = A->Dd.win;
    } else {
      if (!is_finite(s.tof_min_s) || !is_finite(s.tof_max_s) || !(s.tof_max_s > s.tof_min_s))
        return fail(MCV_EINVAL, who + "bad time window");
      d.win = tof_window(s.tof_min_s, s.tof_max_s, A->Dd.win.n_tof);
    }
    d.seed = s.seed;
    d.sim_id = s.sim_id;
    d.first_id = s.first_id;
    d.n = s.n;
    d.hist = s.hist.counts;
    d.tallies = s.hist.tallies;
    if (s.hist.events) {
      st = event_sink(s.hist.events, s.sim_id, &d.ev);
      if (st != MCV_OK) return fail(st, who + mcv_last_error());
      im->ev = 1;
    }
    if (total > kMaxNeutrons - s.n) return fail(MCV_EINVAL, "too many neutrons in the batch");
    total += s.n;
    ns = std::max(ns, d.S.ns);
    if (d.S.wide) bvk = 1;
    if (k == 0)
      first = d.S;
    else if (std::memcmp(&first, &d.S, sizeof(first)) != 0)
      same = 0;
    im->n[k] = s.n;
    if (fp_mode == MCV_FP32) {
      mcv::SimP<float> f;
      std::memset(&f, 0, sizeof(f));
      cast_sample(d.S, &f.S);
      cast_beam(d.B, &f.B);
      f.win = d.win;
      f.seed = d.seed;
      f.sim_id = d.sim_id;
      f.first_id = d.first_id;
      f.n = d.n;
      f.hist = d.hist;
      f.tallies = d.tallies;
      f.ev = d.ev;
      put_sim(im, k, f);
    } else {
      put_sim(im, k, d);
    }
  }
  // every detected packet starts at a scattering point in one of the samples
  set_det_miss_bounds(r_s, &A->Dd);
  cast_detector(A->Dd, &A->Df);
  im->ns = ns <= 1 ? 1 : (ns == 2 ? 2 : 4);
  im->bvk = bvk;
  im->ss = same;
  im->total_n = total;
  if (same) {
    // the shared sample goes into the kernel's parameter blocks
    A->Sd = first;
    cast_sample(first, &A->Sf);
  }
  return MCV_OK;
}

// number of work items of a batch for a chunk size
int64_t count_items(const std::vector<int64_t>& n, int64_t chunk) {
  int64_t k = 0;
  for (int64_t m : n) k += (m + chunk - 1) / chunk;
  return k;
}

// Device layout of a batch: the item counters (nsims, padded to 256 bytes), SimP[nsims],
// nstart[nsims + 1].
size_t counters_bytes(const BatchImage& im) {
  return ((im.n.size() * sizeof(unsigned long long) + 255) / 256) * 256;
}

size_t device_bytes(const BatchImage& im) {
  return counters_bytes(im) + im.sims.size() + (im.n.size() + 1) * sizeof(int64_t);
}

void point_args(void* base, const BatchImage& im, int64_t chunk, mcv::BatchArgs* Q) {
  unsigned char* b = static_cast<unsigned char*>(base);
  Q->next = reinterpret_cast<unsigned long long*>(b);
  Q->sims = b + counters_bytes(im);
  Q->nstart = reinterpret_cast<const int64_t*>(b + counters_bytes(im) + im.sims.size());
  Q->nsims = im.nsims;
  Q->chunk = chunk;
  Q->total = im.total_n;
}

// host image of the whole device block (counters zero)
std::vector<unsigned char> device_image(const BatchImage& im) {
  std::vector<unsigned char> out(device_bytes(im), 0);
  std::vector<int64_t> nstart(im.n.size() + 1, 0);
  for (size_t k = 0; k < im.n.size(); ++k) nstart[k + 1] = nstart[k] + im.n[k];
  std::memcpy(out.data() + counters_bytes(im), im.sims.data(), im.sims.size());
  std::memcpy(out.data() + counters_bytes(im) + im.sims.size(), nstart.data(),
              nstart.size() * sizeof(int64_t));
  return out;
}

// default work-item size: about 16 items per resident warp, a multiple of 32 in
// [kMinChunk, kDefaultChunk] (items of one simulation follow each other in a warp without a
// drain, so small items cost little more than their queue counter update)
int64_t default_chunk(int64_t total_n, int64_t warps) {
  int64_t c = total_n / std::max<int64_t>(1, warps * 16);
  c = std::min(std::max(c, kMinChunk), kDefaultChunk);
  return (c / 32) * 32;
}

int grid_of(int sm_count, int blocks_per_sm, int64_t n_items) {
  const int64_t full = (int64_t)sm_count * blocks_per_sm;
  const int64_t need = (n_items + kWarpsPerBlock - 1) / kWarpsPerBlock;
  return (int)std::max<int64_t>(1, std::min(full, need));
}

}  // namespace

struct mcv_batch {
  mcv_ctx* ctx = nullptr;
  mcv::TraceArgs A;
  BatchImage im;
  void* d_block = nullptr;
  mcv::BatchArgs Q;
  int64_t chunk = 0, n_items = 0;
  int blocks_per_sm = 1, max_blocks_per_sm = 1;
  int grid = 1;
};

namespace {

mcv::TraceArgs& zeroed(mcv::TraceArgs& A) {
  std::memset(&A, 0, sizeof(A));
  return A;
}

mcv_ctx::Tuned& tuned_slot(mcv_ctx* ctx, const BatchImage& im) {
  return ctx->tuned[im.fp][ns_index(im.ns)][im.det][im.bvk][im.ss];
}

// uploads the batch's device block and sets the launch arguments for its current chunk
mcv_status upload(mcv_batch* b) {
  const std::vector<unsigned char> img = device_image(b->im);
  cudaError_t e = cudaMemcpy(b->d_block, img.data(), img.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy (batch parameters)");
  point_args(b->d_block, b->im, b->chunk, &b->Q);
  b->n_items = count_items(b->im.n, b->chunk);
  b->grid = grid_of(b->ctx->sm_count, b->blocks_per_sm, b->n_items);
  return MCV_OK;
}

mcv_status launch(mcv_batch* b, const mcv::BatchArgs& Q, int64_t n_items, int grid,
                  cudaStream_t s) {
  if (n_items == 0) return MCV_OK;
  cudaError_t e = cudaMemsetAsync(Q.next, 0, (size_t)Q.nsims * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync (queue counters)");
  e = mcv::launch_batch(b->A, Q, b->im.fp, b->im.ns, b->im.det, b->im.bvk, b->im.ss, b->im.ev,
                        grid, s);
  if (e != cudaSuccess) return cuda_fail(e, "batch kernel launch");
  return MCV_OK;
}

mcv_status occupancy(mcv_ctx* ctx, const BatchImage& im, int* blocks) {
  cudaError_t e = mcv::batch_blocks_per_sm(im.fp, im.ns, im.det, im.bvk, im.ss, im.ev, blocks);
  if (e != cudaSuccess) return cuda_fail(e, "batch kernel occupancy");
  if (*blocks < 1) return fail(MCV_ECUDA, "the batch kernel does not fit on an SM");
  (void)ctx;
  return MCV_OK;
}

}  // namespace

extern "C" {

mcv_status mcv_batch_create(mcv_ctx* ctx, const mcv_sim* sims, int nsims,
                            const mcv_detector* det, int fp_mode, mcv_batch** out) {
  mcv::host::CallRange range_("mcv_batch_create");
  if (!out) return fail(MCV_EINVAL, "out is NULL");
  *out = nullptr;
  mcv_status st = check_ctx(ctx);
  if (st != MCV_OK) return st;
  mcv_batch* b = new mcv_batch();
  b->ctx = ctx;
  zeroed(b->A);
  st = build_image(sims, nsims, det, fp_mode, &b->A, &b->im);
  if (st != MCV_OK) {
    delete b;
    return st;
  }
  b->A.err = ctx->d_err;
  b->A.stop_on_zero = 1;
  st = occupancy(ctx, b->im, &b->max_blocks_per_sm);
  if (st != MCV_OK) {
    delete b;
    return st;
  }
  const mcv_ctx::Tuned& t = tuned_slot(ctx, b->im);
  if (t.chunk > 0) {
    b->chunk = t.chunk;
    b->blocks_per_sm = std::min(t.blocks_per_sm, b->max_blocks_per_sm);
  } else {
    b->blocks_per_sm = b->max_blocks_per_sm;
    b->chunk = default_chunk(b->im.total_n,
                             (int64_t)ctx->sm_count * b->blocks_per_sm * kWarpsPerBlock);
  }
  cudaError_t e = cudaMalloc(&b->d_block, device_bytes(b->im));
  if (e != cudaSuccess) {
    delete b;
    return alloc_fail("cannot allocate the batch's parameter block");
  }
  st = upload(b);
  if (st != MCV_OK) {
    cudaFree(b->d_block);
    delete b;
    return st;
  }
  *out = b;
  return MCV_OK;
}

mcv_status mcv_batch_run(mcv_batch* b, void* stream) {
  mcv::host::CallRange range_("mcv_batch_run");
  if (!b) return fail(MCV_EINVAL, "batch is NULL");
  mcv_status st = check_ctx(b->ctx);
  if (st != MCV_OK) return st;
  return launch(b, b->Q, b->n_items, b->grid, static_cast<cudaStream_t>(stream));
}

mcv_status mcv_batch_shape(const mcv_batch* b, int64_t* chunk, int* blocks_per_sm, int* grid,
                           int64_t* n_items) {
  if (!b) return fail(MCV_EINVAL, "batch is NULL");
  if (chunk) *chunk = b->chunk;
  if (blocks_per_sm) *blocks_per_sm = b->blocks_per_sm;
  if (grid) *grid = b->grid;
  if (n_items) *n_items = b->n_items;
  return MCV_OK;
}

mcv_status mcv_batch_destroy(mcv_batch* b) {
  if (!b) return MCV_OK;
  cudaSetDevice(b->ctx->device);
  cudaDeviceSynchronize();
  cudaFree(b->d_block);
  delete b;
  return MCV_OK;
}

mcv_status mcv_batch_tune(mcv_batch* b, int64_t trial_neutrons, void* stream) {
  mcv::host::CallRange range_("mcv_batch_tune");
  if (!b) return fail(MCV_EINVAL, "batch is NULL");
  mcv_status st = check_ctx(b->ctx);
  if (st != MCV_OK) return st;
  if (b->im.total_n == 0) return MCV_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (trial_neutrons <= 0) trial_neutrons = 20000000;
  const int64_t trial_total = std::min(trial_neutrons, b->im.total_n);
  // the trial batch: the same simulations with proportionally fewer neutrons, all into one
  // scratch histogram and tally block
  BatchImage tr = b->im;
  double* scratch = nullptr;
  const int64_t nb = b->A.Dd.n_bins;
  cudaError_t e = cudaMalloc(&scratch, (size_t)(nb + MCV_NTALLY) * sizeof(double));
  if (e != cudaSuccess) return alloc_fail("cannot allocate the tuner's scratch histogram");
  e = cudaMemsetAsync(scratch, 0, (size_t)(nb + MCV_NTALLY) * sizeof(double), s);
  tr.total_n = 0;
  for (int k = 0; k < tr.nsims; ++k) {
    int64_t m = 0;
    if (b->im.n[k] > 0)
      m = std::max<int64_t>(1, (int64_t)((double)b->im.n[k] * trial_total / b->im.total_n));
    tr.n[k] = m;
    tr.total_n += m;
    unsigned char* p = tr.sims.data() + (size_t)k * tr.sim_bytes;
    if (tr.fp == MCV_FP32) {
      mcv::SimP<float>* q = reinterpret_cast<mcv::SimP<float>*>(p);
      q->n = m;
      q->hist = scratch;
      q->tallies = scratch + nb;
      q->ev = mcv::EvSink{};
    } else {
      mcv::SimP<double>* q = reinterpret_cast<mcv::SimP<double>*>(p);
      q->n = m;
      q->hist = scratch;
      q->tallies = scratch + nb;
      q->ev = mcv::EvSink{};
    }
  }
  void* d_trial = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&d_trial, device_bytes(tr));
  if (e == cudaSuccess) {
    const std::vector<unsigned char> img = device_image(tr);
    e = cudaMemcpyAsync(d_trial, img.data(), img.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&ev1);
  float best_ms = -1.0f;
  int64_t best_chunk = b->chunk;
  int best_blocks = b->blocks_per_sm;
  // candidate work-item sizes of the full batch; the trial uses them scaled by its fraction
  // of the neutrons, which keeps the number of items per warp (the load balance at the end)
  const double frac = (double)tr.total_n / (double)b->im.total_n;
  const int64_t chunks[] = {512, 1024, 2048, 4096, 8192};
  st = MCV_OK;
  for (int64_t chunk : chunks) {
    if (e != cudaSuccess || st != MCV_OK) break;
    const int64_t tc = std::max<int64_t>(32, ((int64_t)(chunk * frac) / 32) * 32);
    mcv::BatchArgs Q;
    point_args(d_trial, tr, tc, &Q);
    const int64_t items = count_items(tr.n, tc);
    for (int bps = b->max_blocks_per_sm; bps >= std::max(1, b->max_blocks_per_sm - 1); --bps) {
      const int grid = grid_of(b->ctx->sm_count, bps, items);
      st = launch(b, Q, items, grid, s);  // warm-up
      if (st != MCV_OK) break;
      e = cudaEventRecord(ev0, s);
      if (e == cudaSuccess) st = launch(b, Q, items, grid, s);
      if (st != MCV_OK) break;
      if (e == cudaSuccess) e = cudaEventRecord(ev1, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(ev1);
      float ms = 0.0f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev0, ev1);
      if (e != cudaSuccess) break;
      if (best_ms < 0.0f || ms < best_ms) {
        best_ms = ms;
        best_chunk = chunk;
        best_blocks = bps;
      }
    }
  }
  if (e == cudaSuccess && st == MCV_OK) e = cudaStreamSynchronize(s);
  if (ev0) cudaEventDestroy(ev0);
  if (ev1) cudaEventDestroy(ev1);
  if (d_trial) cudaFree(d_trial);
  cudaFree(scratch);
  if (st != MCV_OK) return st;
  if (e != cudaSuccess) return cuda_fail(e, "batch tuning");
  b->chunk = best_chunk;
  b->blocks_per_sm = best_blocks;
  mcv_ctx::Tuned& t = tuned_slot(b->ctx, b->im);
  t.chunk = best_chunk;
  t.blocks_per_sm = best_blocks;
  return upload(b);
}

mcv_status mcv_trace_batch(mcv_ctx* ctx, const mcv_sim* sims, int nsims,
                           const mcv_detector* det, int fp_mode, void* stream) {
  mcv::host::CallRange range_("mcv_trace_batch");
  mcv_status st = check_ctx(ctx);
  if (st != MCV_OK) return st;
  mcv_batch b;
  b.ctx = ctx;
  zeroed(b.A);
  st = build_image(sims, nsims, det, fp_mode, &b.A, &b.im);
  if (st != MCV_OK) return st;
  b.A.err = ctx->d_err;
  b.A.stop_on_zero = 1;
  if (b.im.total_n == 0) return MCV_OK;
  st = occupancy(ctx, b.im, &b.max_blocks_per_sm);
  if (st != MCV_OK) return st;
  const mcv_ctx::Tuned& t = tuned_slot(ctx, b.im);
  if (t.chunk > 0) {
    b.chunk = t.chunk;
    b.blocks_per_sm = std::min(t.blocks_per_sm, b.max_blocks_per_sm);
  } else {
    b.blocks_per_sm = b.max_blocks_per_sm;
    b.chunk = default_chunk(b.im.total_n, (int64_t)ctx->sm_count * b.blocks_per_sm * kWarpsPerBlock);
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const std::vector<unsigned char> img = device_image(b.im);
  void* d = nullptr;
  cudaError_t e = cudaMallocAsync(&d, img.size(), s);
  if (e != cudaSuccess) return alloc_fail("cannot allocate the batch's parameter block");
  // pageable source: the copy has taken the host bytes when the call returns
  e = cudaMemcpyAsync(d, img.data(), img.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    point_args(d, b.im, b.chunk, &b.Q);
    const int64_t items = count_items(b.im.n, b.chunk);
    st = launch(&b, b.Q, items, grid_of(ctx->sm_count, b.blocks_per_sm, items), s);
  }
  cudaError_t ef = cudaFreeAsync(d, s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync (batch parameters)");
  if (st != MCV_OK) return st;
  if (ef != cudaSuccess) return cuda_fail(ef, "cudaFreeAsync");
  return MCV_OK;
}

}  // extern "C"
