// mcv_grad_noalloc: the loss and its adjoint gradient (mcv_grad) for callers that cannot
// allocate device memory -- code that runs where cudaMalloc is not allowed or not wanted:
// inside a captured CUDA graph, under a memory pool owned by someone else, in a process whose
// allocator is locked down, or from a language runtime that only hands out the buffers it
// manages.  Those callers pass the inputs and outputs; the work buffers mcv_grad takes from
// its context or from the caller (the device error word and dchi2/dI per histogram bin)
// live here instead, in one file-scope device array that every GPU loading the library
// holds until the process exits.
#include <atomic>
#include <cmath>
#include <cstring>
#include <string>

#include <cuda_runtime.h>

#include "mcv_host.h"

namespace {

// dchi2/dI for up to kMaxBins bins, preceded by the device error word (256-byte aligned)
constexpr int64_t kMaxBins = MCV_NOALLOC_MAX_BINS;
constexpr int64_t kHeader = 32;  // doubles: the error word and padding
static __device__ __align__(256) double g_noalloc_scratch[kHeader + kMaxBins];

mcv_status noalloc_fail(mcv_status st, const std::string& msg) {
  mcv::set_last_error(msg);
  return st;
}

// Device address of the array on each device.  The address belongs to the module loaded in
// the device's current context; it is looked up again on every call made outside stream
// capture (a context created anew, after cudaDeviceReset, may hold the module elsewhere) and
// kept for calls made during capture, where no lookup is done.
constexpr int kMaxDevices = 64;
std::atomic<double*> g_scratch_addr[kMaxDevices];

mcv_status scratch_of(int device, cudaStream_t stream, double** out) {
  if (device < 0 || device >= kMaxDevices)
    return noalloc_fail(MCV_EINVAL, "device index out of range");
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(stream, &cap);
  if (e != cudaSuccess)
    return noalloc_fail(MCV_ECUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(e));
  double* addr = g_scratch_addr[device].load();
  if (cap == cudaStreamCaptureStatusNone || !addr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess)
      return noalloc_fail(MCV_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    addr = static_cast<double*>(p);
    g_scratch_addr[device].store(addr);
  }
  *out = addr;
  return MCV_OK;
}

}  // namespace

namespace mcv {
// parameter blocks and error message of the C ABI (mcv_api.cu)
mcv_status build_trace_args_for_grad(const mcv_sample* sample, const mcv_beam_params* beam,
                                     const mcv_detector* det, TraceArgs* A);
}  // namespace mcv

extern "C" {

mcv_status mcv_grad_noalloc(const mcv_sample* sample, const mcv_beam_params* beam,
                            const mcv_detector* det, uint32_t seed, uint32_t sim_id,
                            int64_t first_id, int64_t n, const double* target, double scale_c,
                            int grad_scatterer, mcv_hist* hist, double* loss, double* dsqe,
                            double* dsig, void* stream) {
  mcv::host::CallRange range_("mcv_grad_noalloc");
  mcv::TraceArgs A;
  std::memset(&A, 0, sizeof(A));
  mcv_status st = mcv::build_trace_args_for_grad(sample, beam, det, &A);
  if (st != MCV_OK) return st;
  if (A.Dd.n_bins > kMaxBins)
    return noalloc_fail(MCV_EINVAL, "the histogram has " + std::to_string(A.Dd.n_bins) +
                                        " bins; mcv_grad_noalloc holds at most " +
                                        std::to_string(kMaxBins));
  if (n < 0 || n > ((int64_t)1 << 40) || first_id < 0 || first_id > (((int64_t)1 << 62) - n))
    return noalloc_fail(MCV_EINVAL, "bad neutron range");
  if (!target || !loss || !dsig || !hist || !hist->counts)
    return noalloc_fail(MCV_EINVAL, "needs target, hist->counts, loss and dsig");
  if (A.Sd.has_sqe && !dsqe) return noalloc_fail(MCV_EINVAL, "needs dsqe for an S(Q,E) sample");
  if (grad_scatterer < 0 || grad_scatterer >= A.Sd.ns)
    return noalloc_fail(MCV_EINVAL, "grad_scatterer out of range");
  if (!(A.Sd.s[grad_scatterer].sig_s > 0.0))
    return noalloc_fail(MCV_EINVAL, "the differentiated scatterer needs a positive cross section");
  if (!std::isfinite(scale_c)) return noalloc_fail(MCV_EINVAL, "scale_c is not finite");
  int device = 0;
  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess) return noalloc_fail(MCV_ECUDA, cudaGetErrorString(e));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* scratch = nullptr;
  st = scratch_of(device, s, &scratch);
  if (st != MCV_OK) return st;
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) return noalloc_fail(MCV_ECUDA, cudaGetErrorString(e));
  double* g = scratch + kHeader;
  // the outputs start at zero; the dchi2/dI bins are all overwritten; the error word keeps
  // what earlier calls found until mcv_sync(NULL, stream) reads and clears it
  e = mcv::launch_zero(hist->counts, A.Dd.n_bins, sms * 8, s);
  if (e == cudaSuccess && hist->tallies) e = mcv::launch_zero(hist->tallies, MCV_NTALLY, 1, s);
  if (e == cudaSuccess) e = mcv::launch_zero(loss, 1, 1, s);
  if (e == cudaSuccess) e = mcv::launch_zero(dsig, 2, 1, s);
  if (e == cudaSuccess && A.Sd.has_sqe) e = mcv::launch_zero(dsqe, (int64_t)A.Sd.nq * A.Sd.ne, sms * 8, s);
  if (e != cudaSuccess) return noalloc_fail(MCV_ECUDA, cudaGetErrorString(e));
  A.seed = seed;
  A.sim_id = sim_id;
  A.keys = mcv::host::philox_keys(seed, sim_id);
  A.first_id = first_id;
  A.n = n;
  A.err = reinterpret_cast<int*>(scratch);
  A.gs = grad_scatterer;
  const int fp = sample->fp_mode;
  const int threads = mcv::trace_threads();
  auto grid_of = [&](int per_sm) {
    const int64_t full = (int64_t)sms * per_sm;
    const int64_t need = (n + threads - 1) / threads;
    const int64_t gsz = need < full ? need : full;
    return (int)(gsz < 1 ? 1 : gsz);
  };
  if (n > 0) {
    A.hist = hist->counts;
    A.tallies = hist->tallies;
    A.stop_on_zero = 1;
    int occ = 0;
    e = mcv::trace_blocks_per_sm(fp, A.Sd.ns, A.Dd.kind, A.Sd.wide, &occ);
    if (e != cudaSuccess || occ < 1) occ = 1;
    e = mcv::launch_trace(A, fp, A.Dd.kind, grid_of(occ), s);
    if (e != cudaSuccess) return noalloc_fail(MCV_ECUDA, cudaGetErrorString(e));
  }
  e = mcv::launch_chi2(hist->counts, target, scale_c, A.Dd.n_bins, g, loss,
                       reinterpret_cast<int*>(scratch), sms * 8, s);
  if (e != cudaSuccess) return noalloc_fail(MCV_ECUDA, cudaGetErrorString(e));
  if (n > 0) {
    A.hist = nullptr;
    A.tallies = nullptr;
    A.stop_on_zero = 0;
    A.g = g;
    A.dsqe = A.Sd.has_sqe ? dsqe : nullptr;
    A.dsig = dsig;
    int occ_a = 0;
    e = mcv::adjoint_blocks_per_sm(fp, A.Sd.ns, A.Dd.kind, A.Sd.wide, &occ_a);
    if (e != cudaSuccess || occ_a < 1) occ_a = 1;
    e = mcv::launch_adjoint(A, fp, A.Dd.kind, grid_of(occ_a), s);
    if (e != cudaSuccess) return noalloc_fail(MCV_ECUDA, cudaGetErrorString(e));
  }
  return MCV_OK;
}

}  // extern "C"

namespace mcv {

mcv_status noalloc_sync(cudaStream_t stream) {
  cudaError_t e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess)
    return noalloc_fail(MCV_ECUDA, std::string("cudaStreamSynchronize: ") + cudaGetErrorString(e));
  int device = 0;
  e = cudaGetDevice(&device);
  if (e != cudaSuccess) return noalloc_fail(MCV_ECUDA, cudaGetErrorString(e));
  double* scratch = nullptr;
  mcv_status st = scratch_of(device, stream, &scratch);
  if (st != MCV_OK) return st;
  int flag = 0;
  e = cudaMemcpy(&flag, scratch, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess)
    return noalloc_fail(MCV_ECUDA, std::string("cudaMemcpy: ") + cudaGetErrorString(e));
  if (flag) {
    e = cudaMemset(scratch, 0, sizeof(int));
    if (e != cudaSuccess)
      return noalloc_fail(MCV_ECUDA, std::string("cudaMemset: ") + cudaGetErrorString(e));
    return noalloc_fail(MCV_EDEVICE,
                        "mcv_grad_noalloc: a kernel found an out-of-range index or a target "
                        "bin that is negative or not finite");
  }
  return MCV_OK;
}

}  // namespace mcv
