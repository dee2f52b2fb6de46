// Host-side pieces of the C ABI shared by its translation units (mcv_api.cu, mcv_batch.cu):
// the context, the error message, and the conversion of the public descriptions (mcv.h)
// into the kernels' parameter blocks.
#pragma once

#include <cstdint>
#include <string>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "mcv_launch.h"

struct mcv_ctx {
  int device;
  int sm_count;
  int* d_err;          // device error flag (kernels set it; mcv_sync reads and clears it)
  int occ[2][3][3][2]; // cached blocks per SM of the fused kernel: [fp][ns 1,2,4][det][bvk]
  int occ_adj[2][3][3][2];  // the same for the adjoint kernel
  // batched launch chosen by mcv_batch_tune for a kind of batch: neutrons per work item and
  // blocks per SM (0: not tuned yet); [fp][ns 1,2,4][det][bvk][one sample for all]
  struct Tuned {
    int64_t chunk;
    int blocks_per_sm;
  } tuned[2][3][3][2][2];
};

namespace mcv {
namespace host {

constexpr int64_t kMaxNeutrons = (int64_t)1 << 40;

mcv_status fail(mcv_status st, const std::string& msg);
mcv_status cuda_fail(cudaError_t e, const char* where);
// An NVTX range around one call of the C ABI, named after the call: a profiler's timeline
// shows the library's calls around their kernels (with no tool attached, a push and a pop
// cost a few nanoseconds).
struct CallRange {
  explicit CallRange(const char* name) { nvtxRangePushA(name); }
  ~CallRange() { nvtxRangePop(); }
  CallRange(const CallRange&) = delete;
  CallRange& operator=(const CallRange&) = delete;
};

// A device allocation that failed: MCV_ENOMEM, with CUDA's record of the failure cleared
// (cudaGetLastError), so that the next launch on this thread does not report it again.
mcv_status alloc_fail(const std::string& msg);
bool is_finite(double v);
mcv_status check_ctx(mcv_ctx* ctx);
int ns_index(int ns);

mcv_status build_beam(const mcv_beam_params* b, BeamP<double>* B);
mcv_status build_sample(const mcv_sample* s, SampleP<double>* S);
mcv_status build_detector(const mcv_detector* d, DetP<double>* D);
TofWin tof_window(double tof_min_s, double tof_max_s, int n_tof);
PhiloxKeys philox_keys(uint32_t seed, uint32_t sim_id);
void set_miss_bounds(const SampleP<double>& S, BeamP<double>* B);
double sample_radius(const SampleP<double>& S);
void set_det_miss_bounds(double r_s, DetP<double>* D);
void cast_beam(const BeamP<double>& d, BeamP<float>* f);
void cast_sample(const SampleP<double>& d, SampleP<float>* f);
void cast_detector(const DetP<double>& d, DetP<float>* f);
void cast_all(TraceArgs* A);
// the device sink of an event list (checks its arrays); tag: the simulation's sim_id
mcv_status event_sink(const mcv_event_list* l, uint32_t tag, EvSink* out);

}  // namespace host

// mcv_sync without a context: waits for `stream`, then reports and clears the device error
// word of mcv_grad_noalloc on the current device (mcv_noalloc.cu)
mcv_status noalloc_sync(cudaStream_t stream);

}  // namespace mcv
