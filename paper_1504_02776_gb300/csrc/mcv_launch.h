// Host-side entry points of the kernels (mcv_fp32.cu, mcv_fp64.cu, mcv_batch_fp32.cu,
// mcv_batch_fp64.cu, mcv_misc.cu), used by the C ABI.
#pragma once

#include <string>

#include <cuda_runtime.h>

#include "mcv_params.h"

namespace mcv {

struct EventsArgs {
  int32_t* pixel;
  double* tof;
  double* w_det;
  int64_t* bin;
};

int trace_threads();
cudaError_t trace_blocks_per_sm(int fp_mode, int ns, int det, int bvk, int* blocks);
cudaError_t launch_trace(const TraceArgs& A, int fp_mode, int det, int grid, cudaStream_t s);
cudaError_t launch_beam(const TraceArgs& A, int fp_mode, int grid, cudaStream_t s);
cudaError_t launch_detect(const TraceArgs& A, const EventsArgs& E, int fp_mode, int det, int grid,
                          cudaStream_t s);
cudaError_t launch_zero(double* p, int64_t n, int grid, cudaStream_t s);
// chi-squared loss into *loss (accumulated); g (optional) receives dchi2/dI per bin; err
// (optional) is set when a target bin is negative or not finite
cudaError_t launch_chi2(const double* hist, const double* target, double c, int64_t nb,
                        double* g, double* loss, int* err, int grid, cudaStream_t s);
cudaError_t launch_adjoint(const TraceArgs& A, int fp_mode, int det, int grid, cudaStream_t s);
// the paper's recursive estimator (one neutron per thread, grid-stride)
cudaError_t launch_paper(const TraceArgs& A, int fp_mode, int det, int grid, cudaStream_t s);
cudaError_t adjoint_blocks_per_sm(int fp_mode, int ns, int det, int bvk, int* blocks);
// batched launch: blocks per SM of its kernel (also sets the kernel's shared-memory limit;
// call before the first launch of a shape), and the launch itself.  ss: every simulation
// has the sample in A (kept in kernel parameter space).
// ev: some simulation appends to an event list (the kernels that can)
cudaError_t batch_blocks_per_sm(int fp_mode, int ns, int det, int bvk, int ss, int ev,
                                int* blocks);
cudaError_t launch_batch(const TraceArgs& A, const BatchArgs& Q, int fp_mode, int ns, int det,
                         int bvk, int ss, int ev, int grid, cudaStream_t s);
// random FP64 atomic adds (mcv_bench_atomics)
cudaError_t launch_atomics(double* hist, int64_t nb, int64_t n_adds, uint64_t seed, int grid,
                           cudaStream_t s);
// sets the message mcv_last_error() returns to the calling thread
void set_last_error(const std::string& msg);

}  // namespace mcv
