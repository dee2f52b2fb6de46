// Tables of the coherent elastic powder kernel (host code): the reflections sorted by
// decreasing lattice spacing (ties in input order), so that the reflections a wavelength can
// excite (lambda < 2 d) form a prefix of the list.  A reflection's cross section at
// wavelength lambda, lambda^3 w / (4 sin theta_B) with sin theta_B = lambda / 2d, is
// lambda^2 w d / 2: the table holds the prefix sums of w d, so that the sum over the allowed
// reflections and the choice among them need no per-reflection arithmetic.
// Device layout (mcv_bragg::tables): d[n], C[n] (C[r] = sum of w d over reflections 0..r) as
// doubles (FP64 kernels), then d[n], C[n] as floats (FP32 kernels).
#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include <cuda_runtime.h>

#include "mcv_host.h"

namespace {
constexpr int kMaxReflections = 1 << 16;
}

extern "C" {

int64_t mcv_bragg_table_bytes(int n) {
  if (n < 1 || n > kMaxReflections) return 0;
  return (int64_t)n * 2 * (int64_t)(sizeof(double) + sizeof(float));
}

mcv_status mcv_bragg_build(const double* d_A, const double* w, int n, mcv_bragg* out,
                           void* tables, int64_t bytes, void* stream) {
  mcv::host::CallRange range_("mcv_bragg_build");
  using mcv::host::fail;
  using mcv::host::is_finite;
  if (!d_A || !w || !out || !tables) return fail(MCV_EINVAL, "mcv_bragg_build needs d_A, w, out, tables");
  const int64_t need = mcv_bragg_table_bytes(n);
  if (need == 0) return fail(MCV_EINVAL, "n must be 1..65536");
  if (bytes < need) return fail(MCV_EINVAL, "the table buffer is too small");
  for (int i = 0; i < n; ++i) {
    if (!(d_A[i] > 0) || !is_finite(d_A[i])) return fail(MCV_EINVAL, "spacings must be finite and > 0");
    if (!(w[i] >= 0) || !is_finite(w[i])) return fail(MCV_EINVAL, "strengths must be finite and >= 0");
  }
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return d_A[a] > d_A[b]; });
  std::vector<unsigned char> buf((size_t)need);
  double* dd = reinterpret_cast<double*>(buf.data());
  double* dc = dd + n;
  float* fd = reinterpret_cast<float*>(dc + n);
  float* fc = fd + n;
  double sum = 0.0;
  for (int r = 0; r < n; ++r) {
    dd[r] = d_A[order[r]];
    sum += w[order[r]] * dd[r];
    dc[r] = sum;
    fd[r] = (float)dd[r];
    fc[r] = (float)dc[r];
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(tables, buf.data(), (size_t)need, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return mcv::host::cuda_fail(e, "cudaMemcpyAsync");
  e = cudaStreamSynchronize(s);  // `buf` must outlive the copy
  if (e != cudaSuccess) return mcv::host::cuda_fail(e, "cudaStreamSynchronize");
  out->tables = tables;
  out->n = n;
  return MCV_OK;
}

}  // extern "C"
