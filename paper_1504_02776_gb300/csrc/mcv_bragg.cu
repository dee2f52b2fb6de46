// Tables of the coherent elastic powder kernel (host code): the reflections sorted by
// decreasing lattice spacing (ties in input order), so that the reflections a wavelength can
// excite (lambda < 2 d) form a prefix of the list.
// Device layout (mcv_bragg::tables): d[n], w[n] as doubles (FP64 kernels), then d[n], w[n]
// as floats (FP32 kernels).
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
  double* dw = dd + n;
  float* fd = reinterpret_cast<float*>(dw + n);
  float* fw = fd + n;
  for (int r = 0; r < n; ++r) {
    dd[r] = d_A[order[r]];
    dw[r] = w[order[r]];
    fd[r] = (float)dd[r];
    fw[r] = (float)dw[r];
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
