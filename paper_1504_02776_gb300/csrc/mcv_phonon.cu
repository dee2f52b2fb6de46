// Tables of the incoherent phonon kernel (host code): the phonon expansion of the incoherent
// scattering function of a harmonic cubic crystal from its density of states,
//   S(Q,E) = e^{-2W} [delta(E) + sum_{n=1}^{N} (2W)^n/n! A_n(E)],
//   A_1(E) = Z(|E|)/(|E| gamma_0) (n_B(|E|) + 1 for E > 0, n_B(|E|) for E < 0),
//   A_n = A_1 * A_{n-1},  gamma_0 = sum coth(E/2kT) Z(E)/E,  2W = hbar^2 Q^2 gamma_0 / 2M
// (the paper's supplement, "Scattering kernels used in the examples": its incoherent
// single-phonon and multi-phonon forms are the n = 1 and n >= 2 terms).  The density of
// states is a histogram of mode energies j de, so A_1 is a set of masses on the grid E = i de
// and each A_n an exact discrete convolution on it.
//
// Device layout (mcv_phonon::tables), T = (2J + 1) + M + M + (N - 1) M values with M = 2NJ + 1:
//   cumulative masses of A_1 over i = -J..J, cumulative masses of the multi-phonon sampling
//   mixture B = (A_2 + ... + A_N)/(N - 1) over i = -NJ..NJ, the masses of B, and A_n for
//   n = 2..N (row n - 2) -- first as T doubles (the FP64 kernels), then as T floats (FP32).
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "mcv_host.h"

namespace {

constexpr int kMaxOrder = 16;
constexpr int kMaxModes = 1 << 16;

int64_t table_count(int J, int N) {
  const int64_t M = 2 * (int64_t)N * J + 1;
  return (2 * (int64_t)J + 1) + 2 * M + (int64_t)(N - 1) * M;
}

}  // namespace

extern "C" {

int64_t mcv_phonon_table_bytes(int n_modes, int n_max) {
  if (n_modes < 1 || n_modes > kMaxModes || n_max < 2 || n_max > kMaxOrder) return 0;
  return table_count(n_modes, n_max) * (int64_t)(sizeof(double) + sizeof(float));
}

mcv_status mcv_phonon_build(const double* dos_z, mcv_phonon* ph, void* tables, int64_t bytes,
                            void* stream) {
  mcv::host::CallRange range_("mcv_phonon_build");
  using mcv::host::fail;
  using mcv::host::is_finite;
  if (!dos_z || !ph || !tables) return fail(MCV_EINVAL, "mcv_phonon_build needs dos_z, ph, tables");
  const int J = ph->n_modes, N = ph->n_max;
  const int64_t need = mcv_phonon_table_bytes(J, N);
  if (need == 0) return fail(MCV_EINVAL, "n_modes must be 1..65536 and n_max 2..16");
  if (bytes < need) return fail(MCV_EINVAL, "the table buffer is too small");
  if (!(ph->de_mev > 0) || !is_finite(ph->de_mev) || !(ph->mass_u > 0) ||
      !is_finite(ph->mass_u) || !(ph->temperature_K > 0) || !is_finite(ph->temperature_K))
    return fail(MCV_EINVAL, "bad phonon energy step, mass or temperature");
  double psum = 0.0;
  for (int c = 0; c < 3; ++c) {
    if (!(ph->p[c] > 0) || !is_finite(ph->p[c]))
      return fail(MCV_EINVAL, "channel probabilities must be positive");
    psum += ph->p[c];
  }
  if (std::fabs(psum - 1.0) > 1e-12) return fail(MCV_EINVAL, "channel probabilities must sum to 1");
  double zsum = 0.0;
  for (int j = 0; j < J; ++j) {
    if (!(dos_z[j] >= 0) || !is_finite(dos_z[j]))
      return fail(MCV_EINVAL, "density of states values must be finite and >= 0");
    zsum += dos_z[j];
  }
  if (!(zsum > 0)) return fail(MCV_EINVAL, "the density of states is empty");
  const double kBoltzmann = 1.380649e-23, kAtomicMass = 1.66053906660e-27;
  const double mev_per_j = 1.0 / (mcv::kElemCharge * 1e-3);
  const double kT = kBoltzmann * ph->temperature_K * mev_per_j;
  const double de = ph->de_mev;
  // gamma_0 and the Debye-Waller coefficient c_w (2W = c_w Q^2)
  double gamma0 = 0.0;
  for (int j = 1; j <= J; ++j) {
    const double e = j * de;
    gamma0 += (dos_z[j - 1] / zsum) / (e * std::tanh(e / (2.0 * kT)));
  }
  const double hb2m = mcv::kHbar * mcv::kHbar / (2.0 * ph->mass_u * kAtomicMass) * 1e20 * mev_per_j;
  // A_1 masses on i = -J..J, then A_n = A_1 * A_{n-1} on i = -NJ..NJ
  const int M = 2 * N * J + 1;
  std::vector<double> a1(2 * J + 1, 0.0);
  for (int j = 1; j <= J; ++j) {
    const double e = j * de, w = dos_z[j - 1] / zsum;
    const double nb = 1.0 / std::expm1(e / kT);
    a1[J + j] = w * (nb + 1.0) / (e * gamma0);
    a1[J - j] = w * nb / (e * gamma0);
  }
  std::vector<double> prev(M, 0.0), cur(M, 0.0);
  for (int i = -J; i <= J; ++i) prev[i + N * J] = a1[i + J];
  std::vector<double> an((size_t)(N - 1) * M, 0.0);
  for (int n = 2; n <= N; ++n) {
    for (int i = -n * J; i <= n * J; ++i) {
      double v = 0.0;
      for (int k = -J; k <= J; ++k) {
        const int r = i - k;
        if (r < -(n - 1) * J || r > (n - 1) * J) continue;
        v += a1[k + J] * prev[r + N * J];
      }
      cur[i + N * J] = v;
    }
    std::memcpy(&an[(size_t)(n - 2) * M], cur.data(), sizeof(double) * M);
    prev.swap(cur);
    std::fill(cur.begin(), cur.end(), 0.0);
  }
  // the device tables: cumulative masses of A_1, of B, the masses of B, and A_2..A_N
  const int64_t T = table_count(J, N);
  std::vector<double> t((size_t)T, 0.0);
  double* cdf1 = t.data();
  double* cdfb = cdf1 + (2 * J + 1);
  double* b = cdfb + M;
  double* a = b + M;
  double acc = 0.0;
  for (int i = 0; i < 2 * J + 1; ++i) cdf1[i] = (acc += a1[i]);
  acc = 0.0;
  for (int i = 0; i < M; ++i) {
    double v = 0.0;
    for (int n = 2; n <= N; ++n) v += an[(size_t)(n - 2) * M + i] / (N - 1);
    b[i] = v;
    cdfb[i] = (acc += v);
  }
  std::memcpy(a, an.data(), sizeof(double) * an.size());
  std::vector<unsigned char> buf((size_t)need);
  std::memcpy(buf.data(), t.data(), sizeof(double) * T);
  float* tf = reinterpret_cast<float*>(buf.data() + sizeof(double) * T);
  for (int64_t i = 0; i < T; ++i) tf[i] = (float)t[i];
  cudaError_t e = cudaMemcpyAsync(tables, buf.data(), (size_t)need, cudaMemcpyHostToDevice,
                                  static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return mcv::host::cuda_fail(e, "cudaMemcpyAsync");
  // the pageable source is staged before cudaMemcpyAsync returns; wait all the same, so
  // that `buf` outlives the copy whatever the driver does
  e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return mcv::host::cuda_fail(e, "cudaStreamSynchronize");
  ph->gamma0 = gamma0;
  ph->c_w = hb2m * gamma0;
  ph->tables = tables;
  return MCV_OK;
}

}  // extern "C"
