// Spectral-index map of a cube: the post-processing of the paper's first
// simulation (Section 4), where every pixel spectrum S(nu_l) is fitted, in a
// log scale, by the second-order power law
//   log S(nu) = c + alpha u + beta u^2,   u = log(nu / nu0),
// by least squares over the bands.  The design matrix A = [1, u_l, u_l^2] is
// the same for every pixel, so its pseudo-inverse P = (A^T A)^-1 A^T (3 x L,
// formed on the host in long double) turns each fit into three dot products
// with the log spectrum.  A pixel with any S(nu_l) <= floor has no log-scale
// fit: its three outputs are NaN.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "mf_internal.cuh"

namespace mf {
namespace {

struct Pinv {
  float p[3][MF_MAX_L];
};

__global__ void k_spectral_index(const float* __restrict__ cube, int NN, int L, Pinv P, float floor,
                                 float* __restrict__ c0, float* __restrict__ alpha, float* __restrict__ beta) {
  for (int px = blockIdx.x * blockDim.x + threadIdx.x; px < NN; px += gridDim.x * blockDim.x) {
    float a0 = 0.f, a1 = 0.f, a2 = 0.f;
    bool ok = true;
    for (int l = 0; l < L; l++) {
      const float v = cube[(size_t)l * NN + px];
      ok = ok && v > floor;
      const float lv = logf(v > 0.f ? v : 1.f);
      a0 = fmaf(P.p[0][l], lv, a0);
      a1 = fmaf(P.p[1][l], lv, a1);
      a2 = fmaf(P.p[2][l], lv, a2);
    }
    const float nan = __int_as_float(0x7fc00000);
    if (c0) c0[px] = ok ? a0 : nan;
    if (alpha) alpha[px] = ok ? a1 : nan;
    if (beta) beta[px] = ok ? a2 : nan;
  }
}

// P = (A^T A)^-1 A^T for A = [1, u, u^2]; false when A^T A is singular.
bool pseudo_inverse(const double* nu, int L, double nu0, Pinv* out) {
  long double G[3][3] = {}, u[MF_MAX_L];
  for (int l = 0; l < L; l++) {
    u[l] = std::log((long double)nu[l] / (long double)nu0);
    const long double a[3] = {1.0L, u[l], u[l] * u[l]};
    for (int i = 0; i < 3; i++)
      for (int j = 0; j < 3; j++) G[i][j] += a[i] * a[j];
  }
  // inverse of the symmetric 3 x 3 Gram matrix by cofactors
  long double C[3][3];
  C[0][0] = G[1][1] * G[2][2] - G[1][2] * G[2][1];
  C[0][1] = G[0][2] * G[2][1] - G[0][1] * G[2][2];
  C[0][2] = G[0][1] * G[1][2] - G[0][2] * G[1][1];
  C[1][0] = G[1][2] * G[2][0] - G[1][0] * G[2][2];
  C[1][1] = G[0][0] * G[2][2] - G[0][2] * G[2][0];
  C[1][2] = G[0][2] * G[1][0] - G[0][0] * G[1][2];
  C[2][0] = G[1][0] * G[2][1] - G[1][1] * G[2][0];
  C[2][1] = G[0][1] * G[2][0] - G[0][0] * G[2][1];
  C[2][2] = G[0][0] * G[1][1] - G[0][1] * G[1][0];
  const long double det = G[0][0] * C[0][0] + G[0][1] * C[1][0] + G[0][2] * C[2][0];
  long double scale = 0;
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) scale = std::fmax(scale, std::fabs(G[i][j]));
  if (!(std::fabs(det) > 1e-14L * scale * scale * scale)) return false;
  std::memset(out, 0, sizeof(*out));
  for (int l = 0; l < L; l++) {
    const long double a[3] = {1.0L, u[l], u[l] * u[l]};
    for (int i = 0; i < 3; i++) {
      long double s = 0;
      for (int j = 0; j < 3; j++) s += C[i][j] * a[j];
      out->p[i][l] = (float)(s / det);
    }
  }
  return true;
}

}  // namespace
}  // namespace mf

extern "C" mf_status mf_spectral_index(int N, int L, const float* cube, const double* nu, double nu0, float floor,
                                       float* c0_out, float* alpha_out, float* beta_out, void* stream) {
  if (!cube || !nu || N < 1 || N > 16384 || L < 3 || L > MF_MAX_L || !(nu0 > 0) || !std::isfinite(floor)) return MF_ERR_INVALID;
  if (!c0_out && !alpha_out && !beta_out) return MF_ERR_INVALID;
  for (int l = 0; l < L; l++)
    if (!(nu[l] > 0) || !std::isfinite(nu[l])) return MF_ERR_INVALID;
  mf::Pinv P;
  if (!mf::pseudo_inverse(nu, L, nu0, &P)) return MF_ERR_INVALID;  // fewer than 3 distinct frequencies
  const int NN = N * N;
  const int blocks = (NN + 255) / 256 < 152 * 16 ? (NN + 255) / 256 : 152 * 16;
  mf::k_spectral_index<<<blocks, 256, 0, (cudaStream_t)stream>>>(cube, NN, L, P, floor, c0_out, alpha_out, beta_out);
  return cudaGetLastError() == cudaSuccess ? MF_OK : MF_ERR_CUDA;
}
