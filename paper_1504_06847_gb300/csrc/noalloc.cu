// mf_xstep_noalloc: the step I solve with every intermediate in one static
// device array, for callers that cannot allocate device memory (see mf.h).
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "mf_internal.cuh"

using namespace mf;

namespace {

// Layout for V = N * N * L <= MF_XSTEP_NOALLOC_MAX_VOXELS voxels (floats):
//   work  V      packed half spectrum (V/2 complex)
//   hhat  V      transfer function, unpacked half spectrum
//   yhat  V      F(y)
//   cc    V      conj(hhat) yhat g
//   gg    V/2    g
//   nyq   7 L N  the kx = N/2 columns of hhat, yhat, cc (complex) and g (real)
//   tw    2 N    twiddles exp(-2 pi i k / N)
// With N >= 16, L N = V / N <= kMaxV / 16, and N <= 512 (L >= 2).
constexpr size_t kMaxV = MF_XSTEP_NOALLOC_MAX_VOXELS;
constexpr size_t kMaxNyq = 7 * (kMaxV / 16);
constexpr size_t kMaxN = 2048;
constexpr size_t kScratchFloats = 4 * kMaxV + kMaxV / 2 + kMaxNyq + 2 * kMaxN;  // 2,592,768 floats, 10.4 MB

__device__ __align__(256) float g_xstep_scratch[kScratchFloats];

constexpr int kMaxDevices = 64;
float* g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mutex;

// Device address of the static array on the current device, looked up by the
// first call on that device (with the device current) and kept for later
// calls.  A cudaDeviceReset of that device unloads the module and leaves the
// kept address stale; mf.h states that the entry point is not for use after one.
cudaError_t scratch_for_current_device(float** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_xstep_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<float*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

// tw[k] = exp(-2 pi i k / N): the angle's cosine and sine in FP64, rounded
// once to FP32 (the plans build the same table on the host).
__global__ void k_twiddles(cx<float>* tw, int N) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
    double sn, cs;
    sincospi(-2.0 * (double)k / (double)N, &sn, &cs);
    tw[k].x = (float)cs;
    tw[k].y = (float)sn;
  }
}

}  // namespace

extern "C" mf_status mf_xstep_noalloc(int N, int L, const float* psf, const float* y, const float* b,
                                      const mf_params* prm, float* x_out) {
  if (!psf || !y || !b || !prm || !x_out) return MF_ERR_INVALID;
  if (!pow2(N) || N < 16 || N > 2048 || L < 2 || L > MF_MAX_L) return MF_ERR_INVALID;
  if (!(prm->rho_P > 0 && prm->rho_T > 0 && prm->rho_S > 0 && prm->mu_eps >= 0)) return MF_ERR_INVALID;
  if (prm->wavelet_mask == 0 || (prm->wavelet_mask >> 9) != 0) return MF_ERR_INVALID;
  const size_t V = (size_t)N * N * L;
  if (V > kMaxV) return MF_ERR_TOO_LARGE;
  int n_s = 0;
  for (int bit = 0; bit < 9; bit++) n_s += (prm->wavelet_mask >> bit) & 1u;
  const double rho_bar = prm->mu_eps + prm->rho_S + prm->rho_P + n_s * prm->rho_T;  // Eq. Qlsimp

  float* base = nullptr;
  if (scratch_for_current_device(&base) != cudaSuccess) return MF_ERR_CUDA;
  typedef cx<float> C;
  const size_t nq = (size_t)L * N;  // complex entries of one kx = N/2 column set
  C* work = reinterpret_cast<C*>(base);
  C* hhat = reinterpret_cast<C*>(base + V);
  C* yhat = reinterpret_cast<C*>(base + 2 * V);
  C* cc = reinterpret_cast<C*>(base + 3 * V);
  float* gg = base + 4 * V;
  float* nyq = base + 4 * V + V / 2;
  C* hhat_nyq = reinterpret_cast<C*>(nyq);
  C* yhat_nyq = hhat_nyq + nq;
  C* cc_nyq = yhat_nyq + nq;
  float* gg_nyq = reinterpret_cast<float*>(cc_nyq + nq);
  C* tw = reinterpret_cast<C*>(base + 4 * V + V / 2 + kMaxNyq);

  cudaStream_t s = (cudaStream_t)prm->stream;
  k_twiddles<<<(N + 255) / 256, 256, 0, s>>>(tw, N);
  cudaError_t e = cudaGetLastError();
  // transfer function: F(ifftshift(psf)); the shifted PSF (V floats) waits in
  // the cc region, which is free until the constants are formed, so that x_out
  // is written by the last pass only (x_out may alias psf, y or b)
  float* shifted = reinterpret_cast<float*>(cc);
  if (!e) e = launch_shift_psf<float>(psf, shifted, N, V, s);
  if (!e) e = launch_rows_fwd<float>(shifted, work, N, N * L, tw, s);
  if (!e)
    e = launch_cols<float>(work, N, L, tw, 0, hhat, hhat_nyq, nullptr, nullptr, nullptr, nullptr, nullptr,
                           nullptr, nullptr, nullptr, nullptr, s);
  // F(y), then g and c
  if (!e) e = launch_rows_fwd<float>(y, work, N, N * L, tw, s);
  if (!e)
    e = launch_cols<float>(work, N, L, tw, 0, yhat, yhat_nyq, nullptr, nullptr, nullptr, nullptr, nullptr,
                           nullptr, nullptr, nullptr, nullptr, s);
  if (!e) e = launch_constants<float>(hhat, hhat_nyq, yhat, yhat_nyq, cc, cc_nyq, gg, gg_nyq, N, L, rho_bar, s);
  // x = F^-1(c + g F(b))
  if (!e) e = launch_rows_fwd<float>(b, work, N, N * L, tw, s);
  if (!e)
    e = launch_cols<float>(work, N, L, tw, 1, nullptr, nullptr, cc, cc_nyq, gg, gg_nyq, nullptr, nullptr,
                           nullptr, nullptr, nullptr, s);
  if (!e) e = launch_rows_inv<float>(work, x_out, N, N * L, tw, s);
  return e ? MF_ERR_CUDA : MF_OK;
}
