// Reverse mode of n_iter unrolled iterations of Algorithm 1 (tied penalty
// rho_P = rho_T = rho_V = rho_S = rho): given dL/dX_K for X_K, the X of the
// last step I, returns dL/dy, dL/dmu_s, dL/dmu_nu and dL/drho.
//
// The forward runs from the zero state and checkpoints, for every iteration k,
// X_k and the multipliers and S entering it; the reverse sweep recomputes the
// threshold and positivity decisions from them.  Per iteration (k = K..1):
//   Prox adjoint (k < K): spectral adjoint (steps II, IV, V and duals) and
//     wavelet adjoint (W_k X and W_k b_bar analysed, pointwise adjoint of
//     step III, synthesis of the cotangent of W_k X) give X_bar;
//   step I adjoint: X = Q^-1 (H^T y + b) gives b_bar = Q^-1 X_bar (Q is
//     symmetric), y_bar += H b_bar, rho_bar -= (2 + n_s) <b_bar, X>.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "mf_internal.cuh"
#include "reduce.cuh"

namespace mf {

template <class R>
cudaError_t launch_spectral_bwd(const R* X, const R* GP, const R* Sd, const R* GV, const R* GSd, const R* bb, R* GPc,
                                R* Sc, R* GVc, R* GSc, R* Xc, const R* dctC, int N, int L, R rho, R mu_nu,
                                double* partials, int* nblocks, cudaStream_t s);
template <class R>
cudaError_t launch_wav_analysis_full(const R* src, R* coef, R* tmp, int N, int L, int J, int nd, const int* Ks,
                                     cudaStream_t s);
template <class R>
cudaError_t launch_wav_synthesis_acc(R* coef, R* out, R* tmp, int N, int L, int J, int nd, const int* Ks,
                                     cudaStream_t s);
template <class R>
cudaError_t launch_wav_bwd_point(R* zc, const R* uc, const R* gam_old, R* gc, size_t per_basis, int nd,
                                 const WavSet<R>* ws, R rho, R mu_s, double* partials, int* nblocks,
                                 cudaStream_t s);

namespace {

constexpr int BNT = 256;

__global__ void k_axpy(float* __restrict__ y, const float* __restrict__ x, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] += x[i];
}

// partial rows of scale * <a, b> in slot 2 (d rho)
__global__ void k_dot(const float* __restrict__ a, const float* __restrict__ b, size_t n, double scale,
                      double* __restrict__ partials) {
  double acc = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    acc += (double)a[i] * (double)b[i];
  double q[Q_COUNT];
#pragma unroll
  for (int i = 0; i < Q_COUNT; i++) q[i] = 0.0;
  q[Q_XMIN] = 1e300;
  q[2] = scale * acc;
  block_reduce_write<BNT>(q, partials + (size_t)blockIdx.x * MF_NQ);
}

unsigned grid_for(size_t n) {
  size_t b = (n + BNT - 1) / BNT;
  return (unsigned)(b < 152 * 16 ? (b ? b : 1) : 152 * 16);
}

}  // namespace

// Applies Q^-1 (mode 4) or H (mode 3) to src, result in dst (uses the plan's work buffer).
static cudaError_t apply_filter(mf_plan* p, const float* src, float* dst, int mode, cudaStream_t s) {
  const int N = p->N, L = p->L;
  typedef cx<float> C;
  cudaError_t e = launch_rows_fwd<float>(src, (C*)p->work, N, N * L, (const C*)p->tw, s);
  if (!e)
    e = launch_cols<float>((C*)p->work, N, L, (const C*)p->tw, mode, nullptr, nullptr, nullptr, nullptr,
                           (const float*)p->gg, (const float*)p->gg_nyq, (const C*)p->hhat, (const C*)p->hhat_nyq,
                           nullptr, nullptr, nullptr, s);
  if (!e) e = launch_rows_inv<float>((const C*)p->work, dst, N, N * L, (const C*)p->tw, s);
  return e;
}

}  // namespace mf

using namespace mf;

// Forward pieces of plan.cu reused here.
mf_status mf_internal_prepare_f32(mf_plan* p, const float* y, const mf_params* prm, int n_iter, cudaStream_t s,
                                  WavSet<float>* ws, IterScalars<float>* sc);
cudaError_t mf_internal_iteration_f32(mf_plan* p, const mf_params* prm, const WavSet<float>& ws,
                                      const IterScalars<float>& sc, cudaStream_t s);
void mf_internal_finish(mf_plan* p, const mf_params* prm, int n_iter);

extern "C" mf_status mf_admm_backward(mf_plan* p, const float* y, const mf_params* prm, int n_iter,
                                      const float* dL_dX, float* dL_dy, double* dL_dmu_s, double* dL_dmu_nu,
                                      double* dL_drho) {
  if (!p || !prm || !y || !dL_dX || !dL_dy || n_iter < 1) return MF_ERR_INVALID;
  if (p->dbl || prm->precision != MF_FP32 || prm->warm_start) return MF_ERR_INVALID;
  if (!(prm->rho_P == prm->rho_T && prm->rho_P == prm->rho_V && prm->rho_P == prm->rho_S)) return MF_ERR_INVALID;
  if (p->L > 64 || p->linear || prm->spectral_mask != 1) return MF_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)prm->stream;
  WavSet<float> ws;
  IterScalars<float> sc;
  mf_params fp = *prm;
  fp.resid_every = 0;
  mf_status st = mf_internal_prepare_f32(p, y, &fp, n_iter, s, &ws, &sc);
  if (st != MF_OK) return st;
  const int N = p->N, L = p->L, nd = ws.nd, J = prm->wavelet_levels;
  const size_t V = p->cube, cb = V * sizeof(float);
  int n_s = 0;
  for (int bit = 0; bit < 9; bit++) n_s += (prm->wavelet_mask >> bit) & 1u;
  const float rho = (float)prm->rho_P;

  // checkpoints: per iteration X_k and the multipliers / S entering it
  const size_t per_ck = (size_t)(5 + nd);  // X, GP, Sd, GV, GSd, GT[nd]
  // cotangents and scratch: Xbar, bbar, ybar, GPc, Sc, GVc, GSc, tmp[nd] (the wavelet
  // transforms of all bases at once; its first cube also serves the filters), GTc[nd],
  // coefZ[nd], coefU[nd]
  const size_t nwork = 7 + 4 * (size_t)nd;
  const size_t need = cb * (per_ck * n_iter + nwork);
  if (need > p->bwd_bytes) {
    // the plan keeps this memory for later calls; it grows it when a call needs more
    if (p->bwd_buf) {
      cudaError_t fe = cudaStreamSynchronize(s);
      if (fe == cudaSuccess) fe = cudaFree(p->bwd_buf);
      p->bwd_buf = nullptr;
      p->bwd_bytes = 0;
      if (fe != cudaSuccess) {
        cudaGetLastError();
        p->status = MF_ERR_CUDA;
        return MF_ERR_CUDA;
      }
    }
    if (cudaMalloc(&p->bwd_buf, need) != cudaSuccess) {
      cudaGetLastError();
      p->bwd_buf = nullptr;
      return MF_ERR_OOM;
    }
    p->bwd_bytes = need;
  }
  float* ckp = (float*)p->bwd_buf;
  float* W = ckp + per_ck * n_iter * V;
  float *Xbar = W, *bbar = W + V, *ybar = W + 2 * V;
  float *GPc = W + 3 * V, *Sc = W + 4 * V, *GVc = W + 5 * V, *GSc = W + 6 * V;
  float* tmp = W + 7 * V;
  float* GTc = tmp + nd * V;
  float* coefZ = GTc + nd * V;
  float* coefU = coefZ + nd * V;
  auto slot = [&](int k, int which) { return ckp + ((size_t)k * per_ck + which) * V; };

  cudaError_t e = cudaSuccess;
  // forward with checkpoints (iteration k = 0..n_iter-1 checkpoints X_{k+1} and its input state)
  for (int k = 0; k < n_iter && !e; k++) {
    const float* gt = (const float*)p->GT[p->gt_cur];
    e = cudaMemcpyAsync(slot(k, 1), p->GP, cb, cudaMemcpyDeviceToDevice, s);
    if (!e) e = cudaMemcpyAsync(slot(k, 2), p->Sd, cb, cudaMemcpyDeviceToDevice, s);
    if (!e) e = cudaMemcpyAsync(slot(k, 3), p->GV, cb, cudaMemcpyDeviceToDevice, s);
    if (!e) e = cudaMemcpyAsync(slot(k, 4), p->GSd, cb, cudaMemcpyDeviceToDevice, s);
    if (!e) e = cudaMemcpyAsync(slot(k, 5), gt, cb * nd, cudaMemcpyDeviceToDevice, s);
    if (!e) e = mf_internal_iteration_f32(p, &fp, ws, sc, s);
    if (!e) e = cudaMemcpyAsync(slot(k, 0), p->X, cb, cudaMemcpyDeviceToDevice, s);
  }
  mf_internal_finish(p, &fp, n_iter);

  // reverse sweep
  double* gsum = p->sums;  // [0] d mu_s, [1] d mu_nu, [2] d rho (accumulated by the finalize kernel)
  if (!e) e = cudaMemsetAsync(gsum, 0, MF_NQ * sizeof(double), s);
  if (!e) e = cudaMemcpyAsync(Xbar, dL_dX, cb, cudaMemcpyDeviceToDevice, s);
  if (!e) e = cudaMemsetAsync(ybar, 0, cb, s);
  if (!e) e = cudaMemsetAsync(GPc, 0, cb * 4, s);
  if (!e) e = cudaMemsetAsync(GTc, 0, cb * nd, s);
  int Ks[MF_MAX_BASES];
  for (int i = 0; i < nd; i++) Ks[i] = ws.K[i];
  for (int k = n_iter - 1; k >= 0 && !e; k--) {
    const float* Xk = slot(k, 0);
    if (k < n_iter - 1) {
      int nb = 0;
      e = launch_spectral_bwd<float>(Xk, slot(k, 1), slot(k, 2), slot(k, 3), slot(k, 4), bbar, GPc, Sc, GVc, GSc,
                                     Xbar, (const float*)p->dctC, N, L, rho, (float)prm->mu_nu, p->partials, &nb, s);
      if (!e) e = launch_finalize(p->partials, nb, gsum, 1, s);
      if (!e) e = launch_wav_analysis_full<float>(Xk, coefZ, tmp, N, L, J, nd, Ks, s);
      if (!e) e = launch_wav_analysis_full<float>(bbar, coefU, tmp, N, L, J, nd, Ks, s);
      if (!e)
        e = launch_wav_bwd_point<float>(coefZ, coefU, slot(k, 5), GTc, V, nd, (const WavSet<float>*)p->wset, rho,
                                        (float)prm->mu_s, p->partials, &nb, s);
      if (!e) e = launch_finalize(p->partials, nb, gsum, 1, s);
      if (!e) e = launch_wav_synthesis_acc<float>(coefZ, Xbar, tmp, N, L, J, nd, Ks, s);
    }
    // step I adjoint
    if (!e) e = apply_filter(p, Xbar, bbar, 4, s);
    if (!e) e = apply_filter(p, bbar, tmp, 3, s);
    if (!e) {
      k_axpy<<<grid_for(V), BNT, 0, s>>>(ybar, tmp, V);
      const unsigned g = grid_for(V);
      k_dot<<<g, BNT, 0, s>>>(bbar, Xk, V, -(2.0 + n_s) , p->partials);
      e = cudaGetLastError();
      if (!e) e = launch_finalize(p->partials, (int)g, gsum, 1, s);
    }
  }
  if (!e) e = cudaMemcpyAsync(dL_dy, ybar, cb, cudaMemcpyDeviceToDevice, s);
  double g[MF_NQ];
  if (!e) e = cudaMemcpyAsync(g, gsum, sizeof(g), cudaMemcpyDeviceToHost, s);
  if (!e) e = cudaStreamSynchronize(s);
  if (e) {
    cudaGetLastError();
    p->status = MF_ERR_CUDA;
    return MF_ERR_CUDA;
  }
  p->report_pending = 0;
  if (dL_dmu_s) *dL_dmu_s = g[0];
  if (dL_dmu_nu) *dL_dmu_nu = g[1];
  if (dL_drho) *dL_drho = g[2];
  return MF_OK;
}
