// C ABI of the library (include/mf.h): plans, the ADMM iteration of
// Algorithm 1 as a fixed launch sequence on one stream, state access and the
// FP64 residual report.
//
// One iteration (J wavelet levels, nd distinct bases):
//   rows_fwd(b) -> cols(divide) -> rows_inv -> X                 step I
//   spectral(X, Gamma_P, S, Gamma_V, Gamma_S) -> b               steps II, IV, V, VI
//   wav_ll(j), j = 1..J-1; wav_level(j), j = J..1 -> b += ...    steps III, VI
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <atomic>
#include <cstring>
#include <new>
#include <vector>

#include "mf_internal.cuh"

using namespace mf;

namespace {

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

// Brackets one launch with events when timing is on; counts launches always.
struct Timed {
  mf_plan* p;
  int kid;
  cudaStream_t s;
  int n;
  Timed(mf_plan* p_, int kid_, cudaStream_t s_, int launches = 1) : p(p_), kid(kid_), s(s_), n(launches) {
    if (p->timing) record();
  }
  ~Timed() {
    if (p->timing) record();
    p->launches[kid] += n;
  }
  void record() {
    if (p->ev_used == p->ev_pool.size()) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        p->timing = 0;
        return;
      }
      p->ev_pool.push_back(e);
    }
    cudaEventRecord(p->ev_pool[p->ev_used], s);
    if ((p->ev_used & 1) == 0) p->ev_kernel.push_back(kid);
    p->ev_used++;
  }
};

void fold_timing(mf_plan* p) {
  for (size_t i = 0; i + 1 < p->ev_used; i += 2) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p->ev_pool[i], p->ev_pool[i + 1]) == cudaSuccess)
      p->kernel_ms[p->ev_kernel[i / 2]] += ms;
    else
      cudaGetLastError();
  }
  p->ev_used = 0;
  p->ev_kernel.clear();
}

template <class R>
__global__ void k_shift_psf(const R* __restrict__ psf, R* __restrict__ out, int N, size_t total) {
  // out[l][r][c] = psf[l][(r + N/2) mod N][(c + N/2) mod N]: the peak moves to (0, 0)
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t NN = (size_t)N * N;
    const size_t l = i / NN, rem = i % NN;
    const int r = (int)(rem / N), c = (int)(rem % N);
    out[i] = psf[l * NN + (size_t)((r + N / 2) & (N - 1)) * N + ((c + N / 2) & (N - 1))];
  }
}

struct Alloc {
  mf_plan* p;
  bool ok = true;
  void* get(size_t bytes) {
    if (!ok) return nullptr;
    void* d = nullptr;
    if (cudaMalloc(&d, bytes) != cudaSuccess) {
      ok = false;
      cudaGetLastError();
      return nullptr;
    }
    p->total_bytes += bytes;
    return d;
  }
};

void free_plan_memory(mf_plan* p) {
  void* ptrs[] = {p->X, p->b, p->GP, p->Sd, p->GV, p->GV2, p->Mb2, p->GSd, p->GT[0], p->GT[1], p->work, p->hhat,
                  p->hhat_nyq,
                  p->yhat, p->yhat_nyq, p->cc, p->cc_nyq, p->gg, p->gg_nyq, p->tw, p->dctC, p->scratch,
                  p->partials, p->sums, p->wset, p->dct_tc, p->err, p->bwd_buf, p->dual, p->h2, p->h2_nyq,
                  p->tw2, p->work2, p->big, p->cgv, p->cgs, p->cgpart, p->vis_uv, p->vis_w, p->vis_c0, p->S2,
                  p->vis_phihat, p->vis_twM, p->vis_spec, p->vis_nyq};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  p->bwd_buf = nullptr;
  p->bwd_bytes = 0;
  p->dual = nullptr;
  p->dual_bytes = 0;
  for (cudaEvent_t e : p->ev_pool) cudaEventDestroy(e);
  p->ev_pool.clear();
}

size_t scratch_elems(int N, int L) {
  // LL_j and R_j for j = 1..J-1 (J <= log2 N - 1), MF_MAX_BASES bases
  size_t s = 0;
  for (int M = N / 2; M >= 2; M /= 2) s += (size_t)M * M;
  return 2 * s * MF_MAX_BASES * L;
}

// no_psf: a plan whose step I does not use the circulant transfer function
// (the visibility operator): psf is not read and hhat is zero.
template <class R>
mf_status create(int N, int L, const R* psf, mf_plan** out, bool no_psf = false) {
  if (!out) return MF_ERR_INVALID;
  *out = nullptr;
  if ((!psf && !no_psf) || !is_pow2(N) || N < 16 || N > 2048 || L < 2 || L > MF_MAX_L) return MF_ERR_INVALID;
  if (sizeof(R) == 8 && L > 64) return MF_ERR_INVALID;
  mf_plan* p = new (std::nothrow) mf_plan();
  if (!p) return MF_ERR_OOM;
  static std::atomic<unsigned long long> next_serial{1};
  p->serial = next_serial++;
  p->N = N;
  p->L = L;
  p->dbl = sizeof(R) == 8;
  p->esz = sizeof(R);
  p->cube = (size_t)N * N * L;
  p->report.resid_iter = -1;
  // level tiles: 64 wide for FP32; 32 for FP64, whose 64-wide level kernels spill
  // registers (level 1 at 64 x 64 x 8: 0.54 ms against 0.21 ms per launch)
  p->wav_tile = sizeof(R) == 8 ? 32 : 64;
  const size_t cb = p->cube * sizeof(R);
  const size_t half = (size_t)L * N * (N / 2) * sizeof(cx<R>);
  const size_t nyq = (size_t)L * N * sizeof(cx<R>);
  Alloc a{p};
  p->X = a.get(cb);
  p->b = a.get(cb);
  p->GP = a.get(cb);
  p->Sd = a.get(cb);
  p->GV = a.get(cb);
  p->GSd = a.get(cb);
  p->GV2 = a.get(cb);
  p->Mb2 = a.get(sizeof(R) * L * L);
  p->GT[0] = a.get(cb * MF_MAX_BASES);
  p->GT[1] = a.get(cb * MF_MAX_BASES);
  p->work = a.get(half);
  p->hhat = a.get(half);
  p->hhat_nyq = a.get(nyq);
  p->yhat = a.get(half);
  p->yhat_nyq = a.get(nyq);
  p->cc = a.get(half);
  p->cc_nyq = a.get(nyq);
  p->gg = a.get(half / 2);
  p->gg_nyq = a.get(nyq / 2);
  p->tw = a.get(sizeof(cx<R>) * N);
  p->dctC = a.get(sizeof(R) * L * L);
  p->scratch_bytes = scratch_elems(N, L) * sizeof(R);
  p->scratch = a.get(p->scratch_bytes);
  // partial rows: the largest grid of any kernel that reduces
  size_t cap = (size_t)spectral_blocks<R>(N, L);
  for (int M = N; M >= 4; M /= 2) {
    for (int pref = 32; pref <= 64; pref *= 2) {
      const size_t nb = (size_t)wav_level_blocks<R>(M, L, M == N ? 1 : MF_MAX_BASES, pref);
      if (nb > cap) cap = nb;
    }
  }
  const size_t colblocks = (size_t)L * N;  // upper bound of the column kernel's grid
  if (colblocks > cap) cap = colblocks;
  if ((size_t)MF_AUX_GRID > cap) cap = MF_AUX_GRID;
  if ((size_t)MF_CG_CHUNKS * L > cap) cap = (size_t)MF_CG_CHUNKS * L;  // data-fit partials of a linear plan
  p->partial_cap = cap;
  p->partials = (double*)a.get(cap * MF_NQ * sizeof(double));
  p->sums = (double*)a.get(MF_NQ * sizeof(double));
  p->wset = a.get(sizeof(WavSet<R>));
  p->err = (int*)a.get(sizeof(int));
  if (sizeof(R) == 4 && spectral_tc_lp_of(L) > 0) p->dct_tc = a.get(spectral_tc_operand_elems(L) * sizeof(uint16_t));
  if (!a.ok) {
    free_plan_memory(p);
    delete p;
    return MF_ERR_OOM;
  }
  // host-built tables: twiddles and the DCT-II matrix
  {
    cx<R>* tw = new cx<R>[N];
    for (int k = 0; k < N; k++) {
      const double ang = -2.0 * M_PI * (double)k / (double)N;
      tw[k].x = (R)std::cos(ang);
      tw[k].y = (R)std::sin(ang);
    }
    R* C = new R[(size_t)L * L];
    for (int k = 0; k < L; k++) {
      const double ak = k == 0 ? std::sqrt(1.0 / L) : std::sqrt(2.0 / L);
      for (int l = 0; l < L; l++) C[k * L + l] = (R)(ak * std::cos(M_PI * (2.0 * l + 1.0) * k / (2.0 * L)));
    }
    // change of basis from the DCT domain (where S and Gamma_S live) to the
    // Chebyshev basis of the spectral dictionary: M = C2 C^T (offered for L <= 64)
    std::vector<double> C2((size_t)L * L);
    std::vector<R> Mh((size_t)L * L, (R)0);
    if (L <= 64) chebyshev_matrix(L, C2.data());
    for (int k2 = 0; k2 < L && L <= 64; k2++) {
      for (int k1 = 0; k1 < L; k1++) {
        const double ak = k1 == 0 ? std::sqrt(1.0 / L) : std::sqrt(2.0 / L);
        long double acc = 0;
        for (int l = 0; l < L; l++)
          acc += (long double)C2[(size_t)k2 * L + l] * (ak * std::cos(M_PI * (2.0 * l + 1.0) * k1 / (2.0 * L)));
        Mh[(size_t)k2 * L + k1] = (R)acc;
      }
    }
    cudaError_t e1 = cudaMemcpy(p->tw, tw, sizeof(cx<R>) * N, cudaMemcpyHostToDevice);
    if (e1 == cudaSuccess) e1 = cudaMemcpy(p->Mb2, Mh.data(), sizeof(R) * L * L, cudaMemcpyHostToDevice);
    cudaError_t e2 = cudaMemcpy(p->dctC, C, sizeof(R) * L * L, cudaMemcpyHostToDevice);
    cudaError_t e3 = upload_taps();
    if (e3 == cudaSuccess) e3 = cudaMemset(p->err, 0, sizeof(int));
    if (e3 == cudaSuccess && p->dct_tc) {
      std::vector<uint16_t> ops(spectral_tc_operand_elems(L));
      spectral_tc_build_operands(L, ops.data());
      e3 = cudaMemcpy(p->dct_tc, ops.data(), ops.size() * sizeof(uint16_t), cudaMemcpyHostToDevice);
    }
    delete[] tw;
    delete[] C;
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
      free_plan_memory(p);
      delete p;
      return MF_ERR_CUDA;
    }
  }
  // transfer function of every band: F(ifftshift(psf))
  cudaError_t e = cudaSuccess;
  if (no_psf) {
    e = cudaMemset(p->hhat, 0, half);
    if (e == cudaSuccess) e = cudaMemset(p->hhat_nyq, 0, nyq);
  } else {
    R* shifted = reinterpret_cast<R*>(p->X);
    k_shift_psf<R><<<1024, 256>>>(psf, shifted, N, p->cube);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = launch_rows_fwd<R>(shifted, (cx<R>*)p->work, N, N * L, (const cx<R>*)p->tw, 0);
    if (e == cudaSuccess)
      e = launch_cols<R>((cx<R>*)p->work, N, L, (const cx<R>*)p->tw, 0, (cx<R>*)p->hhat, (cx<R>*)p->hhat_nyq,
                         nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0);
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    free_plan_memory(p);
    delete p;
    return MF_ERR_CUDA;
  }
  *out = p;
  return MF_OK;
}

mf_status check_params(const mf_plan* p, const mf_params* prm, int n_iter, int want_dbl) {
  if (p && prm && p->linear && n_iter >= 1 && prm->cg_iters < 1) return MF_ERR_INVALID;
  if (!p || !prm || n_iter < 1) return MF_ERR_INVALID;
  if (p->dbl != want_dbl) return MF_ERR_INVALID;
  if (!(prm->rho_P > 0 && prm->rho_T > 0 && prm->rho_V > 0 && prm->rho_S > 0)) return MF_ERR_INVALID;
  if (!(prm->mu_eps >= 0 && prm->mu_s >= 0 && prm->mu_nu >= 0)) return MF_ERR_INVALID;
  if (!std::isfinite(prm->mu_eps + prm->mu_s + prm->mu_nu + prm->rho_P + prm->rho_T + prm->rho_V + prm->rho_S))
    return MF_ERR_INVALID;
  const int J = prm->wavelet_levels;
  if (J < 1 || (p->N >> J) < 2) return MF_ERR_INVALID;
  if (prm->wavelet_mask == 0 || (prm->wavelet_mask >> 9) != 0) return MF_ERR_INVALID;
  if (prm->resid_every < 0) return MF_ERR_INVALID;
  if (p->linear && prm->cg_iters < 1) return MF_ERR_INVALID;
  if (prm->spectral_mask < 1 || prm->spectral_mask > 3) return MF_ERR_INVALID;
  if ((prm->spectral_mask & 2) && (p->L > 64 || prm->precision == MF_FP32_DCT_SPLITBF16)) return MF_ERR_INVALID;
  if (p->dbl) {
    if (prm->precision != MF_FP64) return MF_ERR_INVALID;
  } else if (prm->precision == MF_FP32_DCT_SPLITBF16) {
    if (!p->dct_tc) return MF_ERR_INVALID;  // needs L <= 64
  } else if (prm->precision != MF_FP32) {
    return MF_ERR_INVALID;
  }
  return MF_OK;
}

// Distinct bases of the mask: Db1..Db8 in order, Haar folded into Db1 (weight 2)
// or, without Db1, its own K = 1 entry.
template <class R>
WavSet<R> make_wavset(unsigned mask, int* n_s) {
  WavSet<R> ws;
  std::memset(&ws, 0, sizeof(ws));
  int nd = 0, ns = 0;
  for (int K = 1; K <= MF_MAX_K; K++) {
    const bool on = (mask >> (K - 1)) & 1u;
    const bool haar = (K == 1) && ((mask >> 8) & 1u);
    if (!on && !haar) continue;
    const double* h = filter_taps(K);
    ws.K[nd] = K;
    ws.w[nd] = (R)((on ? 1 : 0) + (haar ? 1 : 0));
    for (int n = 0; n < 2 * K; n++) {
      ws.h[nd][n] = (R)h[n];
      const double gv = h[2 * K - 1 - n];
      ws.g[nd][n] = (R)((n & 1) ? -gv : gv);
    }
    ns += (on ? 1 : 0) + (haar ? 1 : 0);
    nd++;
  }
  ws.nd = nd;
  *n_s = ns;
  return ws;
}

template <class R>
cudaError_t spectral_step(mf_plan* p, const IterScalars<R>& sc, int resid, int precision, cudaStream_t s) {
  if (p->spectral_mask & 2)
    return launch_spectral_b2<R>((const R*)p->X, (R*)p->GP, (R*)p->Sd, (R*)p->GV, (R*)p->GV2, (R*)p->GSd, (R*)p->S2,
                                 (R*)p->b,
                                 (const R*)p->dctC, (const R*)p->Mb2, p->spectral_mask & 1, p->N, p->L, sc,
                                 p->partials, resid, s);
  return launch_spectral<R>((const R*)p->X, (R*)p->GP, (R*)p->Sd, (R*)p->GV, (R*)p->GSd, (R*)p->b,
                            (const R*)p->dctC, p->N, p->L, sc, p->partials, resid, s);
}
template <>
cudaError_t spectral_step<float>(mf_plan* p, const IterScalars<float>& sc, int resid, int precision,
                                 cudaStream_t s) {
  if (p->spectral_mask & 2)
    return launch_spectral_b2<float>((const float*)p->X, (float*)p->GP, (float*)p->Sd, (float*)p->GV,
                                     (float*)p->GV2, (float*)p->GSd, (float*)p->S2, (float*)p->b,
                                     (const float*)p->dctC,
                                     (const float*)p->Mb2, p->spectral_mask & 1, p->N, p->L, sc, p->partials, resid,
                                     s);
  if (precision == MF_FP32_DCT_SPLITBF16)
    return launch_spectral_tc((const float*)p->X, (float*)p->GP, (float*)p->Sd, (float*)p->GV, (float*)p->GSd,
                              (float*)p->b, (const uint16_t*)p->dct_tc, p->N, p->L, sc, p->partials, resid, p->err,
                              p->tc_stall, s);
  return launch_spectral<float>((const float*)p->X, (float*)p->GP, (float*)p->Sd, (float*)p->GV, (float*)p->GSd,
                                (float*)p->b, (const float*)p->dctC, p->N, p->L, sc, p->partials, resid, s);
}

template <class R>
int spectral_grid(const mf_plan* p, int precision) {
  return (precision == MF_FP32_DCT_SPLITBF16 && !(p->spectral_mask & 2)) ? spectral_tc_blocks(p->N)
                                                                        : spectral_blocks<R>(p->N, p->L);
}

template <class R>
cudaError_t iteration(mf_plan* p, int J, const WavSet<R>& ws, const WavSet<R>* wsd, const IterScalars<R>& sc,
                      int resid, int precision, cudaStream_t s) {
  const int N = p->N, L = p->L, nd = ws.nd;
  const size_t NN = (size_t)N * N;
  cudaError_t e;
  if (resid) {
    // state entering the iteration, for the dual residual
    Timed t(p, MF_K_DUAL, s);
    if ((e = dual_snapshot<R>(p, s))) return e;
  }
  // step I
  if (p->linear) {
    {
      // conjugate gradients with the linear convolution, started from the previous X
      Timed t(p, MF_K_CG, s);
      if ((e = linear_step_I(p, p->cg_iters, p->rho_bar, s))) return e;
    }
    if (resid) {
      int nb = 0;
      {
        Timed t(p, MF_K_CG, s);
        if ((e = linear_fit(p, (const float*)p->y_cur, p->partials, &nb, s))) return e;
      }
      Timed t(p, MF_K_REDUCE, s);
      if ((e = launch_finalize(p->partials, nb, p->sums, 0, s))) return e;
    }
  } else {
  {
    Timed t(p, MF_K_ROWS_FWD, s);
    if ((e = launch_rows_fwd<R>((const R*)p->b, (cx<R>*)p->work, N, N * L, (const cx<R>*)p->tw, s))) return e;
  }
  {
    Timed t(p, MF_K_COLS, s);
    if ((e = launch_cols<R>((cx<R>*)p->work, N, L, (const cx<R>*)p->tw, resid ? 2 : 1, nullptr, nullptr,
                            (const cx<R>*)p->cc, (const cx<R>*)p->cc_nyq, (const R*)p->gg, (const R*)p->gg_nyq,
                            (const cx<R>*)p->hhat, (const cx<R>*)p->hhat_nyq, (const cx<R>*)p->yhat,
                            (const cx<R>*)p->yhat_nyq, p->partials, s)))
      return e;
  }
  if (resid) {
    Timed t(p, MF_K_REDUCE, s);
    if ((e = launch_finalize(p->partials, cols_blocks<R>(N, L), p->sums, 0, s))) return e;
  }
  {
    Timed t(p, MF_K_ROWS_INV, s);
    if ((e = launch_rows_inv<R>((const cx<R>*)p->work, (R*)p->X, N, N * L, (const cx<R>*)p->tw, s))) return e;
  }
  }
  // steps II, IV, V (+ duals), pointwise part of b
  {
    Timed t(p, MF_K_SPECTRAL, s);
    if ((e = spectral_step<R>(p, sc, resid, precision, s))) return e;
  }
  if (resid) {
    Timed t(p, MF_K_REDUCE, s);
    if ((e = launch_finalize(p->partials, spectral_grid<R>(p, precision), p->sums, 1, s))) return e;
  }
  // step III (+ dual), wavelet part of b
  R* scr = (R*)p->scratch;
  R* LL[MF_MAX_LEVELS + 1] = {nullptr};
  R* RC[MF_MAX_LEVELS + 1] = {nullptr};
  {
    size_t off = 0;
    for (int j = 1; j < J; j++) {
      const size_t m = (size_t)(N >> j) * (N >> j) * MF_MAX_BASES * L;
      LL[j] = scr + off;
      off += m;
      RC[j] = scr + off;
      off += m;
    }
  }
  for (int j = 1; j < J; j++) {
    const int M = N >> (j - 1);
    const R* in = j == 1 ? (const R*)p->X : LL[j - 1];
    const size_t band_stride = j == 1 ? NN : (size_t)M * M;
    const size_t basis_stride = j == 1 ? 0 : (size_t)M * M * L;
    Timed t(p, MF_K_WAV_LL, s);
    if ((e = launch_wav_ll<R>(in, band_stride, basis_stride, LL[j], M, L, nd, wsd, s))) return e;
  }
  const R* gto = (const R*)p->GT[p->gt_cur];
  R* gtn = (R*)p->GT[1 - p->gt_cur];
  for (int j = J; j >= 1; j--) {
    const int M = N >> (j - 1);
    const R* in = j == 1 ? (const R*)p->X : LL[j - 1];
    const R* rco = j == J ? nullptr : RC[j];
    R* outp = j == 1 ? (R*)p->b : RC[j - 1];
    {
      Timed t(p, j == 1 ? MF_K_WAV_LEVEL1 : MF_K_WAV_LEVELJ, s);
      if ((e = launch_wav_level<R>(in, 0, 0, rco, outp, gto, gtn, N, M, L, j == J, nd, wsd, sc, p->partials,
                                   resid, p->wav_tile, p->err, s)))
        return e;
    }
    if (resid) {
      Timed t(p, MF_K_REDUCE, s);
      if ((e = launch_finalize(p->partials, wav_level_blocks<R>(M, L, M == N ? 1 : nd, p->wav_tile), p->sums, 1, s)))
        return e;
    }
  }
  if (resid) {
    // dual residual: acc = d(b - Gamma_P) - dGamma_S - sum_k w_k W_k^T dGamma_T,k, the
    // wavelet term synthesised level by level from the two Gamma_T buffers through
    // the (now free) level scratch RC
    Timed t(p, MF_K_DUAL, s);
    if ((e = dual_spectral<R>(p, s))) return e;
    for (int j = J; j >= 1; j--) {
      const int M = N >> (j - 1);
      const R* rco = j == J ? nullptr : RC[j];
      R* outp = j == 1 ? dual_acc<R>(p) : RC[j - 1];
      if ((e = launch_wav_level<R>(nullptr, 0, 0, rco, outp, gto, gtn, N, M, L, j == J, nd, wsd, sc, nullptr, 2,
                                   p->wav_tile, p->err, s)))
        return e;
    }
    if ((e = dual_norm<R>(p, s))) return e;
  }
  p->gt_cur = 1 - p->gt_cur;
  return cudaSuccess;
}

// Per-call part of an iterate: validation, the wavelet set, Fourier constants
// F(y), g, c and (unless warm) the zero state, enqueued on s.
template <class R>
mf_status prepare(mf_plan* p, const R* y, const mf_params* prm, int n_iter, cudaStream_t s, WavSet<R>* ws_out,
                  IterScalars<R>* sc_out) {
  mf_status st = check_params(p, prm, n_iter, sizeof(R) == 8);
  if (st != MF_OK) return st;
  if (!y) return MF_ERR_INVALID;
  if (p->status != MF_OK) return p->status;
  p->stream = s;
  const int N = p->N, L = p->L;
  int n_s = 0;
  const WavSet<R> ws = make_wavset<R>(prm->wavelet_mask, &n_s);
  const double rho_bar = prm->mu_eps + prm->rho_S + prm->rho_P + n_s * prm->rho_T;  // Eq. Qlsimp
  IterScalars<R> sc;
  sc.rho_P = (R)prm->rho_P;
  sc.rho_T = (R)prm->rho_T;
  sc.rho_V = (R)prm->rho_V;
  sc.rho_S = (R)prm->rho_S;
  sc.tau_T = (R)(prm->mu_s / prm->rho_T);
  sc.tau_V = (R)(prm->mu_nu / prm->rho_V);
  sc.inv_rho_P = (R)(1.0 / prm->rho_P);
  sc.inv_rho_T = (R)(1.0 / prm->rho_T);
  sc.inv_rho_V = (R)(1.0 / prm->rho_V);
  const int m_nu = (prm->spectral_mask & 1) + ((prm->spectral_mask >> 1) & 1);  // bases of W_nu
  sc.inv_VS = (R)(1.0 / (m_nu * prm->rho_V + prm->rho_S));  // step V: m_nu rho_V + rho_S
  if (prm->warm_start && p->nd_state >= 0 && p->nd_state != ws.nd && p->iters_done > 0)
    return MF_ERR_INVALID;  // the stored Gamma_T belongs to another dictionary
  if (prm->warm_start && p->iters_done > 0 && p->spectral_mask != 0 && p->spectral_mask != (int)prm->spectral_mask)
    return MF_ERR_INVALID;  // the stored Gamma_V belongs to another spectral dictionary
  p->spectral_mask = (int)prm->spectral_mask;
  if (!(prm->spectral_mask & 2)) {
    p->s2_valid = 0;  // S2 is kept only while the Chebyshev basis is iterated
  } else if (!p->S2) {
    // S in the Chebyshev basis, kept by the plan from its first use on
    const size_t bytes = p->cube * sizeof(R);
    if (cudaMalloc(&p->S2, bytes) != cudaSuccess) {
      cudaGetLastError();
      p->S2 = nullptr;
      return MF_ERR_OOM;
    }
    p->total_bytes += bytes;
    p->s2_valid = 0;
  }
  if (prm->resid_every > 0 && !p->dual) {
    // snapshots and work cubes of the dual residual, kept by the plan from now on
    const size_t bytes = dual_cubes() * p->cube * sizeof(R);
    if (cudaMalloc(&p->dual, bytes) != cudaSuccess) {
      cudaGetLastError();
      p->dual = nullptr;
      return MF_ERR_OOM;
    }
    p->dual_bytes = bytes;
  }
  cudaError_t e = cudaMemcpyAsync(p->wset, &ws, sizeof(ws), cudaMemcpyHostToDevice, s);
  p->rho_bar = rho_bar;
  p->cg_iters = prm->cg_iters;
  p->y_cur = y;
  if (p->linear) {
    // H^T y of the linear convolution (step I runs conjugate gradients)
    Timed t(p, MF_K_SETUP, s, 1);
    if (!e) e = linear_hty(p, (const float*)y, s);
  } else {
    // constants: F(y), g, c
    Timed t(p, MF_K_SETUP, s, 4);
    if (!e) e = launch_rows_fwd<R>(y, (cx<R>*)p->work, N, N * L, (const cx<R>*)p->tw, s);
    if (!e)
      e = launch_cols<R>((cx<R>*)p->work, N, L, (const cx<R>*)p->tw, 0, (cx<R>*)p->yhat, (cx<R>*)p->yhat_nyq,
                         nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, s);
    if (!e)
      e = launch_constants<R>((const cx<R>*)p->hhat, (const cx<R>*)p->hhat_nyq, (const cx<R>*)p->yhat,
                              (const cx<R>*)p->yhat_nyq, (cx<R>*)p->cc, (cx<R>*)p->cc_nyq, (R*)p->gg,
                              (R*)p->gg_nyq, N, L, rho_bar, s);
  }
  {
    if (!e && !prm->warm_start) {
      const size_t cb = p->cube * sizeof(R);
      void* z[] = {p->X, p->b, p->GP, p->Sd, p->GV, p->GV2, p->GSd};
      for (void* q : z)
        if (!e) e = cudaMemsetAsync(q, 0, cb, s);
      if (!e) e = cudaMemsetAsync(p->GT[p->gt_cur], 0, cb * MF_MAX_BASES, s);
      if (!e && (prm->spectral_mask & 2)) {
        e = cudaMemsetAsync(p->S2, 0, cb, s);  // M S^ of the zero state
        p->s2_valid = 1;
      }
      p->iters_done = 0;
      p->report.resid_iter = -1;
    }
    if (!e && (prm->spectral_mask & 2) && !p->s2_valid) {
      e = launch_s2_from_sd<R>((const R*)p->Mb2, (const R*)p->Sd, (R*)p->S2, N, L, s);
      p->s2_valid = 1;
    }
  }
  if (e) {
    p->status = MF_ERR_CUDA;
    return p->status;
  }
  p->nd_state = ws.nd;
  *ws_out = ws;
  *sc_out = sc;
  return MF_OK;
}

// n_iter iterations enqueued on s (also under stream capture).
template <class R>
cudaError_t run_iterations(mf_plan* p, const mf_params* prm, int n_iter, const WavSet<R>& ws,
                           const IterScalars<R>& sc, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  for (int it = 0; it < n_iter && !e; it++) {
    const int resid = prm->resid_every > 0 && (((it + 1) % prm->resid_every) == 0 || it == n_iter - 1);
    e = iteration<R>(p, prm->wavelet_levels, ws, (const WavSet<R>*)p->wset, sc, resid, prm->precision, s);
    if (!e && resid) {
      p->report_pending = 1;
      p->report.resid_iter = p->iters_done + it + 1;
    }
  }
  return e;
}

void finish(mf_plan* p, const mf_params* prm, int n_iter) {
  p->iters_done += n_iter;
  p->rho_weights[0] = prm->rho_P;
  p->rho_weights[1] = prm->rho_T;
  p->rho_weights[2] = prm->rho_V;
  p->rho_weights[3] = prm->rho_S;
  p->report.iters_done = p->iters_done;
  std::memcpy(&p->last_params, prm, sizeof(mf_params));
}

template <class R>
mf_status iterate(mf_plan* p, const R* y, const mf_params* prm, int n_iter) {
  cudaStream_t s = prm ? (cudaStream_t)prm->stream : nullptr;
  WavSet<R> ws;
  IterScalars<R> sc;
  mf_status st = prepare<R>(p, y, prm, n_iter, s, &ws, &sc);
  if (st != MF_OK) return st;
  if (run_iterations<R>(p, prm, n_iter, ws, sc, s) != cudaSuccess) {
    cudaGetLastError();
    p->status = MF_ERR_CUDA;
    return p->status;
  }
  finish(p, prm, n_iter);
  return MF_OK;
}

// What a captured batch graph depends on: every plan (by serial number, with
// its options and the Gamma_T buffer it starts from: an odd n_iter swaps the
// double buffer), every y pointer, n_iter and every parameter but the stream.
std::vector<unsigned long long> batch_key_of(mf_plan* const* plans, const float* const* ys, int count,
                                             const mf_params* prm, int n_iter) {
  std::vector<unsigned long long> k;
  auto bits = [&](double v) {
    unsigned long long u;
    std::memcpy(&u, &v, sizeof(u));
    k.push_back(u);
  };
  k.push_back((unsigned long long)count);
  k.push_back((unsigned long long)n_iter);
  for (double v : {prm->mu_eps, prm->mu_s, prm->mu_nu, prm->rho_P, prm->rho_T, prm->rho_V, prm->rho_S}) bits(v);
  for (long long v : {(long long)prm->wavelet_levels, (long long)prm->wavelet_mask, (long long)prm->precision,
                      (long long)prm->resid_every, (long long)prm->warm_start, (long long)prm->cg_iters,
                      (long long)prm->spectral_mask})
    k.push_back((unsigned long long)v);
  for (int i = 0; i < count; i++) {
    k.push_back(plans[i]->serial);
    k.push_back((unsigned long long)(uintptr_t)ys[i]);
    k.push_back((unsigned long long)plans[i]->gt_cur);
    k.push_back((unsigned long long)plans[i]->wav_tile);
    k.push_back((unsigned long long)plans[i]->tc_stall);
  }
  return k;
}

// Host-side effects of run_iterations for a replayed graph: the Gamma_T buffer
// swap of every iteration and the residual-report bookkeeping.
void replay_effects(mf_plan* p, const mf_params* prm, int n_iter) {
  for (int it = 0; it < n_iter; it++) {
    const int resid = prm->resid_every > 0 && (((it + 1) % prm->resid_every) == 0 || it == n_iter - 1);
    if (resid) {
      p->report_pending = 1;
      p->report.resid_iter = p->iters_done + it + 1;
    }
    p->gt_cur = 1 - p->gt_cur;
  }
}

// Batched form: every plan's n_iter iterations in one CUDA graph, each cube on
// its own branch, launched once on prm->stream.  A call identical to the
// previous one with the same first plan (same plans, y pointers, n_iter,
// parameters, options and Gamma_T buffer) relaunches that graph instead of
// capturing and instantiating a new one.
mf_status batch_iterate(mf_plan* const* plans, const float* const* ys, int count, const mf_params* prm,
                        int n_iter) {
  if (!plans || !ys || !prm || count < 1 || count > 1024 || n_iter < 1) return MF_ERR_INVALID;
  for (int i = 0; i < count; i++) {
    if (!plans[i] || plans[i]->dbl || !ys[i]) return MF_ERR_INVALID;
    for (int j = 0; j < i; j++)
      if (plans[j] == plans[i]) return MF_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)prm->stream;
  mf_plan* owner = plans[0];
  std::vector<unsigned long long> key = batch_key_of(plans, ys, count, prm, n_iter);
  const bool reuse = owner->batch_exec && owner->batch_stream == s && owner->batch_key == key;
  if (owner->batch_exec && !reuse) {  // the previous batch graph of this owner
    if (cudaStreamSynchronize(owner->batch_stream) != cudaSuccess) return MF_ERR_CUDA;
    cudaGraphExecDestroy((cudaGraphExec_t)owner->batch_exec);
    owner->batch_exec = nullptr;
    owner->batch_key.clear();
  }
  std::vector<WavSet<float>> ws(count);
  std::vector<IterScalars<float>> sc(count);
  for (int i = 0; i < count; i++) {
    mf_status st = prepare<float>(plans[i], ys[i], prm, n_iter, s, &ws[i], &sc[i]);
    if (st != MF_OK) return st;
  }
  if (reuse) {
    if (cudaGraphLaunch((cudaGraphExec_t)owner->batch_exec, s) != cudaSuccess) {
      cudaGetLastError();
      for (int i = 0; i < count; i++) plans[i]->status = MF_ERR_CUDA;
      return MF_ERR_CUDA;
    }
    for (int i = 0; i < count; i++) {
      replay_effects(plans[i], prm, n_iter);
      finish(plans[i], prm, n_iter);
      plans[i]->stream = s;
    }
    return MF_OK;
  }
  // The graph is recorded on a private stream (the caller's may be the legacy
  // default stream, which cannot be captured) and launched on the caller's.
  std::vector<cudaStream_t> side(count, nullptr);
  std::vector<cudaEvent_t> join(count, nullptr);
  cudaEvent_t fork = nullptr;
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<int> timing(count);
  cudaError_t e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
  if (!e) e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  for (int i = 0; i < count && !e; i++) {
    e = cudaStreamCreateWithFlags(&side[i], cudaStreamNonBlocking);
    if (!e) e = cudaEventCreateWithFlags(&join[i], cudaEventDisableTiming);
    timing[i] = plans[i]->timing;
    plans[i]->timing = 0;  // no event brackets inside the graph
  }
  bool capturing = false;
  if (!e) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (!e) {
    capturing = true;
    e = cudaEventRecord(fork, cap);
  }
  for (int i = 0; i < count && !e; i++) {
    e = cudaStreamWaitEvent(side[i], fork, 0);
    if (!e) e = run_iterations<float>(plans[i], prm, n_iter, ws[i], sc[i], side[i]);
    if (!e) e = cudaEventRecord(join[i], side[i]);
    if (!e) e = cudaStreamWaitEvent(cap, join[i], 0);
  }
  if (capturing) {
    cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
    if (!e) e = e2;
  }
  if (!e) e = cudaGraphInstantiate(&exec, graph, 0);
  if (!e) e = cudaGraphLaunch(exec, s);
  for (int i = 0; i < count; i++) {
    plans[i]->timing = timing[i];
  }
  if (graph) cudaGraphDestroy(graph);
  if (fork) cudaEventDestroy(fork);
  if (cap) cudaStreamDestroy(cap);
  for (int i = 0; i < count; i++) {
    if (join[i]) cudaEventDestroy(join[i]);
    if (side[i]) cudaStreamDestroy(side[i]);
  }
  if (e) {
    cudaGetLastError();
    if (exec) cudaGraphExecDestroy(exec);
    for (int i = 0; i < count; i++) plans[i]->status = MF_ERR_CUDA;
    return MF_ERR_CUDA;
  }
  owner->batch_exec = exec;
  owner->batch_stream = s;
  owner->batch_key = key;  // taken before the capture swapped the Gamma_T buffers
  for (int i = 0; i < count; i++) {
    finish(plans[i], prm, n_iter);
    plans[i]->stream = s;
  }
  return MF_OK;
}

void* array_ptr(mf_plan* p, int which, size_t* count) {
  *count = p->cube;
  switch (which) {
    case MF_ARR_X: return p->X;
    case MF_ARR_GAMMA_P: return p->GP;
    case MF_ARR_S_DCT: return p->Sd;
    case MF_ARR_GAMMA_V: return p->GV;
    case MF_ARR_GAMMA_S_DCT: return p->GSd;
    case MF_ARR_GAMMA_V2: return p->GV2;
    case MF_ARR_B: return p->b;
    case MF_ARR_HTY: return p->linear ? p->cgv : nullptr;
    case MF_ARR_GAMMA_T: *count = p->cube * (p->nd_state > 0 ? p->nd_state : MF_MAX_BASES); return p->GT[p->gt_cur];
    default: return nullptr;
  }
}

}  // namespace

namespace mf {
template <class R>
cudaError_t launch_shift_psf(const R* psf, R* out, int N, size_t total, cudaStream_t s) {
  k_shift_psf<R><<<1024, 256, 0, s>>>(psf, out, N, total);
  return cudaGetLastError();
}
template cudaError_t launch_shift_psf<float>(const float*, float*, int, size_t, cudaStream_t);
}  // namespace mf

// Entry points for the reverse pass (backward.cu).
mf_status mf_internal_prepare_f32(mf_plan* p, const float* y, const mf_params* prm, int n_iter, cudaStream_t s,
                                  WavSet<float>* ws, IterScalars<float>* sc) {
  return prepare<float>(p, y, prm, n_iter, s, ws, sc);
}
cudaError_t mf_internal_iteration_f32(mf_plan* p, const mf_params* prm, const WavSet<float>& ws,
                                      const IterScalars<float>& sc, cudaStream_t s) {
  return iteration<float>(p, prm->wavelet_levels, ws, (const WavSet<float>*)p->wset, sc, 0, prm->precision, s);
}
void mf_internal_finish(mf_plan* p, const mf_params* prm, int n_iter) { finish(p, prm, n_iter); }

extern "C" {

void mf_params_default(mf_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->mu_eps = 0.001;
  p->mu_s = 0.05;
  p->mu_nu = 0.01;
  p->rho_P = p->rho_T = p->rho_V = p->rho_S = 1.0;
  p->wavelet_levels = 3;
  p->wavelet_mask = 0x1FF;
  p->precision = MF_FP32;
  p->cg_iters = 20;
  p->spectral_mask = 1;
}

mf_status mf_plan_create(int N, int L, const float* psf_cube, mf_plan** out) {
  return create<float>(N, L, psf_cube, out);
}
mf_status mf_plan_create_f64(int N, int L, const double* psf_cube, mf_plan** out) {
  return create<double>(N, L, psf_cube, out);
}

mf_status mf_plan_create_linear(int N, int L, const float* psf_cube, mf_plan** out) {
  if (!out) return MF_ERR_INVALID;
  *out = nullptr;
  if (!psf_cube || !is_pow2(N) || N < 16 || N > 1024 || L < 2 || L > MF_MAX_L) return MF_ERR_INVALID;
  mf_plan* p = nullptr;
  mf_status st = create<float>(N, L, psf_cube, &p);
  if (st != MF_OK) return st;
  const size_t cb = p->cube * sizeof(float);
  Alloc a{p};
  p->h2 = a.get(4 * cb);
  p->h2_nyq = a.get((size_t)L * 2 * N * sizeof(cx<float>));
  p->tw2 = a.get((size_t)2 * N * sizeof(cx<float>));
  p->work2 = a.get(4 * cb);
  p->big = a.get(4 * cb);
  p->cgv = a.get(4 * cb);
  p->cgs = (double*)a.get((size_t)5 * L * sizeof(double));
  p->cgpart = (double*)a.get((size_t)MF_CG_CHUNKS * L * sizeof(double));
  if (!a.ok) {
    mf_plan_destroy(p);
    return MF_ERR_OOM;
  }
  p->linear = 1;
  if (linear_setup(p, psf_cube) != cudaSuccess) {
    cudaGetLastError();
    mf_plan_destroy(p);
    return MF_ERR_CUDA;
  }
  *out = p;
  return MF_OK;
}

mf_status mf_plan_create_vis(int N, int L, const int* n_vis, const float* uv, const float* weights,
                             mf_plan** out) {
  if (!out) return MF_ERR_INVALID;
  *out = nullptr;
  if (!n_vis || !is_pow2(N) || N < 16 || N > 512 || L < 2 || L > MF_MAX_L) return MF_ERR_INVALID;
  long total = 0;
  for (int l = 0; l < L; l++) {
    if (n_vis[l] < 0) return MF_ERR_INVALID;
    total += n_vis[l];
  }
  if (total > (1L << 30) || (total > 0 && !uv)) return MF_ERR_INVALID;
  mf_plan* p = nullptr;
  mf_status st = create<float>(N, L, nullptr, &p, true);
  if (st != MF_OK) return st;
  const size_t cb = p->cube * sizeof(float);
  Alloc a{p};
  p->h2 = a.get(4 * cb);
  p->h2_nyq = a.get((size_t)L * 2 * N * sizeof(cx<float>));
  p->tw2 = a.get((size_t)2 * N * sizeof(cx<float>));
  p->work2 = a.get(4 * cb);
  p->big = a.get(4 * cb);
  p->cgv = a.get(4 * cb);
  p->cgs = (double*)a.get((size_t)5 * L * sizeof(double));
  p->cgpart = (double*)a.get((size_t)MF_CG_CHUNKS * L * sizeof(double));
  if (total > 0) p->vis_uv = a.get(sizeof(float2) * total);
  if (total > 0 && weights) p->vis_w = a.get(sizeof(float) * total);
  p->vis_c0 = (double*)a.get(sizeof(double));
  p->vis_phihat = a.get(sizeof(float) * N);
  p->vis_twM = a.get((size_t)2 * N * sizeof(cx<float>));
  p->vis_spec = a.get(vis_spec_elems(N) * sizeof(cx<float>));
  p->vis_nyq = a.get((size_t)2 * 2 * N * sizeof(cx<float>));
  if (!a.ok) {
    mf_plan_destroy(p);
    return MF_ERR_OOM;
  }
  p->linear = 1;
  p->vis = 1;
  p->vis_off.assign(L + 1, 0);
  for (int l = 0; l < L; l++) p->vis_off[l + 1] = p->vis_off[l] + n_vis[l];
  cudaError_t e = cudaSuccess;
  if (total > 0) e = cudaMemcpy(p->vis_uv, uv, sizeof(float2) * total, cudaMemcpyDeviceToDevice);
  if (!e && total > 0 && weights) e = cudaMemcpy(p->vis_w, weights, sizeof(float) * total, cudaMemcpyDeviceToDevice);
  if (!e) e = vis_setup(p, n_vis);
  if (e) {
    cudaGetLastError();
    mf_plan_destroy(p);
    return e == cudaErrorInvalidValue ? MF_ERR_INVALID : MF_ERR_CUDA;
  }
  *out = p;
  return MF_OK;
}

mf_status mf_vis_predict(mf_plan* p, const float* x, float* vis_out, void* stream) {
  if (!p || !p->vis || !vis_out) return MF_ERR_INVALID;
  if (p->status != MF_OK) return p->status;
  cudaStream_t s = (cudaStream_t)stream;
  // the call shares the plan's work arrays: it runs after the plan's last work
  if (s != p->stream && cudaStreamSynchronize(p->stream) != cudaSuccess) {
    cudaGetLastError();
    p->status = MF_ERR_CUDA;
    return p->status;
  }
  p->stream = s;
  if (p->vis_off.back() == 0) return MF_OK;
  if (vis_predict(p, x ? x : (const float*)p->X, vis_out, s) != cudaSuccess) {
    cudaGetLastError();
    p->status = MF_ERR_CUDA;
    return p->status;
  }
  return MF_OK;
}

void mf_plan_destroy(mf_plan* p) {
  if (!p) return;
  cudaDeviceSynchronize();
  if (p->batch_exec) cudaGraphExecDestroy((cudaGraphExec_t)p->batch_exec);
  free_plan_memory(p);
  delete p;
}

size_t mf_plan_device_bytes(const mf_plan* p) { return p ? p->total_bytes + p->bwd_bytes + p->dual_bytes : 0; }

mf_status mf_admm_iterate(mf_plan* p, const float* y, const mf_params* prm, int n_iter) {
  return iterate<float>(p, y, prm, n_iter);
}
mf_status mf_admm_iterate_f64(mf_plan* p, const double* y, const mf_params* prm, int n_iter) {
  return iterate<double>(p, y, prm, n_iter);
}

mf_status mf_batch_iterate(mf_plan* const* plans, const float* const* y_cubes, int count, const mf_params* prm,
                           int n_iter) {
  return batch_iterate(plans, y_cubes, count, prm, n_iter);
}

// Device-to-device copy on the plan's stream, complete on return (a plain
// cudaMemcpy between device buffers may return before the copy has finished,
// and the legacy stream it uses is not ordered with non-blocking streams).
static bool copy_d2d(mf_plan* p, void* dst, const void* src, size_t bytes) {
  return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, p->stream) == cudaSuccess &&
         cudaStreamSynchronize(p->stream) == cudaSuccess;
}

mf_status mf_plan_get_array(mf_plan* p, int which, void* dst, size_t* count) {
  if (!p) return MF_ERR_INVALID;
  size_t n = 0;
  void* src = array_ptr(p, which, &n);
  if (!src) return MF_ERR_INVALID;
  if (count) *count = n;
  if (!dst) return count ? MF_OK : MF_ERR_INVALID;
  if (cudaStreamSynchronize(p->stream) != cudaSuccess) return MF_ERR_CUDA;
  if (!copy_d2d(p, dst, src, n * p->esz)) return MF_ERR_CUDA;
  return MF_OK;
}

mf_status mf_plan_set_array(mf_plan* p, int which, const void* src, size_t count) {
  if (!p || !src || which == MF_ARR_HTY) return MF_ERR_INVALID;
  size_t n = 0;
  void* dst = array_ptr(p, which, &n);
  if (which == MF_ARR_GAMMA_T) n = p->cube * MF_MAX_BASES;
  if (!dst || count > n || (which != MF_ARR_GAMMA_T && count != n)) return MF_ERR_INVALID;
  if (cudaStreamSynchronize(p->stream) != cudaSuccess) return MF_ERR_CUDA;
  if (!copy_d2d(p, dst, src, count * p->esz)) return MF_ERR_CUDA;
  if (which == MF_ARR_S_DCT) p->s2_valid = 0;
  if (which == MF_ARR_GAMMA_T) p->nd_state = (int)(count / p->cube);
  return MF_OK;
}

mf_status mf_plan_get_state(mf_plan* p, void* buf, size_t* bytes) {
  if (!p || !bytes) return MF_ERR_INVALID;
  const size_t cb = p->cube * p->esz;
  const size_t need = cb * (7 + MF_MAX_BASES);
  if (!buf) {
    *bytes = need;
    return MF_OK;
  }
  if (*bytes < need) return MF_ERR_INVALID;
  if (cudaStreamSynchronize(p->stream) != cudaSuccess) return MF_ERR_CUDA;
  void* src[] = {p->X, p->b, p->GP, p->Sd, p->GV, p->GV2, p->GSd};
  char* d = (char*)buf;
  for (void* s : src) {
    if (!copy_d2d(p, d, s, cb)) return MF_ERR_CUDA;
    d += cb;
  }
  if (!copy_d2d(p, d, p->GT[p->gt_cur], cb * MF_MAX_BASES)) return MF_ERR_CUDA;
  return MF_OK;
}

mf_status mf_plan_set_state(mf_plan* p, const void* buf, size_t bytes) {
  if (!p || !buf) return MF_ERR_INVALID;
  const size_t cb = p->cube * p->esz;
  if (bytes != cb * (7 + MF_MAX_BASES)) return MF_ERR_INVALID;
  if (cudaStreamSynchronize(p->stream) != cudaSuccess) return MF_ERR_CUDA;
  void* dst[] = {p->X, p->b, p->GP, p->Sd, p->GV, p->GV2, p->GSd};
  const char* s = (const char*)buf;
  for (void* d : dst) {
    if (!copy_d2d(p, d, s, cb)) return MF_ERR_CUDA;
    s += cb;
  }
  if (!copy_d2d(p, p->GT[p->gt_cur], s, cb * MF_MAX_BASES)) return MF_ERR_CUDA;
  if (p->iters_done == 0) p->iters_done = 1;
  p->s2_valid = 0;
  // the dictionaries the state was made with are not recorded in it: the next
  // warm start takes the caller's (the checks against the plan's last call are off)
  p->nd_state = -1;
  p->spectral_mask = 0;
  return MF_OK;
}

mf_status mf_plan_get_report(mf_plan* p, mf_report* r) {
  if (!p || !r) return MF_ERR_INVALID;
  if (cudaStreamSynchronize(p->stream) != cudaSuccess) {
    p->status = MF_ERR_CUDA;
    return p->status;
  }
  {
    int err = 0;
    if (cudaMemcpy(&err, p->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
      p->status = MF_ERR_CUDA;
      return p->status;
    }
    if (err && p->status == MF_OK) p->status = MF_ERR_TIMEOUT;
  }
  if (p->report_pending) {
    double q[MF_NQ];
    if (cudaMemcpy(q, p->sums, sizeof(q), cudaMemcpyDeviceToHost) != cudaSuccess) {
      p->status = MF_ERR_CUDA;
      return p->status;
    }
    const double* w = p->rho_weights;
    p->report.primal_res = q[Q_DGP] / (w[0] * w[0]) + q[Q_DGT] / (w[1] * w[1]) + q[Q_DGV] / (w[2] * w[2]) +
                           q[Q_DGS] / (w[3] * w[3]);
    p->report.dual_gamma = q[Q_DGP] + q[Q_DGT] + q[Q_DGV] + q[Q_DGS];
    const int m_nu = (p->last_params.spectral_mask & 1) + ((p->last_params.spectral_mask >> 1) & 1);
    p->report.dual_res = q[Q_DUALX] + m_nu * w[2] * w[2] * q[Q_DS2];  // rho_V^2 sum_j ||dS W_j||^2
    const mf_params* pr = &p->last_params;
    p->report.objective = q[Q_FIT] + 0.5 * pr->mu_eps * q[Q_X2] + pr->mu_s * q[Q_L1S] + pr->mu_nu * q[Q_L1NU];
    p->report.x_min = q[Q_XMIN];
    p->report.x_norm2 = q[Q_X2];
    p->report_pending = 0;
    bool finite = q[Q_NONFIN] == 0.0;
    for (int i = 0; i < Q_COUNT; i++) finite = finite && std::isfinite(q[i]);
    if (!finite && p->status == MF_OK) p->status = MF_ERR_NONFINITE;
  }
  *r = p->report;
  return p->status;
}

mf_status mf_plan_set_timing(mf_plan* p, int enable) {
  if (!p) return MF_ERR_INVALID;
  if (cudaStreamSynchronize(p->stream) != cudaSuccess) return MF_ERR_CUDA;
  p->ev_used = 0;
  p->ev_kernel.clear();
  for (int k = 0; k < MF_K_COUNT; k++) {
    p->kernel_ms[k] = 0.0;
    p->launches[k] = 0;
  }
  p->timing = enable ? 1 : 0;
  return MF_OK;
}

mf_status mf_plan_get_timing(mf_plan* p, int kernel, double* total_ms, long long* launches) {
  if (!p || kernel < 0 || kernel >= MF_K_COUNT) return MF_ERR_INVALID;
  if (cudaStreamSynchronize(p->stream) != cudaSuccess) return MF_ERR_CUDA;
  fold_timing(p);
  if (total_ms) *total_ms = p->kernel_ms[kernel];
  if (launches) *launches = p->launches[kernel];
  return MF_OK;
}

mf_status mf_plan_set_option(mf_plan* p, int option, int value) {
  if (!p) return MF_ERR_INVALID;
  switch (option) {
    case MF_OPT_WAV_TILE:
      if (value != 32 && value != 64) return MF_ERR_INVALID;
      if (cudaStreamSynchronize(p->stream) != cudaSuccess) return MF_ERR_CUDA;
      p->wav_tile = value;
      return MF_OK;
    case MF_OPT_TEST_TC_STALL:
      if (value < 0) return MF_ERR_INVALID;
      if (cudaStreamSynchronize(p->stream) != cudaSuccess) return MF_ERR_CUDA;
      p->tc_stall = value;
      return MF_OK;
    default: return MF_ERR_INVALID;
  }
}

mf_status mf_plan_clear_status(mf_plan* p) {
  if (!p) return MF_ERR_INVALID;
  if (cudaStreamSynchronize(p->stream) != cudaSuccess) return MF_ERR_CUDA;
  if (cudaMemset(p->err, 0, sizeof(int)) != cudaSuccess) return MF_ERR_CUDA;
  p->status = MF_OK;
  return MF_OK;
}

const char* mf_kernel_name(int kernel) {
  static const char* names[MF_K_COUNT] = {"rows_fwd", "cols_solve", "rows_inv", "spectral", "wav_ll",
                                          "wav_level1", "wav_levelj", "setup", "reduce", "dual", "cg"};
  return (kernel >= 0 && kernel < MF_K_COUNT) ? names[kernel] : "unknown";
}

mf_status mf_spectral_basis(int kind, int L, double* out) {
  if (!out || L < 2 || L > 64) return MF_ERR_INVALID;
  if (kind == MF_SPECTRAL_DCT) {
    for (int k = 0; k < L; k++) {
      const double ak = k == 0 ? std::sqrt(1.0 / L) : std::sqrt(2.0 / L);
      for (int l = 0; l < L; l++) out[k * L + l] = ak * std::cos(M_PI * (2.0 * l + 1.0) * k / (2.0 * L));
    }
    return MF_OK;
  }
  if (kind == MF_SPECTRAL_CHEBYSHEV) {
    chebyshev_matrix(L, out);
    return MF_OK;
  }
  return MF_ERR_INVALID;
}

mf_status mf_wavelet_filter(int K, double* taps, int* len) {
  if (K < 1 || K > MF_MAX_K) return MF_ERR_INVALID;
  if (len) *len = 2 * K;
  if (taps) std::memcpy(taps, filter_taps(K), sizeof(double) * 2 * K);
  return MF_OK;
}

const char* mf_status_string(mf_status s) {
  switch (s) {
    case MF_OK: return "ok";
    case MF_ERR_INVALID: return "invalid argument";
    case MF_ERR_OOM: return "device out of memory";
    case MF_ERR_CUDA: return "CUDA error";
    case MF_ERR_TIMEOUT: return "device wait timed out";
    case MF_ERR_NONFINITE: return "non-finite value in the iterate";
    case MF_ERR_TOO_LARGE: return "cube exceeds the static scratch of the no-allocation entry point";
    default: return "unknown status";
  }
}

}  // extern "C"
