// Internal declarations of the mf library: plan layout, kernel parameter
// blocks and the host launchers of each kernel family.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstddef>
#include <vector>

#include "mf.h"

#define MF_MAX_K 8        // DbK with K <= 8 (Db1..Db8 of the paper's dictionary)
#define MF_MAX_F 16       // 2 * MF_MAX_K taps
#define MF_MAX_BASES 8    // distinct wavelet bases (Haar folds into Db1)
#define MF_MAX_LEVELS 8
#define MF_MAX_L 128
#define MF_NQ 16          // reduction quantities per block partial
#define MF_AUX_GRID (152 * 8)  // largest grid of the grid-stride reduction kernels (dual residual)
#define MF_CG_CHUNKS 64        // blocks per band of the conjugate-gradient reductions

namespace mf {

const double* filter_taps(int K);  // DbK low-pass, 2K taps (daub.cpp)
void chebyshev_matrix(int L, double* out);  // orthonormal Chebyshev basis on L bands, row n = degree n

template <class R> struct cx_t;
template <> struct cx_t<float> { typedef float2 type; };
template <> struct cx_t<double> { typedef double2 type; };
template <class R> using cx = typename cx_t<R>::type;

// Distinct bases of W_s as seen by the kernels: filter half-length K,
// synthesis weight w (2 when Db1 and Haar are both selected), taps.
template <class R>
struct WavSet {
  int nd;
  int K[MF_MAX_BASES];
  R w[MF_MAX_BASES];
  R h[MF_MAX_BASES][MF_MAX_F];
  R g[MF_MAX_BASES][MF_MAX_F];
};

// Scalars of one ADMM iteration.
template <class R>
struct IterScalars {
  R rho_P, rho_T, rho_V, rho_S;
  R tau_T, tau_V;   // mu_s / rho_T, mu_nu / rho_V
  R inv_rho_P, inv_rho_T, inv_rho_V, inv_VS;  // 1/rho_P, 1/rho_T, 1/rho_V, 1/(m_nu rho_V + rho_S)
};

// Reduction slots of the per-block FP64 partials.
enum {
  Q_DGP = 0,   // ||dGamma_P||^2
  Q_DGT,       // ||dGamma_T||^2 (all bases, weights included)
  Q_DGV,       // ||dGamma_V||^2
  Q_DGS,       // ||dGamma_S||^2
  Q_X2,        // ||X||^2
  Q_L1NU,      // ||X W_nu||_1
  Q_L1S,       // ||W_s X||_1 (weights included)
  Q_FIT,       // 1/2 ||Y - H X||^2
  Q_XMIN,      // min X (reduced with min)
  Q_NONFIN,    // count of non-finite values met
  Q_DUALX,     // ||rho_P dP + rho_T W_s^T dT + rho_S dS||^2 (dual residual, X part)
  Q_DS2,       // ||d(S W_nu)||^2
  Q_COUNT
};

}  // namespace mf

struct mf_plan {
  int N, L, dbl;
  size_t esz;        // sizeof real type
  size_t cube;       // N * N * L elements
  // reverse-pass checkpoints and work arrays, kept between calls (grown on demand)
  void* bwd_buf = nullptr;
  size_t bwd_bytes = 0;
  // ADMM state and work arrays (real type, [L][N][N] unless noted)
  void* X;
  void* b;
  void* GP;
  void* Sd;          // S W_nu
  void* GV;          // Gamma_V (DCT basis of the spectral dictionary)
  void* GV2;         // Gamma_V of the Chebyshev basis (spectral_mask bit 1)
  void* S2;          // M S^: S in the Chebyshev basis (plans that used it; derived state)
  int s2_valid;       // S2 equals M S^ (cleared when the state is set from outside)
  void* Mb2;         // L x L change of basis DCT domain -> Chebyshev basis (C2 C^T)
  int spectral_mask; // spectral dictionary of the current call
  void* GSd;         // Gamma_S W_nu
  void* GT[2];       // Gamma_T ping-pong, [MF_MAX_BASES][L][N][N]
  int gt_cur;
  int nd_state;      // distinct bases stored in GT (from the last iterate call)
  void* work;        // packed half spectrum [L][N][N/2] complex
  void* hhat;        // transfer function, unpacked half spectrum [L][N][N/2] complex
  void* hhat_nyq;    // its kx = N/2 column [L][N] complex
  void* yhat;        // F(y), same layout
  void* yhat_nyq;
  void* cc;          // conj(hhat) yhat g
  void* cc_nyq;
  void* gg;          // 1 / ((|hhat|^2 + rho) N^2), real [L][N][N/2]
  void* gg_nyq;      // [L][N]
  void* tw;          // exp(-2 pi i k / N), k < N, complex
  void* dctC;        // L x L orthonormal DCT-II
  void* scratch;     // wavelet LL_j and R_j images
  size_t scratch_bytes;
  double* partials;  // [max_blocks][MF_NQ]
  size_t partial_cap;
  double* sums;      // [MF_NQ] device
  void* wset;        // WavSet of the current call (device)
  void* dct_tc;      // split-BF16 DCT operands of the precision form (device), or null
  int* err;          // device error word (bounded waits that expired)
  void* dual;        // dual-residual snapshots and work cubes (allocated on first use)
  size_t dual_bytes;
  // linear convolution (plans from mf_plan_create_linear): step I by conjugate gradients
  int linear;
  void* h2;          // transfer function of the PSF embedded in 2N x 2N: [L][2N][N] complex
  void* h2_nyq;      // its kx = N column: [L][2N] complex
  void* tw2;         // twiddles of length 2N
  void* work2;       // packed half spectrum at 2N: [L][2N][N] complex
  void* big;         // real 2N x 2N images [L][2N][2N]
  void* cgv;         // H^T y, r, p, q: 4 cubes
  int cg_iters;      // conjugate gradient iterations of the current call
  const void* y_cur; // dirty cube of the current call
  double rho_bar;    // rho of Eq. Qlsimp for the current call
  double* cgs;       // per band: gamma, p.q, alpha, beta, gamma' ([5][L])
  double* cgpart;    // per band and chunk partial sums [L][MF_CG_CHUNKS]
  // visibility operator (plans from mf_plan_create_vis; linear == 1 as well):
  // h2 holds the transfer function of each band's Toeplitz kernel, cgv[0] the dirty image
  int vis;
  std::vector<int> vis_off;  // [L+1] first visibility of each band (host)
  void* vis_uv;      // [total] float2 (u, v) in cells
  void* vis_w;       // [total] weights, or null (all 1)
  double* vis_c0;    // 1/2 sum w |y|^2 of the current call
  void* vis_phihat;  // [N] kernel transform at the image's modes
  void* vis_twM;     // twiddles of length 2N (the dirty image's grid)
  void* vis_spec;    // two planes' half spectra at 2N: [2][2N][N] complex
  void* vis_nyq;     // their kx = N columns: [2][2N] complex
  size_t total_bytes;
  cudaStream_t stream;
  mf_status status;
  int iters_done;
  mf_report report;
  int report_pending;   // sums on the device not yet folded into report
  double rho_weights[4];
  mf_params last_params;
  int wav_tile;         // preferred wavelet tile edge (MF_OPT_WAV_TILE)
  long long tc_stall;   // MF_OPT_TEST_TC_STALL (0: off)
  void* batch_exec;     // last batch graph launched with this plan first (cudaGraphExec_t)
  cudaStream_t batch_stream;
  unsigned long long serial;            // unique per plan created (never reused, unlike addresses)
  std::vector<unsigned long long> batch_key;  // what batch_exec was captured for (see batch_iterate)
  // per-kernel timing
  int timing;
  long long launches[MF_K_COUNT];
  double kernel_ms[MF_K_COUNT];
  std::vector<cudaEvent_t> ev_pool;     // created events, reused
  std::vector<int> ev_kernel;           // kernel id of each recorded pair
  size_t ev_used;                       // events in use (2 per pair)
};

namespace mf {

// ---- launchers (explicitly instantiated for float and double) ----
// Row-wise forward real FFT of `rows` rows of length N: real in -> packed half spectrum out.
template <class R> cudaError_t launch_rows_fwd(const R* in, cx<R>* out, int N, int rows, const cx<R>* tw, cudaStream_t s);
// Column pass on the packed half spectrum of L bands.  mode 0: forward transform only,
// unpacked into (out_main, out_nyq).  mode 1: forward, X = c + g B, inverse, in place.
// mode 2: mode 1 plus the data-fit partials from (hh, yh).  mode 3: X = hh B / N^2 (applies
// H).  mode 4: X = g B (applies Q^-1 without the H^T y term).  mode 5: X = conj(hh) B / N^2
// (applies H^T).
template <class R> cudaError_t launch_cols(cx<R>* work, int N, int L, const cx<R>* tw, int mode,
                                           cx<R>* out_main, cx<R>* out_nyq,
                                           const cx<R>* cc, const cx<R>* cc_nyq,
                                           const R* gg, const R* gg_nyq,
                                           const cx<R>* hh, const cx<R>* hh_nyq,
                                           const cx<R>* yh, const cx<R>* yh_nyq, double* partials,
                                           cudaStream_t s);
template <class R> int cols_blocks(int N, int L);
// Row-wise inverse: packed half spectrum in -> real rows out (scaled by N).
template <class R> cudaError_t launch_rows_inv(const cx<R>* in, R* out, int N, int rows, const cx<R>* tw, cudaStream_t s);
// Zero-padded convolution at transform length M (FP32): rows of (M/2)-wide
// images padded to M (rows = (M/2) L, output rows l M + r), the column pass
// with transfer function hh (mode 3) or its conjugate (mode 5) on the first
// M/2 spatial rows, and the inverse rows cropped to the [0, M/2)^2 region.
cudaError_t launch_rows_fwd_pad(const float* in, cx<float>* out, int M, int rows, const cx<float>* tw,
                                cudaStream_t s);
cudaError_t launch_cols_pruned(cx<float>* work, int M, int L, const cx<float>* tw, int mode, const cx<float>* hh,
                               const cx<float>* hh_nyq, cudaStream_t s);
cudaError_t launch_rows_inv_crop(const cx<float>* in, float* out, int M, int rows, const cx<float>* tw,
                                 cudaStream_t s);
// g and c of the Fourier-diagonal solve.
template <class R> cudaError_t launch_constants(const cx<R>* hh, const cx<R>* hh_nyq, const cx<R>* yh,
                                                const cx<R>* yh_nyq, cx<R>* cc, cx<R>* cc_nyq, R* gg,
                                                R* gg_nyq, int N, int L, double rho_bar, cudaStream_t s);

// Spectral step (positivity, steps IV-V, duals, pointwise part of b).
template <class R> cudaError_t launch_spectral(const R* X, R* GP, R* Sd, R* GV, R* GSd, R* b,
                                               const R* dctC, int N, int L, IterScalars<R> sc,
                                               double* partials, int resid, cudaStream_t s);
template <class R> int spectral_blocks(int N, int L);
// The spectral step with the Chebyshev basis in the dictionary (DCT too when dct_on), L <= 64.
template <class R> cudaError_t launch_spectral_b2(const R* X, R* GP, R* Sd, R* GV, R* GV2, R* GSd, R* S2, R* b,
                                                  const R* dctC, const R* Mb, int dct_on, int N, int L,
                                                  IterScalars<R> sc, double* partials, int resid, cudaStream_t s);
// S2 = M S^ (S in the second spectral basis) from the DCT-domain S, after the
// state was set from outside.
template <class R> cudaError_t launch_s2_from_sd(const R* Mb, const R* Sd, R* S2, int N, int L, cudaStream_t s);

// Wavelet analysis of the low-low band: LL_j (M/2 x M/2) from the M x M input.
template <class R> cudaError_t launch_wav_ll(const R* in, size_t in_band_stride, size_t in_basis_stride,
                                             R* out, int M, int L, int nd, const WavSet<R>* ws, cudaStream_t s);
// Fused level: analysis of the M x M input, thresholds and dual update of the level's
// coefficients, synthesis into the M x M output (or accumulation into b at level 1).
// pref_tile: preferred output tile edge (64 or 32) where the level is large enough.
// resid: 0 plain, 1 with the residual partials, 2 synthesis only (no input, no
// update): the level's coefficients are gt_old - gt_new, rcoarse the low-low
// band below the coarsest level; out receives the synthesis (level 1: added).
template <class R> cudaError_t launch_wav_level(const R* in, size_t in_band_stride, size_t in_basis_stride,
                                                const R* rcoarse, R* out, const R* gt_old, R* gt_new,
                                                int N, int M, int L, int coarsest, int nd, const WavSet<R>* ws,
                                                IterScalars<R> sc, double* partials, int resid, int pref_tile,
                                                int* err, cudaStream_t s);
template <class R> int wav_level_blocks(int M, int L, int nd, int pref_tile);
// Precision form of the spectral step: DCTs as split-BF16 tcgen05 products (L <= 64).
int spectral_tc_lp_of(int L);                        // padded L (16, 32, 48, 64) or 0
size_t spectral_tc_operand_elems(int L);             // BF16 elements of the DCT operands
void spectral_tc_build_operands(int L, uint16_t* out);  // host: C and C^T split hi/lo, core layout
// stall > 0: CTA 0 skips its product and waits at most stall cycles (test of the timeout path).
cudaError_t launch_spectral_tc(const float* X, float* GP, float* Sd, float* GV, float* GSd, float* b,
                               const uint16_t* bmats, int N, int L, IterScalars<float> sc, double* partials,
                               int resid, int* err, long long stall, cudaStream_t s);
int spectral_tc_blocks(int N);

// Copies the Daubechies tap tables into the wavelet kernels' constant memory
// (current device; the values are the same for every plan).
cudaError_t upload_taps();

// ifftshift of a PSF cube (peak from (N/2, N/2) to (0, 0)).
template <class R> cudaError_t launch_shift_psf(const R* psf, R* out, int N, size_t total, cudaStream_t s);

cudaError_t launch_finalize(const double* partials, int nblocks, double* sums, int accumulate, cudaStream_t s);

// Step I of a linear-convolution plan (cg.cu): transfer function and twiddles at
// 2N (plan creation), H^T y (per call), the conjugate gradient solve (per
// iteration) and the data-fit partials 1/2 ||y - H X||^2 (residual iterations).
cudaError_t linear_setup(mf_plan* p, const float* psf);
cudaError_t linear_hty(mf_plan* p, const float* y, cudaStream_t s);
cudaError_t linear_step_I(mf_plan* p, int cg_iters, double rho_bar, cudaStream_t s);
cudaError_t linear_fit(mf_plan* p, const float* y, double* partials, int* nblocks, cudaStream_t s);

// Visibility operator (vis.cu): plan-time Toeplitz kernels (into h2), the
// per-call dirty image Re(Phi^H W y) (into cgv) and 1/2 sum w |y|^2, and the
// data-fit partials from A X (residual iterations).
size_t vis_spec_elems(int N);
cudaError_t vis_setup(mf_plan* p, const int* counts);
cudaError_t vis_dirty(mf_plan* p, const float* y, cudaStream_t s);
cudaError_t vis_fit(mf_plan* p, const float* ax, double* partials, int* nblocks, cudaStream_t s);
cudaError_t vis_predict(mf_plan* p, const float* x, float* out, cudaStream_t s);

// Dual residual of residual iterations (dual.cu): cubes of p->dual, the
// snapshot taken before step I, and the reduction after the iteration.
size_t dual_cubes();
template <class R> cudaError_t dual_snapshot(mf_plan* p, cudaStream_t s);
// After the iteration: the spectral part of acc and ||dS||^2 (dual_spectral),
// the wavelet part added into acc by the level kernels' synthesis-only mode,
// then ||acc||^2 (dual_norm).
template <class R> cudaError_t dual_spectral(mf_plan* p, cudaStream_t s);
template <class R> R* dual_acc(mf_plan* p);
template <class R> cudaError_t dual_norm(mf_plan* p, cudaStream_t s);

}  // namespace mf
