/*
 * mf.h -- C ABI of the GB300 (sm_103a) spatio-spectral ADMM deconvolution
 * (Ferrari et al., arXiv:1504.06847, "Multi-frequency image reconstruction
 * for radio interferometry. A regularized inverse problem approach").
 *
 * Problem (Section 2, Eqs. nbmodel, wbmodel, costreg, eq:RegAll):
 *   y_l = H_l x_l + n_l for every band l = 0..L-1, H_l the circular
 *   convolution by band l's PSF, and
 *   min_X 1/2 ||Y - H X||^2 + 1_{R+}(X) + mu_eps/2 ||X||_F^2
 *         + mu_s ||W_s X||_1 + mu_nu ||X W_nu||_1,
 * solved by the ADMM of Section 3 (Algorithm 1, steps I-VI) with
 *   W_s  = union of orthonormal periodic 2-D wavelet bases (Db1..Db8 and Haar,
 *          Section 4), J levels of the separable Mallat transform;
 *   W_nu = orthonormal DCT-II along the band axis (Section 4), m_nu = 1;
 *   step I solved with the Fourier filter (|h_l|^2 + rho)^-1 (Section 3,
 *          Eq. Qlsimp, rho = mu_eps + rho_S + rho_P + n_s rho_T).
 *
 * Conventions shared by every entry point:
 *   - Cubes are [L][N][N] row-major (band images contiguous; a pixel spectrum
 *     has stride N*N), in the plan's real type (float, or double for the
 *     *_f64 plans).  Unless stated otherwise pointers are DEVICE pointers of
 *     the current CUDA device.
 *   - PSF: each band's PSF has its peak at pixel (N/2, N/2); the operator is
 *     (H x)[i] = sum_j psf[(i - j + N/2) mod N] x[j] in 2-D (circular), and H^T
 *     uses the conjugate transfer function.
 *   - N must be a power of two in [16, 2048]; L in [2, 128].  The wavelet
 *     levels J >= 1 with N / 2^J >= 2.
 *   - Asynchrony: iterate calls enqueue work on params->stream and return;
 *     the first error is latched in the plan and returned by later calls.
 *   - No C++ exception crosses this interface.
 */
#ifndef MF_H
#define MF_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mf_plan mf_plan;

typedef enum {
  MF_OK = 0,
  MF_ERR_INVALID = 1,   /* bad argument; nothing was enqueued */
  MF_ERR_OOM = 2,       /* device allocation failed */
  MF_ERR_CUDA = 3,      /* a CUDA call or launch failed */
  MF_ERR_TIMEOUT = 4,   /* a bounded device wait expired */
  MF_ERR_NONFINITE = 5, /* a NaN/Inf was seen by a residual reduction */
  MF_ERR_TOO_LARGE = 6  /* the cube exceeds MF_XSTEP_NOALLOC_MAX_VOXELS */
} mf_status;

typedef enum {
  MF_FP32 = 0,                 /* FP32 cube, FP32 DCT */
  MF_FP64 = 1,                 /* FP64 plan (created with mf_plan_create_f64) */
  MF_FP32_DCT_SPLITBF16 = 2    /* FP32 cube, DCT as split-BF16 tensor-core products (L <= 64) */
} mf_precision;

/* Regularisation and penalty parameters (Section 3 and the settings of Section 4). */
typedef struct {
  double mu_eps, mu_s, mu_nu;        /* mu_epsilon, mu_s, mu_nu (Eq. eq:RegAll) */
  double rho_P, rho_T, rho_V, rho_S; /* augmented Lagrangian penalties (Eqs. admm1/admm2) */
  int wavelet_levels;                /* J (default 3) */
  unsigned wavelet_mask;             /* bit K-1: DbK (K = 1..8); bit 8: Haar. default 0x1FF */
  int precision;                     /* mf_precision */
  int resid_every;                   /* 0: never; k: FP64 residuals/objective every k-th iteration
                                        and on the last one */
  int warm_start;                    /* 0: zero state first (Algorithm 1); 1: continue */
  void* stream;                      /* cudaStream_t; NULL = legacy default stream */
  int cg_iters;                      /* plans from mf_plan_create_linear and _vis: conjugate
                                        gradient iterations of step I per band (>= 1, default 20) */
  unsigned spectral_mask;            /* spectral dictionary W_nu, a union of orthonormal bases
                                        (step V divides by m_nu rho_V + rho_S): bit 0 the DCT,
                                        bit 1 the Chebyshev basis (mf_spectral_basis); default 1.
                                        Masks with bit 1 need L <= 64 and MF_FP32 or MF_FP64. */
} mf_params;

/* Filled by mf_plan_get_report, FP64 sums over the cube, measured after the
 * dual update of the last residual iteration (the residuals of the stopping
 * rule Section 3 takes from Boyd et al. 2011, Sec. 3.3, for the two-block
 * split (X, V) | (P, T, S) of Algorithm 1; d = change over that iteration):
 *   primal_res = ||P-X||^2 + ||T-W_s X||^2 + ||V-S W_nu||^2 + ||S-X||^2
 *              = sum_c ||dGamma_c||^2 / rho_c^2;
 *   dual_res   = ||rho_P dP + rho_T W_s^T dT + rho_S dS||^2 + rho_V^2 ||dS W_nu||^2;
 *   objective  = 1/2||Y-HX||^2 + mu_eps/2||X||^2 + mu_s||W_s X||_1 + mu_nu||X W_nu||_1;
 *   x_min      = min(X) (X may carry small negatives; P is its projection).
 * A plan's first call with resid_every > 0 allocates 3 more cubes for the
 * dual residual's snapshots and work array (kept until the plan is destroyed). */
typedef struct {
  int iters_done;
  int resid_iter;      /* iteration index the residual fields refer to (-1: none) */
  double primal_res;
  double dual_gamma;   /* sum_c ||dGamma_c||^2 (unweighted) */
  double objective;
  double x_min;
  double x_norm2;
  double dual_res;
} mf_report;

/* Defaults: mu_eps 0.001, mu_s 0.05, mu_nu 0.01, all rho 1, J 3, mask 0x1FF,
 * MF_FP32, resid_every 0, warm_start 0, stream NULL, cg_iters 20, spectral_mask 1. */
void mf_params_default(mf_params* p);

/* Creates a plan for N x N x L cubes.  psf_cube: device [L][N][N] float; it is
 * read during the call only (the plan keeps its transfer function).  On
 * success *out owns all device memory of the plan (see mf_plan_device_bytes).
 * Errors: MF_ERR_INVALID (sizes, NULL), MF_ERR_OOM, MF_ERR_CUDA. */
mf_status mf_plan_create(int N, int L, const float* psf_cube, mf_plan** out);
/* Same with an FP64 plan (all cubes double); L <= 64. */
mf_status mf_plan_create_f64(int N, int L, const double* psf_cube, mf_plan** out);

/* An FP32 plan whose H_l is the LINEAR ("same"-size) convolution by each
 * band's PSF -- (H x)[i] = sum_{j in [0,N)^2} psf[i - j + (N/2, N/2)] x[j], the
 * PSF zero outside its N x N support, no wrap-around -- for which
 * Q_l = H_l^T H_l + rho I (Eq. Qlsimp) is no longer a convolution.  Step I then
 * runs prm->cg_iters conjugate gradient iterations per band (the solver that
 * Algorithm 1's comment names), started from the previous X: H and H^T are
 * applied exactly through 2N x 2N FFTs (zero padding).  Every other step is as
 * in mf_plan_create; the report's data-fit term is formed in the image domain.
 * N is a power of two in [16, 1024].  The plan holds 17 cubes more than a
 * circular plan (transfer function and work arrays at 2N, the CG vectors).
 * mf_admm_backward rejects it.  Errors: MF_ERR_INVALID, MF_ERR_OOM, MF_ERR_CUDA. */
mf_status mf_plan_create_linear(int N, int L, const float* psf_cube, mf_plan** out);

/* An FP32 plan for the visibility-domain form of the model (Section 2, last
 * paragraph): y_l are the complex visibilities of band l and H_l maps the sky
 * to them,
 *   (Phi_l x)_m = sum_{r,c} x[r][c] exp(-2 pi i (u_m (c - N/2) + v_m (r - N/2)) / N),
 * with the data-fit term 1/2 sum_m w_m |y_m - (Phi_l x)_m|^2.  x being real,
 * Q_l = Re(Phi_l^H W Phi_l) + rho I (Eq. Qlsimp with H_l = Phi_l) and the
 * right-hand side of Eq. matB has Re(Phi_l^H W y_l) for H^T y.  Step I runs
 * prm->cg_iters conjugate gradient iterations per band from the previous X
 * (as for mf_plan_create_linear); Re(Phi^H W Phi) is applied as the Toeplitz
 * convolution it is (one 2N x 2N FFT round trip), whose kernel the plan
 * computes here by gridding (a type-1 non-uniform FFT, exponential-of-
 * semicircle kernel, width 8, oversampling 2); the dirty image Re(Phi^H W y)
 * is computed the same way at the start of every mf_admm_iterate call.
 *   n_vis   : host [L], visibilities per band (>= 0)
 *   uv      : device float [sum n_vis][2], (u_m, v_m) in cells of the N x N
 *             image's Fourier grid, band after band; |u|, |v| < N/2
 *   weights : device float [sum n_vis], w_m >= 0, or NULL (all 1)
 * Both are copied (the caller keeps its buffers).  mf_admm_iterate on this plan
 * takes y_cube = device float [sum n_vis][2], the complex visibilities
 * (re, im), in the same order.  N is a power of two in [16, 512].
 * The gridding adds the visibilities' contributions with FP32 atomics, so the
 * last bits of the Toeplitz kernel and of the dirty image (and of the X that
 * follows) depend on the order the additions land in: results agree to
 * rounding from run to run, not bit for bit (circular and linear plans are
 * bitwise reproducible).
 * mf_admm_backward rejects it.  Errors: MF_ERR_INVALID (sizes, NULL, a uv
 * point or weight out of range or not finite), MF_ERR_OOM, MF_ERR_CUDA. */
mf_status mf_plan_create_vis(int N, int L, const int* n_vis, const float* uv, const float* weights,
                             mf_plan** out);

/* Model visibilities of a plan from mf_plan_create_vis: vis_out = Phi_l x_l for
 * every band (the operator of mf_plan_create_vis, Section 2's last paragraph),
 * by a type-2 non-uniform FFT with the same gridding kernel: x divided by the
 * kernel's transform on the 2x oversampled grid, the grid's FFT, interpolation
 * at each uv point (about 1e-7 of sum |x| from the exact sum).
 *   x       : device float [L][N][N], or NULL for the plan's X
 *   vis_out : device float [sum n_vis][2] (re, im), the plan's visibility order
 *   stream  : cudaStream_t; the call first waits for the plan's last stream
 *             (it uses the plan's work arrays) and becomes the plan's stream
 * Asynchronous.  Errors: MF_ERR_INVALID (not a visibility plan, NULL vis_out),
 * the plan's latched status, MF_ERR_CUDA. */
mf_status mf_vis_predict(mf_plan* p, const float* x, float* vis_out, void* stream);
/* Frees everything the plan owns; NULL is a no-op.  Synchronises the device. */
void mf_plan_destroy(mf_plan* p);
size_t mf_plan_device_bytes(const mf_plan* p);

/* Runs n_iter >= 1 iterations of Algorithm 1 on the dirty cube y_cube
 * (device [L][N][N] float, read during the enqueued work; for a plan from
 * mf_plan_create_vis, the visibilities described there).  Constants
 * H^T y and the Fourier filter are recomputed on every call.  Returns
 * MF_ERR_INVALID for bad parameters (rho <= 0, mu < 0, J, mask, precision
 * not matching the plan), otherwise the plan's latched status. */
mf_status mf_admm_iterate(mf_plan* p, const float* y_cube, const mf_params* prm, int n_iter);
mf_status mf_admm_iterate_f64(mf_plan* p, const double* y_cube, const mf_params* prm, int n_iter);

/* Batched form: runs n_iter iterations of Algorithm 1 on each of `count`
 * independent FP32 plans (cubes of any N and L; no plan may appear twice),
 * plan i on the dirty cube y_cubes[i] (device pointers), as ONE CUDA graph
 * launch on prm->stream in which every cube is its own branch.  A call
 * identical to the previous batch call with the same plans[0] (same plans in
 * the same order, y pointers, n_iter, parameters and stream, plan options, and
 * each plan's Gamma_T buffer, which an odd n_iter swaps) relaunches the graph
 * captured then; any other call captures and instantiates a new graph (host
 * cost), which plans[0] keeps until its next batch call or its destruction.
 * The per-call constants (F(y), the filter, H^T y) are enqueued before the
 * graph on every call.  Per-plan results, state access and
 * reports are as after mf_admm_iterate.  Per-kernel event timing is suspended
 * inside the graph.  Errors: MF_ERR_INVALID, MF_ERR_CUDA (latched in every plan). */
mf_status mf_batch_iterate(mf_plan* const* plans, const float* const* y_cubes, int count, const mf_params* prm,
                           int n_iter);

/* Differentiable form (reverse mode of the unrolled iteration).  Runs n_iter
 * iterations of Algorithm 1 from the zero state on y_cube with the four
 * penalties tied (prm->rho_P = rho_T = rho_V = rho_S = rho; FP32 plan,
 * MF_FP32, L <= 64, warm_start 0), checkpointing every iteration, then sweeps
 * back: given dL_dX = dL/dX (device [L][N][N]) for the X of the last step I,
 * writes dL/dy into dL_dy (device [L][N][N]) and dL/dmu_s, dL/dmu_nu, dL/drho
 * into the host doubles (any may be NULL).  Subgradients: the derivative of
 * max(0, t) and of the soft threshold in t is 1 only where the inequality is
 * strict.  Needs device memory for the checkpoints ((5 + nd) cubes per
 * iteration) and (7 + 4 nd) work cubes (nd = distinct bases, at most 8): the
 * plan allocates it on the first call, keeps it for later calls, grows it
 * when a call needs more and frees it with the plan.  Synchronises
 * prm->stream before returning; afterwards the plan holds the forward's
 * final state.
 * Errors: MF_ERR_INVALID, MF_ERR_OOM, MF_ERR_CUDA. */
mf_status mf_admm_backward(mf_plan* p, const float* y_cube, const mf_params* prm, int n_iter, const float* dL_dX,
                           float* dL_dy, double* dL_dmu_s, double* dL_dmu_nu, double* dL_drho);

/* Which state array to read or write (all [L][N][N] unless noted). */
typedef enum {
  MF_ARR_X = 0,        /* X after the last step I (Algorithm 1 returns X) */
  MF_ARR_GAMMA_P = 1,  /* Gamma_P */
  MF_ARR_S_DCT = 2,    /* S W_nu: S in the DCT domain (row k = DCT frequency) */
  MF_ARR_GAMMA_V = 3,  /* Gamma_V (DCT domain) */
  MF_ARR_GAMMA_S_DCT = 4, /* Gamma_S W_nu */
  MF_ARR_B = 5,        /* right-hand side of Eq. matB without the H^T Y term */
  MF_ARR_GAMMA_T = 6,  /* Gamma_T: [nd][L][N][N], nd distinct bases in mask order
                          (Db1..Db8, Haar folded into Db1 when both are on),
                          each band in the in-place Mallat layout */
  MF_ARR_GAMMA_V2 = 7, /* Gamma_V of the Chebyshev spectral basis (its coefficient domain) */
  MF_ARR_HTY = 8       /* plans from mf_plan_create_linear / _vis: H^T y of the last call
                          (Re(Phi^H W y) for visibilities); get only */
} mf_array;

/* Device-to-device copies of a state array (dst/src: device, plan's real
 * type).  *count receives the element count when dst is NULL.  The copy runs
 * on the plan's last stream after its work and is complete on return. */
mf_status mf_plan_get_array(mf_plan* p, int which, void* dst, size_t* count);
mf_status mf_plan_set_array(mf_plan* p, int which, const void* src, size_t count);

/* Whole ADMM state (every array above, Gamma_V2 included) as one opaque device buffer for
 * checkpoint and warm restart.  With buf == NULL *bytes receives the size.  The
 * buffer does not record the dictionaries it was made with: after
 * mf_plan_set_state (into the same plan or a new one of the same N, L and type)
 * the next warm start continues with the wavelet and spectral dictionaries the
 * caller passes, which must be those the state was made with. */
mf_status mf_plan_get_state(mf_plan* p, void* buf, size_t* bytes);
mf_status mf_plan_set_state(mf_plan* p, const void* buf, size_t bytes);

/* Synchronises the plan's stream and fills *r.  Returns the latched status. */
mf_status mf_plan_get_report(mf_plan* p, mf_report* r);

/* Kernels of one iteration, for per-kernel timing and launch counts. */
typedef enum {
  MF_K_ROWS_FWD = 0,   /* step I: forward row FFT of b */
  MF_K_COLS = 1,       /* step I: column FFT, Fourier-diagonal divide, inverse column FFT */
  MF_K_ROWS_INV = 2,   /* step I: inverse row FFT into X */
  MF_K_SPECTRAL = 3,   /* steps II, IV, V and their duals, pointwise part of b */
  MF_K_WAV_LL = 4,     /* step III: low-low analysis of the coarser levels */
  MF_K_WAV_LEVEL1 = 5, /* step III: finest level, every basis, adds into b */
  MF_K_WAV_LEVELJ = 6, /* step III: coarser fused levels */
  MF_K_SETUP = 7,      /* per-call constants: F(y), g, c; zeroing of the state */
  MF_K_REDUCE = 8,     /* FP64 fold of the residual partials */
  MF_K_DUAL = 9,       /* dual residual: snapshot before step I, reduction after the iteration */
  MF_K_CG = 10,        /* step I of a linear or visibility plan: conjugate gradients, 2N FFTs */
  MF_K_COUNT = 11
} mf_kernel;

/* Per-kernel CUDA-event timing of the plan's launches on its stream (off by
 * default; each timed launch is bracketed by two events).  Enabling resets the
 * accumulators.  mf_plan_get_timing synchronises the stream and returns, for
 * one kernel, the summed duration in ms (0 when timing is off) and the launch
 * count (always counted since the plan was created or timing was enabled). */
mf_status mf_plan_set_timing(mf_plan* p, int enable);
mf_status mf_plan_get_timing(mf_plan* p, int kernel, double* total_ms, long long* launches);
const char* mf_kernel_name(int kernel);

/* Options of a plan (each call synchronises the plan's last stream).
 *   MF_OPT_WAV_TILE: output tile edge of the fused wavelet level kernels,
 *                    64 (default of FP32 plans) or 32 (default of FP64 plans,
 *                    whose 64-wide kernels spill registers); levels smaller than the tile use
 *                    the largest tile that fits.  Launch shape only: every
 *                    value computes the same arithmetic per element in the
 *                    same order, so results are bitwise identical.
 *   MF_OPT_TEST_TC_STALL: for tests of the failure path only.  A value v > 0
 *                    makes CTA 0 of every later split-BF16 spectral launch
 *                    skip its tensor-core product and its commit and give
 *                    up on the completion wait after v SM cycles, with
 *                    nothing in flight: the kernel records the expiry in the
 *                    plan's device error word, frees its tensor memory and
 *                    returns, and mf_plan_get_report returns MF_ERR_TIMEOUT.
 *                    0 (default) turns it off. */
typedef enum { MF_OPT_WAV_TILE = 0, MF_OPT_TEST_TC_STALL = 1 } mf_option;
mf_status mf_plan_set_option(mf_plan* p, int option, int value);

/* Synchronises the plan's last stream and clears its latched status and device
 * error word, so that a plan whose bounded device wait expired (or whose
 * reduction saw a non-finite value) accepts work again.  The state arrays may
 * be inconsistent after such a failure: restart from the zero state
 * (warm_start = 0) or restore a saved state. */
mf_status mf_plan_clear_status(mf_plan* p);

/* Host copy (row-major L x L, double) of a basis of the spectral dictionary:
 * MF_SPECTRAL_DCT, the orthonormal DCT-II (row k = frequency k), or
 * MF_SPECTRAL_CHEBYSHEV, the Chebyshev polynomials Section 4 suggests, made
 * orthonormal on the L equispaced bands (the discrete Chebyshev / Gram
 * polynomials; row n = degree n, positive leading coefficient), computed as
 * the eigenvectors of their difference equation.  2 <= L <= 64. */
typedef enum { MF_SPECTRAL_DCT = 0, MF_SPECTRAL_CHEBYSHEV = 1 } mf_spectral;
mf_status mf_spectral_basis(int kind, int L, double* out);

/* Host copy of the library's low-pass filter DbK (K = 1..8, 2K taps, double),
 * built at load time from Daubechies' spectral factorisation. */
mf_status mf_wavelet_filter(int K, double* taps_host, int* len);

const char* mf_status_string(mf_status s);

/*
 * Spectral-index map (the post-processing of the paper's first simulation,
 * Section 4): every pixel spectrum of cube is fitted, in a log scale, by the
 * second-order power law
 *   log S(nu) = c + alpha log(nu/nu0) + beta log^2(nu/nu0)
 * by least squares over the L >= 3 bands.
 *   cube       : device [L][N][N] float (e.g. X after mf_admm_iterate)
 *   nu         : host, L band frequencies (> 0, at least 3 distinct); nu0 > 0
 *   floor      : a pixel with any S(nu_l) <= floor has no log-scale fit and
 *                gets NaN in all three outputs
 *   c0_out, alpha_out, beta_out : device [N][N] float outputs (any may be NULL,
 *                not all)
 *   stream     : cudaStream_t (NULL = legacy default); the call enqueues one
 *                kernel and returns.
 * Errors: MF_ERR_INVALID (sizes, frequencies), MF_ERR_CUDA.
 */
mf_status mf_spectral_index(int N, int L, const float* cube, const double* nu, double nu0, float floor,
                            float* c0_out, float* alpha_out, float* beta_out, void* stream);

/*
 * Step I without any allocation: x = (H^T H + rho I)^-1 (H^T y + b) per band,
 * rho = mu_eps + rho_S + rho_P + n_s rho_T with n_s the number of bases in
 * prm->wavelet_mask -- the same solve, on the same kernels, as the first step
 * of an mf_admm_iterate iteration whose right-hand side (MF_ARR_B) is b.
 *
 * The paper has no counterpart: this entry point exists for callers that may
 * not allocate device memory at all -- code running where cudaMalloc is
 * unavailable or forbidden (inside another library's allocator hook, under a
 * caller-owned memory pool or budget, or a real-time path that must not block
 * on the allocator).  Plans need cudaMalloc; this call does not.  Its working memory is one file-scope static __device__
 * array of about 10.4 MB (MF_XSTEP_NOALLOC_MAX_VOXELS = 2^19 voxels:
 * e.g. 256 x 256 x 8 or 128 x 128 x 32), which every GPU that loads the
 * library holds until the process exits.  Larger cubes return
 * MF_ERR_TOO_LARGE before any device work.
 *
 *   psf_cube, y_cube, b_cube : device [L][N][N] float inputs (read only)
 *   x_out                    : device [L][N][N] float output, written by the
 *                              last kernel only, so it may alias psf_cube,
 *                              y_cube or b_cube (an in-place solve)
 *   prm                      : mu_eps, rho_P, rho_T, rho_S, wavelet_mask and
 *                              stream are read; other fields are ignored.
 * All pointers belong to the current device.  The first call on a device
 * looks up the static array's device address (cudaGetSymbolAddress) with
 * that device current and keeps it; make that first call before any stream
 * capture, and do not use this entry point on a device after a
 * cudaDeviceReset of it (the kept address is then stale).  Every call shares
 * the one array, which keeps the last call's contents (each call overwrites
 * everything it reads), so calls whose work overlaps on the GPU -- on
 * different streams or host threads -- race; serialise them.  The call copies
 * nothing from the host: it enqueues kernels on prm->stream and returns;
 * errors: MF_ERR_INVALID, MF_ERR_TOO_LARGE, MF_ERR_CUDA.
 */
#define MF_XSTEP_NOALLOC_MAX_VOXELS (1u << 19)
mf_status mf_xstep_noalloc(int N, int L, const float* psf_cube, const float* y_cube, const float* b_cube,
                           const mf_params* prm, float* x_out);

#ifdef __cplusplus
}
#endif
#endif /* MF_H */
