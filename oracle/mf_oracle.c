/*
 * FP64 CPU oracle for the spatio-spectral ADMM deconvolution of
 * Ferrari et al., "Multi-frequency image reconstruction for radio
 * interferometry. A regularized inverse problem approach" (arXiv:1504.06847).
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg load this library.  It shares no code with the CUDA path.
 *
 * It is a plain, slow transcription of Algorithm 1 (Section 3) in IEEE
 * double precision, built without fast-math and without FMA contraction:
 *
 *   repeat
 *     for every band l:  b_l from Eq. matB,  solve Q_l x_l = b_l  (Eq. linsystemX,
 *                        Q_l = H_l^T H_l + rho I by Eq. Qlsimp, solved with the
 *                        Fourier filter (|h_l|^2 + rho)^-1 of Section 3)
 *     P <- max(0, X - Gamma_P / rho_P)                          (step II)
 *     T <- S_{mu_s/rho_T}(W_s X - Gamma_T / rho_T)              (step III)
 *     V <- S_{mu_nu/rho_V}(S W_nu - Gamma_V / rho_V)   old S    (step IV)
 *     S <- ((Gamma_V + rho_V V) W_nu^T - Gamma_S + rho_S X)
 *          / (m_nu rho_V + rho_S)                               (step V)
 *     Gamma_P += rho_P (P - X);  Gamma_T += rho_T (T - W_s X);
 *     Gamma_V += rho_V (V - S W_nu);  Gamma_S += rho_S (S - X)  (step VI)
 *
 * Readings where the paper is silent:
 *   - H_l is a circular convolution by the band's PSF, whose peak sits at
 *     pixel (N/2, N/2): (H x)[i] = sum_j psf[(i - j + N/2) mod N] x[j].
 *   - W_s is the union of nb orthonormal periodic 2-D wavelet bases; each is
 *     the separable Mallat transform with J levels (rows and columns of the
 *     current approximation block at each level), analysis
 *     a_i = sum_n h_n x[(2i+n) mod M], d_i = sum_n g_n x[(2i+n) mod M],
 *     g_n = (-1)^n h_{F-1-n}.  Coefficients are stored in place: after a level
 *     on the top-left M x M block, column c < M/2 of a row holds the low-pass
 *     output and c >= M/2 the high-pass output (and likewise for rows).
 *   - W_nu is the orthonormal DCT-II along the band axis, so m_nu = 1:
 *     (X W_nu)[k] = sum_l C[k][l] X[l] with C[k][l] = a_k cos(pi (2l+1) k / (2L)).
 *   - S_r(0) = 0.
 *   - Two other forms of H_l, each with step I by conjugate gradients (the
 *     solver Algorithm 1's comment names): the linear ("same"-size)
 *     convolution by the PSF, and the operator from the sky to sampled
 *     visibilities of Section 2's last paragraph (both described below).
 *
 * Layout: every cube is [L][N][N] row-major; the wavelet-domain arrays T and
 * Gamma_T are [nb][L][N][N] (basis-major), each band in the in-place layout above.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define ORC_MAXF 16
#define ORC_MAXB 16

/* ------------------------------------------------------------------------ */
/* FFT: iterative radix-2 Cooley-Tukey, unnormalised, sign -1 forward.       */
/* ------------------------------------------------------------------------ */

static void fft_line(double* re, double* im, int n, int inverse,
                     const double* twr, const double* twi) {
  for (int i = 1, j = 0; i < n; i++) {
    int bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) {
      double t = re[i]; re[i] = re[j]; re[j] = t;
      t = im[i]; im[i] = im[j]; im[j] = t;
    }
  }
  for (int len = 2; len <= n; len <<= 1) {
    int half = len >> 1, step = n / len;
    for (int i = 0; i < n; i += len) {
      for (int k = 0; k < half; k++) {
        double wr = twr[k * step];
        double wi = inverse ? -twi[k * step] : twi[k * step];
        int a = i + k, b = i + k + half;
        double vr = re[b] * wr - im[b] * wi;
        double vi = re[b] * wi + im[b] * wr;
        re[b] = re[a] - vr; im[b] = im[a] - vi;
        re[a] = re[a] + vr; im[a] = im[a] + vi;
      }
    }
  }
}

static void twiddles(int n, double* twr, double* twi) {
  for (int k = 0; k < n / 2; k++) {
    twr[k] = cos(2.0 * M_PI * (double)k / (double)n);
    twi[k] = -sin(2.0 * M_PI * (double)k / (double)n);
  }
}

/* In-place 2-D DFT of one N x N complex image (rows, then columns). */
static void fft2_image(double* re, double* im, int N, int inverse,
                       const double* twr, const double* twi, double* lr, double* li) {
  for (int r = 0; r < N; r++) fft_line(re + (long)r * N, im + (long)r * N, N, inverse, twr, twi);
  for (int c = 0; c < N; c++) {
    for (int r = 0; r < N; r++) { lr[r] = re[(long)r * N + c]; li[r] = im[(long)r * N + c]; }
    fft_line(lr, li, N, inverse, twr, twi);
    for (int r = 0; r < N; r++) { re[(long)r * N + c] = lr[r]; im[(long)r * N + c] = li[r]; }
  }
}

/* Exported: 2-D DFT of `count` N x N images, in place.  sign -1 forward,
 * +1 inverse (unnormalised). */
void orc_fft2(double* re, double* im, int N, int count, int sign) {
  double* twr = malloc(sizeof(double) * (N / 2 + 1));
  double* twi = malloc(sizeof(double) * (N / 2 + 1));
  twiddles(N, twr, twi);
#pragma omp parallel for schedule(dynamic, 1)
  for (int i = 0; i < count; i++) {
    double* lr = malloc(sizeof(double) * N);
    double* li = malloc(sizeof(double) * N);
    fft2_image(re + (long)i * N * N, im + (long)i * N * N, N, sign > 0, twr, twi, lr, li);
    free(lr); free(li);
  }
  free(twr); free(twi);
}

/* ------------------------------------------------------------------------ */
/* Periodic orthonormal wavelet transform.                                  */
/* ------------------------------------------------------------------------ */

static double hp_tap(const double* h, int F, int n) {
  double v = h[F - 1 - n];
  return (n & 1) ? -v : v;
}

/* a_i = sum_n h_n x[(2i+n) mod M],  d_i = sum_n g_n x[(2i+n) mod M]. */
static void dwt1_analysis(const double* x, int M, double* a, double* d, const double* h, int F) {
  for (int i = 0; i < M / 2; i++) {
    double sa = 0.0, sd = 0.0;
    for (int n = 0; n < F; n++) {
      double v = x[(2 * i + n) % M];
      sa += h[n] * v;
      sd += hp_tap(h, F, n) * v;
    }
    a[i] = sa;
    d[i] = sd;
  }
}

/* The transpose of dwt1_analysis: every (i, n) term sends its weight back to
 * the sample it was read from. */
static void dwt1_synthesis(const double* a, const double* d, int M, double* x, const double* h, int F) {
  for (int m = 0; m < M; m++) x[m] = 0.0;
  for (int i = 0; i < M / 2; i++) {
    for (int n = 0; n < F; n++) {
      x[(2 * i + n) % M] += h[n] * a[i] + hp_tap(h, F, n) * d[i];
    }
  }
}

/* One 2-D level on the top-left M x M block of an N x N image: every row,
 * then every column.  buf holds 2M doubles. */
static void level_analysis(double* img, int N, int M, const double* h, int F, double* buf) {
  double* line = buf;
  double* out = buf + M;
  for (int r = 0; r < M; r++) {
    double* row = img + (long)r * N;
    memcpy(line, row, sizeof(double) * M);
    dwt1_analysis(line, M, out, out + M / 2, h, F);
    memcpy(row, out, sizeof(double) * M);
  }
  for (int c = 0; c < M; c++) {
    for (int r = 0; r < M; r++) line[r] = img[(long)r * N + c];
    dwt1_analysis(line, M, out, out + M / 2, h, F);
    for (int r = 0; r < M; r++) img[(long)r * N + c] = out[r];
  }
}

/* Transpose of level_analysis: columns back first, then rows. */
static void level_synthesis(double* img, int N, int M, const double* h, int F, double* buf) {
  double* line = buf;
  double* out = buf + M;
  for (int c = 0; c < M; c++) {
    for (int r = 0; r < M; r++) line[r] = img[(long)r * N + c];
    dwt1_synthesis(line, line + M / 2, M, out, h, F);
    for (int r = 0; r < M; r++) img[(long)r * N + c] = out[r];
  }
  for (int r = 0; r < M; r++) {
    double* row = img + (long)r * N;
    memcpy(line, row, sizeof(double) * M);
    dwt1_synthesis(line, line + M / 2, M, out, h, F);
    memcpy(row, out, sizeof(double) * M);
  }
}

/* z = W x for one N x N image, J levels. */
static void dwt2(const double* x, double* z, int N, int J, const double* h, int F, double* buf) {
  memcpy(z, x, sizeof(double) * N * N);
  for (int j = 1; j <= J; j++) level_analysis(z, N, N >> (j - 1), h, F, buf);
}

/* x = W^T z for one N x N image, J levels. */
static void idwt2(const double* z, double* x, int N, int J, const double* h, int F, double* buf) {
  memcpy(x, z, sizeof(double) * N * N);
  for (int j = J; j >= 1; j--) level_synthesis(x, N, N >> (j - 1), h, F, buf);
}

/* Exported: `count` images, analysis (dir = +1) or synthesis (dir = -1). */
void orc_dwt2(const double* in, double* out, int N, int count, int J,
              const double* h, int F, int dir) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int i = 0; i < count; i++) {
    double* buf = malloc(sizeof(double) * 2 * N);
    if (dir > 0) dwt2(in + (long)i * N * N, out + (long)i * N * N, N, J, h, F, buf);
    else idwt2(in + (long)i * N * N, out + (long)i * N * N, N, J, h, F, buf);
    free(buf);
  }
}

/* ------------------------------------------------------------------------ */
/* DCT-II (orthonormal) along the band axis.                                 */
/* ------------------------------------------------------------------------ */

void orc_dct_matrix(int L, double* C) {
  for (int k = 0; k < L; k++) {
    double a = (k == 0) ? sqrt(1.0 / L) : sqrt(2.0 / L);
    for (int l = 0; l < L; l++) C[k * L + l] = a * cos(M_PI * (2.0 * l + 1.0) * k / (2.0 * L));
  }
}

/* ------------------------------------------------------------------------ */
/* Problem description.                                                      */
/* ------------------------------------------------------------------------ */

#define ORC_MAXNU 4

/* The spectral dictionary W_nu is a union of m_nu orthonormal bases (Section
 * 3, step V: W_nu W_nu^T = m_nu I): Cnu holds m_nu L x L matrices, basis j's
 * coefficient k of a spectrum s being sum_l Cnu[(j L + k) L + l] s[l].  V and
 * Gamma_V are [m_nu][L][N][N]. */
typedef struct {
  int N, L, J, nb;
  int F[ORC_MAXB];
  double h[ORC_MAXB][ORC_MAXF];
  double mu_eps, mu_s, mu_nu, rho_P, rho_T, rho_V, rho_S;
  int mnu;
  const double* Cnu;
} problem;

static int load_problem(problem* pb, int N, int L, int J, int nb, const int* F,
                        const double* h, const double* prm) {
  if (nb < 1 || nb > ORC_MAXB) return 1;
  pb->N = N; pb->L = L; pb->J = J; pb->nb = nb;
  for (int k = 0; k < nb; k++) {
    if (F[k] < 2 || F[k] > ORC_MAXF || (F[k] & 1)) return 1;
    pb->F[k] = F[k];
    for (int n = 0; n < ORC_MAXF; n++) pb->h[k][n] = h[k * ORC_MAXF + n];
  }
  pb->mu_eps = prm[0]; pb->mu_s = prm[1]; pb->mu_nu = prm[2];
  pb->rho_P = prm[3]; pb->rho_T = prm[4]; pb->rho_V = prm[5]; pb->rho_S = prm[6];
  /* prm[7] = m_nu, then the m_nu spectral basis matrices (L x L each) */
  pb->mnu = (int)prm[7];
  if (pb->mnu < 1 || pb->mnu > ORC_MAXNU) return 1;
  pb->Cnu = prm + 8;
  return 0;
}

static double soft(double t, double r) {
  /* S_r(t) = t max(0, 1 - r/|t|), with S_r(0) = 0 */
  if (t == 0.0) return 0.0;
  double f = 1.0 - r / fabs(t);
  return f > 0.0 ? t * f : 0.0;
}

/* ------------------------------------------------------------------------ */
/* Set-up: hhat = F(ifftshift(psf)),  yhat = F(y),  H^T y.                   */
/* ------------------------------------------------------------------------ */

int orc_setup(int N, int L, const double* psf, const double* y,
              double* hre, double* him, double* yre, double* yim, double* HtY) {
  long NN = (long)N * N;
  for (int l = 0; l < L; l++) {
    for (int r = 0; r < N; r++)
      for (int c = 0; c < N; c++) {
        /* h[r][c] = psf[(r + N/2) mod N][(c + N/2) mod N] (peak moved to (0,0)) */
        hre[l * NN + (long)r * N + c] = psf[l * NN + (long)((r + N / 2) % N) * N + (c + N / 2) % N];
        him[l * NN + (long)r * N + c] = 0.0;
        yre[l * NN + (long)r * N + c] = y[l * NN + (long)r * N + c];
        yim[l * NN + (long)r * N + c] = 0.0;
      }
  }
  orc_fft2(hre, him, N, L, -1);
  orc_fft2(yre, yim, N, L, -1);
  /* H^T y = F^-1(conj(hhat) yhat) / N^2 */
  double* tr = malloc(sizeof(double) * NN * L);
  double* ti = malloc(sizeof(double) * NN * L);
  for (long i = 0; i < NN * L; i++) {
    tr[i] = hre[i] * yre[i] + him[i] * yim[i];
    ti[i] = hre[i] * yim[i] - him[i] * yre[i];
  }
  orc_fft2(tr, ti, N, L, +1);
  for (long i = 0; i < NN * L; i++) HtY[i] = tr[i] / (double)NN;
  free(tr); free(ti);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Step I: b from Eq. matB, then x_l = Q_l^-1 b_l.                           */
/* ------------------------------------------------------------------------ */

/* b = H^T Y + W_s^T (Gamma_T + rho_T T) + Gamma_P + rho_P P + Gamma_S + rho_S S */
static void make_b(const problem* pb, const double* HtY, const double* P, const double* T,
                   const double* S, const double* GP, const double* GT, const double* GS,
                   double* b) {
  int N = pb->N, L = pb->L;
  long NN = (long)N * N;
#pragma omp parallel for schedule(dynamic, 1)
  for (int l = 0; l < L; l++) {
    double* u = malloc(sizeof(double) * NN);
    double* w = malloc(sizeof(double) * NN);
    double* buf = malloc(sizeof(double) * 2 * N);
    double* bl = b + l * NN;
    for (long i = 0; i < NN; i++) {
      long q = l * NN + i;
      bl[i] = HtY[q] + GP[q] + pb->rho_P * P[q] + GS[q] + pb->rho_S * S[q];
    }
    for (int k = 0; k < pb->nb; k++) {
      long off = ((long)k * L + l) * NN;
      for (long i = 0; i < NN; i++) u[i] = GT[off + i] + pb->rho_T * T[off + i];
      idwt2(u, w, N, pb->J, pb->h[k], pb->F[k], buf);
      for (long i = 0; i < NN; i++) bl[i] += w[i];
    }
    free(u); free(w); free(buf);
  }
}

static double rho_bar(const problem* pb) {
  /* Eq. Qlsimp: rho = mu_eps + rho_S + rho_P + n_s rho_T */
  return pb->mu_eps + pb->rho_S + pb->rho_P + pb->nb * pb->rho_T;
}

/* x_l = F^-1( F(b_l) / (|hhat_l|^2 + rho) ) / N^2.  If dfit is not NULL it
 * receives per band 1/2 ||y_l - H_l x_l||^2 (Parseval). */
static void solve_x(const problem* pb, const double* hre, const double* him,
                    const double* yre, const double* yim, const double* b, double* X,
                    double* dfit) {
  int N = pb->N, L = pb->L;
  long NN = (long)N * N;
  double rho = rho_bar(pb);
  double* twr = malloc(sizeof(double) * (N / 2 + 1));
  double* twi = malloc(sizeof(double) * (N / 2 + 1));
  twiddles(N, twr, twi);
#pragma omp parallel for schedule(dynamic, 1)
  for (int l = 0; l < L; l++) {
    double* re = malloc(sizeof(double) * NN);
    double* im = malloc(sizeof(double) * NN);
    double* lr = malloc(sizeof(double) * N);
    double* li = malloc(sizeof(double) * N);
    for (long i = 0; i < NN; i++) { re[i] = b[l * NN + i]; im[i] = 0.0; }
    fft2_image(re, im, N, 0, twr, twi, lr, li);
    double fit = 0.0;
    for (long i = 0; i < NN; i++) {
      long q = l * NN + i;
      double den = hre[q] * hre[q] + him[q] * him[q] + rho;
      re[i] /= den;
      im[i] /= den;
      if (dfit) {
        double rr = yre[q] - (hre[q] * re[i] - him[q] * im[i]);
        double ri = yim[q] - (hre[q] * im[i] + him[q] * re[i]);
        fit += rr * rr + ri * ri;
      }
    }
    if (dfit) dfit[l] = 0.5 * fit / (double)NN;
    fft2_image(re, im, N, 1, twr, twi, lr, li);
    for (long i = 0; i < NN; i++) X[l * NN + i] = re[i] / (double)NN;
    free(re); free(im); free(lr); free(li);
  }
  free(twr); free(twi);
}

/* ------------------------------------------------------------------------ */
/* Step I for a non-circulant H: linear convolution and conjugate gradients. */
/* ------------------------------------------------------------------------ */

/*
 * Reading for a PSF that does not wrap around the image: H_l is the linear
 * ("same"-size) 2-D convolution
 *   (H x)[i] = sum_{j in [0,N)^2} psf[i - j + (N/2, N/2)] x[j],  psf = 0 outside [0,N)^2,
 * and Q_l = H_l^T H_l + rho I is no longer a convolution, so step I is solved
 * with the conjugate gradient algorithm that Algorithm 1's comment names
 * (Hestenes-Stiefel), one system per band, started from the previous X and
 * run for a fixed number of iterations.  H and H^T are applied exactly through
 * a 2N x 2N FFT: with x embedded at [0,N)^2 and the PSF at offsets
 * (u - N/2) mod 2N, the circular convolution of size 2N has no wrap-around on
 * the cropped [0,N)^2 output.
 */
/*
 * Visibility-domain operator (Section 2, last paragraph: y_l are the sampled
 * visibilities and H_l maps the sky to them).  Reading: band l has the
 * visibilities m in [voff[l], voff[l+1]) at uv coordinates (u_m, v_m), in
 * cells of the N x N image's Fourier grid, with weights w_m >= 0, and
 *   (Phi_l x)_m = sum_{r,c} x[r][c] exp(-2 pi i (u_m (c - N/2) + v_m (r - N/2)) / N)
 * (phase centre at pixel (N/2, N/2), column index along u).  The data-fit term
 * is 1/2 sum_m w_m |y_m - (Phi_l x)_m|^2 and, x being real, step I's matrix is
 * Q_l = Re(Phi_l^H W Phi_l) + rho I with right-hand side Re(Phi_l^H W y_l) + b_l.
 */
typedef struct {
  const int* voff;     /* [L+1] */
  const double* u;     /* [voff[L]] uv coordinates, cells */
  const double* v;
  const double* w;     /* weights */
  const double* yre;   /* visibilities */
  const double* yim;
} vis_data;

typedef struct {
  const double* h2re;  /* [L][2N][2N] transfer function of the embedded PSF */
  const double* h2im;
  const double* y;     /* dirty cube [L][N][N], for the data-fit term */
  int cg_iters;
  const vis_data* vis; /* not NULL: H_l is the visibility operator instead */
} lin_op;

/* out = H x (adjoint = 0) or H^T x (adjoint = 1) for one band; buffers re, im hold (2N)^2 each. */
static void lin_apply_band(int N, const double* h2re, const double* h2im, const double* x, double* out, int adjoint,
                           double* re, double* im, const double* twr, const double* twi, double* lr, double* li) {
  int M = 2 * N;
  long MM = (long)M * M;
  for (long i = 0; i < MM; i++) { re[i] = 0.0; im[i] = 0.0; }
  for (int r = 0; r < N; r++)
    for (int c = 0; c < N; c++) re[(long)r * M + c] = x[(long)r * N + c];
  fft2_image(re, im, M, 0, twr, twi, lr, li);
  for (long i = 0; i < MM; i++) {
    double hr = h2re[i], hi = adjoint ? -h2im[i] : h2im[i];
    double vr = re[i] * hr - im[i] * hi;
    double vi = re[i] * hi + im[i] * hr;
    re[i] = vr;
    im[i] = vi;
  }
  fft2_image(re, im, M, 1, twr, twi, lr, li);
  for (int r = 0; r < N; r++)
    for (int c = 0; c < N; c++) out[(long)r * N + c] = re[(long)r * M + c] / (double)MM;
}

/* Transfer functions of the embedded PSFs and H^T y. */
int orc_linear_setup(int N, int L, const double* psf, const double* y, double* h2re, double* h2im, double* HtY) {
  int M = 2 * N;
  long MM = (long)M * M, NN = (long)N * N;
  for (long i = 0; i < MM * L; i++) { h2re[i] = 0.0; h2im[i] = 0.0; }
  for (int l = 0; l < L; l++)
    for (int u = 0; u < N; u++)
      for (int v = 0; v < N; v++) {
        int r = ((u - N / 2) % M + M) % M, c = ((v - N / 2) % M + M) % M;
        h2re[l * MM + (long)r * M + c] = psf[l * NN + (long)u * N + v];
      }
  orc_fft2(h2re, h2im, M, L, -1);
  double* twr = malloc(sizeof(double) * (M / 2 + 1));
  double* twi = malloc(sizeof(double) * (M / 2 + 1));
  twiddles(M, twr, twi);
#pragma omp parallel for schedule(dynamic, 1)
  for (int l = 0; l < L; l++) {
    double *re = malloc(sizeof(double) * MM), *im = malloc(sizeof(double) * MM);
    double *lr = malloc(sizeof(double) * M), *li = malloc(sizeof(double) * M);
    lin_apply_band(N, h2re + l * MM, h2im + l * MM, y + l * NN, HtY + l * NN, 1, re, im, twr, twi, lr, li);
    free(re); free(im); free(lr); free(li);
  }
  free(twr); free(twi);
  return 0;
}

/* H x (adjoint 0) or H^T x (adjoint 1) for every band. */
void orc_linear_apply(int N, int L, const double* h2re, const double* h2im, const double* x, double* out,
                      int adjoint) {
  int M = 2 * N;
  long MM = (long)M * M, NN = (long)N * N;
  double* twr = malloc(sizeof(double) * (M / 2 + 1));
  double* twi = malloc(sizeof(double) * (M / 2 + 1));
  twiddles(M, twr, twi);
#pragma omp parallel for schedule(dynamic, 1)
  for (int l = 0; l < L; l++) {
    double *re = malloc(sizeof(double) * MM), *im = malloc(sizeof(double) * MM);
    double *lr = malloc(sizeof(double) * M), *li = malloc(sizeof(double) * M);
    lin_apply_band(N, h2re + l * MM, h2im + l * MM, x + l * NN, out + l * NN, adjoint, re, im, twr, twi, lr, li);
    free(re); free(im); free(lr); free(li);
  }
  free(twr); free(twi);
}

/* e^{-2 pi i f (n - N/2) / N} for n in [0, N): the phases of one uv coordinate f along a pixel axis */
static void vis_phases(int N, double f, double* cr, double* ci) {
  for (int n = 0; n < N; n++) {
    double a = -2.0 * M_PI * f * (double)(n - N / 2) / (double)N;
    cr[n] = cos(a);
    ci[n] = sin(a);
  }
}

/* t = Phi_l x for band l (t indexed from the band's first visibility); buf holds 4N doubles */
static void vis_forward_band(int N, const vis_data* vd, int l, const double* x, double* tre, double* tim,
                             double* buf) {
  double *exr = buf, *exi = buf + N, *eyr = buf + 2 * N, *eyi = buf + 3 * N;
  for (int m = vd->voff[l]; m < vd->voff[l + 1]; m++) {
    vis_phases(N, vd->u[m], exr, exi);
    vis_phases(N, vd->v[m], eyr, eyi);
    double sr = 0.0, si = 0.0;
    for (int r = 0; r < N; r++) {
      double ar = 0.0, ai = 0.0; /* sum over the row of x[r][c] e_u[c] */
      for (int c = 0; c < N; c++) {
        ar += x[(long)r * N + c] * exr[c];
        ai += x[(long)r * N + c] * exi[c];
      }
      sr += ar * eyr[r] - ai * eyi[r];
      si += ar * eyi[r] + ai * eyr[r];
    }
    tre[m - vd->voff[l]] = sr;
    tim[m - vd->voff[l]] = si;
  }
}

/* out = Re(Phi_l^H W z) for band l (z indexed from the band's first visibility) */
static void vis_adjoint_band(int N, const vis_data* vd, int l, const double* zre, const double* zim, double* out,
                             double* buf) {
  double *exr = buf, *exi = buf + N, *eyr = buf + 2 * N, *eyi = buf + 3 * N;
  for (long i = 0; i < (long)N * N; i++) out[i] = 0.0;
  for (int m = vd->voff[l]; m < vd->voff[l + 1]; m++) {
    vis_phases(N, vd->u[m], exr, exi);
    vis_phases(N, vd->v[m], eyr, eyi);
    double wt = vd->w ? vd->w[m] : 1.0;
    double cr = wt * zre[m - vd->voff[l]], ci = wt * zim[m - vd->voff[l]];
    for (int r = 0; r < N; r++) {
      /* a + ib = w z conj(e_v[r]); out[r][c] += Re((a + ib) conj(e_u[c])) */
      double a = cr * eyr[r] + ci * eyi[r];
      double b = ci * eyr[r] - cr * eyi[r];
      for (int c = 0; c < N; c++) out[(long)r * N + c] += a * exr[c] + b * exi[c];
    }
  }
}

static int vis_max_count(const vis_data* vd, int L) {
  int mx = 1;
  for (int l = 0; l < L; l++)
    if (vd->voff[l + 1] - vd->voff[l] > mx) mx = vd->voff[l + 1] - vd->voff[l];
  return mx;
}

/* HtY = Re(Phi^H W y) for every band. */
int orc_vis_setup(int N, int L, const int* voff, const double* u, const double* v, const double* w,
                  const double* yre, const double* yim, double* HtY) {
  vis_data vd = {voff, u, v, w, yre, yim};
  for (int l = 0; l < L; l++)
    if (voff[l + 1] < voff[l]) return 1;
#pragma omp parallel for schedule(dynamic, 1)
  for (int l = 0; l < L; l++) {
    double* buf = malloc(sizeof(double) * 4 * N);
    vis_adjoint_band(N, &vd, l, yre + voff[l], yim + voff[l], HtY + (long)l * N * N, buf);
    free(buf);
  }
  return 0;
}

/* Phi x (adjoint 0: x real [L][N][N] -> (zre, zim) [voff[L]]) or Re(Phi^H W z) (adjoint 1: z -> x). */
void orc_vis_apply(int N, int L, const int* voff, const double* u, const double* v, const double* w, double* x,
                   double* zre, double* zim, int adjoint) {
  vis_data vd = {voff, u, v, w, NULL, NULL};
#pragma omp parallel for schedule(dynamic, 1)
  for (int l = 0; l < L; l++) {
    double* buf = malloc(sizeof(double) * 4 * N);
    double* xl = x + (long)l * N * N;
    if (adjoint) vis_adjoint_band(N, &vd, l, zre + voff[l], zim + voff[l], xl, buf);
    else vis_forward_band(N, &vd, l, xl, zre + voff[l], zim + voff[l], buf);
    free(buf);
  }
}

static double dot(const double* a, const double* b, long n) {
  double s = 0.0;
  for (long i = 0; i < n; i++) s += a[i] * b[i];
  return s;
}

/*
 * Conjugate gradients on Q_l x_l = b_l, Q_l = H_l^T H_l + rho I, for every band,
 * from the x given (updated in place), `iters` iterations:
 *   r = b - Q x, p = r, g = r.r;
 *   repeat: q = Q p, a = g / p.q, x += a p, r -= a q, g' = r.r, p = r + (g'/g) p, g = g'.
 * A zero residual or a zero p.q ends the band's iterations (the system is solved).
 * If dfit is not NULL it receives per band 1/2 ||y_l - H_l x_l||^2 for the final x.
 */
/* Per-band work buffers of the normal operator H_l^T H_l (or Re(Phi_l^H W Phi_l)). */
typedef struct {
  double *re, *im, *lr, *li, *t; /* linear convolution: (2N)^2 FFT image, FFT line, H x */
  double *zr, *zi, *buf;         /* visibilities: Phi x, phase tables */
} normal_ws;

static void normal_ws_alloc(normal_ws* ws, int N, const lin_op* lo, int L) {
  long M = 2L * N, NN = (long)N * N;
  memset(ws, 0, sizeof(*ws));
  if (lo->vis) {
    int mx = vis_max_count(lo->vis, L);
    ws->zr = malloc(sizeof(double) * mx);
    ws->zi = malloc(sizeof(double) * mx);
    ws->buf = malloc(sizeof(double) * 4 * N);
  } else {
    ws->re = malloc(sizeof(double) * M * M);
    ws->im = malloc(sizeof(double) * M * M);
    ws->lr = malloc(sizeof(double) * M);
    ws->li = malloc(sizeof(double) * M);
    ws->t = malloc(sizeof(double) * NN);
  }
}

static void normal_ws_free(normal_ws* ws) {
  free(ws->re); free(ws->im); free(ws->lr); free(ws->li); free(ws->t);
  free(ws->zr); free(ws->zi); free(ws->buf);
}

/* q = H_l^T H_l x for band l */
static void normal_band(int N, const lin_op* lo, int l, const double* x, double* q, normal_ws* ws,
                        const double* twr, const double* twi) {
  if (lo->vis) {
    vis_forward_band(N, lo->vis, l, x, ws->zr, ws->zi, ws->buf);
    vis_adjoint_band(N, lo->vis, l, ws->zr, ws->zi, q, ws->buf);
  } else {
    long MM = 4L * N * N;
    const double* hr = lo->h2re + l * MM;
    const double* hi = lo->h2im + l * MM;
    lin_apply_band(N, hr, hi, x, ws->t, 0, ws->re, ws->im, twr, twi, ws->lr, ws->li);
    lin_apply_band(N, hr, hi, ws->t, q, 1, ws->re, ws->im, twr, twi, ws->lr, ws->li);
  }
}

/* 1/2 ||y_l - H_l x||^2 (linear convolution) or 1/2 sum_m w_m |y_m - (Phi_l x)_m|^2 */
static double data_fit_band(int N, const lin_op* lo, int l, const double* x, normal_ws* ws, const double* twr,
                            const double* twi) {
  double f = 0.0;
  if (lo->vis) {
    const vis_data* vd = lo->vis;
    vis_forward_band(N, vd, l, x, ws->zr, ws->zi, ws->buf);
    for (int m = vd->voff[l]; m < vd->voff[l + 1]; m++) {
      double dr = vd->yre[m] - ws->zr[m - vd->voff[l]], di = vd->yim[m] - ws->zi[m - vd->voff[l]];
      f += (vd->w ? vd->w[m] : 1.0) * (dr * dr + di * di);
    }
  } else {
    long NN = (long)N * N, MM = 4L * N * N;
    lin_apply_band(N, lo->h2re + l * MM, lo->h2im + l * MM, x, ws->t, 0, ws->re, ws->im, twr, twi, ws->lr, ws->li);
    for (long i = 0; i < NN; i++) {
      double d = lo->y[l * NN + i] - ws->t[i];
      f += d * d;
    }
  }
  return 0.5 * f;
}

static void solve_cg(const problem* pb, const lin_op* lo, const double* b, double* X, double* dfit) {
  int N = pb->N, L = pb->L, M = 2 * N;
  long NN = (long)N * N;
  double rho = pb->mu_eps + pb->rho_S + pb->rho_P + pb->nb * pb->rho_T; /* Eq. Qlsimp */
  double* twr = malloc(sizeof(double) * (M / 2 + 1));
  double* twi = malloc(sizeof(double) * (M / 2 + 1));
  twiddles(M, twr, twi);
#pragma omp parallel for schedule(dynamic, 1)
  for (int l = 0; l < L; l++) {
    normal_ws ws;
    normal_ws_alloc(&ws, N, lo, L);
    double *r = malloc(sizeof(double) * NN), *p = malloc(sizeof(double) * NN), *q = malloc(sizeof(double) * NN);
    double* x = X + l * NN;
    const double* bl = b + l * NN;
    /* r = b - Q x */
    normal_band(N, lo, l, x, q, &ws, twr, twi);
    for (long i = 0; i < NN; i++) {
      r[i] = bl[i] - (q[i] + rho * x[i]);
      p[i] = r[i];
    }
    double g = dot(r, r, NN);
    for (int it = 0; it < lo->cg_iters && g > 0.0; it++) {
      normal_band(N, lo, l, p, q, &ws, twr, twi);
      for (long i = 0; i < NN; i++) q[i] += rho * p[i];
      double pq = dot(p, q, NN);
      if (!(pq > 0.0)) break;
      double a = g / pq;
      for (long i = 0; i < NN; i++) {
        x[i] += a * p[i];
        r[i] -= a * q[i];
      }
      double g2 = dot(r, r, NN);
      double beta = g2 / g;
      for (long i = 0; i < NN; i++) p[i] = r[i] + beta * p[i];
      g = g2;
    }
    if (dfit) dfit[l] = data_fit_band(N, lo, l, x, &ws, twr, twi);
    normal_ws_free(&ws);
    free(r); free(p); free(q);
  }
  free(twr); free(twi);
}

/* Step I alone with CG: X (in: start, out: result) for right-hand side b (including H^T y). */
int orc_solve_cg(int N, int L, int J, int nb, const int* F, const double* h, const double* prm, const double* h2re,
                 const double* h2im, int cg_iters, const double* b, double* X) {
  problem pb;
  if (load_problem(&pb, N, L, J, nb, F, h, prm)) return 1;
  lin_op lo = {h2re, h2im, NULL, cg_iters, NULL};
  solve_cg(&pb, &lo, b, X, NULL);
  return 0;
}

/* Step I alone with CG for the visibility operator (see vis_data). */
int orc_solve_cg_vis(int N, int L, int J, int nb, const int* F, const double* h, const double* prm, const int* voff,
                     const double* u, const double* v, const double* w, int cg_iters, const double* b, double* X) {
  problem pb;
  if (load_problem(&pb, N, L, J, nb, F, h, prm)) return 1;
  vis_data vd = {voff, u, v, w, NULL, NULL};
  lin_op lo = {NULL, NULL, NULL, cg_iters, &vd};
  solve_cg(&pb, &lo, b, X, NULL);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Steps II-VI.                                                              */
/* ------------------------------------------------------------------------ */

/* Z receives W_k X for every basis (needed again by the Gamma_T update). */
static void primal_dual(const problem* pb, const double* X, double* P, double* T, double* V,
                        double* S, double* GP, double* GT, double* GV, double* GS, double* Z) {
  int N = pb->N, L = pb->L, nb = pb->nb;
  long NN = (long)N * N, V_ = NN * L;

  /* Step II: P <- max(0, X - Gamma_P / rho_P) */
#pragma omp parallel for
  for (long i = 0; i < V_; i++) {
    double pt = X[i] - GP[i] / pb->rho_P;
    P[i] = pt > 0.0 ? pt : 0.0;
  }

  /* Step III: T <- S_{mu_s/rho_T}(W_s X - Gamma_T / rho_T) */
  double tauT = pb->mu_s / pb->rho_T;
#pragma omp parallel for collapse(2) schedule(dynamic, 1)
  for (int k = 0; k < nb; k++) {
    for (int l = 0; l < L; l++) {
      double* buf = malloc(sizeof(double) * 2 * N);
      long off = ((long)k * L + l) * NN;
      dwt2(X + l * NN, Z + off, N, pb->J, pb->h[k], pb->F[k], buf);
      for (long i = 0; i < NN; i++) T[off + i] = soft(Z[off + i] - GT[off + i] / pb->rho_T, tauT);
      free(buf);
    }
  }

  /* Steps IV and V, one pixel spectrum at a time (uses the old S in IV):
   *   V_j = S_{mu_nu/rho_V}(S W_j - Gamma_Vj / rho_V) for every basis j,
   *   S = (sum_j (Gamma_Vj + rho_V V_j) W_j^T - Gamma_S + rho_S X) / (m_nu rho_V + rho_S). */
  double tauV = pb->mu_nu / pb->rho_V;
  int mnu = pb->mnu;
#pragma omp parallel for schedule(static)
  for (long p = 0; p < NN; p++) {
    double s[256], u[256], v[256];
    for (int l = 0; l < L; l++) u[l] = 0.0;
    for (int j = 0; j < mnu; j++) {
      const double* C = pb->Cnu + (long)j * L * L;
      const double* GVj = GV + (long)j * V_;
      double* Vj = V + (long)j * V_;
      for (int k = 0; k < L; k++) {
        double sw = 0.0;
        for (int l = 0; l < L; l++) sw += C[k * L + l] * S[l * NN + p];
        v[k] = soft(sw - GVj[k * NN + p] / pb->rho_V, tauV);
        Vj[k * NN + p] = v[k];
      }
      for (int l = 0; l < L; l++) {
        double acc = 0.0;
        for (int k = 0; k < L; k++) acc += C[k * L + l] * (GVj[k * NN + p] + pb->rho_V * v[k]);
        u[l] += acc;
      }
    }
    for (int l = 0; l < L; l++)
      s[l] = (u[l] - GS[l * NN + p] + pb->rho_S * X[l * NN + p]) / ((double)mnu * pb->rho_V + pb->rho_S);
    for (int l = 0; l < L; l++) S[l * NN + p] = s[l];
  }

  /* Step VI: dual updates (Gamma_V with the new S). */
#pragma omp parallel for
  for (long i = 0; i < V_; i++) {
    GP[i] += pb->rho_P * (P[i] - X[i]);
    GS[i] += pb->rho_S * (S[i] - X[i]);
  }
#pragma omp parallel for
  for (long i = 0; i < V_ * nb; i++) GT[i] += pb->rho_T * (T[i] - Z[i]);
#pragma omp parallel for schedule(static)
  for (long p = 0; p < NN; p++) {
    for (int j = 0; j < mnu; j++) {
      const double* C = pb->Cnu + (long)j * L * L;
      for (int k = 0; k < L; k++) {
        double sw = 0.0;
        for (int l = 0; l < L; l++) sw += C[k * L + l] * S[l * NN + p];
        GV[(long)j * V_ + k * NN + p] += pb->rho_V * (V[(long)j * V_ + k * NN + p] - sw);
      }
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Exported entry points.                                                    */
/* ------------------------------------------------------------------------ */

/* Step I alone: X = Q^-1 b (b includes H^T Y). */
int orc_solve(int N, int L, int J, int nb, const int* F, const double* h, const double* prm,
              const double* hre, const double* him, const double* b, double* X) {
  problem pb;
  if (load_problem(&pb, N, L, J, nb, F, h, prm)) return 1;
  solve_x(&pb, hre, him, NULL, NULL, b, X, NULL);
  return 0;
}

/* Eq. matB alone. */
int orc_make_b(int N, int L, int J, int nb, const int* F, const double* h, const double* prm,
               const double* HtY, const double* P, const double* T, const double* S,
               const double* GP, const double* GT, const double* GS, double* b) {
  problem pb;
  if (load_problem(&pb, N, L, J, nb, F, h, prm)) return 1;
  make_b(&pb, HtY, P, T, S, GP, GT, GS, b);
  return 0;
}

/* Steps II-VI alone, given the new X. */
int orc_primal_dual(int N, int L, int J, int nb, const int* F, const double* h, const double* prm,
                    const double* X, double* P, double* T, double* V, double* S,
                    double* GP, double* GT, double* GV, double* GS) {
  problem pb;
  if (load_problem(&pb, N, L, J, nb, F, h, prm)) return 1;
  if (L > 256) return 1;
  double* Z = malloc(sizeof(double) * (long)nb * L * N * N);
  primal_dual(&pb, X, P, T, V, S, GP, GT, GV, GS, Z);
  free(Z);
  return 0;
}

#define ORC_NHIST 8

static double sumsq_diff(const double* a, const double* b, long n) {
  double s = 0.0;
  for (long i = 0; i < n; i++) { double d = a[i] - b[i]; s += d * d; }
  return s;
}

/*
 * Algorithm 1 for n_iter iterations from the given state (all zero for the
 * paper's initialisation).  If hist is not NULL it receives ORC_NHIST values
 * per iteration, measured after the iteration's dual update:
 *   [0] primal residual^2  ||P-X||^2 + ||T-W_sX||^2 + ||V-SW_nu||^2 + ||S-X||^2
 *   [1] dual residual^2    ||rho_P dP + rho_T W_s^T dT + rho_S dS||^2 + rho_V^2 ||dS W_nu||^2
 *   [2] merit  rho_P||dP||^2 + rho_T||dT||^2 + (m_nu rho_V+rho_S)||dS||^2 + sum_c ||dGamma_c||^2/rho_c
 *   [3] objective  1/2||Y-HX||^2 + mu_eps/2||X||^2 + mu_s||W_sX||_1 + mu_nu||XW_nu||_1
 *   [4] min(X)
 *   [5] ||X||^2
 *   [6] ||dGamma_P||^2 + ||dGamma_T||^2 + ||dGamma_V||^2 + ||dGamma_S||^2
 *   [7] unused (0)
 * (d = change over the iteration; the residuals follow Boyd et al. for the
 * two-block split (X, V) | (P, T, S).)
 */
static int iterate_impl(int N, int L, int J, int nb, const int* F, const double* h, const double* prm,
                        const double* hre, const double* him, const double* yre, const double* yim, const lin_op* lo,
                        const double* HtY, double* X, double* P, double* T, double* V, double* S, double* GP,
                        double* GT, double* GV, double* GS, int n_iter, double* hist) {
  problem pb;
  if (load_problem(&pb, N, L, J, nb, F, h, prm)) return 1;
  if (L > 256) return 1;
  long NN = (long)N * N, V_ = NN * L, VT = V_ * nb, VV = V_ * pb.mnu;
  double* b = malloc(sizeof(double) * V_);
  double* Z = malloc(sizeof(double) * VT);
  double* dfit = malloc(sizeof(double) * L);
  double *P0 = NULL, *T0 = NULL, *S0 = NULL, *GP0 = NULL, *GT0 = NULL, *GV0 = NULL, *GS0 = NULL;
  if (hist) {
    P0 = malloc(sizeof(double) * V_); T0 = malloc(sizeof(double) * VT);
    S0 = malloc(sizeof(double) * V_); GP0 = malloc(sizeof(double) * V_);
    GT0 = malloc(sizeof(double) * VT); GV0 = malloc(sizeof(double) * VV);
    GS0 = malloc(sizeof(double) * V_);
  }
  for (int it = 0; it < n_iter; it++) {
    if (hist) {
      memcpy(P0, P, sizeof(double) * V_); memcpy(T0, T, sizeof(double) * VT);
      memcpy(S0, S, sizeof(double) * V_); memcpy(GP0, GP, sizeof(double) * V_);
      memcpy(GT0, GT, sizeof(double) * VT); memcpy(GV0, GV, sizeof(double) * VV);
      memcpy(GS0, GS, sizeof(double) * V_);
    }
    make_b(&pb, HtY, P, T, S, GP, GT, GS, b);
    if (lo) solve_cg(&pb, lo, b, X, hist ? dfit : NULL);
    else solve_x(&pb, hre, him, yre, yim, b, X, hist ? dfit : NULL);
    primal_dual(&pb, X, P, T, V, S, GP, GT, GV, GS, Z);
    if (!hist) continue;

    double* hh = hist + (long)it * ORC_NHIST;
    for (int q = 0; q < ORC_NHIST; q++) hh[q] = 0.0;
    /* primal residual */
    double r2 = sumsq_diff(P, X, V_) + sumsq_diff(T, Z, VT) + sumsq_diff(S, X, V_);
    for (int j = 0; j < pb.mnu; j++) {
      const double* C = pb.Cnu + (long)j * L * L;
      for (long p = 0; p < NN; p++)
        for (int k = 0; k < L; k++) {
          double sw = 0.0;
          for (int l = 0; l < L; l++) sw += C[k * L + l] * S[l * NN + p];
          double d = V[(long)j * V_ + k * NN + p] - sw;
          r2 += d * d;
        }
    }
    hh[0] = r2;
    /* dual residual: needs W_s^T dT */
    double s2 = 0.0, dS2 = 0.0;
    {
      double* u = malloc(sizeof(double) * NN);
      double* w = malloc(sizeof(double) * NN);
      double* acc = malloc(sizeof(double) * NN);
      double* buf = malloc(sizeof(double) * 2 * N);
      for (int l = 0; l < L; l++) {
        for (long i = 0; i < NN; i++) {
          long q = l * NN + i;
          acc[i] = pb.rho_P * (P[q] - P0[q]) + pb.rho_S * (S[q] - S0[q]);
        }
        for (int k = 0; k < nb; k++) {
          long off = ((long)k * L + l) * NN;
          for (long i = 0; i < NN; i++) u[i] = pb.rho_T * (T[off + i] - T0[off + i]);
          idwt2(u, w, N, pb.J, pb.h[k], pb.F[k], buf);
          for (long i = 0; i < NN; i++) acc[i] += w[i];
        }
        for (long i = 0; i < NN; i++) s2 += acc[i] * acc[i];
      }
      free(u); free(w); free(acc); free(buf);
      /* rho_V^2 sum_j ||dS W_j||^2 = m_nu rho_V^2 ||dS||^2 (orthonormal bases) */
      dS2 = sumsq_diff(S, S0, V_);
      s2 += pb.mnu * pb.rho_V * pb.rho_V * dS2;
    }
    hh[1] = s2;
    double dGP = sumsq_diff(GP, GP0, V_), dGT = sumsq_diff(GT, GT0, VT);
    double dGV = sumsq_diff(GV, GV0, VV), dGS = sumsq_diff(GS, GS0, V_);
    hh[2] = pb.rho_P * sumsq_diff(P, P0, V_) + pb.rho_T * sumsq_diff(T, T0, VT) +
            (pb.mnu * pb.rho_V + pb.rho_S) * dS2 + dGP / pb.rho_P + dGT / pb.rho_T + dGV / pb.rho_V +
            dGS / pb.rho_S;
    /* objective */
    double fit = 0.0, x2 = 0.0, l1s = 0.0, l1n = 0.0, xmin = X[0];
    for (int l = 0; l < L; l++) fit += dfit[l];
    for (long i = 0; i < V_; i++) { x2 += X[i] * X[i]; if (X[i] < xmin) xmin = X[i]; }
    for (long i = 0; i < VT; i++) l1s += fabs(Z[i]);
    for (int j = 0; j < pb.mnu; j++) {
      const double* C = pb.Cnu + (long)j * L * L;
      for (long p = 0; p < NN; p++)
        for (int k = 0; k < L; k++) {
          double xw = 0.0;
          for (int l = 0; l < L; l++) xw += C[k * L + l] * X[l * NN + p];
          l1n += fabs(xw);
        }
    }
    hh[3] = fit + 0.5 * pb.mu_eps * x2 + pb.mu_s * l1s + pb.mu_nu * l1n;
    hh[4] = xmin;
    hh[5] = x2;
    hh[6] = dGP + dGT + dGV + dGS;
  }
  free(b); free(Z); free(dfit);
  if (hist) { free(P0); free(T0); free(S0); free(GP0); free(GT0); free(GV0); free(GS0); }
  return 0;
}

/* Algorithm 1 with the circular H of the workloads: step I by the Fourier filter. */
int orc_iterate(int N, int L, int J, int nb, const int* F, const double* h, const double* prm,
                const double* hre, const double* him, const double* yre, const double* yim,
                const double* HtY, double* X, double* P, double* T, double* V, double* S,
                double* GP, double* GT, double* GV, double* GS, int n_iter, double* hist) {
  return iterate_impl(N, L, J, nb, F, h, prm, hre, him, yre, yim, NULL, HtY, X, P, T, V, S, GP, GT, GV, GS, n_iter,
                      hist);
}

/* Algorithm 1 with the linear H (see orc_linear_setup): step I by cg_iters conjugate
 * gradient iterations per band from the previous X; the history's data-fit term
 * is formed in the image domain. */
int orc_iterate_linear(int N, int L, int J, int nb, const int* F, const double* h, const double* prm,
                       const double* h2re, const double* h2im, const double* y, int cg_iters, const double* HtY,
                       double* X, double* P, double* T, double* V, double* S, double* GP, double* GT, double* GV,
                       double* GS, int n_iter, double* hist) {
  lin_op lo = {h2re, h2im, y, cg_iters, NULL};
  return iterate_impl(N, L, J, nb, F, h, prm, NULL, NULL, NULL, NULL, &lo, HtY, X, P, T, V, S, GP, GT, GV, GS, n_iter,
                      hist);
}

/* Algorithm 1 with the visibility operator (see vis_data): step I by cg_iters conjugate
 * gradient iterations per band from the previous X, HtY = Re(Phi^H W y) (orc_vis_setup);
 * the history's data-fit term is formed in the visibility domain. */
int orc_iterate_vis(int N, int L, int J, int nb, const int* F, const double* h, const double* prm, const int* voff,
                    const double* u, const double* v, const double* w, const double* yre, const double* yim,
                    int cg_iters, const double* HtY, double* X, double* P, double* T, double* V, double* S,
                    double* GP, double* GT, double* GV, double* GS, int n_iter, double* hist) {
  vis_data vd = {voff, u, v, w, yre, yim};
  lin_op lo = {NULL, NULL, NULL, cg_iters, &vd};
  return iterate_impl(N, L, J, nb, F, h, prm, NULL, NULL, NULL, NULL, &lo, HtY, X, P, T, V, S, GP, GT, GV, GS, n_iter,
                      hist);
}
