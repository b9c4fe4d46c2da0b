// The visibility-domain operator of Section 2 (last paragraph): y_l are the
// visibilities sampled at uv points (u_m, v_m) and H_l maps the sky to them,
//   (Phi_l x)_m = sum_{r,c} x[r][c] exp(-2 pi i (u_m (c - N/2) + v_m (r - N/2)) / N),
// with weights w_m in the data-fit term 1/2 sum_m w_m |y_m - (Phi_l x)_m|^2.
// x being real, step I's matrix is Q_l = Re(Phi_l^H W Phi_l) + rho I and its
// right-hand side Re(Phi_l^H W y_l) + b_l (Eqs. linsystemX, matB with H_l = Phi_l).
//
// Q_l is not diagonalised by the image FFT (the uv points are off the grid),
// so step I runs the plan's conjugate gradients (cg.cu).  Its operator is a
// Toeplitz matrix: Re(Phi^H W Phi)[p][q] = kr(p - q) with
//   k(d) = sum_m w_m exp(2 pi i (u_m d_x + v_m d_y) / N),  kr = Re k,
// for d in (-N, N)^2, so Q_l p is one circular convolution of size 2N (the
// kernel embedded at offsets d mod 2N, p at [0,N)^2, the output cropped to
// [0,N)^2): one 2N FFT round trip per CG iteration, no gridding in the loop.
//
// The forward operator itself (model visibilities, mf_vis_predict) is the
// type-2 transform with the same kernel: the image divided by the kernel's
// transform on the oversampled grid, its FFT, and interpolation at each point.
//
// k (once per plan) and the dirty image d = Re(Phi^H W y) (once per call) are
// type-1 non-uniform FFTs, computed by gridding with the "exponential of
// semicircle" kernel phi(z) = exp(beta (sqrt(1 - z^2) - 1)) (Barnett, Magland
// and af Klinteberg, SIAM J. Sci. Comput. 2019): spread each visibility onto
// an oversampled grid (factor 2, kernel width VW cells), FFT the grid with
// the plan's own real FFT kernels, keep the wanted modes and divide them by
// the kernel's Fourier transform (computed on the host by Gauss-Legendre
// quadrature).  With VW = 8 the approximation error is about 1e-7 of
// sum_m w_m |c_m|, below FP32 rounding of the result.
//
// The data-fit term of the objective is 1/2 x^T (Q_l - rho I) x - x^T d + 1/2 sum_m w_m |y_m|^2.
// The CG operator's 2N convolution skips the padding zeros and the discarded
// outputs (cg.cu, conv2n).

#include <cmath>
#include <vector>

#include "mf_internal.cuh"
#include "reduce.cuh"

namespace mf {
namespace {

constexpr int VW = 8;                  // kernel width in fine-grid cells
constexpr double VBETA = 2.30 * VW;    // shape parameter for oversampling 2
constexpr int VNT = 256;

using C = cx<float>;

__device__ __forceinline__ float es_kernel(float z) {
  const float t = 1.0f - z * z;
  return t > 0.0f ? expf((float)VBETA * (sqrtf(t) - 1.0f)) : 0.0f;
}

// grid [G][G] (and the imaginary plane at grid + G*G when y is given) +=
// c_m phi(2 (j_y - g_y) / VW) phi(2 (j_x - g_x) / VW) over the VW x VW cells
// nearest the visibility's grid point g = scale (u_m, v_m), periodically.
// c_m = w_m (y == nullptr) or w_m y_m.  One thread per visibility and kernel row.
__global__ void __launch_bounds__(VNT) k_vis_spread(const float2* __restrict__ uv, const float* __restrict__ w,
                                                    const float2* __restrict__ y, int count, int G, float scale,
                                                    float* __restrict__ grid) {
  const long t = blockIdx.x * (long)VNT + threadIdx.x;
  if (t >= (long)count * VW) return;
  const int m = (int)(t / VW), row = (int)(t % VW);
  const float2 q = uv[m];
  const float gx = q.x * scale, gy = q.y * scale;  // exact: scale is a power of two
  const float jx0 = ceilf(gx - 0.5f * VW), jy = ceilf(gy - 0.5f * VW) + (float)row;
  const float py = es_kernel((jy - gy) * (2.0f / VW));
  float cr = w ? w[m] : 1.0f, ci = 0.0f;
  if (y) {
    const float2 v = y[m];
    ci = cr * v.y;
    cr = cr * v.x;
  }
  const int iy = (((int)jy % G) + G) % G;
  float* rp = grid + (size_t)iy * G;
#pragma unroll
  for (int c = 0; c < VW; c++) {
    const float jx = jx0 + (float)c;
    const float ph = py * es_kernel((jx - gx) * (2.0f / VW));
    const int ix = (((int)jx % G) + G) % G;
    atomicAdd(rp + ix, cr * ph);
    if (y) atomicAdd(rp + (size_t)G * G + ix, ci * ph);
  }
}

// F(ky, kx) of a real G x G image from the forward half spectrum (main
// [G][G/2], kx = G/2 column in nyq [G]): F(ky, kx) = conj(F(-ky, -kx)) above G/2.
__device__ __forceinline__ float2 spec_at(const C* __restrict__ main, const C* __restrict__ nyq, int G, int ky,
                                          int kx) {
  const int h = G / 2;
  if (kx < h) {
    const C z = main[(size_t)ky * h + kx];
    return make_float2(z.x, z.y);
  }
  if (kx == h) {
    const C z = nyq[ky];
    return make_float2(z.x, z.y);
  }
  const C z = main[(size_t)((G - ky) % G) * h + (G - kx)];
  return make_float2(z.x, -z.y);
}

// Toeplitz kernel of one band, embedded in its 2N x 2N image: out[e] = kr(d)
// for the offset d = e (mod 2N) in (-N, N)^2, 0 where a component is -N.
// Modes d of the grid (G = 4N) spectrum: the e^{+i} sum is the conjugate of
// the forward FFT of the real grid, so kr(d) = Re F(d) / (phi^(d_y) phi^(d_x)).
__global__ void __launch_bounds__(VNT) k_vis_kernel_embed(const C* __restrict__ main, const C* __restrict__ nyq,
                                                          const float* __restrict__ phihat, int N,
                                                          float* __restrict__ out) {
  const int M = 2 * N, G = 4 * N;
  const long t = blockIdx.x * (long)VNT + threadIdx.x;
  if (t >= (long)M * M) return;
  const int ey = (int)(t / M), ex = (int)(t % M);
  const int dy = ey < N ? ey : ey - M, dx = ex < N ? ex : ex - M;
  float v = 0.0f;
  if (dy != -N && dx != -N) {
    const float2 f = spec_at(main, nyq, G, (dy + G) % G, (dx + G) % G);
    v = f.x / (phihat[dy + N] * phihat[dx + N]);
  }
  out[t] = v;
}

// Dirty image of one band: d[r][c] = Re sum_m w_m y_m e^{+2 pi i (u (c - N/2) + v (r - N/2)) / N}
// from the two planes (real and imaginary parts of w y, G = 2N) of the grid:
// Re F+(k) = Re Fre(k) + Im Fim(k) with F the forward FFT of each plane.
__global__ void __launch_bounds__(VNT) k_vis_dirty_gather(const C* __restrict__ main, const C* __restrict__ nyq,
                                                          const float* __restrict__ phihat, int N,
                                                          float* __restrict__ out) {
  const int G = 2 * N, h = G / 2;
  const long t = blockIdx.x * (long)VNT + threadIdx.x;
  if (t >= (long)N * N) return;
  const int r = (int)(t / N), c = (int)(t % N);
  const int ky = (r - N / 2 + G) % G, kx = (c - N / 2 + G) % G;
  const float2 fr = spec_at(main, nyq, G, ky, kx);
  const float2 fi = spec_at(main + (size_t)G * h, nyq + G, G, ky, kx);
  out[t] = (fr.x + fi.y) / (phihat[r] * phihat[c]);
}

// Forward operator (type-2 non-uniform FFT, the same kernel): the image's
// modes k = (r - N/2, c - N/2), divided by phi^(k_y) phi^(k_x), at k mod G of a
// real G x G grid (G = 2N), zero elsewhere; one thread per grid cell.
__global__ void __launch_bounds__(VNT) k_vis_modes(const float* __restrict__ x, const float* __restrict__ phihat,
                                                   int N, float* __restrict__ grid) {
  const int G = 2 * N;
  const long t = blockIdx.x * (long)VNT + threadIdx.x;
  if (t >= (long)G * G) return;
  const int gy = (int)(t / G), gx = (int)(t % G);
  // grid index -> mode -> image index (rows and columns N/2 .. G - N/2 - 1 are empty)
  const int r = gy < N / 2 ? gy + N / 2 : gy - G + N / 2;
  const int c = gx < N / 2 ? gx + N / 2 : gx - G + N / 2;
  float v = 0.0f;
  if (r >= 0 && r < N && c >= 0 && c < N) v = x[(size_t)r * N + c] / (phihat[r] * phihat[c]);
  grid[t] = v;
}

// (Phi x)_m = sum over the VW x VW cells j nearest g = 2 (u_m, v_m) of
// phi(2 (j_y - g_y) / VW) phi(2 (j_x - g_x) / VW) F(j), F the forward DFT of the
// mode grid (sum_k grid_k e^{-2 pi i k.j / G}); one thread per visibility.
__global__ void __launch_bounds__(VNT) k_vis_interp(const float2* __restrict__ uv, const C* __restrict__ main,
                                                    const C* __restrict__ nyq, int count, int G, float scale,
                                                    float2* __restrict__ out) {
  const int m = blockIdx.x * VNT + threadIdx.x;
  if (m >= count) return;
  const float2 q = uv[m];
  const float gx = q.x * scale, gy = q.y * scale;
  const float jx0 = ceilf(gx - 0.5f * VW), jy0 = ceilf(gy - 0.5f * VW);
  float px[VW];
#pragma unroll
  for (int c = 0; c < VW; c++) px[c] = es_kernel((jx0 + (float)c - gx) * (2.0f / VW));
  float sr = 0.0f, si = 0.0f;
  for (int a = 0; a < VW; a++) {
    const float jy = jy0 + (float)a;
    const float py = es_kernel((jy - gy) * (2.0f / VW));
    const int iy = (((int)jy % G) + G) % G;
    float rr = 0.0f, ri = 0.0f;
#pragma unroll
    for (int c = 0; c < VW; c++) {
      const int ix = (((int)(jx0 + (float)c) % G) + G) % G;
      const float2 f = spec_at(main, nyq, G, iy, ix);
      rr = fmaf(px[c], f.x, rr);
      ri = fmaf(px[c], f.y, ri);
    }
    sr = fmaf(py, rr, sr);
    si = fmaf(py, ri, si);
  }
  out[m] = make_float2(sr, si);
}

// 1/2 sum_m w_m |y_m|^2 in FP64, one block, fixed order
__global__ void __launch_bounds__(1024) k_vis_norm(const float* __restrict__ w, const float2* __restrict__ y,
                                                    int count, double* __restrict__ out) {
  __shared__ double red[1024];
  double s = 0.0;
  for (int m = threadIdx.x; m < count; m += 1024) {
    const float2 v = y[m];
    s += (double)(w ? w[m] : 1.0f) * ((double)v.x * v.x + (double)v.y * v.y);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = 512; k > 0; k >>= 1) {
    if ((int)threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = 0.5 * red[0];
}

// Plan-time check of the uv points and weights: |u|, |v| < N/2 (the grid's
// band: every point then lies inside the oversampled grids), w >= 0, all finite.
__global__ void k_vis_check(const float2* __restrict__ uv, const float* __restrict__ w, int count, float half,
                            int* __restrict__ bad) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < count; m += gridDim.x * blockDim.x) {
    const float2 q = uv[m];
    const bool ok = fabsf(q.x) < half && fabsf(q.y) < half && (!w || w[m] >= 0.0f) && isfinite(q.x) &&
                    isfinite(q.y) && (!w || isfinite(w[m]));
    if (!ok) atomicOr(bad, 1);
  }
}

// Data-fit partials 1/2 x.(A x) - x.d per band and chunk (A x: ax, [L][N][N]),
// plus 1/2 sum w |y|^2 in the first block.
__global__ void __launch_bounds__(VNT) k_vis_fit(const float* __restrict__ X, const float* __restrict__ ax_cube,
                                                 const float* __restrict__ d, const double* __restrict__ c0, int N,
                                                 double* __restrict__ partials) {
  const int band = blockIdx.y;
  const size_t NN = (size_t)N * N;
  float s = 0.0f;
  for (size_t e = blockIdx.x * (size_t)VNT + threadIdx.x; e < NN; e += (size_t)gridDim.x * VNT) {
    const size_t i = (size_t)band * NN + e;
    const float x = X[i];
    const float ax = ax_cube[i];
    s = fmaf(x, fmaf(0.5f, ax, -d[i]), s);
  }
  float q[Q_COUNT];
#pragma unroll
  for (int k = 0; k < Q_COUNT; k++) q[k] = 0.0f;
  q[Q_XMIN] = NoMin<float>::v;
  q[Q_FIT] = s;
  double* row = partials + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * MF_NQ;
  block_reduce_write<VNT>(q, row);
  // the thread that wrote the row's Q_FIT slot adds the constant term
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == Q_FIT) row[Q_FIT] += *c0;
}

unsigned blocks_for(long n) { return (unsigned)((n + VNT - 1) / VNT); }

// Gauss-Legendre nodes and weights on [-1, 1] (Newton's method on the
// three-term recurrence of the Legendre polynomials).
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& wt) {
  x.resize(n);
  wt.resize(n);
  for (int i = 0; i < n; i++) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; it++) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; k++) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      const double dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) {
        // derivative at the converged node for the weight
        double q0 = 1.0, q1 = z;
        for (int k = 2; k <= n; k++) {
          const double q2 = ((2.0 * k - 1.0) * z * q1 - (k - 1.0) * q0) / k;
          q0 = q1;
          q1 = q2;
        }
        const double d = n * (z * q1 - q0) / (z * z - 1.0);
        wt[i] = 2.0 / ((1.0 - z * z) * d * d);
        break;
      }
    }
    x[i] = z;
  }
}

// phi^(k) = (VW/2) int_{-1}^{1} phi(z) cos(pi k VW z / G) dz for the K modes
// k in [-K/2, K/2) of a grid of size G = 2K (index k + K/2).
std::vector<float> phihat_table(int K) {
  std::vector<double> z, wt;
  gauss_legendre(64, z, wt);
  const int G = 2 * K;
  std::vector<float> out(K);
  for (int i = 0; i < K; i++) {
    const double k = i - K / 2;
    double s = 0.0;
    for (size_t j = 0; j < z.size(); j++)
      s += wt[j] * std::exp(VBETA * (std::sqrt(1.0 - z[j] * z[j]) - 1.0)) * std::cos(M_PI * k * VW * z[j] / G);
    out[i] = (float)(0.5 * VW * s);
  }
  return out;
}

// Forward half spectrum of `planes` real G x G images at grid (contiguous):
// rows into work, columns into spec / spec_nyq.
cudaError_t grid_fft(const float* grid, int G, int planes, C* work, C* spec, C* spec_nyq, const C* twG,
                     cudaStream_t s) {
  cudaError_t e = launch_rows_fwd<float>(grid, work, G, G * planes, twG, s);
  if (!e)
    e = launch_cols<float>(work, G, planes, twG, 0, spec, spec_nyq, nullptr, nullptr, nullptr, nullptr, nullptr,
                           nullptr, nullptr, nullptr, nullptr, s);
  return e;
}

std::vector<C> twiddles(int G) {
  std::vector<C> h(G);
  for (int k = 0; k < G; k++) {
    const double ang = -2.0 * M_PI * (double)k / (double)G;
    h[k].x = (float)std::cos(ang);
    h[k].y = (float)std::sin(ang);
  }
  return h;
}

}  // namespace

size_t vis_spec_elems(int N) { return (size_t)2 * (2 * N) * N; }

// Plan-time part: the plan's arrays vis_uv, vis_w (counts[], uv and w copied
// by the caller), vis_phihat, vis_twM, tw2 are allocated; this fills the
// tables, checks the uv points and builds the transfer function h2 of every
// band's Toeplitz kernel.  cudaErrorInvalidValue: a uv point or weight is out of range.
cudaError_t vis_setup(mf_plan* p, const int* counts) {
  const int N = p->N, L = p->L, M = 2 * N, G = 4 * N;
  const int total = p->vis_off[L];
  std::vector<float> ph_n = phihat_table(N);
  cudaError_t e = cudaMemcpy(p->vis_phihat, ph_n.data(), sizeof(float) * N, cudaMemcpyHostToDevice);
  std::vector<C> twm = twiddles(M);
  if (!e) e = cudaMemcpy(p->vis_twM, twm.data(), sizeof(C) * M, cudaMemcpyHostToDevice);
  if (!e) e = cudaMemcpy(p->tw2, twm.data(), sizeof(C) * M, cudaMemcpyHostToDevice);
  if (e) return e;
  if (total > 0) {
    int* bad = nullptr;
    int hbad = 0;
    e = cudaMalloc(&bad, sizeof(int));
    if (!e) e = cudaMemset(bad, 0, sizeof(int));
    if (!e) {
      k_vis_check<<<256, 256>>>((const float2*)p->vis_uv, (const float*)p->vis_w, total, 0.5f * N, bad);
      e = cudaGetLastError();
    }
    if (!e) e = cudaMemcpy(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(bad);
    if (e) return e;
    if (hbad) return cudaErrorInvalidValue;
  }
  // the Toeplitz kernels, band by band on a 4N grid (temporary buffers)
  std::vector<float> ph_k = phihat_table(M);
  std::vector<C> twg = twiddles(G);
  float* phk = nullptr;
  float* grid = nullptr;
  C* work = nullptr;
  C* spec = nullptr;
  C* spec_nyq = nullptr;
  C* twG = nullptr;
  e = cudaMalloc(&phk, sizeof(float) * M);
  if (!e) e = cudaMemcpy(phk, ph_k.data(), sizeof(float) * M, cudaMemcpyHostToDevice);
  if (!e) e = cudaMalloc(&grid, sizeof(float) * (size_t)G * G);
  if (!e) e = cudaMalloc(&work, sizeof(C) * (size_t)G * (G / 2));
  if (!e) e = cudaMalloc(&spec, sizeof(C) * (size_t)G * (G / 2));
  if (!e) e = cudaMalloc(&spec_nyq, sizeof(C) * G);
  if (!e) e = cudaMalloc(&twG, sizeof(C) * G);
  if (!e) e = cudaMemcpy(twG, twg.data(), sizeof(C) * G, cudaMemcpyHostToDevice);
  for (int l = 0; l < L && !e; l++) {
    const int cnt = counts[l];
    e = cudaMemset(grid, 0, sizeof(float) * (size_t)G * G);
    if (!e && cnt > 0) {
      k_vis_spread<<<blocks_for((long)cnt * VW), VNT>>>((const float2*)p->vis_uv + p->vis_off[l],
                                                         p->vis_w ? (const float*)p->vis_w + p->vis_off[l] : nullptr,
                                                         nullptr, cnt, G, 4.0f, grid);
      e = cudaGetLastError();
    }
    if (!e) e = grid_fft(grid, G, 1, work, spec, spec_nyq, twG, 0);
    if (!e) {
      k_vis_kernel_embed<<<blocks_for((long)M * M), VNT>>>(spec, spec_nyq, phk, N,
                                                             (float*)p->big + (size_t)l * M * M);
      e = cudaGetLastError();
    }
  }
  // transfer function of every band's embedded kernel (the MODE 3 filter of the 2N convolution)
  if (!e) e = launch_rows_fwd<float>((const float*)p->big, (C*)p->work2, M, M * L, (const C*)p->tw2, 0);
  if (!e)
    e = launch_cols<float>((C*)p->work2, M, L, (const C*)p->tw2, 0, (C*)p->h2, (C*)p->h2_nyq, nullptr, nullptr,
                           nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0);
  if (!e) e = cudaDeviceSynchronize();
  cudaFree(phk);
  cudaFree(grid);
  cudaFree(work);
  cudaFree(spec);
  cudaFree(spec_nyq);
  cudaFree(twG);
  return e;
}

// d = Re(Phi^H W y) into the first cube of cgv, and 1/2 sum w |y|^2, for the
// visibilities y (interleaved complex, concatenated by band).  Scratch: the two
// grid planes (2 (2N)^2 floats) in big and their row transforms (4 N^2
// complex) in work2 (both hold 4 N^2 L >= 8 N^2 floats), the spectra in vis_spec.
cudaError_t vis_dirty(mf_plan* p, const float* y, cudaStream_t s) {
  const int N = p->N, L = p->L, G = 2 * N;
  const int total = p->vis_off[L];
  float* grid = (float*)p->big;
  C* work = (C*)p->work2;
  C* spec = (C*)p->vis_spec;
  C* spec_nyq = (C*)p->vis_nyq;
  cudaError_t e = cudaSuccess;
  k_vis_norm<<<1, 1024, 0, s>>>((const float*)p->vis_w, (const float2*)y, total, p->vis_c0);
  e = cudaGetLastError();
  for (int l = 0; l < L && !e; l++) {
    const int cnt = p->vis_off[l + 1] - p->vis_off[l];
    e = cudaMemsetAsync(grid, 0, sizeof(float) * 2 * (size_t)G * G, s);
    if (!e && cnt > 0) {
      k_vis_spread<<<blocks_for((long)cnt * VW), VNT, 0, s>>>(
          (const float2*)p->vis_uv + p->vis_off[l], p->vis_w ? (const float*)p->vis_w + p->vis_off[l] : nullptr,
          (const float2*)y + p->vis_off[l], cnt, G, 2.0f, grid);
      e = cudaGetLastError();
    }
    if (!e) e = grid_fft(grid, G, 2, work, spec, spec_nyq, (const C*)p->vis_twM, s);
    if (!e) {
      k_vis_dirty_gather<<<blocks_for((long)N * N), VNT, 0, s>>>(spec, spec_nyq, (const float*)p->vis_phihat, N,
                                                                  (float*)p->cgv + (size_t)l * N * N);
      e = cudaGetLastError();
    }
  }
  return e;
}

// out = Phi x for every band (x: [L][N][N]; out: the plan's visibility order),
// band by band through big (the mode grid), work2 (row transforms) and vis_spec.
cudaError_t vis_predict(mf_plan* p, const float* x, float* out, cudaStream_t s) {
  const int N = p->N, L = p->L, G = 2 * N;
  float* grid = (float*)p->big;
  C* work = (C*)p->work2;
  C* spec = (C*)p->vis_spec;
  C* spec_nyq = (C*)p->vis_nyq;
  cudaError_t e = cudaSuccess;
  for (int l = 0; l < L && !e; l++) {
    const int cnt = p->vis_off[l + 1] - p->vis_off[l];
    if (cnt == 0) continue;
    k_vis_modes<<<blocks_for((long)G * G), VNT, 0, s>>>(x + (size_t)l * N * N, (const float*)p->vis_phihat, N,
                                                          grid);
    e = cudaGetLastError();
    if (!e) e = grid_fft(grid, G, 1, work, spec, spec_nyq, (const C*)p->vis_twM, s);
    if (!e) {
      k_vis_interp<<<blocks_for(cnt), VNT, 0, s>>>((const float2*)p->vis_uv + p->vis_off[l], spec, spec_nyq, cnt,
                                                    G, 2.0f, (float2*)out + p->vis_off[l]);
      e = cudaGetLastError();
    }
  }
  return e;
}

cudaError_t vis_fit(mf_plan* p, const float* ax, double* partials, int* nblocks, cudaStream_t s) {
  const dim3 g(MF_CG_CHUNKS, p->L);
  k_vis_fit<<<g, VNT, 0, s>>>((const float*)p->X, ax, (const float*)p->cgv, p->vis_c0, p->N, partials);
  *nblocks = MF_CG_CHUNKS * p->L;
  return cudaGetLastError();
}

}  // namespace mf
