// Step I of Algorithm 1 for a linear (non-circulant) convolution H: the
// conjugate gradient solve that Algorithm 1's comment names for
// Q_l x_l = b_l (Eqs. linsystemX, matQ, Qlsimp: Q_l = H_l^T H_l + rho I), one
// system per band (the ForPar over l), started from the previous X:
//   r = (H^T y + b) - Q X,  p = r,  g = r.r
//   repeat cg_iters times:  q = Q p,  a = g / p.q,  X += a p,  r -= a q,
//                           g' = r.r,  p = r + (g'/g) p,  g = g'
// (a band whose residual or p.q reaches zero keeps its X from then on).
//
// H is the "same"-size linear convolution by the band's PSF (peak at
// (N/2, N/2), zero outside its N x N support): x is embedded in a 2N x 2N
// image at [0,N)^2, the PSF at offsets (u - N/2) mod 2N, and the circular
// convolution of size 2N -- the plan's own FFT kernels at 2N -- has no
// wrap-around on the [0,N)^2 output.  Q p = crop(H^T pad(crop(H pad(p)))) +
// rho p.  The transforms skip the known zeros and the discarded outputs: the
// row pass reads the N x N image as the padded one, the column pass works on
// the first N spatial rows only, the inverse row pass writes only [0,N)^2
// (conv2n), so pad and crop cost no pass of their own.
//
// Per-band dot products: each band's elements are summed by MF_CG_CHUNKS
// blocks in the cube's precision per thread and FP64 across threads and
// blocks, in a fixed order; the per-band scalars stay on the device, so the
// whole solve is enqueued without a host round trip.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "mf_internal.cuh"
#include "reduce.cuh"

namespace mf {
namespace {

constexpr int CNT = 256;
typedef cx<float> C;

unsigned grid_of(size_t n) {
  const size_t b = (n + CNT - 1) / CNT;
  return (unsigned)(b < 152 * 16 ? (b ? b : 1) : 152 * 16);
}

// the PSF of band l at offsets (u - N/2) mod 2N of a 2N x 2N image
__global__ void k_embed_psf(const float* __restrict__ psf, float* __restrict__ dst, int N, int L) {
  const int M = 2 * N;
  const size_t MM = (size_t)M * M, total = MM * L;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t l = i / MM, rem = i - l * MM;
    const int r = (int)(rem / M), c = (int)(rem - (size_t)r * M);
    const int u = (r + N / 2) & (M - 1), v = (c + N / 2) & (M - 1);
    dst[i] = (u < N && v < N) ? psf[(l * N + u) * N + v] : 0.f;
  }
}

// Element e of band l's [0,N)^2 region: thread walk over a band with stride
// CNT * MF_CG_CHUNKS; blockIdx.y = band, blockIdx.x = chunk.
#define CG_BAND_LOOP(N, body)                                                                \
  {                                                                                          \
    const int l = blockIdx.y;                                                                \
    const size_t NN = (size_t)(N) * (N);                                                     \
    for (size_t e = blockIdx.x * (size_t)CNT + threadIdx.x; e < NN; e += (size_t)CNT * gridDim.x) { \
      const size_t o = l * NN + e;                                                           \
      body                                                                                   \
    }                                                                                        \
  }

// block sum of v (FP32 per thread, FP64 across warps) into part[band][chunk]
__device__ __forceinline__ void band_partial(float v, double* part) {
  __shared__ double red[CNT / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < CNT / 32; w++) s += red[w];
    part[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = s;
  }
}

// r = (H^T y + b) - (t + rho X), p = r, with t = H^T H X; partial r.r
__global__ void __launch_bounds__(CNT) k_cg_init(const float* __restrict__ t, const float* __restrict__ hty,
                                                 const float* __restrict__ b, const float* __restrict__ X,
                                                 float* __restrict__ r, float* __restrict__ p, int N, float rho,
                                                 double* __restrict__ part) {
  float s = 0.f;
  CG_BAND_LOOP(N, {
    const float v = (hty[o] + b[o]) - (t[o] + rho * X[o]);
    r[o] = v;
    p[o] = v;
    s = fmaf(v, v, s);
  });
  band_partial(s, part);
}

// q = t + rho p, t = H^T H p; partial p.q
__global__ void __launch_bounds__(CNT) k_cg_q(const float* __restrict__ t, const float* __restrict__ p,
                                              float* __restrict__ q, int N, float rho, double* __restrict__ part) {
  float s = 0.f;
  CG_BAND_LOOP(N, {
    const float v = t[o] + rho * p[o];
    q[o] = v;
    s = fmaf(p[o], v, s);
  });
  band_partial(s, part);
}

// X += a p, r -= a q; partial r.r
__global__ void __launch_bounds__(CNT) k_cg_step(float* __restrict__ X, float* __restrict__ r,
                                                 const float* __restrict__ p, const float* __restrict__ q,
                                                 const double* __restrict__ cgs, int N, int L,
                                                 double* __restrict__ part) {
  const float a = (float)cgs[2 * L + blockIdx.y];
  float s = 0.f;
  CG_BAND_LOOP(N, {
    const float x = fmaf(a, p[o], X[o]);
    const float v = fmaf(-a, q[o], r[o]);
    X[o] = x;
    r[o] = v;
    s = fmaf(v, v, s);
  });
  band_partial(s, part);
}

// p = r + beta p
__global__ void __launch_bounds__(CNT) k_cg_dir(const float* __restrict__ r, float* __restrict__ p,
                                                const double* __restrict__ cgs, int N, int L) {
  const float bt = (float)cgs[3 * L + blockIdx.y];
  CG_BAND_LOOP(N, { p[o] = fmaf(bt, p[o], r[o]); });
}

// Per-band scalars from the chunk partials (fixed order), one thread per band.
// cgs rows: 0 gamma, 1 p.q, 2 alpha, 3 beta, 4 done flag.
//   kind 0: gamma = sum (after init), done = (gamma == 0)
//   kind 1: p.q = sum; alpha = gamma / p.q unless done or p.q <= 0 (then done, alpha = 0)
//   kind 2: g' = sum; beta = done ? 0 : g' / gamma; gamma = g'; done |= (g' == 0)
__global__ void k_cg_scalars(const double* __restrict__ part, int chunks, double* __restrict__ cgs, int L,
                             int kind) {
  for (int l = threadIdx.x; l < L; l += blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < chunks; c++) s += part[(size_t)l * chunks + c];
    double* g = cgs + l;
    double* pq = cgs + L + l;
    double* al = cgs + 2 * L + l;
    double* bt = cgs + 3 * L + l;
    double* done = cgs + 4 * L + l;
    if (kind == 0) {
      *g = s;
      *done = s > 0.0 ? 0.0 : 1.0;
      *al = 0.0;
      *bt = 0.0;
    } else if (kind == 1) {
      *pq = s;
      if (*done == 0.0 && s > 0.0) {
        *al = *g / s;
      } else {
        *done = 1.0;
        *al = 0.0;
      }
    } else {
      if (*done == 0.0) {
        *bt = s / *g;
        *g = s;
        if (!(s > 0.0)) *done = 1.0;
      } else {
        *bt = 0.0;
      }
    }
  }
}

// 1/2 (y - H X)^2 partials into the Q_FIT slot, t = H X
__global__ void __launch_bounds__(CNT) k_cg_fit(const float* __restrict__ t, const float* __restrict__ y, int N,
                                                double* __restrict__ partials) {
  float s = 0.f;
  CG_BAND_LOOP(N, {
    const float d = y[o] - t[o];
    s = fmaf(d, d, s);
  });
  float q[Q_COUNT];
#pragma unroll
  for (int i = 0; i < Q_COUNT; i++) q[i] = 0.f;
  q[Q_XMIN] = NoMin<float>::v;
  q[Q_FIT] = 0.5f * s;
  block_reduce_write<CNT>(q, partials + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * MF_NQ);
}

// dst [L][N][N] = [0,N)^2 region of the circular 2N convolution of src [L][N][N]
// (zero-padded) by the band's transfer function h2: mode 3 (H, or the
// Toeplitz kernel of a visibility plan) or 5 (H^T)
cudaError_t conv2n(mf_plan* p, const float* src, float* dst, int mode, cudaStream_t s) {
  const int M = 2 * p->N, rows = p->N * p->L;
  cudaError_t e = launch_rows_fwd_pad(src, (C*)p->work2, M, rows, (const C*)p->tw2, s);
  if (!e) e = launch_cols_pruned((C*)p->work2, M, p->L, (const C*)p->tw2, mode, (const C*)p->h2, (const C*)p->h2_nyq, s);
  if (!e) e = launch_rows_inv_crop((const C*)p->work2, dst, M, rows, (const C*)p->tw2, s);
  return e;
}

// the operator's output cube (the first cube of big; the second is the linear
// operator's intermediate H src)
float* op_out(mf_plan* p) { return (float*)p->big; }

// op_out <- H^T H src (linear convolution) or Re(Phi^H W Phi) src (visibilities, vis.cu)
cudaError_t apply_hth(mf_plan* p, const float* src, cudaStream_t s) {
  if (p->vis) return conv2n(p, src, op_out(p), 3, s);
  float* mid = op_out(p) + p->cube;
  cudaError_t e = conv2n(p, src, mid, 3, s);
  if (!e) e = conv2n(p, mid, op_out(p), 5, s);
  return e;
}

}  // namespace

cudaError_t linear_setup(mf_plan* p, const float* psf) {
  const int N = p->N, L = p->L, M = 2 * N;
  std::vector<C> tw(M);
  for (int k = 0; k < M; k++) {
    const double ang = -2.0 * M_PI * (double)k / (double)M;
    tw[k].x = (float)std::cos(ang);
    tw[k].y = (float)std::sin(ang);
  }
  cudaError_t e = cudaMemcpy(p->tw2, tw.data(), sizeof(C) * M, cudaMemcpyHostToDevice);
  if (e) return e;
  const size_t big_n = (size_t)4 * p->cube;
  k_embed_psf<<<grid_of(big_n), CNT>>>(psf, (float*)p->big, N, L);
  if ((e = cudaGetLastError())) return e;
  if ((e = launch_rows_fwd<float>((const float*)p->big, (C*)p->work2, M, M * L, (const C*)p->tw2, 0))) return e;
  if ((e = launch_cols<float>((C*)p->work2, M, L, (const C*)p->tw2, 0, (C*)p->h2, (C*)p->h2_nyq, nullptr, nullptr,
                              nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0)))
    return e;
  return cudaDeviceSynchronize();
}

cudaError_t linear_hty(mf_plan* p, const float* y, cudaStream_t s) {
  if (p->vis) return vis_dirty(p, y, s);
  return conv2n(p, y, (float*)p->cgv, 5, s);  // H^T y
}

cudaError_t linear_step_I(mf_plan* p, int cg_iters, double rho_bar, cudaStream_t s) {
  const int N = p->N, L = p->L;
  const size_t V = p->cube;
  float* hty = (float*)p->cgv;
  float* r = hty + V;
  float* pv = r + V;
  float* q = pv + V;
  float* X = (float*)p->X;
  const dim3 g(MF_CG_CHUNKS, L);
  const float rho = (float)rho_bar;
  cudaError_t e = apply_hth(p, X, s);
  if (!e) {
    k_cg_init<<<g, CNT, 0, s>>>(op_out(p), hty, (const float*)p->b, X, r, pv, N, rho, p->cgpart);
    k_cg_scalars<<<1, 128, 0, s>>>(p->cgpart, MF_CG_CHUNKS, p->cgs, L, 0);
    e = cudaGetLastError();
  }
  for (int it = 0; it < cg_iters && !e; it++) {
    e = apply_hth(p, pv, s);
    if (e) break;
    k_cg_q<<<g, CNT, 0, s>>>(op_out(p), pv, q, N, rho, p->cgpart);
    k_cg_scalars<<<1, 128, 0, s>>>(p->cgpart, MF_CG_CHUNKS, p->cgs, L, 1);
    k_cg_step<<<g, CNT, 0, s>>>(X, r, pv, q, p->cgs, N, L, p->cgpart);
    k_cg_scalars<<<1, 128, 0, s>>>(p->cgpart, MF_CG_CHUNKS, p->cgs, L, 2);
    k_cg_dir<<<g, CNT, 0, s>>>(r, pv, p->cgs, N, L);
    e = cudaGetLastError();
  }
  return e;
}

cudaError_t linear_fit(mf_plan* p, const float* y, double* partials, int* nblocks, cudaStream_t s) {
  cudaError_t e = conv2n(p, (const float*)p->X, op_out(p), 3, s);  // H X (or A X for visibilities)
  if (e) return e;
  if (p->vis) return vis_fit(p, op_out(p), partials, nblocks, s);
  const dim3 g(MF_CG_CHUNKS, p->L);
  k_cg_fit<<<g, CNT, 0, s>>>(op_out(p), y, p->N, partials);
  *nblocks = MF_CG_CHUNKS * p->L;
  return cudaGetLastError();
}

}  // namespace mf
