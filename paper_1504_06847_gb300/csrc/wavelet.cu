// Step III of Algorithm 1 with its dual update (step VI) and the wavelet term
// of the next right-hand side (Eq. matB), for every basis W_k of the
// dictionary W_s (Section 4: Db1..Db8 and Haar, orthonormal, periodic):
//   Z = W_k X,  T = S_{mu_s/rho_T}(Z - Gamma_T / rho_T),
//   Gamma_T += rho_T (T - Z),  b += W_k^T (Gamma_T + rho_T T).
// W_k is the J-level separable Mallat transform: at level j the top-left
// M x M block (M = N / 2^(j-1)) is filtered along rows and columns with
// a_i = sum_n h_n x[(2i+n) mod M], d_i = sum_n g_n x[(2i+n) mod M],
// g_n = (-1)^n h_{2K-1-n}; coefficients stay in place (low-pass half first).
//
// Because synthesis is linear, W_k^T U splits level by level:
//   R_{j-1} = level-j synthesis of (R_j as the low-low band, U's detail bands),
// with R_J the thresholded coarsest low-low band and R_0 the contribution to b.
// Per iteration:
//   wav_ll(j)    LL_j = low-low analysis of LL_{j-1}            j = 1..J-1 (LL_0 = X)
//   wav_level(j) analysis of LL_{j-1} over the tile plus halo, threshold and
//                dual update of level j's coefficients, synthesis into R_{j-1}
//                j = J..1; level 1 runs every basis in one CTA and adds the
//                weighted sum into b.
// Gamma_T is double-buffered: a tile reads old values in its halo while the
// neighbouring tile writes new ones.
#include <cuda_runtime.h>

#include "mf_internal.cuh"
#include "reduce.cuh"

namespace mf {

constexpr int WNT = 256;
constexpr int WT = 32;                       // output tile edge of the fused level kernel
constexpr int IHM = WT + 4 * MF_MAX_K - 4;   // input tile edge (halo for K = 8)
constexpr int CWM = WT / 2 + MF_MAX_K - 1;   // coefficient tile edge
constexpr int OPT = WT * WT / WNT;           // output pixels per thread
constexpr int LT = 32;                       // output tile edge of the low-low kernel
constexpr int LIM = 2 * LT + 2 * MF_MAX_K - 2;

template <class R> __device__ __forceinline__ R soft_w(R t, R tau) {
  const R a = fabs(t) - tau;
  return a > (R)0 ? copysign(a, t) : (R)0;
}

// Loads rows/cols [r0, r0 + H) x [c0, c0 + W) of an M x M image (periodic) into
// dst with pitch P.
template <class R>
__device__ __forceinline__ void load_tile(const R* __restrict__ img, int M, int r0, int c0, int H, int W, R* dst,
                                          int P) {
  for (int e = threadIdx.x; e < H * W; e += WNT) {
    const int r = e / W, c = e % W;
    dst[r * P + c] = img[(size_t)((r0 + r) & (M - 1)) * M + ((c0 + c) & (M - 1))];
  }
}

// Fused level on one output tile for the basis with half-length K.
// in: input tile (pitch IHM), loaded for half-length Kin >= K; off = 2 (Kin - K).
// Coefficients of this level live in the top-left M x M block of the band's
// Gamma_T image (pitch N).  rco: the M/2 x M/2 coarse reconstruction used as the
// low-low band (nullptr at the coarsest level, whose low-low band is thresholded).
template <class R, int K, int RESID, class Emit>
__device__ __forceinline__ void level_tile(const R* in, int off, int T, R* ra, R* rd, R* sb,
                                           const R* __restrict__ h, const R* __restrict__ g, int M, int y0, int x0,
                                           const R* __restrict__ gto, R* __restrict__ gtn, int N,
                                           const R* __restrict__ rco, const IterScalars<R>& sc, R w, double* q,
                                           Emit emit) {
  constexpr int F = 2 * K;
  const int CW = T / 2 + K - 1;
  const int IH = T + 4 * K - 4;
  const int tid = threadIdx.x;
  R hr[F], gr[F];
#pragma unroll
  for (int n = 0; n < F; n++) {
    hr[n] = h[n];
    gr[n] = g[n];
  }
  // 1. row analysis of IH input rows into CW low and CW high coefficients
  for (int e = tid; e < IH * CW; e += WNT) {
    const int r = e / CW, c = e % CW;
    const R* src = in + (off + r) * IHM + off + 2 * c;
    R a = 0, d = 0;
#pragma unroll
    for (int n = 0; n < F; n++) {
      const R v = src[n];
      a = fma(hr[n], v, a);
      d = fma(gr[n], v, d);
    }
    ra[r * CWM + c] = a;
    rd[r * CWM + c] = d;
  }
  __syncthreads();
  // 2. column analysis: four sub-bands of CW x CW coefficients
  for (int e = tid; e < CW * CW; e += WNT) {
    const int i = e / CW, c = e % CW;
    R s00 = 0, s01 = 0, s10 = 0, s11 = 0;
#pragma unroll
    for (int n = 0; n < F; n++) {
      const R va = ra[(2 * i + n) * CWM + c], vd = rd[(2 * i + n) * CWM + c];
      s00 = fma(hr[n], va, s00);
      s10 = fma(gr[n], va, s10);
      s01 = fma(hr[n], vd, s01);
      s11 = fma(gr[n], vd, s11);
    }
    sb[0 * CWM * CWM + i * CWM + c] = s00;  // top-left: low rows of low columns
    sb[1 * CWM * CWM + i * CWM + c] = s01;  // top-right
    sb[2 * CWM * CWM + i * CWM + c] = s10;  // bottom-left
    sb[3 * CWM * CWM + i * CWM + c] = s11;  // bottom-right
  }
  __syncthreads();
  // 3. threshold and dual update; sb becomes U = Gamma_T+ + rho_T T+
  const int Mh = M / 2;
  const int ci0 = y0 / 2 - (K - 1), cj0 = x0 / 2 - (K - 1);
  const int own0 = K - 1, own1 = K - 1 + T / 2;
  for (int e = tid; e < 4 * CW * CW; e += WNT) {
    const int qd = e / (CW * CW), rr = e % (CW * CW);
    const int i = rr / CW, c = rr % CW;
    const int gi = (ci0 + i) & (Mh - 1), gc = (cj0 + c) & (Mh - 1);
    R* cell = sb + qd * CWM * CWM + i * CWM + c;
    if (qd == 0 && rco != nullptr) {
      *cell = rco[(size_t)gi * Mh + gc];
    } else {
      const size_t pos = (size_t)(gi + (qd >> 1) * Mh) * N + gc + (qd & 1) * Mh;
      const R z = *cell;
      const R gam = gto[pos];
      const R tt = z - gam * sc.inv_rho_T;
      const R tp = soft_w<R>(tt, sc.tau_T);
      const R gn = gam + sc.rho_T * (tp - z);
      *cell = gn + sc.rho_T * tp;
      if (i >= own0 && i < own1 && c >= own0 && c < own1) {
        gtn[pos] = gn;
        if (RESID) {
          const double dg = (double)gn - (double)gam;
          q[Q_DGT] += (double)w * dg * dg;
          q[Q_L1S] += (double)w * fabs((double)z);
          if (!isfinite(gn)) q[Q_NONFIN] += 1.0;
        }
      }
    }
  }
  __syncthreads();
  // 4. column synthesis into T rows of CW low (ra) and CW high (rd) coefficients
  const R* U00 = sb;
  const R* U01 = sb + CWM * CWM;
  const R* U10 = sb + 2 * CWM * CWM;
  const R* U11 = sb + 3 * CWM * CWM;
  for (int e = tid; e < T * CW; e += WNT) {
    const int m = e / CW, c = e % CW;
    const int par = m & 1;
    R lo = 0, hi = 0;
#pragma unroll
    for (int n2 = 0; n2 < K; n2++) {
      const int n = 2 * n2 + par;
      const R hn = par ? hr[2 * n2 + 1] : hr[2 * n2];
      const R gn = par ? gr[2 * n2 + 1] : gr[2 * n2];
      const int i = ((m - n) >> 1) + K - 1;
      lo = fma(hn, U00[i * CWM + c], fma(gn, U10[i * CWM + c], lo));
      hi = fma(hn, U01[i * CWM + c], fma(gn, U11[i * CWM + c], hi));
    }
    ra[m * CWM + c] = lo;
    rd[m * CWM + c] = hi;
  }
  __syncthreads();
  // 5. row synthesis of the T x T output tile
#pragma unroll
  for (int s = 0; s < OPT; s++) {
    const int e = tid + s * WNT;
    if (e < T * T) {
      const int m = e / T, x = e % T;
      const int par = x & 1;
      R v = 0;
#pragma unroll
      for (int n2 = 0; n2 < K; n2++) {
        const int n = 2 * n2 + par;
        const R hn = par ? hr[2 * n2 + 1] : hr[2 * n2];
        const R gn = par ? gr[2 * n2 + 1] : gr[2 * n2];
        const int c = ((x - n) >> 1) + K - 1;
        v = fma(hn, ra[m * CWM + c], fma(gn, rd[m * CWM + c], v));
      }
      emit(s, m, x, v);
    }
  }
}

#define MF_K_SWITCH(Kv, ...)                              \
  switch (Kv) {                                           \
    case 1: { constexpr int KK = 1; __VA_ARGS__; } break; \
    case 2: { constexpr int KK = 2; __VA_ARGS__; } break; \
    case 3: { constexpr int KK = 3; __VA_ARGS__; } break; \
    case 4: { constexpr int KK = 4; __VA_ARGS__; } break; \
    case 5: { constexpr int KK = 5; __VA_ARGS__; } break; \
    case 6: { constexpr int KK = 6; __VA_ARGS__; } break; \
    case 7: { constexpr int KK = 7; __VA_ARGS__; } break; \
    default: { constexpr int KK = 8; __VA_ARGS__; } break; \
  }

template <class R>
__device__ __forceinline__ R* level_smem(R*& ra, R*& rd, R*& sb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* in = reinterpret_cast<R*>(smem_raw);
  ra = in + IHM * IHM;
  rd = ra + IHM * CWM;
  sb = rd + IHM * CWM;
  return in;
}

// Level 1 (M = N): every basis in one CTA on the same X tile; b += sum_k w_k W_k^T U_k.
template <class R, int RESID>
__global__ void __launch_bounds__(WNT) k_wav_level1(const R* __restrict__ X, R* __restrict__ b,
                                                     const R* __restrict__ gto, R* __restrict__ gtn,
                                                     const R* __restrict__ rco, int N, int L, int coarsest,
                                                     const WavSet<R>* __restrict__ ws, IterScalars<R> sc,
                                                     double* __restrict__ partials) {
  R *ra, *rd, *sb;
  R* in = level_smem<R>(ra, rd, sb);
  const int T = N < WT ? N : WT;
  const int tpd = N / T;
  const int band = blockIdx.y;
  const int y0 = (blockIdx.x / tpd) * T, x0 = (blockIdx.x % tpd) * T;
  const size_t NN = (size_t)N * N;
  load_tile<R>(X + band * NN, N, y0 - 2 * MF_MAX_K + 2, x0 - 2 * MF_MAX_K + 2, T + 4 * MF_MAX_K - 4,
               T + 4 * MF_MAX_K - 4, in, IHM);
  __syncthreads();
  double q[Q_COUNT];
#pragma unroll
  for (int i = 0; i < Q_COUNT; i++) q[i] = 0.0;
  q[Q_XMIN] = 1e300;
  R acc[OPT];
#pragma unroll
  for (int s = 0; s < OPT; s++) acc[s] = 0;
  for (int k = 0; k < ws->nd; k++) {
    const size_t gofs = ((size_t)k * L + band) * NN;
    const R* rc = coarsest ? nullptr : rco + ((size_t)k * L + band) * (NN / 4);
    const R w = ws->w[k];
    auto emit = [&](int s, int, int, R v) { acc[s] = fma(w, v, acc[s]); };
    MF_K_SWITCH(ws->K[k], (level_tile<R, KK, RESID>(in, 2 * (MF_MAX_K - KK), T, ra, rd, sb, ws->h[k], ws->g[k], N, y0,
                                                   x0, gto + gofs, gtn + gofs, N, rc, sc, w, q, emit)));
    __syncthreads();
  }
#pragma unroll
  for (int s = 0; s < OPT; s++) {
    const int e = threadIdx.x + s * WNT;
    if (e < T * T) {
      const int m = e / T, x = e % T;
      const size_t o = band * NN + (size_t)(y0 + m) * N + x0 + x;
      b[o] = b[o] + acc[s];
    }
  }
  if (RESID) block_reduce_write<WNT>(q, partials + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * MF_NQ);
}

// Level j >= 2 (M = N / 2^(j-1)): one basis per CTA; writes R_{j-1} (M x M).
template <class R, int RESID>
__global__ void __launch_bounds__(WNT) k_wav_levelj(const R* __restrict__ in_img, R* __restrict__ out_img,
                                                     const R* __restrict__ gto, R* __restrict__ gtn,
                                                     const R* __restrict__ rco, int N, int M, int L, int coarsest,
                                                     const WavSet<R>* __restrict__ ws, IterScalars<R> sc,
                                                     double* __restrict__ partials) {
  R *ra, *rd, *sb;
  R* in = level_smem<R>(ra, rd, sb);
  const int T = M < WT ? M : WT;
  const int tpd = M / T;
  const int band = blockIdx.y, k = blockIdx.z;
  const int y0 = (blockIdx.x / tpd) * T, x0 = (blockIdx.x % tpd) * T;
  const size_t MM = (size_t)M * M;
  const R* src = in_img + ((size_t)k * L + band) * MM;
  R* dst = out_img + ((size_t)k * L + band) * MM;
  const size_t gofs = ((size_t)k * L + band) * (size_t)N * N;
  const R* rc = coarsest ? nullptr : rco + ((size_t)k * L + band) * (MM / 4);
  double q[Q_COUNT];
#pragma unroll
  for (int i = 0; i < Q_COUNT; i++) q[i] = 0.0;
  q[Q_XMIN] = 1e300;
  const R w = ws->w[k];
  auto emit = [&](int, int m, int x, R v) { dst[(size_t)(y0 + m) * M + x0 + x] = v; };
  MF_K_SWITCH(ws->K[k], {
    load_tile<R>(src, M, y0 - 2 * KK + 2, x0 - 2 * KK + 2, T + 4 * KK - 4, T + 4 * KK - 4, in, IHM);
    __syncthreads();
    level_tile<R, KK, RESID>(in, 0, T, ra, rd, sb, ws->h[k], ws->g[k], M, y0, x0, gto + gofs, gtn + gofs, N, rc, sc,
                             w, q, emit);
  });
  if (RESID)
    block_reduce_write<WNT>(
        q, partials + (((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x) * MF_NQ);
}

// Low-low analysis: LL_j (M/2 x M/2) of the M x M input, for one basis per CTA
// or (shared input, in_basis_stride == 0) for every basis in one CTA.
template <class R, int K>
__device__ __forceinline__ void ll_tile(const R* in, R* a, int TO, const R* __restrict__ h, R* __restrict__ dst,
                                        int Mo, int oy, int ox) {
  constexpr int F = 2 * K;
  R hr[F];
#pragma unroll
  for (int n = 0; n < F; n++) hr[n] = h[n];
  const int IH = 2 * TO + F - 2;
  for (int e = threadIdx.x; e < IH * TO; e += WNT) {
    const int r = e / TO, c = e % TO;
    const R* src = in + r * LIM + 2 * c;
    R s = 0;
#pragma unroll
    for (int n = 0; n < F; n++) s = fma(hr[n], src[n], s);
    a[r * LT + c] = s;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < TO * TO; e += WNT) {
    const int i = e / TO, c = e % TO;
    R s = 0;
#pragma unroll
    for (int n = 0; n < F; n++) s = fma(hr[n], a[(2 * i + n) * LT + c], s);
    dst[(size_t)(oy + i) * Mo + ox + c] = s;
  }
  __syncthreads();
}

template <class R>
__global__ void __launch_bounds__(WNT) k_wav_ll(const R* __restrict__ in_img, size_t in_band_stride,
                                                 size_t in_basis_stride, R* __restrict__ out, int M, int L,
                                                 const WavSet<R>* __restrict__ ws) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* in = reinterpret_cast<R*>(smem_raw);
  R* a = in + LIM * LIM;
  const int Mo = M / 2;
  const int TO = Mo < LT ? Mo : LT;
  const int tpd = Mo / TO;
  const int band = blockIdx.y;
  const int oy = (blockIdx.x / tpd) * TO, ox = (blockIdx.x % tpd) * TO;
  const size_t MMo = (size_t)Mo * Mo;
  if (in_basis_stride == 0) {
    const R* src = in_img + band * in_band_stride;
    load_tile<R>(src, M, 2 * oy, 2 * ox, 2 * TO + 2 * MF_MAX_K - 2, 2 * TO + 2 * MF_MAX_K - 2, in, LIM);
    __syncthreads();
    for (int k = 0; k < ws->nd; k++) {
      R* dst = out + ((size_t)k * L + band) * MMo;
      MF_K_SWITCH(ws->K[k], (ll_tile<R, KK>(in, a, TO, ws->h[k], dst, Mo, oy, ox)));
    }
  } else {
    const int k = blockIdx.z;
    const R* src = in_img + band * in_band_stride + k * in_basis_stride;
    R* dst = out + ((size_t)k * L + band) * MMo;
    MF_K_SWITCH(ws->K[k], {
      load_tile<R>(src, M, 2 * oy, 2 * ox, 2 * TO + 2 * KK - 2, 2 * TO + 2 * KK - 2, in, LIM);
      __syncthreads();
      ll_tile<R, KK>(in, a, TO, ws->h[k], dst, Mo, oy, ox);
    });
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <class R>
int wav_level_blocks(int M, int L, int nd) {
  const int T = M < WT ? M : WT;
  const int tiles = (M / T) * (M / T);
  return tiles * L * nd;
}

template <class R>
cudaError_t launch_wav_ll(const R* in, size_t in_band_stride, size_t in_basis_stride, R* out, int M, int L, int nd,
                          const WavSet<R>* ws, cudaStream_t s) {
  const int Mo = M / 2;
  const int TO = Mo < LT ? Mo : LT;
  const int tiles = (Mo / TO) * (Mo / TO);
  const size_t sm = sizeof(R) * (LIM * LIM + LIM * LT);
  cudaError_t e = cudaFuncSetAttribute(k_wav_ll<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  dim3 grid(tiles, L, in_basis_stride == 0 ? 1 : nd);
  k_wav_ll<R><<<grid, WNT, sm, s>>>(in, in_band_stride, in_basis_stride, out, M, L, ws);
  return cudaGetLastError();
}

template <class R>
cudaError_t launch_wav_level(const R* in, size_t, size_t, const R* rcoarse, R* out, const R* gt_old, R* gt_new,
                             int N, int M, int L, int coarsest, int nd, const WavSet<R>* ws, IterScalars<R> sc,
                             double* partials, int resid, cudaStream_t s) {
  const int T = M < WT ? M : WT;
  const int tiles = (M / T) * (M / T);
  const size_t sm = sizeof(R) * (IHM * IHM + 2 * IHM * CWM + 4 * CWM * CWM);
  cudaError_t e;
  if (M == N) {
    dim3 grid(tiles, L);
    if (resid) {
      e = cudaFuncSetAttribute(k_wav_level1<R, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
      k_wav_level1<R, 1><<<grid, WNT, sm, s>>>(in, out, gt_old, gt_new, rcoarse, N, L, coarsest, ws, sc, partials);
    } else {
      e = cudaFuncSetAttribute(k_wav_level1<R, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
      k_wav_level1<R, 0><<<grid, WNT, sm, s>>>(in, out, gt_old, gt_new, rcoarse, N, L, coarsest, ws, sc, partials);
    }
  } else {
    dim3 grid(tiles, L, nd);
    if (resid) {
      e = cudaFuncSetAttribute(k_wav_levelj<R, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
      k_wav_levelj<R, 1><<<grid, WNT, sm, s>>>(in, out, gt_old, gt_new, rcoarse, N, M, L, coarsest, ws, sc,
                                               partials);
    } else {
      e = cudaFuncSetAttribute(k_wav_levelj<R, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
      k_wav_levelj<R, 0><<<grid, WNT, sm, s>>>(in, out, gt_old, gt_new, rcoarse, N, M, L, coarsest, ws, sc,
                                               partials);
    }
  }
  return cudaGetLastError();
}

#define INST(R)                                                                                               \
  template int wav_level_blocks<R>(int, int, int);                                                           \
  template cudaError_t launch_wav_ll<R>(const R*, size_t, size_t, R*, int, int, int, const WavSet<R>*,            \
                                        cudaStream_t);                                                          \
  template cudaError_t launch_wav_level<R>(const R*, size_t, size_t, const R*, R*, const R*, R*, int, int, int,   \
                                           int, int, const WavSet<R>*, IterScalars<R>, double*, int, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace mf
