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

#include <type_traits>

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
constexpr int LIMP = LIM + 1;                // pitch (in pairs) of the row-pair layout of the low-low input
constexpr int LTP = LT + 2;                  // pitch of the packed low-low row-analysis buffer
constexpr int LL_IN = (LIM / 2) * LIMP * 2 > LIM * LIM ? (LIM / 2) * LIMP * 2 : LIM * LIM;  // input region
constexpr int LL_A = LIM * LTP;              // row-analysis region (>= LIM * LT)

// Daubechies taps by half-length K (the same numbers for every plan):
// low-pass h_n and high-pass g_n = (-1)^n h_{2K-1-n}.  With K and n known at
// compile time the FMAs read them straight from the constant bank.
__constant__ float c_hf[MF_MAX_K + 1][MF_MAX_F];
__constant__ float c_gf[MF_MAX_K + 1][MF_MAX_F];
__constant__ double c_hd[MF_MAX_K + 1][MF_MAX_F];
__constant__ double c_gd[MF_MAX_K + 1][MF_MAX_F];

template <class R> struct Taps;
template <> struct Taps<float> {
  static __device__ __forceinline__ float h(int K, int n) { return c_hf[K][n]; }
  static __device__ __forceinline__ float g(int K, int n) { return c_gf[K][n]; }
};
template <> struct Taps<double> {
  static __device__ __forceinline__ double h(int K, int n) { return c_hd[K][n]; }
  static __device__ __forceinline__ double g(int K, int n) { return c_gd[K][n]; }
};

cudaError_t upload_tap_pairs();

cudaError_t upload_taps() {
  float hf[MF_MAX_K + 1][MF_MAX_F] = {}, gf[MF_MAX_K + 1][MF_MAX_F] = {};
  double hd[MF_MAX_K + 1][MF_MAX_F] = {}, gd[MF_MAX_K + 1][MF_MAX_F] = {};
  for (int K = 1; K <= MF_MAX_K; K++) {
    const double* h = filter_taps(K);
    for (int n = 0; n < 2 * K; n++) {
      const double gv = (n & 1) ? -h[2 * K - 1 - n] : h[2 * K - 1 - n];
      hd[K][n] = h[n];
      gd[K][n] = gv;
      hf[K][n] = (float)h[n];
      gf[K][n] = (float)gv;
    }
  }
  cudaError_t e = cudaMemcpyToSymbol(c_hf, hf, sizeof(hf));
  if (!e) e = cudaMemcpyToSymbol(c_gf, gf, sizeof(gf));
  if (!e) e = cudaMemcpyToSymbol(c_hd, hd, sizeof(hd));
  if (!e) e = cudaMemcpyToSymbol(c_gd, gd, sizeof(gd));
  if (!e) e = upload_tap_pairs();
  return e;
}

template <class R> __device__ __forceinline__ R soft_w(R t, R tau) {
  const R a = fabs(t) - tau;
  return a > (R)0 ? copysign(a, t) : (R)0;
}

// Asynchronous global -> shared copy of one element (cp.async: the thread does
// not wait for the data, so all of a tile's copies are in flight at once).
template <class R>
__device__ __forceinline__ void cp_async_elem(R* dst, const R* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src),
               "n"((int)sizeof(R))
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Loads rows/cols [r0, r0 + H) x [c0, c0 + W) of an M x M image (periodic) into
// dst with pitch P.  The caller synchronises the CTA before reading dst.
template <class R>
__device__ __forceinline__ void load_tile(const R* __restrict__ img, int M, int r0, int c0, int H, int W, R* dst,
                                          int P) {
  for (int e = threadIdx.x; e < H * W; e += WNT) {
    const int r = e / W, c = e % W;
    cp_async_elem(dst + r * P + c, img + (size_t)((r0 + r) & (M - 1)) * M + ((c0 + c) & (M - 1)));
  }
  cp_async_wait_all();
}

// Fused level on one output tile for the basis with half-length K.
// in: input tile (pitch IHM), loaded for half-length Kin >= K; off = 2 (Kin - K).
// Coefficients of this level live in the top-left M x M block of the band's
// Gamma_T image (pitch N).  rco: the M/2 x M/2 coarse reconstruction used as the
// low-low band (nullptr at the coarsest level, whose low-low band is thresholded).
// RESID: 0 plain, 1 with the residual terms, 2 synthesis only (no input tile):
// the level's coefficients are gto - gtn (the change of Gamma_T over the
// iteration, negated), with rco as the low-low band below the coarsest level.
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
  for (int e = tid; e < (RESID == 2 ? 0 : IH * CW); e += WNT) {
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
  for (int e = tid; e < (RESID == 2 ? 0 : CW * CW); e += WNT) {
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
    } else if (RESID == 2) {
      const size_t pos = (size_t)(gi + (qd >> 1) * Mh) * N + gc + (qd & 1) * Mh;
      *cell = gto[pos] - gtn[pos];
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
        if (RESID == 1) {
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
  if (RESID != 2)
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
  if (RESID == 1) block_reduce_write<WNT>(q, partials + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * MF_NQ);
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
  const R* src = RESID == 2 ? nullptr : in_img + ((size_t)k * L + band) * MM;
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
    if (RESID != 2) load_tile<R>(src, M, y0 - 2 * KK + 2, x0 - 2 * KK + 2, T + 4 * KK - 4, T + 4 * KK - 4, in, IHM);
    __syncthreads();
    level_tile<R, KK, RESID>(in, 0, T, ra, rd, sb, ws->h[k], ws->g[k], M, y0, x0, gto + gofs, gtn + gofs, N, rc, sc,
                             w, q, emit);
  });
  if (RESID == 1)
    block_reduce_write<WNT>(
        q, partials + (((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x) * MF_NQ);
}

// Residual terms of one basis on one tile, per thread, in the cube's precision
// (the block reduction takes them to FP64 across warps), returned by value so
// that they stay in registers across the non-inlined per-basis calls.
template <class R>
struct LevelSums {
  R dgt = 0, l1s = 0, bad = 0;
  __device__ void add(const LevelSums& o) {
    dgt += o.dgt;
    l1s += o.l1s;
    bad += o.bad;
  }
};

// ---------------------------------------------------------------------------
// T x T output tiles (T = 64 or 32, M >= T): compile-time shapes, runs of RB
// outputs per thread along the filter direction, odd shared-memory pitches so
// that consecutive rows fall in different banks.
// ---------------------------------------------------------------------------
template <int T>
struct TC {
  static constexpr int RB = 4;                                  // outputs per run
  static constexpr int IR = T + 4 * MF_MAX_K - 4;               // input rows / columns (halo for K = 8)
  static constexpr int CWM = T / 2 + MF_MAX_K - 1;              // largest coefficient tile edge
  static constexpr int NRM = (CWM + RB - 1) / RB;               // runs per coefficient line
  static constexpr int NVM = 2 * RB - 2 + 2 * MF_MAX_K;         // inputs of one analysis run
  static constexpr int RD = 2 * RB * (NRM - 1) + NVM;           // extent read by the analysis runs
  static constexpr int IP = (RD > IR ? RD : IR) | 1;            // input pitch
  static constexpr int CR = RD > IR ? RD : IR;                  // rows of the row-analysis buffers
  static constexpr int CP = (RB * NRM) | 1;                     // coefficient pitch
  static constexpr int SR = RB * NRM;                           // rows of each sub-band buffer
  static constexpr int SBQ = SR * CP;                           // stride between sub-band buffers
  static constexpr int SMEM = IR * IP + 2 * CR * CP + 4 * SBQ;  // elements
  static constexpr int BP = T + 1;                              // pitch of the level-1 b accumulator
  static constexpr int SMEM1 = SMEM + T * BP;
  static constexpr int OPI = (T * T / WNT) < 8 ? (T * T / WNT) : 8;  // outputs of one synthesis item
  static constexpr int IPT = T * T / (WNT * OPI);                    // synthesis items per thread
  static constexpr int MINB = T == 64 ? 2 : 4;                       // CTAs per SM
  // the synthesis-only mode (RESID == 2) has no input tile: IN fewer elements
  // of shared memory, and one more FP32 CTA per SM for the 64 x 64 tiles
  static constexpr int IN = IR * IP;
  static constexpr int MINB_SYN = T == 64 ? 3 : 4;
  // the pair planes that follow the input tile start on a 16-byte boundary
  static_assert((IR * IP) % 2 == 0, "input tile size must keep the pair planes aligned");
};

// CTAs per SM that the level kernels' register budget is set for (FP64 keeps
// the plain count in the synthesis-only mode: 80 registers would spill)
template <class R, int T, int RESID>
constexpr int level_minb() {
  return RESID == 2 && sizeof(R) == 4 ? TC<T>::MINB_SYN : TC<T>::MINB;
}

// Shared memory of the T x T level kernels: the input tile, then the pair
// plane of the row analysis / column synthesis (CR x CP pairs), then the two
// sub-band pair planes (SR x CP pairs each); level 1 adds its accumulator.
// Without an input tile (WITH_IN false) the pair planes start the layout.
template <class R, int T, bool WITH_IN>
__device__ __forceinline__ R* tile_smem(R*& ra, R*& sb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* in = reinterpret_cast<R*>(smem_raw);
  ra = in + (WITH_IN ? TC<T>::IN : 0);
  sb = ra + 2 * TC<T>::CR * TC<T>::CP;
  return in;
}

// Pairs of values that travel together through one level: the {low, high}
// outputs of the row analysis, the {top-left, top-right} and {bottom-left,
// bottom-right} sub-bands of the column analysis, and the {low, high} parts of
// the column synthesis.  For FP32 a pair is one 64-bit register and shared
// memory word, and each filter tap is one packed FMA (fma.rn.f32x2, two IEEE
// FMAs with round-to-nearest) on both members.
template <class R> struct V2;
template <> struct V2<float> { typedef float2 T; };
template <> struct V2<double> { typedef double2 T; };

__device__ __forceinline__ float2 mk2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 mk2(double a, double b) { return make_double2(a, b); }

__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n\t.reg .b64 pa, pb, pc, pd;\n\t"
      "mov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\tmov.b64 pc, {%6, %7};\n\t"
      "fma.rn.f32x2 pd, pa, pb, pc;\n\tmov.b64 {%0, %1}, pd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}
__device__ __forceinline__ double2 fma2(double2 a, double2 b, double2 c) {
  return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}

// Tap pairs by half-length K: {h_n, h_n}, {g_n, g_n} and {h_n, g_n}.
__constant__ float2 c_hh2f[MF_MAX_K + 1][MF_MAX_F];
__constant__ float2 c_gg2f[MF_MAX_K + 1][MF_MAX_F];
__constant__ float2 c_hg2f[MF_MAX_K + 1][MF_MAX_F];
__constant__ double2 c_hh2d[MF_MAX_K + 1][MF_MAX_F];
__constant__ double2 c_gg2d[MF_MAX_K + 1][MF_MAX_F];
__constant__ double2 c_hg2d[MF_MAX_K + 1][MF_MAX_F];

template <class R> struct Taps2;
template <> struct Taps2<float> {
  static __device__ __forceinline__ float2 hh(int K, int n) { return c_hh2f[K][n]; }
  static __device__ __forceinline__ float2 gg(int K, int n) { return c_gg2f[K][n]; }
  static __device__ __forceinline__ float2 hg(int K, int n) { return c_hg2f[K][n]; }
};
template <> struct Taps2<double> {
  static __device__ __forceinline__ double2 hh(int K, int n) { return c_hh2d[K][n]; }
  static __device__ __forceinline__ double2 gg(int K, int n) { return c_gg2d[K][n]; }
  static __device__ __forceinline__ double2 hg(int K, int n) { return c_hg2d[K][n]; }
};

cudaError_t upload_tap_pairs() {
  float2 hhf[MF_MAX_K + 1][MF_MAX_F] = {}, ggf[MF_MAX_K + 1][MF_MAX_F] = {}, hgf[MF_MAX_K + 1][MF_MAX_F] = {};
  double2 hhd[MF_MAX_K + 1][MF_MAX_F] = {}, ggd[MF_MAX_K + 1][MF_MAX_F] = {}, hgd[MF_MAX_K + 1][MF_MAX_F] = {};
  for (int K = 1; K <= MF_MAX_K; K++) {
    const double* h = filter_taps(K);
    for (int n = 0; n < 2 * K; n++) {
      const double gv = (n & 1) ? -h[2 * K - 1 - n] : h[2 * K - 1 - n];
      hhd[K][n] = make_double2(h[n], h[n]);
      ggd[K][n] = make_double2(gv, gv);
      hgd[K][n] = make_double2(h[n], gv);
      hhf[K][n] = make_float2((float)h[n], (float)h[n]);
      ggf[K][n] = make_float2((float)gv, (float)gv);
      hgf[K][n] = make_float2((float)h[n], (float)gv);
    }
  }
  cudaError_t e = cudaMemcpyToSymbol(c_hh2f, hhf, sizeof(hhf));
  if (!e) e = cudaMemcpyToSymbol(c_gg2f, ggf, sizeof(ggf));
  if (!e) e = cudaMemcpyToSymbol(c_hg2f, hgf, sizeof(hgf));
  if (!e) e = cudaMemcpyToSymbol(c_hh2d, hhd, sizeof(hhd));
  if (!e) e = cudaMemcpyToSymbol(c_gg2d, ggd, sizeof(ggd));
  if (!e) e = cudaMemcpyToSymbol(c_hg2d, hgd, sizeof(hgd));
  return e;
}

// One basis (half-length K) on one T x T output tile.  in: input tile with
// pitch TC<T>::IP, loaded for half-length Kin >= K at offset off = 2 (Kin - K).
// rpair: TC<T>::CR x TC<T>::CP pairs (row analysis, then column synthesis);
// spair: two TC<T>::SR x TC<T>::CP planes of sub-band pairs.
// emit(s, m, x, v[OPI]) receives output row m, columns x..x+OPI-1 for the
// thread's item s (fixed across calls); after_rows() runs once the input tile
// has been consumed (all threads past the row analysis).
template <class R, int T, int K, int RESID, class Emit, class AfterRows>
__device__ __forceinline__ LevelSums<R> level_tile_t(const R* in, int off, R* rpair, R* spair, int M, int y0,
                                                     int x0, const R* __restrict__ gto, R* __restrict__ gtn, int N,
                                                     const R* __restrict__ rco, const IterScalars<R>& sc, R w,
                                                     Emit emit, AfterRows after_rows) {
  LevelSums<R> sums;
  typedef TC<T> C;
  typedef typename V2<R>::T P;
  constexpr int F = 2 * K;
  constexpr int CW = T / 2 + K - 1;     // coefficients per tile edge (with the synthesis halo)
  constexpr int IH = T + 4 * K - 4;     // input rows used
  constexpr int RB = C::RB;             // outputs per thread run
  constexpr int B_IP = C::IP, B_CP = C::CP, OPI = C::OPI;
  constexpr int NRUN = (CW + RB - 1) / RB;
  constexpr int NV = 2 * RB - 2 + F;    // inputs of a run of RB analysis outputs
  constexpr int NU = RB / 2 + K - 1;    // coefficients of a run of RB synthesis outputs
  P* rp = reinterpret_cast<P*>(rpair);
  P* top = reinterpret_cast<P*>(spair);  // {top-left, top-right}: low rows of the low / high columns
  P* bot = top + C::SR * B_CP;           // {bottom-left, bottom-right}: high rows
  const int tid = threadIdx.x;
  // 1. row analysis: row r, coefficient pairs {low, high} RB j..RB j+RB-1;
  //    consecutive threads take consecutive rows (none in the synthesis-only
  //    mode, RESID == 2, which has no input tile; see level_tile)
  for (int it = tid; it < (RESID == 2 ? 0 : IH * NRUN); it += WNT) {
    const int r = it % IH, j = it / IH;
    const R* src = in + (off + r) * B_IP + off + 2 * RB * j;
    R v[NV];
#pragma unroll
    for (int t = 0; t < NV; t++) v[t] = src[t];
    P* dst = rp + r * B_CP + RB * j;
#pragma unroll
    for (int c = 0; c < RB; c++) {
      P acc = mk2((R)0, (R)0);
#pragma unroll
      for (int n = 0; n < F; n++) acc = fma2(Taps2<R>::hg(K, n), mk2(v[2 * c + n], v[2 * c + n]), acc);
      dst[c] = acc;
    }
  }
  __syncthreads();
  after_rows();  // the input tile is free from here on
  // 2. column analysis of column c of both row-analysis outputs into coefficient
  //    rows RB2 j..RB2 j+RB2-1 of the four sub-bands, fused with 3. threshold and
  //    dual update of those coefficients.  The item issues its global loads (old
  //    Gamma_T, or the coarse reconstruction that replaces the low-low band below
  //    the coarsest level) before its FMAs.  Offsets are 32-bit within the band.
  {
    // rows per item: chosen per filter length so that the items fill whole
    // rounds of the CTA's threads (CW * ceil(CW / RB2) close to a multiple of WNT)
    constexpr int RB2 = K == 1 ? 4 : K <= 4 ? 5 : K == 5 ? 6 : 3;
    constexpr int NRUN2 = (CW + RB2 - 1) / RB2, NV2 = 2 * RB2 - 2 + F;
    static_assert(RB2 * NRUN2 <= C::SR, "rows written");
    static_assert(2 * RB2 * (NRUN2 - 1) + NV2 <= C::CR, "rows read");
    const int Mh = M / 2;
    const int ci0 = y0 / 2 - (K - 1), cj0 = x0 / 2 - (K - 1);
    const int MhN = Mh * N;
    if constexpr (RESID == 2) {
      // synthesis only: the four sub-bands are gto - gtn (rco as the low-low band)
      for (int it = tid; it < CW * NRUN2; it += WNT) {
        const int c = it % CW, j = it / CW;
        const int gc = (cj0 + c) & (Mh - 1);
#pragma unroll
        for (int i = 0; i < RB2; i++) {
          const int row = RB2 * j + i;
          R tl = 0, tr = 0, bl = 0, br = 0;
          if (row < CW) {
            const int gi = (ci0 + row) & (Mh - 1);
            const int go = gi * N + gc;
            tl = rco != nullptr ? rco[gi * Mh + gc] : gto[go] - gtn[go];
            tr = gto[go + Mh] - gtn[go + Mh];
            bl = gto[go + MhN] - gtn[go + MhN];
            br = gto[go + MhN + Mh] - gtn[go + MhN + Mh];
          }
          top[row * B_CP + c] = mk2(tl, tr);
          bot[row * B_CP + c] = mk2(bl, br);
        }
      }
    } else
    for (int it = tid; it < CW * NRUN2; it += WNT) {
      const int c = it % CW, j = it / CW;
      const int gc = (cj0 + c) & (Mh - 1);
      const bool own_c = (unsigned)(c - (K - 1)) < (unsigned)(T / 2);
      R gtl[RB2], gtr[RB2], gbl[RB2], gbr[RB2];
      int go[RB2];
#pragma unroll
      for (int i = 0; i < RB2; i++) {
        const int row = RB2 * j + i;
        const int gi = (ci0 + row) & (Mh - 1);
        go[i] = gi * N + gc;
        gtl[i] = gtr[i] = gbl[i] = gbr[i] = (R)0;
        if (row < CW) {
          gtl[i] = rco != nullptr ? rco[gi * Mh + gc] : gto[go[i]];
          gtr[i] = gto[go[i] + Mh];
          gbl[i] = gto[go[i] + MhN];
          gbr[i] = gto[go[i] + MhN + Mh];
        }
      }
      const P* col = rp + 2 * RB2 * j * B_CP + c;
      P v[NV2];
#pragma unroll
      for (int t = 0; t < NV2; t++) v[t] = col[t * B_CP];
      // residual terms of the item's owned coefficients, in the cube's precision,
      // folded into the FP64 sums once per item
      R r_dg = 0, r_l1 = 0;
      bool r_bad = false;
      auto update = [&](R z, R gam, bool own, int pos) -> R {
        const R tp = soft_w<R>(z - gam * sc.inv_rho_T, sc.tau_T);
        const R gn = gam + sc.rho_T * (tp - z);
        if (own) {
          gtn[pos] = gn;
          if (RESID == 1) {
            const R dg = gn - gam;
            r_dg = fma(dg, dg, r_dg);
            r_l1 += fabs(z);
            r_bad |= !isfinite(gn);
          }
        }
        return gn + sc.rho_T * tp;
      };
#pragma unroll
      for (int i = 0; i < RB2; i++) {
        P lo = mk2((R)0, (R)0), hi = mk2((R)0, (R)0);
#pragma unroll
        for (int n = 0; n < F; n++) {
          lo = fma2(Taps2<R>::hh(K, n), v[2 * i + n], lo);
          hi = fma2(Taps2<R>::gg(K, n), v[2 * i + n], hi);
        }
        const int row = RB2 * j + i;
        const bool own = own_c && (unsigned)(row - (K - 1)) < (unsigned)(T / 2);
        const R tl = rco != nullptr ? gtl[i] : update(lo.x, gtl[i], own, go[i]);
        top[row * B_CP + c] = mk2(tl, update(lo.y, gtr[i], own, go[i] + Mh));
        bot[row * B_CP + c] = mk2(update(hi.x, gbl[i], own, go[i] + MhN), update(hi.y, gbr[i], own, go[i] + MhN + Mh));
      }
      if (RESID == 1) {
        sums.dgt = fma(w, r_dg, sums.dgt);
        sums.l1s = fma(w, r_l1, sums.l1s);
        if (r_bad) sums.bad += (R)1;
      }
    }
  }
  __syncthreads();
  // 4. column synthesis: output rows RB j.. of coefficient column c; the pair
  //    {low part, high part} comes from {TL, TR} and {BL, BR} with the same taps
  for (int it = tid; it < CW * (T / RB); it += WNT) {
    const int c = it % CW, j = it / CW;
    const P* ut = top + (RB / 2) * j * B_CP + c;
    const P* ub = bot + (RB / 2) * j * B_CP + c;
    P ua[NU], ud[NU];
#pragma unroll
    for (int ii = 0; ii < NU; ii++) {
      ua[ii] = ut[ii * B_CP];
      ud[ii] = ub[ii * B_CP];
    }
    P* dst = rp + RB * j * B_CP + c;
#pragma unroll
    for (int t = 0; t < RB; t++) {
      const int par = t & 1;
      P acc = mk2((R)0, (R)0);
#pragma unroll
      for (int n2 = 0; n2 < K; n2++) {
        const int n = 2 * n2 + par;
        const int ii = (t - par) / 2 - n2 + K - 1;
        acc = fma2(Taps2<R>::hh(K, n), ua[ii], fma2(Taps2<R>::gg(K, n), ud[ii], acc));
      }
      dst[t * B_CP] = acc;
    }
  }
  __syncthreads();
  // 5. row synthesis: output row m, columns OPI j..OPI j+OPI-1 (runs of RS) from
  //    the {low, high} pairs with the {h, g} tap pairs; consecutive threads take
  //    consecutive rows
  {
    constexpr int RS = OPI < RB ? OPI : RB;
    constexpr int NS = RS / 2 + K - 1;
#pragma unroll
    for (int s = 0; s < C::IPT; s++) {
      const int it = tid + s * WNT;
      const int m = it % T, j = it / T;
      R out[OPI];
#pragma unroll
      for (int hh = 0; hh < OPI / RS; hh++) {
        const P* cl = rp + m * B_CP + (OPI / 2) * j + (RS / 2) * hh;
        P u[NS];
#pragma unroll
        for (int ii = 0; ii < NS; ii++) u[ii] = cl[ii];
#pragma unroll
        for (int t = 0; t < RS; t++) {
          const int par = t & 1;
          P acc = mk2((R)0, (R)0);
#pragma unroll
          for (int n2 = 0; n2 < K; n2++) {
            const int n = 2 * n2 + par;
            const int ii = (t - par) / 2 - n2 + K - 1;
            acc = fma2(Taps2<R>::hg(K, n), u[ii], acc);
          }
          out[RS * hh + t] = acc.x + acc.y;
        }
      }
      emit(s, m, OPI * j, out);
    }
  }
  return sums;
}

__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Issues L2 prefetches for the level coefficients (and the coarse
// reconstruction) that level_tile_t will read for a basis of half-length K.
template <class R, int T>
__device__ __forceinline__ void prefetch_level(int K, const R* gto, const R* rco, int M, int N, int y0, int x0) {
  const int CW = T / 2 + K - 1;
  const int Mh = M / 2;
  const int ci0 = y0 / 2 - (K - 1), cj0 = x0 / 2 - (K - 1);
  // one prefetch per 32 coefficients of a row (128 bytes of floats)
  const int chunks = (CW + 31) / 32;
  for (int e = threadIdx.x; e < 4 * CW * chunks; e += WNT) {
    const int row = e / chunks, ch = e % chunks;
    const int qd = row / CW, i = row % CW;
    const int gi = (ci0 + i) & (Mh - 1), gc = (cj0 + 32 * ch) & (Mh - 1);
    if (qd == 0 && rco != nullptr) prefetch_l2(rco + (size_t)gi * Mh + gc);
    else if (gto != nullptr) prefetch_l2(gto + (size_t)(gi + (qd >> 1) * Mh) * N + gc + (qd & 1) * Mh);
  }
}

template <class R, int T>
__device__ __forceinline__ void load_tile_t(const R* __restrict__ img, int M, int r0, int c0, int H, R* dst) {
  for (int r = threadIdx.x >> 5; r < H; r += WNT / 32) {
    const R* src = img + (size_t)((r0 + r) & (M - 1)) * M;
    for (int c = threadIdx.x & 31; c < H; c += 32) cp_async_elem(dst + r * TC<T>::IP + c, src + ((c0 + c) & (M - 1)));
  }
}

// One basis of level 1 on a T x T tile, adding w W_k^T U_k into the shared
// accumulator.  Not inlined: each filter length keeps its taps as constant-bank
// operands instead of having all lengths' taps hoisted into registers across
// the loop over bases.
template <class R, int T, int K, int RESID>
__device__ __noinline__ LevelSums<R> level1_basis(const R* in, R* ra, R* sb, R* bacc, int N, int y0, int x0,
                                                  const R* __restrict__ gto, R* __restrict__ gtn,
                                                  const R* __restrict__ rco, IterScalars<R> sc, R w) {
  auto emit = [&](int, int m, int x, const R* v) {
    R* a = bacc + m * TC<T>::BP + x;
#pragma unroll
    for (int t = 0; t < TC<T>::OPI; t++) a[t] = fma(w, v[t], a[t]);
  };
  return level_tile_t<R, T, K, RESID>(in, 2 * (MF_MAX_K - K), ra, sb, N, y0, x0, gto, gtn, N, rco, sc, w, emit,
                                      [] {});
}

template <class R, int T, int RESID>
__global__ void __launch_bounds__(WNT, level_minb<R, T, RESID>()) k_wav_level1_t(const R* __restrict__ X, R* __restrict__ b,
                                                                  const R* __restrict__ gto, R* __restrict__ gtn,
                                                                  const R* __restrict__ rco, int N, int L,
                                                                  int coarsest, const WavSet<R>* __restrict__ ws,
                                                                  IterScalars<R> sc,
                                                                  double* __restrict__ partials) {
  typedef TC<T> C;
  R *ra, *sb;
  R* in = tile_smem<R, T, RESID != 2>(ra, sb);
  const int tpd = N / T;
  const int band = blockIdx.y;
  const int y0 = (blockIdx.x / tpd) * T, x0 = (blockIdx.x % tpd) * T;
  const size_t NN = (size_t)N * N;
  if (RESID != 2) load_tile_t<R, T>(X + band * NN, N, y0 - 2 * MF_MAX_K + 2, x0 - 2 * MF_MAX_K + 2, C::IR, in);
  cp_async_wait_all();
  for (int r = threadIdx.x; r < T * (T / 32); r += WNT)  // the b tile read at the end
    prefetch_l2(b + band * NN + (size_t)(y0 + r / (T / 32)) * N + x0 + 32 * (r % (T / 32)));
  if (ws->nd > 0)
    prefetch_level<R, T>(ws->K[0], gto + (size_t)band * NN, coarsest ? nullptr : rco + (size_t)band * (NN / 4), N,
                         N, y0, x0);
  LevelSums<R> tot;
  // the weighted sum over bases accumulates in shared memory; each thread owns
  // the same outputs for every basis
  R* bacc = sb + 4 * C::SBQ;
  for (int e = threadIdx.x; e < T * C::BP; e += WNT) bacc[e] = 0;
  __syncthreads();
  const int nd = ws->nd;
  for (int k = 0; k < nd; k++) {
    const size_t gofs = ((size_t)k * L + band) * NN;
    const R* rc = coarsest ? nullptr : rco + ((size_t)k * L + band) * (NN / 4);
    const R w = ws->w[k];
    if (k + 1 < nd) {
      const size_t g1 = ((size_t)(k + 1) * L + band) * NN;
      prefetch_level<R, T>(ws->K[k + 1], gto + g1,
                           coarsest ? nullptr : rco + ((size_t)(k + 1) * L + band) * (NN / 4), N, N, y0, x0);
      if (RESID == 2) prefetch_level<R, T>(ws->K[k + 1], gtn + g1, nullptr, N, N, y0, x0);
    }
    MF_K_SWITCH(ws->K[k], (tot.add(level1_basis<R, T, KK, RESID>(in, ra, sb, bacc, N, y0, x0, gto + gofs,
                                                                 gtn + gofs, rc, sc, w))));
    __syncthreads();
  }
  for (int e = threadIdx.x; e < T * T; e += WNT) {
    const int m = e / T, x = e % T;
    R* dst = b + band * NN + (size_t)(y0 + m) * N + x0 + x;
    *dst += bacc[m * C::BP + x];
  }
  if (RESID == 1) {
    R qr[Q_COUNT];  // FP32 plans take the FP32 warp stage of the reduction
#pragma unroll
    for (int i = 0; i < Q_COUNT; i++) qr[i] = 0;
    qr[Q_XMIN] = NoMin<R>::v;
    qr[Q_DGT] = tot.dgt;
    qr[Q_L1S] = tot.l1s;
    qr[Q_NONFIN] = tot.bad;
    block_reduce_write<WNT>(qr, partials + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * MF_NQ);
  }
}

// One basis of a coarser level on a T x T tile (its input tile already in
// shared memory); writes the level's synthesis into R_{j-1} and, once the tile
// is consumed, starts the asynchronous copy of the next basis's tile (next_src,
// half-length next_K; none when next_src is null).  Not inlined (see
// level1_basis).
template <class R, int T, int K, int RESID>
__device__ __noinline__ LevelSums<R> levelj_basis(R* in, R* ra, R* sb, R* __restrict__ dst, int M, int y0, int x0,
                                                  const R* __restrict__ gto, R* __restrict__ gtn, int N,
                                                  const R* __restrict__ rco, IterScalars<R> sc, R w,
                                                  const R* __restrict__ next_src, int next_K) {
  auto emit = [&](int, int m, int x, const R* v) {
    R* o = dst + (size_t)(y0 + m) * M + x0 + x;
#pragma unroll
    for (int t = 0; t < TC<T>::OPI; t++) o[t] = v[t];
  };
  auto after_rows = [&] {
    if (next_src != nullptr)
      load_tile_t<R, T>(next_src, M, y0 - 2 * next_K + 2, x0 - 2 * next_K + 2, T + 4 * next_K - 4, in);
  };
  return level_tile_t<R, T, K, RESID>(in, 0, ra, sb, M, y0, x0, gto, gtn, N, rco, sc, w, emit, after_rows);
}

// L2 prefetch of a basis's input tile at a coarser level.
template <class R, int T>
__device__ __forceinline__ void prefetch_tile(const R* src, int M, int K, int y0, int x0) {
  const int H = T + 4 * K - 4, r0 = y0 - 2 * K + 2, c0 = x0 - 2 * K + 2;
  const int chunks = (H + 31) / 32;
  for (int e = threadIdx.x; e < H * chunks; e += WNT) {
    const int r = e / chunks, ch = e % chunks;
    prefetch_l2(src + (size_t)((r0 + r) & (M - 1)) * M + ((c0 + 32 * ch) & (M - 1)));
  }
}

// Coarser level j >= 2 (M = N / 2^(j-1)): the bases of one group (blockIdx.z;
// one group unless the grid would be too small to fill the GPU) in one CTA, in
// turn, with the next basis's tile and coefficients prefetched; writes R_{j-1}.
template <class R, int T, int RESID>
__global__ void __launch_bounds__(WNT, level_minb<R, T, RESID>()) k_wav_levelj_t(const R* __restrict__ in_img,
                                                                  R* __restrict__ out_img,
                                                                  const R* __restrict__ gto, R* __restrict__ gtn,
                                                                  const R* __restrict__ rco, int N, int M, int L,
                                                                  int coarsest, const WavSet<R>* __restrict__ ws,
                                                                  IterScalars<R> sc,
                                                                  double* __restrict__ partials) {
  R *ra, *sb;
  R* in = tile_smem<R, T, RESID != 2>(ra, sb);
  const int tpd = M / T;
  const int band = blockIdx.y;
  const int y0 = (blockIdx.x / tpd) * T, x0 = (blockIdx.x % tpd) * T;
  const size_t MM = (size_t)M * M, NN = (size_t)N * N;
  LevelSums<R> tot;
  // this CTA's bases: group blockIdx.z of gridDim.z equal groups
  const int per = (ws->nd + gridDim.z - 1) / gridDim.z;
  const int kb = blockIdx.z * per;
  const int ke = kb + per < ws->nd ? kb + per : ws->nd;
  auto src_of = [&](int k) { return RESID == 2 ? (const R*)nullptr : in_img + ((size_t)k * L + band) * MM; };
  auto rc_of = [&](int k) { return coarsest ? (const R*)nullptr : rco + ((size_t)k * L + band) * (MM / 4); };
  if (kb < ke) {
    const int K0 = ws->K[kb];
    if (RESID != 2) load_tile_t<R, T>(src_of(kb), M, y0 - 2 * K0 + 2, x0 - 2 * K0 + 2, T + 4 * K0 - 4, in);
    prefetch_level<R, T>(K0, gto + ((size_t)kb * L + band) * NN, rc_of(kb), M, N, y0, x0);
    if (RESID == 2) prefetch_level<R, T>(K0, gtn + ((size_t)kb * L + band) * NN, nullptr, M, N, y0, x0);
  }
  for (int k = kb; k < ke; k++) {
    const bool more = k + 1 < ke;
    if (more) {
      if (RESID != 2) prefetch_tile<R, T>(src_of(k + 1), M, ws->K[k + 1], y0, x0);
      prefetch_level<R, T>(ws->K[k + 1], gto + ((size_t)(k + 1) * L + band) * NN, rc_of(k + 1), M, N, y0, x0);
      if (RESID == 2)
        prefetch_level<R, T>(ws->K[k + 1], gtn + ((size_t)(k + 1) * L + band) * NN, nullptr, M, N, y0, x0);
    }
    cp_async_wait_all();  // this basis's tile
    __syncthreads();
    const size_t gofs = ((size_t)k * L + band) * NN;
    R* dst = out_img + ((size_t)k * L + band) * MM;
    MF_K_SWITCH(ws->K[k], (tot.add(levelj_basis<R, T, KK, RESID>(in, ra, sb, dst, M, y0, x0, gto + gofs,
                                                                 gtn + gofs, N, rc_of(k), sc, ws->w[k],
                                                                 more ? src_of(k + 1) : nullptr,
                                                                 more ? ws->K[k + 1] : 0))));
    __syncthreads();
  }
  if (RESID == 1) {
    R qr[Q_COUNT];  // FP32 plans take the FP32 warp stage of the reduction
#pragma unroll
    for (int i = 0; i < Q_COUNT; i++) qr[i] = 0;
    qr[Q_XMIN] = NoMin<R>::v;
    qr[Q_DGT] = tot.dgt;
    qr[Q_L1S] = tot.l1s;
    qr[Q_NONFIN] = tot.bad;
    block_reduce_write<WNT>(
        qr, partials + (((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x) * MF_NQ);
  }
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
  if (TO == LT) {
    // rows: 8 consecutive low-pass outputs per thread from 14 + F inputs
    for (int it = threadIdx.x; it < IH * (LT / 8); it += WNT) {
      const int r = it / (LT / 8), j = it % (LT / 8);
      const R* src = in + r * LIM + 16 * j;
      R v[14 + F];
#pragma unroll
      for (int t = 0; t < 14 + F; t++) v[t] = src[t];
#pragma unroll
      for (int c = 0; c < 8; c++) {
        R acc = 0;
#pragma unroll
        for (int n = 0; n < F; n++) acc = fma(hr[n], v[2 * c + n], acc);
        a[r * LT + 8 * j + c] = acc;
      }
    }
    __syncthreads();
    // columns: 4 consecutive outputs per thread from 6 + F inputs
    for (int it = threadIdx.x; it < LT * (LT / 4); it += WNT) {
      const int c = it % LT, j = it / LT;
      const R* col = a + 8 * j * LT + c;
      R v[6 + F];
#pragma unroll
      for (int t = 0; t < 6 + F; t++) v[t] = col[t * LT];
#pragma unroll
      for (int i = 0; i < 4; i++) {
        R acc = 0;
#pragma unroll
        for (int n = 0; n < F; n++) acc = fma(hr[n], v[2 * i + n], acc);
        dst[(size_t)(oy + 4 * j + i) * Mo + ox + c] = acc;
      }
    }
    __syncthreads();
    return;
  }
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

// Loads an H x H tile (H even) of an M x M image (periodic) in the row-pair
// layout of the packed low-low analysis: element (r, c) is member r % 2 of
// pair (r / 2) LIMP + c.
template <class R>
__device__ __forceinline__ void load_tile_rowpairs(const R* __restrict__ img, int M, int r0, int c0, int H, R* dst) {
  // one warp per row, lanes along the row
  for (int r = threadIdx.x >> 5; r < H; r += WNT / 32) {
    const R* src = img + (size_t)((r0 + r) & (M - 1)) * M;
    R* d = dst + (r >> 1) * LIMP * 2 + (r & 1);
    for (int c = threadIdx.x & 31; c < H; c += 32) cp_async_elem(d + 2 * c, src + ((c0 + c) & (M - 1)));
  }
  cp_async_wait_all();
}

// Low-low analysis of one LT x LT output tile on packed pairs: the row pass
// filters two input rows at once ({row 2p, row 2p + 1} pairs), the column pass
// two adjacent columns at once; one fma.rn.f32x2 per tap.
template <class R, int K>
__device__ __forceinline__ void ll_tile_packed(const R* in, R* a, R* __restrict__ dst, int Mo, int oy, int ox) {
  typedef typename V2<R>::T P;
  constexpr int F = 2 * K;
  constexpr int IH = 2 * LT + F - 2;  // input rows and columns used (even)
  constexpr int RO = 4;               // row pass: outputs per item
  constexpr int NVR = 2 * RO - 2 + F;
  constexpr int RC = 2;               // column pass: output rows per item
  constexpr int NVC = 2 * RC - 2 + F;
  const P* pin = reinterpret_cast<const P*>(in);
  // rows: row pair p, low-pass outputs RO j..RO j+RO-1; consecutive threads take consecutive pairs
  for (int it = threadIdx.x; it < (IH / 2) * (LT / RO); it += WNT) {
    const int p = it % (IH / 2), j = it / (IH / 2);
    const P* src = pin + p * LIMP + 2 * RO * j;
    P v[NVR];
#pragma unroll
    for (int t = 0; t < NVR; t++) v[t] = src[t];
    P o[RO];
#pragma unroll
    for (int c = 0; c < RO; c++) {
      P acc = mk2((R)0, (R)0);
#pragma unroll
      for (int n = 0; n < F; n++) acc = fma2(Taps2<R>::hh(K, n), v[2 * c + n], acc);
      o[c] = acc;  // {row 2p, row 2p + 1} of output column RO j + c
    }
    P* d0 = reinterpret_cast<P*>(a + (2 * p) * LTP + RO * j);
    P* d1 = reinterpret_cast<P*>(a + (2 * p + 1) * LTP + RO * j);
#pragma unroll
    for (int c = 0; c < RO; c += 2) {
      d0[c / 2] = mk2(o[c].x, o[c + 1].x);
      d1[c / 2] = mk2(o[c].y, o[c + 1].y);
    }
  }
  __syncthreads();
  // columns: column pair q, output rows RC j..RC j+RC-1; consecutive threads take consecutive pairs
  for (int it = threadIdx.x; it < (LT / 2) * (LT / RC); it += WNT) {
    const int q = it % (LT / 2), j = it / (LT / 2);
    const P* col = reinterpret_cast<const P*>(a + 2 * RC * j * LTP + 2 * q);
    P v[NVC];
#pragma unroll
    for (int t = 0; t < NVC; t++) v[t] = col[t * (LTP / 2)];
#pragma unroll
    for (int i = 0; i < RC; i++) {
      P acc = mk2((R)0, (R)0);
#pragma unroll
      for (int n = 0; n < F; n++) acc = fma2(Taps2<R>::hh(K, n), v[2 * i + n], acc);
      *reinterpret_cast<P*>(dst + (size_t)(oy + RC * j + i) * Mo + ox + 2 * q) = acc;
    }
  }
  __syncthreads();
}

template <class R>
__global__ void __launch_bounds__(WNT) k_wav_ll(const R* __restrict__ in_img, size_t in_band_stride,
                                                 size_t in_basis_stride, R* __restrict__ out, int M, int L,
                                                 const WavSet<R>* __restrict__ ws) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* in = reinterpret_cast<R*>(smem_raw);
  R* a = in + LL_IN;
  const int Mo = M / 2;
  const int TO = Mo < LT ? Mo : LT;
  const int tpd = Mo / TO;
  const int band = blockIdx.y;
  const int oy = (blockIdx.x / tpd) * TO, ox = (blockIdx.x % tpd) * TO;
  const size_t MMo = (size_t)Mo * Mo;
  if (TO == LT) {
    // full LT x LT tiles: the packed form
    if (in_basis_stride == 0) {
      load_tile_rowpairs<R>(in_img + band * in_band_stride, M, 2 * oy, 2 * ox, LIM, in);
      __syncthreads();
      for (int k = 0; k < ws->nd; k++) {
        R* dst = out + ((size_t)k * L + band) * MMo;
        MF_K_SWITCH(ws->K[k], (ll_tile_packed<R, KK>(in, a, dst, Mo, oy, ox)));
      }
    } else {
      const int k = blockIdx.z;
      const R* src = in_img + band * in_band_stride + k * in_basis_stride;
      R* dst = out + ((size_t)k * L + band) * MMo;
      MF_K_SWITCH(ws->K[k], {
        load_tile_rowpairs<R>(src, M, 2 * oy, 2 * ox, 2 * LT + 2 * KK - 2, in);
        __syncthreads();
        ll_tile_packed<R, KK>(in, a, dst, Mo, oy, ox);
      });
    }
    return;
  }
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
// Reverse mode (unrolled iterations): plain periodic level transforms on full
// coefficient arrays, one thread per output, and the adjoint of the
// threshold / dual step.  Taps come from the constant tables with a runtime K.
// ---------------------------------------------------------------------------
// Half-lengths of the bases of one launch (basis k = blockIdx.y).
struct KList {
  int K[MF_MAX_BASES];
};

// Row analysis of one level of one basis: tmp row r = [a_0..a_{M/2-1}, d_0..].
template <class R, int K>
__device__ __forceinline__ void ana_rows_k(const R* __restrict__ src, int sp, size_t ss, R* __restrict__ tmp, int M,
                                           int nimg) {
  constexpr int F = 2 * K;
  const size_t total = (size_t)nimg * M * (M / 2);
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % (M / 2));
    const int r = (int)((e / (M / 2)) % M);
    const size_t img = e / ((size_t)M * (M / 2));
    const R* row = src + img * ss + (size_t)r * sp;
    R a = 0, d = 0;
#pragma unroll
    for (int n = 0; n < F; n++) {
      const R v = row[(2 * i + n) & (M - 1)];
      a = fma(Taps<R>::h(K, n), v, a);
      d = fma(Taps<R>::g(K, n), v, d);
    }
    R* t = tmp + img * (size_t)M * M + (size_t)r * M;
    t[i] = a;
    t[M / 2 + i] = d;
  }
}

// Column analysis of tmp into the level's M x M block of dst (pitch dp).
template <class R, int K>
__device__ __forceinline__ void ana_cols_k(const R* __restrict__ tmp, int M, int nimg, R* __restrict__ dst, int dp,
                                           size_t ds) {
  constexpr int F = 2 * K;
  const size_t total = (size_t)nimg * (M / 2) * M;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % M);
    const int i = (int)((e / M) % (M / 2));
    const size_t img = e / ((size_t)M * (M / 2));
    const R* t = tmp + img * (size_t)M * M + c;
    R a = 0, d = 0;
#pragma unroll
    for (int n = 0; n < F; n++) {
      const R v = t[(size_t)((2 * i + n) & (M - 1)) * M];
      a = fma(Taps<R>::h(K, n), v, a);
      d = fma(Taps<R>::g(K, n), v, d);
    }
    R* o = dst + img * ds + c;
    o[(size_t)i * dp] = a;
    o[(size_t)(M / 2 + i) * dp] = d;
  }
}

// Column synthesis of the level's M x M block of src (pitch sp) into tmp.
template <class R, int K>
__device__ __forceinline__ void syn_cols_k(const R* __restrict__ src, int sp, size_t ss, R* __restrict__ tmp, int M,
                                           int nimg) {
  const size_t total = (size_t)nimg * M * M;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % M);
    const int m = (int)((e / M) % M);
    const size_t img = e / ((size_t)M * M);
    const R* col = src + img * ss + c;
    R v = 0;
#pragma unroll
    for (int n2 = 0; n2 < K; n2++) {
      const int n = 2 * n2 + (m & 1);
      const int i = ((m - n) >> 1) & (M / 2 - 1);
      v = fma(Taps<R>::h(K, n), col[(size_t)i * sp], v);
      v = fma(Taps<R>::g(K, n), col[(size_t)(M / 2 + i) * sp], v);
    }
    tmp[img * (size_t)M * M + (size_t)m * M + c] = v;
  }
}

// Row synthesis of output (m, x) of one basis's tmp.
template <class R, int K>
__device__ __forceinline__ R syn_row_point(const R* __restrict__ row, int M, int x) {
  R v = 0;
#pragma unroll
  for (int n2 = 0; n2 < K; n2++) {
    const int n = 2 * n2 + (x & 1);
    const int i = ((x - n) >> 1) & (M / 2 - 1);
    v = fma(Taps<R>::h(K, n), row[i], v);
    v = fma(Taps<R>::g(K, n), row[M / 2 + i], v);
  }
  return v;
}

template <class R>
__global__ void k_ana_rows(const R* __restrict__ src, size_t src_bs, int sp, size_t ss, R* __restrict__ tmp,
                           size_t tmp_bs, int M, int nimg, KList ks) {
  const int k = blockIdx.y;
  MF_K_SWITCH(ks.K[k], (ana_rows_k<R, KK>(src + k * src_bs, sp, ss, tmp + k * tmp_bs, M, nimg)));
}

template <class R>
__global__ void k_ana_cols(const R* __restrict__ tmp, size_t tmp_bs, int M, int nimg, R* __restrict__ dst,
                           size_t dst_bs, int dp, size_t ds, KList ks) {
  const int k = blockIdx.y;
  MF_K_SWITCH(ks.K[k], (ana_cols_k<R, KK>(tmp + k * tmp_bs, M, nimg, dst + k * dst_bs, dp, ds)));
}

template <class R>
__global__ void k_syn_cols(const R* __restrict__ src, size_t src_bs, int sp, size_t ss, R* __restrict__ tmp,
                           size_t tmp_bs, int M, int nimg, KList ks) {
  const int k = blockIdx.y;
  MF_K_SWITCH(ks.K[k], (syn_cols_k<R, KK>(src + k * src_bs, sp, ss, tmp + k * tmp_bs, M, nimg)));
}

// Row synthesis into the level's block of each basis's coefficient array (j > 1).
template <class R>
__global__ void k_syn_rows(const R* __restrict__ tmp, size_t tmp_bs, int M, int nimg, R* __restrict__ dst,
                           size_t dst_bs, int dp, size_t ds, KList ks) {
  const int k = blockIdx.y;
  const size_t total = (size_t)nimg * M * M;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(e % M);
    const int m = (int)((e / M) % M);
    const size_t img = e / ((size_t)M * M);
    const R* row = tmp + k * tmp_bs + img * (size_t)M * M + (size_t)m * M;
    R v = 0;
    MF_K_SWITCH(ks.K[k], (v = syn_row_point<R, KK>(row, M, x)));
    dst[k * dst_bs + img * ds + (size_t)m * dp + x] = v;
  }
}

// Level-1 row synthesis of every basis, summed and added into out (pitch M).
template <class R>
__global__ void k_syn_rows_sum(const R* __restrict__ tmp, size_t tmp_bs, int nd, int M, int nimg,
                               R* __restrict__ out, KList ks) {
  const size_t total = (size_t)nimg * M * M;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(e % M);
    const int m = (int)((e / M) % M);
    const size_t img = e / ((size_t)M * M);
    R v = 0;
    for (int k = 0; k < nd; k++) {
      const R* row = tmp + k * tmp_bs + img * (size_t)M * M + (size_t)m * M;
      MF_K_SWITCH(ks.K[k], (v += syn_row_point<R, KK>(row, M, x)));
    }
    out[e] += v;
  }
}

// Adjoint of step III and its dual update for one coefficient, with the
// forward recomputed from z = (W_k X) and the old multiplier gam:
//   T~ = z - gam/rho, T = S_tau(T~), tau = mu_s/rho,
//   Gamma_T' = gam + rho (T - z),  U = Gamma_T' + rho T.
// In: g1 = cotangent of Gamma_T', ub = cotangent of U (= w_k W_k b_bar).
// Out: cotangent of z (into zc) and of gam (into gc); d mu_s and d rho partials.
template <class R>
__global__ void k_wav_bwd_point(R* __restrict__ zc, const R* __restrict__ uc, const R* __restrict__ gam_old,
                                R* __restrict__ gc, size_t per_basis, int nd, const WavSet<R>* __restrict__ ws,
                                R rho, R mu_s, double* __restrict__ partials) {
  const size_t total = per_basis * nd;
  // the forward's constants (formed in FP64, rounded once); each element's terms in
  // the cube's precision, summed in FP64 (one add per element: FP64 multiplies and
  // divisions per element are slow)
  const R inv_rho = (R)(1.0 / (double)rho), tau = (R)((double)mu_s / (double)rho);
  const R inv_rho2 = inv_rho * inv_rho;
  double dmu_r = 0, drho_r = 0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / per_basis);
    const R w = ws->w[k];
    const R z = zc[e], gam = gam_old[e], g1 = gc[e], ub = w * uc[e];
    const R tt = z - gam * inv_rho;
    const bool m = fabs(tt) > tau;
    const R sg = tt > 0 ? (R)1 : (tt < 0 ? (R)-1 : (R)0);
    const R t = m ? tt - tau * sg : (R)0;
    const R tb = rho * g1 + 2 * rho * ub;
    const R ttb = m ? tb : (R)0;
    const R taub = m ? -sg * tb : (R)0;
    zc[e] = -rho * g1 - rho * ub + ttb;
    gc[e] = g1 + ub - ttb * inv_rho;
    dmu_r += (double)taub;
    drho_r += (double)(g1 * (t - z) + ub * (2 * t - z) + (ttb * gam - taub * mu_s) * inv_rho2);
  }
  const double dmu = dmu_r * (double)inv_rho, drho = drho_r;
  double q[Q_COUNT];
#pragma unroll
  for (int i = 0; i < Q_COUNT; i++) q[i] = 0.0;
  q[Q_XMIN] = 1e300;
  q[0] = dmu;
  q[2] = drho;
  block_reduce_write<WNT>(q, partials + (size_t)blockIdx.x * MF_NQ);
}

static unsigned simple_grid(size_t total) {
  size_t b = (total + WNT - 1) / WNT;
  return (unsigned)(b < 152 * 32 ? (b ? b : 1) : 152 * 32);
}

// Reverse-mode transforms over full coefficient arrays; every basis of a level
// in one launch (grid y = basis), so tmp holds nd cubes (basis stride L N^2).
template <class R>
cudaError_t launch_wav_analysis_full(const R* src, R* coef, R* tmp, int N, int L, int J, int nd,
                                     const int* Ks, cudaStream_t s) {
  const size_t NN = (size_t)N * N, cube = (size_t)L * NN;
  KList ks{};
  for (int k = 0; k < nd; k++) ks.K[k] = Ks[k];
  for (int j = 1; j <= J; j++) {
    const int M = N >> (j - 1);
    const dim3 g(simple_grid((size_t)L * M * (M / 2)), nd);
    if (j == 1) k_ana_rows<R><<<g, WNT, 0, s>>>(src, 0, N, NN, tmp, cube, M, L, ks);
    else k_ana_rows<R><<<g, WNT, 0, s>>>(coef, cube, N, NN, tmp, cube, M, L, ks);
    k_ana_cols<R><<<g, WNT, 0, s>>>(tmp, cube, M, L, coef, cube, N, NN, ks);
  }
  return cudaGetLastError();
}

template <class R>
cudaError_t launch_wav_synthesis_acc(R* coef, R* out, R* tmp, int N, int L, int J, int nd, const int* Ks,
                                     cudaStream_t s) {
  const size_t NN = (size_t)N * N, cube = (size_t)L * NN;
  KList ks{};
  for (int k = 0; k < nd; k++) ks.K[k] = Ks[k];
  for (int j = J; j >= 1; j--) {
    const int M = N >> (j - 1);
    const dim3 g(simple_grid((size_t)L * M * M), nd);
    k_syn_cols<R><<<g, WNT, 0, s>>>(coef, cube, N, NN, tmp, cube, M, L, ks);
    if (j == 1) k_syn_rows_sum<R><<<simple_grid((size_t)L * M * M), WNT, 0, s>>>(tmp, cube, nd, M, L, out, ks);
    else k_syn_rows<R><<<g, WNT, 0, s>>>(tmp, cube, M, L, coef, cube, N, NN, ks);
  }
  return cudaGetLastError();
}

template <class R>
cudaError_t launch_wav_bwd_point(R* zc, const R* uc, const R* gam_old, R* gc, size_t per_basis, int nd,
                                 const WavSet<R>* ws, R rho, R mu_s, double* partials, int* nblocks,
                                 cudaStream_t s) {
  const unsigned g = simple_grid(per_basis * nd);
  *nblocks = (int)g;
  k_wav_bwd_point<R><<<g, WNT, 0, s>>>(zc, uc, gam_old, gc, per_basis, nd, ws, rho, mu_s, partials);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
// Output tile edge of the fused level kernels: the largest of the allowed
// sizes (pref, 32, or the generic small-tile path) that divides M.
static int level_tile_edge(int M, int pref) {
  if (pref >= 64 && M >= 64) return 64;
  if (M >= 32) return 32;
  return M < WT ? M : WT;
}

// Basis groups of a coarser level with T = 64 / 32 tiles: enough CTAs for about
// eight waves of two per SM, at most one group per basis.
static int levelj_groups(int tiles, int L, int nd) {
  const int target = 152 * 2 * 8;
  const int g = (target + tiles * L - 1) / (tiles * L);
  return g < 1 ? 1 : (g > nd ? nd : g);
}

template <class R>
int wav_level_blocks(int M, int L, int nd, int pref) {
  const int T = level_tile_edge(M, pref);
  const int tiles = (M / T) * (M / T);
  // the T = 64 / 32 kernels loop over a group of bases in a CTA (level 1: all, nd = 1 here)
  return T >= 32 ? tiles * L * levelj_groups(tiles, L, nd) : tiles * L * nd;
}

template <class R>
cudaError_t launch_wav_ll(const R* in, size_t in_band_stride, size_t in_basis_stride, R* out, int M, int L, int nd,
                          const WavSet<R>* ws, cudaStream_t s) {
  const int Mo = M / 2;
  const int TO = Mo < LT ? Mo : LT;
  const int tiles = (Mo / TO) * (Mo / TO);
  const size_t sm = sizeof(R) * (LL_IN + LL_A);
  cudaError_t e = cudaFuncSetAttribute(k_wav_ll<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  dim3 grid(tiles, L, in_basis_stride == 0 ? 1 : nd);
  k_wav_ll<R><<<grid, WNT, sm, s>>>(in, in_band_stride, in_basis_stride, out, M, L, ws);
  return cudaGetLastError();
}

template <class R, class Kern, class... Args>
static cudaError_t launch_k(Kern kern, dim3 grid, size_t sm, cudaStream_t s, Args... args) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  kern<<<grid, WNT, sm, s>>>(args...);
  return cudaGetLastError();
}

template <class R, int T>
static cudaError_t launch_level_t(const R* in, const R* rcoarse, R* out, const R* gt_old, R* gt_new, int N, int M,
                                  int L, int coarsest, int nd, const WavSet<R>* ws, IterScalars<R> sc,
                                  double* partials, int resid, cudaStream_t s) {
  const int tiles = (M / T) * (M / T);
  if (M == N) {
    dim3 grid(tiles, L);
    const size_t sm1 = sizeof(R) * TC<T>::SMEM1;
    if (resid == 2)
      return launch_k<R>(k_wav_level1_t<R, T, 2>, grid, sm1 - sizeof(R) * TC<T>::IN, s, in, out, gt_old, gt_new, rcoarse, N, L, coarsest, ws,
                         sc, partials);
    if (resid)
      return launch_k<R>(k_wav_level1_t<R, T, 1>, grid, sm1, s, in, out, gt_old, gt_new, rcoarse, N, L, coarsest, ws,
                         sc, partials);
    return launch_k<R>(k_wav_level1_t<R, T, 0>, grid, sm1, s, in, out, gt_old, gt_new, rcoarse, N, L, coarsest, ws,
                       sc, partials);
  }
  dim3 grid(tiles, L, levelj_groups(tiles, L, nd));
  const size_t sm = sizeof(R) * TC<T>::SMEM;
  if (resid == 2)
    return launch_k<R>(k_wav_levelj_t<R, T, 2>, grid, sm - sizeof(R) * TC<T>::IN, s, in, out, gt_old, gt_new, rcoarse, N, M, L, coarsest, ws,
                       sc, partials);
  if (resid)
    return launch_k<R>(k_wav_levelj_t<R, T, 1>, grid, sm, s, in, out, gt_old, gt_new, rcoarse, N, M, L, coarsest, ws,
                       sc, partials);
  return launch_k<R>(k_wav_levelj_t<R, T, 0>, grid, sm, s, in, out, gt_old, gt_new, rcoarse, N, M, L, coarsest, ws,
                     sc, partials);
}

template <class R>
cudaError_t launch_wav_level(const R* in, size_t, size_t, const R* rcoarse, R* out, const R* gt_old, R* gt_new,
                             int N, int M, int L, int coarsest, int nd, const WavSet<R>* ws, IterScalars<R> sc,
                             double* partials, int resid, int pref_tile, int*, cudaStream_t s) {
  const int T = level_tile_edge(M, pref_tile);
  if (T == 64)
    return launch_level_t<R, 64>(in, rcoarse, out, gt_old, gt_new, N, M, L, coarsest, nd, ws, sc, partials, resid, s);
  if (T == 32)
    return launch_level_t<R, 32>(in, rcoarse, out, gt_old, gt_new, N, M, L, coarsest, nd, ws, sc, partials, resid, s);
  const int tiles = (M / T) * (M / T);
  const size_t sm = sizeof(R) * (IHM * IHM + 2 * IHM * CWM + 4 * CWM * CWM);
  if (M == N) {
    dim3 grid(tiles, L);
    if (resid == 2)
      return launch_k<R>(k_wav_level1<R, 2>, grid, sm, s, in, out, gt_old, gt_new, rcoarse, N, L, coarsest, ws, sc,
                         partials);
    if (resid)
      return launch_k<R>(k_wav_level1<R, 1>, grid, sm, s, in, out, gt_old, gt_new, rcoarse, N, L, coarsest, ws, sc,
                         partials);
    return launch_k<R>(k_wav_level1<R, 0>, grid, sm, s, in, out, gt_old, gt_new, rcoarse, N, L, coarsest, ws, sc,
                       partials);
  }
  dim3 grid(tiles, L, nd);
  if (resid == 2)
    return launch_k<R>(k_wav_levelj<R, 2>, grid, sm, s, in, out, gt_old, gt_new, rcoarse, N, M, L, coarsest, ws, sc,
                       partials);
  if (resid)
    return launch_k<R>(k_wav_levelj<R, 1>, grid, sm, s, in, out, gt_old, gt_new, rcoarse, N, M, L, coarsest, ws, sc,
                       partials);
  return launch_k<R>(k_wav_levelj<R, 0>, grid, sm, s, in, out, gt_old, gt_new, rcoarse, N, M, L, coarsest, ws, sc,
                     partials);
}

#define INST(R)                                                                                               \
  template int wav_level_blocks<R>(int, int, int, int);                                                           \
  template cudaError_t launch_wav_ll<R>(const R*, size_t, size_t, R*, int, int, int, const WavSet<R>*,            \
                                        cudaStream_t);                                                          \
  template cudaError_t launch_wav_level<R>(const R*, size_t, size_t, const R*, R*, const R*, R*, int, int, int,   \
                                           int, int, const WavSet<R>*, IterScalars<R>, double*, int, int, int*,  \
                                           cudaStream_t);
INST(float)
INST(double)
#undef INST

template cudaError_t launch_wav_analysis_full<float>(const float*, float*, float*, int, int, int, int, const int*,
                                                     cudaStream_t);
template cudaError_t launch_wav_synthesis_acc<float>(float*, float*, float*, int, int, int, int, const int*,
                                                     cudaStream_t);
template cudaError_t launch_wav_synthesis_acc<double>(double*, double*, double*, int, int, int, int, const int*,
                                                      cudaStream_t);
template cudaError_t launch_wav_bwd_point<float>(float*, const float*, const float*, float*, size_t, int,
                                                 const WavSet<float>*, float, float, double*, int*, cudaStream_t);

}  // namespace mf
