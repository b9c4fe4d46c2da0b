// Steps II, IV, V and the matching duals of step VI (Algorithm 1), one pixel
// spectrum (the L values of a row of X) at a time, and the pointwise part of
// the next right-hand side (Eq. matB):
//   P~ = X - Gamma_P / rho_P,  P = max(0, P~),  Gamma_P += rho_P (P - X)      (II, VI)
//   V  = S_{mu_nu/rho_V}(S W_nu - Gamma_V / rho_V)              old S        (IV)
//   S  = ((Gamma_V + rho_V V) W_nu^T - Gamma_S + rho_S X) / (rho_V + rho_S)  (V, m_nu = 1)
//   Gamma_V += rho_V (V - S W_nu),  Gamma_S += rho_S (S - X)       new S     (VI)
//   b = Gamma_P + rho_P P + Gamma_S + rho_S S
// W_nu is the orthonormal DCT-II (Section 4), so S and Gamma_S are kept in the
// DCT domain (S W_nu, Gamma_S W_nu): step V becomes pointwise there and an
// iteration needs two length-L DCTs per pixel (X W_nu forward, and
// (Gamma_S + rho_S S) back), each a (pixels x L) . (L x L) contraction done here
// as a register-tiled FP32 product out of shared memory.
#include <cuda_runtime.h>

#include "mf_internal.cuh"
#include "reduce.cuh"

namespace mf {

constexpr int SP_NT = 256;

template <class R> struct V4;
template <> struct V4<float> {
  static __device__ __forceinline__ void ld(const float* p, float* v) {
    float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  }
  static __device__ __forceinline__ void st(float* p, const float* v) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
};
template <> struct V4<double> {
  static __device__ __forceinline__ void ld(const double* p, double* v) {
    double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
  static __device__ __forceinline__ void st(double* p, const double* v) {
    reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
  }
};

template <class R> __device__ __forceinline__ R soft_thr(R t, R tau) {
  const R a = fabs(t) - tau;
  return a > (R)0 ? copysign(a, t) : (R)0;
}

template <class R> __device__ __forceinline__ bool finite_(R v) { return isfinite(v); }

template <class R, int LP, int RESID>
__global__ void __launch_bounds__(SP_NT) k_spectral(const R* __restrict__ X, R* __restrict__ GP, R* __restrict__ Sd,
                                                     R* __restrict__ GV, R* __restrict__ GSd, R* __restrict__ b,
                                                     const R* __restrict__ dctC, int NN, int L, IterScalars<R> sc,
                                                     double* __restrict__ partials) {
  constexpr int PT = 4096 / LP;   // pixels per CTA
  constexpr int TP = PT / 4;      // thread columns (4 pixels each)
  static_assert((LP / 4) * TP == SP_NT, "tile");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* C = reinterpret_cast<R*>(smem_raw);   // C[k][l]
  R* CT = C + LP * LP;                      // CT[l][k]
  R* T = CT + LP * LP;                      // tile [LP][PT]: X, then U
  const int tid = threadIdx.x;
  const int tk = tid / TP, tp = tid % TP;
  const int p0 = blockIdx.x * PT;

  for (int e = tid; e < LP * LP; e += SP_NT) {
    const int k = e / LP, l = e % LP;
    const R v = (k < L && l < L) ? dctC[k * L + l] : (R)0;
    C[k * LP + l] = v;
    CT[l * LP + k] = v;
  }
  for (int e = tid; e < LP * (PT / 4); e += SP_NT) {
    const int l = e / (PT / 4), p = 4 * (e % (PT / 4));
    R v[4] = {0, 0, 0, 0};
    if (l < L && p0 + p < NN) V4<R>::ld(X + (size_t)l * NN + p0 + p, v);
    V4<R>::st(T + l * PT + p, v);
  }
  __syncthreads();

  const int kb = 4 * tk, pb = 4 * tp;
  const bool pix_ok = p0 + pb < NN;
  R xr[4][4];
#pragma unroll
  for (int a = 0; a < 4; a++) V4<R>::ld(T + (kb + a) * PT + pb, xr[a]);

  // x^[k][p] = sum_l C[k][l] X[l][p]
  R acc[4][4] = {};
#pragma unroll 4
  for (int l = 0; l < LP; l++) {
    R c4[4], x4[4];
    V4<R>::ld(CT + l * LP + kb, c4);
    V4<R>::ld(T + l * PT + pb, x4);
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
      for (int c = 0; c < 4; c++) acc[a][c] = fma(c4[a], x4[c], acc[a][c]);
  }

  // residual terms of this thread's 16 voxels, summed in the cube's precision and
  // folded into the FP64 partial rows once (FP64 arithmetic per voxel is slow)
  R r_dgv = 0, r_dgs = 0, r_l1 = 0, r_dgp = 0, r_x2 = 0, r_xmin = (R)3.0e38;
  bool r_bad = false;

  // DCT-domain part of steps IV, V and VI
  R u[4][4];
#pragma unroll
  for (int a = 0; a < 4; a++) {
    const int k = kb + a;
    if (k < L && pix_ok) {
      const size_t o = (size_t)k * NN + p0 + pb;
      R s[4], gv[4], gs[4];
      V4<R>::ld(Sd + o, s);
      V4<R>::ld(GV + o, gv);
      V4<R>::ld(GSd + o, gs);
#pragma unroll
      for (int c = 0; c < 4; c++) {
        const R xh = acc[a][c];
        const R v = soft_thr<R>(s[c] - gv[c] * sc.inv_rho_V, sc.tau_V);
        const R sn = (gv[c] + sc.rho_V * v - gs[c] + sc.rho_S * xh) * sc.inv_VS;
        const R gvn = gv[c] + sc.rho_V * (v - sn);
        const R gsn = gs[c] + sc.rho_S * (sn - xh);
        if (RESID) {
          const R dv = gvn - gv[c], ds = gsn - gs[c];
          r_dgv = fma(dv, dv, r_dgv);
          r_dgs = fma(ds, ds, r_dgs);
          r_l1 += fabs(xh);
          r_bad |= !finite_<R>(gvn) || !finite_<R>(gsn);
        }
        s[c] = sn;
        gv[c] = gvn;
        gs[c] = gsn;
        u[a][c] = gsn + sc.rho_S * sn;
      }
      V4<R>::st(Sd + o, s);
      V4<R>::st(GV + o, gv);
      V4<R>::st(GSd + o, gs);
    } else {
#pragma unroll
      for (int c = 0; c < 4; c++) u[a][c] = (R)0;
    }
  }
  __syncthreads();
#pragma unroll
  for (int a = 0; a < 4; a++) V4<R>::st(T + (kb + a) * PT + pb, u[a]);
  __syncthreads();

  // (Gamma_S + rho_S S)[l][p] = sum_k C[k][l] U[k][p]
  R bs[4][4] = {};
#pragma unroll 4
  for (int k = 0; k < LP; k++) {
    R c4[4], u4[4];
    V4<R>::ld(C + k * LP + kb, c4);
    V4<R>::ld(T + k * PT + pb, u4);
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
      for (int c = 0; c < 4; c++) bs[a][c] = fma(c4[a], u4[c], bs[a][c]);
  }

  // pixel-domain part: step II, Gamma_P, and b
#pragma unroll
  for (int a = 0; a < 4; a++) {
    const int l = kb + a;
    if (l < L && pix_ok) {
      const size_t o = (size_t)l * NN + p0 + pb;
      R gp[4], bo[4];
      V4<R>::ld(GP + o, gp);
#pragma unroll
      for (int c = 0; c < 4; c++) {
        const R x = xr[a][c];
        const R pt = x - gp[c] * sc.inv_rho_P;
        const R pp = pt > (R)0 ? pt : (R)0;
        const R gpn = gp[c] + sc.rho_P * (pp - x);
        if (RESID) {
          const R d = gpn - gp[c];
          r_dgp = fma(d, d, r_dgp);
          r_x2 = fma(x, x, r_x2);
          r_xmin = x < r_xmin ? x : r_xmin;
          r_bad |= !finite_<R>(x) || !finite_<R>(gpn);
        }
        gp[c] = gpn;
        bo[c] = gpn + sc.rho_P * pp + bs[a][c];
      }
      V4<R>::st(GP + o, gp);
      V4<R>::st(b + o, bo);
    }
  }
  if (RESID) {
    // in the cube's precision: FP32 plans take the FP32 warp stage of the reduction
    R q[Q_COUNT];
#pragma unroll
    for (int i = 0; i < Q_COUNT; i++) q[i] = 0;
    q[Q_DGV] = r_dgv;
    q[Q_DGS] = r_dgs;
    q[Q_L1NU] = r_l1;
    q[Q_DGP] = r_dgp;
    q[Q_X2] = r_x2;
    q[Q_XMIN] = r_xmin < (R)3.0e38 ? r_xmin : (R)1e300;
    q[Q_NONFIN] = r_bad ? (R)1 : (R)0;
    block_reduce_write<SP_NT>(q, partials + (size_t)blockIdx.x * MF_NQ);
  }
}

// The spectral step with a second spectral basis in the dictionary (Section 3,
// step V with m_nu orthonormal bases; the Chebyshev basis of Section 4): the
// dictionary is {DCT, B2} (DCT_ON) or {B2} alone.  S and Gamma_S stay in the
// DCT domain, so basis 2's coefficients of a spectrum in that domain are
// M (.) with M = C2 C^T (M[k2][k1]):
//   V2 = S_{mu_nu/rho_V}(M S^ - Gamma_V2 / rho_V)                   (IV, old S)
//   S^+ = ((Gamma_V + rho_V V) + M^T (Gamma_V2 + rho_V V2) - Gamma_S^ + rho_S X^)
//         / (m_nu rho_V + rho_S)                                     (V)
//   Gamma_V2 += rho_V (V2 - M S^+)                                   (VI, new S)
// and the DCT terms as in k_spectral when DCT_ON.  The plan keeps S2 = M S^ (S
// in the second basis) beside S^: the old one is read for step IV, the new one
// (computed for step VI anyway) written, so two L x L products per pixel
// spectrum are added (M^T Q2, M S^+), each staged through the shared tile.
template <class R, int LP, int RESID, bool DCT_ON>
__global__ void __launch_bounds__(SP_NT) k_spectral_b2(const R* __restrict__ X, R* __restrict__ GP, R* __restrict__ Sd,
                                                        R* __restrict__ GV, R* __restrict__ GV2, R* __restrict__ GSd,
                                                        R* __restrict__ S2, R* __restrict__ b,
                                                        const R* __restrict__ dctC, const R* __restrict__ Mb, int NN,
                                                        int L, IterScalars<R> sc, double* __restrict__ partials) {
  constexpr int PT = 4096 / LP;
  constexpr int TP = PT / 4;
  static_assert((LP / 4) * TP == SP_NT, "tile");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* C = reinterpret_cast<R*>(smem_raw);  // C[k][l]
  R* CT = C + LP * LP;                     // CT[l][k]
  R* M = CT + LP * LP;                     // M[k2][k1]
  R* MT = M + LP * LP;                     // MT[k1][k2]
  R* T = MT + LP * LP;                     // tile [LP][PT]
  const int tid = threadIdx.x;
  const int tk = tid / TP, tp = tid % TP;
  const int p0 = blockIdx.x * PT;
  for (int e = tid; e < LP * LP; e += SP_NT) {
    const int k = e / LP, l = e % LP;
    const R v = (k < L && l < L) ? dctC[k * L + l] : (R)0;
    C[k * LP + l] = v;
    CT[l * LP + k] = v;
    const R m = (k < L && l < L) ? Mb[k * L + l] : (R)0;
    M[k * LP + l] = m;
    MT[l * LP + k] = m;
  }
  auto load_tile = [&](const R* src) {
    for (int e = tid; e < LP * (PT / 4); e += SP_NT) {
      const int l = e / (PT / 4), p = 4 * (e % (PT / 4));
      R v[4] = {0, 0, 0, 0};
      if (l < L && p0 + p < NN) V4<R>::ld(src + (size_t)l * NN + p0 + p, v);
      V4<R>::st(T + l * PT + p, v);
    }
  };
  {
    // L2 prefetch of the tile's rows of the state arrays read after the first
    // product (S2, Gamma_V2, S, Gamma_S, Gamma_P, Gamma_V): one per 128-byte line
    constexpr int LINES = (PT * (int)sizeof(R) + 127) / 128;
    const R* arr[6] = {S2, GV2, Sd, GSd, GP, DCT_ON ? GV : Sd};
    for (int e = tid; e < (DCT_ON ? 6 : 5) * L * LINES; e += SP_NT) {
      const int a = e / (L * LINES), r = e % (L * LINES);
      const int l = r / LINES, ln = r % LINES;
      asm volatile("prefetch.global.L2 [%0];" ::"l"(arr[a] + (size_t)l * NN + p0 + ln * (128 / (int)sizeof(R))));
    }
  }
  // out[a][c] = sum_l A[kb + a][l] T[l][pb + c], with AT = A transposed in shared memory
  auto product = [&](const R* AT, R (&out)[4][4], int kb, int pb) {
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
      for (int c = 0; c < 4; c++) out[a][c] = 0;
#pragma unroll 4
    for (int l = 0; l < LP; l++) {
      R c4[4], x4[4];
      V4<R>::ld(AT + l * LP + kb, c4);
      V4<R>::ld(T + l * PT + pb, x4);
#pragma unroll
      for (int a = 0; a < 4; a++)
#pragma unroll
        for (int c = 0; c < 4; c++) out[a][c] = fma(c4[a], x4[c], out[a][c]);
    }
  };
  auto store_tile = [&](const R (&v)[4][4], int kb, int pb) {
#pragma unroll
    for (int a = 0; a < 4; a++) V4<R>::st(T + (kb + a) * PT + pb, v[a]);
  };
  load_tile(X);
  __syncthreads();
  const int kb = 4 * tk, pb = 4 * tp;
  const bool pix_ok = p0 + pb < NN;
  R xr[4][4];
#pragma unroll
  for (int a = 0; a < 4; a++) V4<R>::ld(T + (kb + a) * PT + pb, xr[a]);
  R xh[4][4];
  product(CT, xh, kb, pb);  // X^ = C X
  R r_dgv = 0, r_dgs = 0, r_l1 = 0, r_dgp = 0, r_x2 = 0, r_xmin = NoMin<R>::v;
  bool r_bad = false;
  if (RESID) {
    // ||X W_2||_1 = sum |M X^| (and |X^| when the DCT is in the dictionary)
    __syncthreads();
    store_tile(xh, kb, pb);
    __syncthreads();
    R mx[4][4];
    product(MT, mx, kb, pb);
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
      for (int c = 0; c < 4; c++)
        if (kb + a < L && pix_ok) r_l1 += fabs(mx[a][c]) + (DCT_ON ? fabs(xh[a][c]) : (R)0);
  }
  // basis-2 coefficients of the old S (kept by the plan)
  R v2[4][4], g2[4][4], q2[4][4];
  {
    R w2[4][4];
#pragma unroll
    for (int a = 0; a < 4; a++) {
      const int k = kb + a;
      if (k < L && pix_ok) {
        V4<R>::ld(GV2 + (size_t)k * NN + p0 + pb, g2[a]);
        V4<R>::ld(S2 + (size_t)k * NN + p0 + pb, w2[a]);
      } else {
        for (int c = 0; c < 4; c++) g2[a][c] = w2[a][c] = 0;
      }
#pragma unroll
      for (int c = 0; c < 4; c++) {
        v2[a][c] = soft_thr<R>(w2[a][c] - g2[a][c] * sc.inv_rho_V, sc.tau_V);
        q2[a][c] = (k < L && pix_ok) ? g2[a][c] + sc.rho_V * v2[a][c] : (R)0;
      }
    }
  }
  __syncthreads();
  store_tile(q2, kb, pb);
  __syncthreads();
  R z[4][4];
  product(M, z, kb, pb);  // M^T Q2 in the DCT domain: sum_k2 M[k2][k1] Q2[k2]
  // DCT-domain part of steps IV, V and VI
  R u[4][4], sn_t[4][4];
#pragma unroll
  for (int a = 0; a < 4; a++) {
    const int k = kb + a;
#pragma unroll
    for (int c = 0; c < 4; c++) u[a][c] = sn_t[a][c] = (R)0;
    if (k < L && pix_ok) {
      const size_t o = (size_t)k * NN + p0 + pb;
      R s[4], gv[4], gs[4];
      V4<R>::ld(Sd + o, s);
      V4<R>::ld(GSd + o, gs);
      if (DCT_ON) V4<R>::ld(GV + o, gv);
#pragma unroll
      for (int c = 0; c < 4; c++) {
        R q1 = 0, v1 = 0;
        if (DCT_ON) {
          v1 = soft_thr<R>(s[c] - gv[c] * sc.inv_rho_V, sc.tau_V);
          q1 = gv[c] + sc.rho_V * v1;
        }
        const R sn = (q1 + z[a][c] - gs[c] + sc.rho_S * xh[a][c]) * sc.inv_VS;
        const R gsn = gs[c] + sc.rho_S * (sn - xh[a][c]);
        if (DCT_ON) {
          const R gvn = gv[c] + sc.rho_V * (v1 - sn);
          if (RESID) {
            const R dv = gvn - gv[c];
            r_dgv = fma(dv, dv, r_dgv);
            r_bad |= !finite_<R>(gvn);
          }
          gv[c] = gvn;
        }
        if (RESID) {
          const R ds = gsn - gs[c];
          r_dgs = fma(ds, ds, r_dgs);
          r_bad |= !finite_<R>(gsn);
        }
        s[c] = sn;
        gs[c] = gsn;
        sn_t[a][c] = sn;
        u[a][c] = gsn + sc.rho_S * sn;
      }
      V4<R>::st(Sd + o, s);
      V4<R>::st(GSd + o, gs);
      if (DCT_ON) V4<R>::st(GV + o, gv);
    }
  }
  // Gamma_V2 with the new S
  __syncthreads();
  store_tile(sn_t, kb, pb);
  __syncthreads();
  {
    R m2[4][4];
    product(MT, m2, kb, pb);
#pragma unroll
    for (int a = 0; a < 4; a++) {
      const int k = kb + a;
      if (k < L && pix_ok) {
        R gn[4];
        V4<R>::st(S2 + (size_t)k * NN + p0 + pb, m2[a]);  // S2 of the new S
#pragma unroll
        for (int c = 0; c < 4; c++) {
          gn[c] = g2[a][c] + sc.rho_V * (v2[a][c] - m2[a][c]);
          if (RESID) {
            const R d = gn[c] - g2[a][c];
            r_dgv = fma(d, d, r_dgv);
            r_bad |= !finite_<R>(gn[c]);
          }
        }
        V4<R>::st(GV2 + (size_t)k * NN + p0 + pb, gn);
      }
    }
  }
  __syncthreads();
  store_tile(u, kb, pb);
  __syncthreads();
  R bs[4][4];
  product(C, bs, kb, pb);  // (Gamma_S + rho_S S)[l] = sum_k C[k][l] U[k]
  // pixel-domain part: step II, Gamma_P, and b
#pragma unroll
  for (int a = 0; a < 4; a++) {
    const int l = kb + a;
    if (l < L && pix_ok) {
      const size_t o = (size_t)l * NN + p0 + pb;
      R gp[4], bo[4];
      V4<R>::ld(GP + o, gp);
#pragma unroll
      for (int c = 0; c < 4; c++) {
        const R x = xr[a][c];
        const R pt = x - gp[c] * sc.inv_rho_P;
        const R pp = pt > (R)0 ? pt : (R)0;
        const R gpn = gp[c] + sc.rho_P * (pp - x);
        if (RESID) {
          const R d = gpn - gp[c];
          r_dgp = fma(d, d, r_dgp);
          r_x2 = fma(x, x, r_x2);
          r_xmin = x < r_xmin ? x : r_xmin;
          r_bad |= !finite_<R>(x) || !finite_<R>(gpn);
        }
        gp[c] = gpn;
        bo[c] = gpn + sc.rho_P * pp + bs[a][c];
      }
      V4<R>::st(GP + o, gp);
      V4<R>::st(b + o, bo);
    }
  }
  if (RESID) {
    R q[Q_COUNT];
#pragma unroll
    for (int i = 0; i < Q_COUNT; i++) q[i] = 0;
    q[Q_DGV] = r_dgv;
    q[Q_DGS] = r_dgs;
    q[Q_L1NU] = r_l1;
    q[Q_DGP] = r_dgp;
    q[Q_X2] = r_x2;
    q[Q_XMIN] = r_xmin;
    q[Q_NONFIN] = r_bad ? (R)1 : (R)0;
    block_reduce_write<SP_NT>(q, partials + (size_t)blockIdx.x * MF_NQ);
  }
}

template <class R, int LP, bool DCT_ON>
static cudaError_t spectral_b2_lp(const R* X, R* GP, R* Sd, R* GV, R* GV2, R* GSd, R* S2, R* b, const R* dctC,
                                  const R* Mb, int N, int L, IterScalars<R> sc, double* partials, int resid,
                                  cudaStream_t s) {
  constexpr int PT = 4096 / LP;
  const int NN = N * N;
  const int blocks = (NN + PT - 1) / PT;
  const size_t sm = sizeof(R) * (4 * LP * LP + LP * PT);
  cudaError_t e;
  if (resid) {
    e = cudaFuncSetAttribute(k_spectral_b2<R, LP, 1, DCT_ON>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_spectral_b2<R, LP, 1, DCT_ON><<<blocks, SP_NT, sm, s>>>(X, GP, Sd, GV, GV2, GSd, S2, b, dctC, Mb, NN, L, sc,
                                                               partials);
  } else {
    e = cudaFuncSetAttribute(k_spectral_b2<R, LP, 0, DCT_ON>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_spectral_b2<R, LP, 0, DCT_ON><<<blocks, SP_NT, sm, s>>>(X, GP, Sd, GV, GV2, GSd, S2, b, dctC, Mb, NN, L, sc,
                                                               partials);
  }
  return cudaGetLastError();
}

template <class R, bool DCT_ON>
static cudaError_t spectral_b2_dispatch(const R* X, R* GP, R* Sd, R* GV, R* GV2, R* GSd, R* S2, R* b, const R* dctC,
                                        const R* Mb, int N, int L, IterScalars<R> sc, double* partials, int resid,
                                        cudaStream_t s);

// Adjoint of the spectral step (steps II, IV, V and their duals, and the
// pointwise part of b) for the tied penalty rho, with the forward recomputed
// from its inputs (X, old Gamma_P, S^, Gamma_V, Gamma_S^).  In: bb = cotangent
// of b; cotangents of the outputs Gamma_P', S^', Gamma_V', Gamma_S^' in
// GPc, Sc, GVc, GSc (overwritten with the cotangents of the old values).
// Out: Xc = cotangent of X from this step; d mu_nu and d rho partials.
template <class R, int LP>
__global__ void __launch_bounds__(SP_NT) k_spectral_bwd(const R* __restrict__ X, const R* __restrict__ GP,
                                                         const R* __restrict__ Sd, const R* __restrict__ GV,
                                                         const R* __restrict__ GSd, const R* __restrict__ bb,
                                                         R* __restrict__ GPc, R* __restrict__ Sc, R* __restrict__ GVc,
                                                         R* __restrict__ GSc, R* __restrict__ Xc,
                                                         const R* __restrict__ dctC, int NN, int L, R rho, R mu_nu,
                                                         double* __restrict__ partials) {
  constexpr int PT = 4096 / LP;
  constexpr int TP = PT / 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* C = reinterpret_cast<R*>(smem_raw);
  R* CT = C + LP * LP;
  R* T1 = CT + LP * LP;  // X, then the cotangent of X^
  R* T2 = T1 + LP * PT;  // b_bar
  const int tid = threadIdx.x;
  const int tk = tid / TP, tp = tid % TP;
  const int p0 = blockIdx.x * PT;
  for (int e = tid; e < LP * LP; e += SP_NT) {
    const int k = e / LP, l = e % LP;
    const R v = (k < L && l < L) ? dctC[k * L + l] : (R)0;
    C[k * LP + l] = v;
    CT[l * LP + k] = v;
  }
  for (int e = tid; e < LP * (PT / 4); e += SP_NT) {
    const int l = e / (PT / 4), p = 4 * (e % (PT / 4));
    R v[4] = {0, 0, 0, 0}, w[4] = {0, 0, 0, 0};
    if (l < L && p0 + p < NN) {
      V4<R>::ld(X + (size_t)l * NN + p0 + p, v);
      V4<R>::ld(bb + (size_t)l * NN + p0 + p, w);
    }
    V4<R>::st(T1 + l * PT + p, v);
    V4<R>::st(T2 + l * PT + p, w);
  }
  __syncthreads();
  const int kb = 4 * tk, pb = 4 * tp;
  const bool pix_ok = p0 + pb < NN;
  R xr[4][4], br[4][4];
#pragma unroll
  for (int a = 0; a < 4; a++) {
    V4<R>::ld(T1 + (kb + a) * PT + pb, xr[a]);
    V4<R>::ld(T2 + (kb + a) * PT + pb, br[a]);
  }
  R xh[4][4] = {}, gh[4][4] = {};
#pragma unroll 4
  for (int l = 0; l < LP; l++) {
    R c4[4], x4[4], b4[4];
    V4<R>::ld(CT + l * LP + kb, c4);
    V4<R>::ld(T1 + l * PT + pb, x4);
    V4<R>::ld(T2 + l * PT + pb, b4);
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
      for (int c = 0; c < 4; c++) {
        xh[a][c] = fma(c4[a], x4[c], xh[a][c]);
        gh[a][c] = fma(c4[a], b4[c], gh[a][c]);
      }
  }
  // each voxel's gradient terms in the cube's precision, summed in FP64 (one add per
  // term: FP64 multiplies per voxel are slow)
  double dmunu_r = 0, drho_r = 0;
  const R irho = (R)1 / rho, tauv = mu_nu / rho;
  R xhb[4][4];
#pragma unroll
  for (int a = 0; a < 4; a++) {
    const int k = kb + a;
#pragma unroll
    for (int c = 0; c < 4; c++) xhb[a][c] = 0;
    if (k < L && pix_ok) {
      const size_t o = (size_t)k * NN + p0 + pb;
      R s[4], gv[4], gs[4], sc_[4], gvc[4], gsc[4];
      V4<R>::ld(Sd + o, s);
      V4<R>::ld(GV + o, gv);
      V4<R>::ld(GSd + o, gs);
      V4<R>::ld(Sc + o, sc_);
      V4<R>::ld(GVc + o, gvc);
      V4<R>::ld(GSc + o, gsc);
#pragma unroll
      for (int c = 0; c < 4; c++) {
        // forward recomputation
        const R vt = s[c] - gv[c] * irho;
        const bool mv = fabs(vt) > tauv;
        const R sv = vt > 0 ? (R)1 : (vt < 0 ? (R)-1 : (R)0);
        const R v = mv ? vt - tauv * sv : (R)0;
        const R sn = (gv[c] + rho * v - gs[c] + rho * xh[a][c]) * ((R)0.5 * irho);
        // cotangents of the outputs
        const R A1 = gsc[c] + gh[a][c];         // Gamma_S^'
        const R A2 = sc_[c] + rho * gh[a][c];   // S^' (outside the duals)
        const R C1 = gvc[c];                    // Gamma_V'
        drho_r += (double)(gh[a][c] * sn);
        const R Sb = A2 - rho * C1 + rho * A1;  // total on S^'
        R Vb = rho * C1 + (R)0.5 * Sb;
        drho_r += (double)(C1 * (v - sn) + A1 * (sn - xh[a][c]) +
                Sb * ((v + xh[a][c]) * ((R)0.5 * irho) - sn * irho));
        const R vtb = mv ? Vb : (R)0;
        const R taub = mv ? -sv * Vb : (R)0;
        dmunu_r += (double)(taub * irho);
        drho_r += (double)((vtb * gv[c] - taub * mu_nu) * irho * irho);
        sc_[c] = vtb;
        gvc[c] = C1 + (R)0.5 * Sb * irho - vtb * irho;
        gsc[c] = A1 - (R)0.5 * Sb * irho;
        xhb[a][c] = -rho * A1 + (R)0.5 * Sb;
      }
      V4<R>::st(Sc + o, sc_);
      V4<R>::st(GVc + o, gvc);
      V4<R>::st(GSc + o, gsc);
    }
  }
  __syncthreads();
#pragma unroll
  for (int a = 0; a < 4; a++) V4<R>::st(T1 + (kb + a) * PT + pb, xhb[a]);
  __syncthreads();
  R xs[4][4] = {};
#pragma unroll 4
  for (int k = 0; k < LP; k++) {
    R c4[4], u4[4];
    V4<R>::ld(C + k * LP + kb, c4);
    V4<R>::ld(T1 + k * PT + pb, u4);
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
      for (int c = 0; c < 4; c++) xs[a][c] = fma(c4[a], u4[c], xs[a][c]);
  }
#pragma unroll
  for (int a = 0; a < 4; a++) {
    const int l = kb + a;
    if (l < L && pix_ok) {
      const size_t o = (size_t)l * NN + p0 + pb;
      R gp[4], gpc[4], out[4];
      V4<R>::ld(GP + o, gp);
      V4<R>::ld(GPc + o, gpc);
#pragma unroll
      for (int c = 0; c < 4; c++) {
        const R x = xr[a][c];
        const R pt = x - gp[c] * irho;
        const bool mp = pt > 0;
        const R pp = mp ? pt : (R)0;
        const R B1 = gpc[c] + br[a][c];  // Gamma_P' (its own cotangent plus b's)
        const R Pb = rho * br[a][c] + rho * B1;
        const R ptb = mp ? Pb : (R)0;
        drho_r += (double)(br[a][c] * pp + B1 * (pp - x) + ptb * gp[c] * irho * irho);
        out[c] = xs[a][c] + ptb - rho * B1;
        gpc[c] = B1 - ptb * irho;
      }
      V4<R>::st(GPc + o, gpc);
      V4<R>::st(Xc + o, out);
    }
  }
  double q[Q_COUNT];
#pragma unroll
  for (int i = 0; i < Q_COUNT; i++) q[i] = 0.0;
  q[Q_XMIN] = 1e300;
  q[1] = dmunu_r;
  q[2] = drho_r;
  block_reduce_write<SP_NT>(q, partials + (size_t)blockIdx.x * MF_NQ);
}

template <class R, int LP>
static cudaError_t spectral_bwd_lp(const R* X, const R* GP, const R* Sd, const R* GV, const R* GSd, const R* bb,
                                   R* GPc, R* Sc, R* GVc, R* GSc, R* Xc, const R* dctC, int N, int L, R rho,
                                   R mu_nu, double* partials, int* nblocks, cudaStream_t s) {
  constexpr int PT = 4096 / LP;
  const int NN = N * N;
  const int blocks = (NN + PT - 1) / PT;
  *nblocks = blocks;
  const size_t sm = sizeof(R) * (2 * LP * LP + 2 * LP * PT);
  cudaError_t e = cudaFuncSetAttribute(k_spectral_bwd<R, LP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_spectral_bwd<R, LP><<<blocks, SP_NT, sm, s>>>(X, GP, Sd, GV, GSd, bb, GPc, Sc, GVc, GSc, Xc, dctC, NN, L, rho,
                                                  mu_nu, partials);
  return cudaGetLastError();
}

template <class R, int LP>
static cudaError_t spectral_lp(const R* X, R* GP, R* Sd, R* GV, R* GSd, R* b, const R* dctC, int N, int L,
                               IterScalars<R> sc, double* partials, int resid, cudaStream_t s) {
  constexpr int PT = 4096 / LP;
  const int NN = N * N;
  const int blocks = (NN + PT - 1) / PT;
  const size_t sm = sizeof(R) * (2 * LP * LP + LP * PT);
  cudaError_t e;
  if (resid) {
    e = cudaFuncSetAttribute(k_spectral<R, LP, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_spectral<R, LP, 1><<<blocks, SP_NT, sm, s>>>(X, GP, Sd, GV, GSd, b, dctC, NN, L, sc, partials);
  } else {
    e = cudaFuncSetAttribute(k_spectral<R, LP, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_spectral<R, LP, 0><<<blocks, SP_NT, sm, s>>>(X, GP, Sd, GV, GSd, b, dctC, NN, L, sc, partials);
  }
  return cudaGetLastError();
}

static int padded_L(int L) {
  int lp = 8;
  while (lp < L) lp *= 2;
  return lp;
}

template <class R>
int spectral_blocks(int N, int L) {
  const int PT = 4096 / padded_L(L);
  return (N * N + PT - 1) / PT;
}

template <class R>
cudaError_t launch_spectral(const R* X, R* GP, R* Sd, R* GV, R* GSd, R* b, const R* dctC, int N, int L,
                            IterScalars<R> sc, double* partials, int resid, cudaStream_t s) {
  switch (padded_L(L)) {
    case 8: return spectral_lp<R, 8>(X, GP, Sd, GV, GSd, b, dctC, N, L, sc, partials, resid, s);
    case 16: return spectral_lp<R, 16>(X, GP, Sd, GV, GSd, b, dctC, N, L, sc, partials, resid, s);
    case 32: return spectral_lp<R, 32>(X, GP, Sd, GV, GSd, b, dctC, N, L, sc, partials, resid, s);
    case 64: return spectral_lp<R, 64>(X, GP, Sd, GV, GSd, b, dctC, N, L, sc, partials, resid, s);
    case 128:
      if (sizeof(R) == 8) return cudaErrorInvalidValue;
      return spectral_lp<R, 128>(X, GP, Sd, GV, GSd, b, dctC, N, L, sc, partials, resid, s);
    default: return cudaErrorInvalidValue;
  }
}

template <class R>
cudaError_t launch_spectral_bwd(const R* X, const R* GP, const R* Sd, const R* GV, const R* GSd, const R* bb, R* GPc,
                                R* Sc, R* GVc, R* GSc, R* Xc, const R* dctC, int N, int L, R rho, R mu_nu,
                                double* partials, int* nblocks, cudaStream_t s) {
  switch (padded_L(L)) {
    case 8: return spectral_bwd_lp<R, 8>(X, GP, Sd, GV, GSd, bb, GPc, Sc, GVc, GSc, Xc, dctC, N, L, rho, mu_nu,
                                         partials, nblocks, s);
    case 16: return spectral_bwd_lp<R, 16>(X, GP, Sd, GV, GSd, bb, GPc, Sc, GVc, GSc, Xc, dctC, N, L, rho, mu_nu,
                                           partials, nblocks, s);
    case 32: return spectral_bwd_lp<R, 32>(X, GP, Sd, GV, GSd, bb, GPc, Sc, GVc, GSc, Xc, dctC, N, L, rho, mu_nu,
                                           partials, nblocks, s);
    case 64: return spectral_bwd_lp<R, 64>(X, GP, Sd, GV, GSd, bb, GPc, Sc, GVc, GSc, Xc, dctC, N, L, rho, mu_nu,
                                           partials, nblocks, s);
    default: return cudaErrorInvalidValue;
  }
}
template cudaError_t launch_spectral_bwd<float>(const float*, const float*, const float*, const float*,
                                                const float*, const float*, float*, float*, float*, float*, float*,
                                                const float*, int, int, float, float, double*, int*, cudaStream_t);

template cudaError_t launch_spectral<float>(const float*, float*, float*, float*, float*, float*, const float*, int,
                                            int, IterScalars<float>, double*, int, cudaStream_t);
template cudaError_t launch_spectral<double>(const double*, double*, double*, double*, double*, double*,
                                             const double*, int, int, IterScalars<double>, double*, int,
                                             cudaStream_t);
template int spectral_blocks<float>(int, int);
template int spectral_blocks<double>(int, int);

template <class R, bool DCT_ON>
static cudaError_t spectral_b2_dispatch(const R* X, R* GP, R* Sd, R* GV, R* GV2, R* GSd, R* S2, R* b, const R* dctC,
                                        const R* Mb, int N, int L, IterScalars<R> sc, double* partials, int resid,
                                        cudaStream_t s) {
  switch (padded_L(L)) {
    case 8: return spectral_b2_lp<R, 8, DCT_ON>(X, GP, Sd, GV, GV2, GSd, S2, b, dctC, Mb, N, L, sc, partials, resid, s);
    case 16: return spectral_b2_lp<R, 16, DCT_ON>(X, GP, Sd, GV, GV2, GSd, S2, b, dctC, Mb, N, L, sc, partials, resid, s);
    case 32: return spectral_b2_lp<R, 32, DCT_ON>(X, GP, Sd, GV, GV2, GSd, S2, b, dctC, Mb, N, L, sc, partials, resid, s);
    case 64: return spectral_b2_lp<R, 64, DCT_ON>(X, GP, Sd, GV, GV2, GSd, S2, b, dctC, Mb, N, L, sc, partials, resid, s);
    default: return cudaErrorInvalidValue;
  }
}

// S2[k][p] = sum_l M[k][l] S^[l][p]: one thread per (band k, pixel p), pixels
// fastest (coalesced); used only when the state was set from outside.
template <class R>
__global__ void k_s2_from_sd(const R* __restrict__ Mb, const R* __restrict__ Sd, R* __restrict__ S2, size_t NN,
                             int L) {
  const size_t total = NN * L;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(i / NN);
    const size_t pix = i - (size_t)k * NN;
    R acc = 0;
    for (int l = 0; l < L; l++) acc = fma(Mb[k * L + l], Sd[(size_t)l * NN + pix], acc);
    S2[i] = acc;
  }
}

template <class R>
cudaError_t launch_s2_from_sd(const R* Mb, const R* Sd, R* S2, int N, int L, cudaStream_t s) {
  const size_t total = (size_t)N * N * L;
  const size_t blocks = (total + 255) / 256;
  k_s2_from_sd<R><<<(unsigned)(blocks < 152 * 32 ? blocks : 152 * 32), 256, 0, s>>>(Mb, Sd, S2, (size_t)N * N, L);
  return cudaGetLastError();
}
template cudaError_t launch_s2_from_sd<float>(const float*, const float*, float*, int, int, cudaStream_t);
template cudaError_t launch_s2_from_sd<double>(const double*, const double*, double*, int, int, cudaStream_t);

template <class R>
cudaError_t launch_spectral_b2(const R* X, R* GP, R* Sd, R* GV, R* GV2, R* GSd, R* S2, R* b, const R* dctC, const R* Mb,
                               int dct_on, int N, int L, IterScalars<R> sc, double* partials, int resid,
                               cudaStream_t s) {
  if (dct_on) return spectral_b2_dispatch<R, true>(X, GP, Sd, GV, GV2, GSd, S2, b, dctC, Mb, N, L, sc, partials, resid, s);
  return spectral_b2_dispatch<R, false>(X, GP, Sd, GV, GV2, GSd, S2, b, dctC, Mb, N, L, sc, partials, resid, s);
}
template cudaError_t launch_spectral_b2<float>(const float*, float*, float*, float*, float*, float*, float*, float*,
                                               const float*, const float*, int, int, int, IterScalars<float>,
                                               double*, int, cudaStream_t);
template cudaError_t launch_spectral_b2<double>(const double*, double*, double*, double*, double*, double*, double*, double*,
                                                const double*, const double*, int, int, int, IterScalars<double>,
                                                double*, int, cudaStream_t);

// FP64 fold of the per-block partials into sums[MF_NQ]: a fixed thread count
// and a fixed tree order, so the result does not depend on scheduling.
constexpr int FIN_NT = 256;
__global__ void __launch_bounds__(FIN_NT) k_finalize(const double* __restrict__ partials, int nblocks,
                                                      double* __restrict__ sums, int accumulate) {
  __shared__ double red[Q_COUNT][FIN_NT];
  double v[Q_COUNT];
#pragma unroll
  for (int q = 0; q < Q_COUNT; q++) v[q] = (q == Q_XMIN) ? 1e300 : 0.0;
  for (int i = threadIdx.x; i < nblocks; i += FIN_NT) {
#pragma unroll
    for (int q = 0; q < Q_COUNT; q++) {
      const double x = partials[(size_t)i * MF_NQ + q];
      v[q] = (q == Q_XMIN) ? fmin(v[q], x) : v[q] + x;
    }
  }
#pragma unroll
  for (int q = 0; q < Q_COUNT; q++) red[q][threadIdx.x] = v[q];
  __syncthreads();
  for (int w = FIN_NT / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
#pragma unroll
      for (int q = 0; q < Q_COUNT; q++) {
        const double a = red[q][threadIdx.x], c = red[q][threadIdx.x + w];
        red[q][threadIdx.x] = (q == Q_XMIN) ? fmin(a, c) : a + c;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x < Q_COUNT) {
    const int q = threadIdx.x;
    const double r = red[q][0];
    if (accumulate) sums[q] = (q == Q_XMIN) ? fmin(sums[q], r) : sums[q] + r;
    else sums[q] = r;
  }
}

cudaError_t launch_finalize(const double* partials, int nblocks, double* sums, int accumulate, cudaStream_t s) {
  k_finalize<<<1, FIN_NT, 0, s>>>(partials, nblocks, sums, accumulate);
  return cudaGetLastError();
}

}  // namespace mf
