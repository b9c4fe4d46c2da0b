// Dual residual of the ADMM of Section 3 (the stopping criterion it cites:
// Boyd et al. 2011, Sec. 3.3), computed on residual iterations.
//
// For the two-block split (X, V) | (P, T, S) of Algorithm 1 the dual residual
// is s = rho A^T B (z+ - z), z = (P, T, S), whose squared norm is
//   ||rho_P dP + rho_T W_s^T dT + rho_S dS||^2 + rho_V^2 ||dS W_nu||^2.
// P and T are never stored by the iteration, so the first term is formed from
// what is: the right-hand side of Eq. matB without H^T Y,
//   b = Gamma_P + rho_P P + Gamma_S + rho_S S + W_s^T (Gamma_T + rho_T T),
// gives
//   rho_P dP + rho_T W_s^T dT + rho_S dS = d(b - Gamma_P) - dGamma_S - W_s^T dGamma_T.
// Before step I the plan keeps pre = b - Gamma_P and the DCT-domain S W_nu and
// Gamma_S W_nu; after the iteration
//   acc = (b - Gamma_P) - pre - (dGamma_S W_nu) W_nu^T          (per pixel spectrum)
//   acc -= w_k W_k^T (Gamma_T,k+ - Gamma_T,k)                    (each distinct basis)
// and the report's dual residual is ||acc||^2 + rho_V^2 ||d(S W_nu)||^2 (W_nu
// orthonormal).  Both Gamma_T buffers are complete states, so the change of
// every coefficient is at hand without extra storage.
#include <cuda_runtime.h>

#include "mf_internal.cuh"
#include "reduce.cuh"

namespace mf {

template <class R>
cudaError_t launch_wav_synthesis_acc(R* coef, R* out, R* tmp, int N, int L, int J, int nd, const int* Ks,
                                     cudaStream_t s);

namespace {

constexpr int DNT = 256;
constexpr int DPIX = 32;  // pixels per tile of the spectral part

unsigned capped_grid(size_t items) {
  const size_t cap = MF_AUX_GRID;
  return (unsigned)(items < cap ? (items ? items : 1) : cap);
}

template <class R>
__global__ void k_dual_snap(const R* __restrict__ b, const R* __restrict__ GP, R* __restrict__ pre, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    pre[i] = b[i] - GP[i];
}

// acc (in pre) = (b - Gamma_P) - pre - sum_k C[k][l] d(Gamma_S W_nu)[k]; ||d(S W_nu)||^2 partials.
// Tiles of DPIX pixels; thread (g, p): pixel p of the tile, band / frequency rows g, g + 8, ...
template <class R>
__global__ void __launch_bounds__(DNT) k_dual_spec(const R* __restrict__ b, const R* __restrict__ GP,
                                                    R* __restrict__ pre, const R* __restrict__ Sd,
                                                    const R* __restrict__ Sd0, const R* __restrict__ GSd,
                                                    const R* __restrict__ GSd0, const R* __restrict__ dctC, int NN,
                                                    int L, double* __restrict__ partials) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* C = reinterpret_cast<R*>(smem_raw);  // C[k][l]
  R* dG = C + L * L;                       // [L][DPIX]
  const int p = threadIdx.x % DPIX, g = threadIdx.x / DPIX;
  constexpr int NG = DNT / DPIX;
  for (int e = threadIdx.x; e < L * L; e += DNT) C[e] = dctC[e];
  R ds2 = 0;
  bool bad = false;
  for (int t = blockIdx.x; t < NN / DPIX; t += gridDim.x) {
    const size_t px = (size_t)t * DPIX + p;
    __syncthreads();  // the previous tile's dG is consumed
    for (int k = g; k < L; k += NG) {
      const size_t o = (size_t)k * NN + px;
      dG[k * DPIX + p] = GSd[o] - GSd0[o];
      const R d = Sd[o] - Sd0[o];
      ds2 = fma(d, d, ds2);
    }
    __syncthreads();
    for (int l = g; l < L; l += NG) {
      const size_t o = (size_t)l * NN + px;
      R a = (b[o] - GP[o]) - pre[o];
      for (int k = 0; k < L; k++) a = fma(-C[k * L + l], dG[k * DPIX + p], a);
      pre[o] = a;
      bad |= !isfinite(a);
    }
  }
  R q[Q_COUNT];
#pragma unroll
  for (int i = 0; i < Q_COUNT; i++) q[i] = 0;
  q[Q_XMIN] = NoMin<R>::v;
  q[Q_DS2] = ds2;
  q[Q_NONFIN] = bad ? (R)1 : (R)0;
  block_reduce_write<DNT>(q, partials + (size_t)blockIdx.x * MF_NQ);
}

// work = -w (Gamma_T+ - Gamma_T) of one basis (all levels of every band)
template <class R>
__global__ void k_dual_gdiff(const R* __restrict__ gn, const R* __restrict__ go, R* __restrict__ work, R w,
                             size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    work[i] = -w * (gn[i] - go[i]);
}

template <class R>
__global__ void __launch_bounds__(DNT) k_dual_norm(const R* __restrict__ acc, size_t n,
                                                    double* __restrict__ partials) {
  R s = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    s = fma(acc[i], acc[i], s);
  R q[Q_COUNT];
#pragma unroll
  for (int i = 0; i < Q_COUNT; i++) q[i] = 0;
  q[Q_XMIN] = NoMin<R>::v;
  q[Q_DUALX] = s;
  block_reduce_write<DNT>(q, partials + (size_t)blockIdx.x * MF_NQ);
}

}  // namespace

size_t dual_cubes() { return 5; }  // pre, S W_nu and Gamma_S W_nu snapshots, basis work cube, synthesis scratch

template <class R>
cudaError_t dual_snapshot(mf_plan* p, cudaStream_t s) {
  R* base = (R*)p->dual;
  const size_t V = p->cube;
  k_dual_snap<R><<<capped_grid((V + DNT - 1) / DNT), DNT, 0, s>>>((const R*)p->b, (const R*)p->GP, base, V);
  cudaError_t e = cudaGetLastError();
  if (!e) e = cudaMemcpyAsync(base + V, p->Sd, V * sizeof(R), cudaMemcpyDeviceToDevice, s);
  if (!e) e = cudaMemcpyAsync(base + 2 * V, p->GSd, V * sizeof(R), cudaMemcpyDeviceToDevice, s);
  return e;
}

template <class R>
cudaError_t dual_finish(mf_plan* p, const R* gt_old, const R* gt_new, int J, int nd, const int* Ks, const R* w,
                        cudaStream_t s) {
  R* base = (R*)p->dual;
  const size_t V = p->cube;
  const int N = p->N, L = p->L, NN = N * N;
  R *pre = base, *Sd0 = base + V, *GSd0 = base + 2 * V, *work = base + 3 * V, *tmp = base + 4 * V;
  const size_t sm = sizeof(R) * ((size_t)L * L + (size_t)L * DPIX);
  cudaError_t e = cudaFuncSetAttribute(k_dual_spec<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e) return e;
  const unsigned gs = capped_grid((size_t)NN / DPIX);
  k_dual_spec<R><<<gs, DNT, sm, s>>>((const R*)p->b, (const R*)p->GP, pre, (const R*)p->Sd, Sd0, (const R*)p->GSd,
                                     GSd0, (const R*)p->dctC, NN, L, p->partials);
  if ((e = cudaGetLastError())) return e;
  if ((e = launch_finalize(p->partials, (int)gs, p->sums, 1, s))) return e;
  for (int k = 0; k < nd && !e; k++) {
    const unsigned g = capped_grid((V + DNT - 1) / DNT);
    k_dual_gdiff<R><<<g, DNT, 0, s>>>(gt_new + (size_t)k * V, gt_old + (size_t)k * V, work, w[k], V);
    e = cudaGetLastError();
    if (!e) e = launch_wav_synthesis_acc<R>(work, pre, tmp, N, L, J, 1, Ks + k, s);
  }
  if (e) return e;
  const unsigned gn = capped_grid((V + DNT - 1) / DNT);
  k_dual_norm<R><<<gn, DNT, 0, s>>>(pre, V, p->partials);
  if ((e = cudaGetLastError())) return e;
  return launch_finalize(p->partials, (int)gn, p->sums, 1, s);
}

template cudaError_t dual_snapshot<float>(mf_plan*, cudaStream_t);
template cudaError_t dual_snapshot<double>(mf_plan*, cudaStream_t);
template cudaError_t dual_finish<float>(mf_plan*, const float*, const float*, int, int, const int*, const float*,
                                        cudaStream_t);
template cudaError_t dual_finish<double>(mf_plan*, const double*, const double*, int, int, const int*,
                                         const double*, cudaStream_t);

}  // namespace mf
