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
//   acc += sum_k w_k W_k^T (Gamma_T,k - Gamma_T,k+)              (every distinct basis)
// and the report's dual residual is ||acc||^2 + m_nu rho_V^2 ||d(S W_nu)||^2
// (orthonormal spectral bases).  Both Gamma_T buffers are complete states, so
// the change of every coefficient is at hand without extra storage; the
// synthesis runs the fused level kernels in their synthesis-only mode
// (wavelet.cu), level by level, through the level scratch of the iteration.
#include <cuda_runtime.h>

#include "mf_internal.cuh"
#include "reduce.cuh"

namespace mf {

namespace {

constexpr int DNT = 256;
constexpr int DPIX = 32;  // pixels per tile of the spectral part

// four consecutive values from a 16-byte aligned shared-memory address
__device__ __forceinline__ void ld4(const float* a, float (&v)[4]) {
  const float4 t = *reinterpret_cast<const float4*>(a);
  v[0] = t.x;
  v[1] = t.y;
  v[2] = t.z;
  v[3] = t.w;
}
__device__ __forceinline__ void ld4(const double* a, double (&v)[4]) {
  const double2 t0 = reinterpret_cast<const double2*>(a)[0], t1 = reinterpret_cast<const double2*>(a)[1];
  v[0] = t0.x;
  v[1] = t0.y;
  v[2] = t1.x;
  v[3] = t1.y;
}

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
// acc = (b - Gamma_P) - pre - (dGamma_S W_nu) W_nu^T per pixel spectrum, and
// ||dS||^2.  A tile is DPIX pixels; warp g of the NG warps owns the bands
// l = g + j NG (j < ROWS) of every pixel and accumulates them together, reading
// each dGamma_S value once; the DCT matrix is laid out [k][g][j] in shared
// memory so that a warp's coefficients of one k are contiguous (vector loads,
// the same address for every lane).
template <class R, int ROWS>
__global__ void __launch_bounds__(DNT) k_dual_spec(const R* __restrict__ b, const R* __restrict__ GP,
                                                    R* __restrict__ pre, const R* __restrict__ Sd,
                                                    const R* __restrict__ Sd0, const R* __restrict__ GSd,
                                                    const R* __restrict__ GSd0, const R* __restrict__ dctC, int NN,
                                                    int L, double* __restrict__ partials) {
  constexpr int NG = DNT / DPIX;
  static_assert(ROWS % 4 == 0, "vector loads of the coefficients");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* C2 = reinterpret_cast<R*>(smem_raw);  // [L][NG][ROWS]: C[k][g + j NG]
  R* dG = C2 + (size_t)L * NG * ROWS;      // [L][DPIX]
  const int p = threadIdx.x % DPIX, g = threadIdx.x / DPIX;
  for (int e = threadIdx.x; e < L * NG * ROWS; e += DNT) {
    const int k = e / (NG * ROWS), rem = e % (NG * ROWS);
    const int l = rem / ROWS + (rem % ROWS) * NG;
    C2[e] = l < L ? dctC[k * L + l] : (R)0;
  }
  R ds2 = 0;
  bool bad = false;
  for (int t = blockIdx.x; t < NN / DPIX; t += gridDim.x) {
    const size_t px = (size_t)t * DPIX + p;
    __syncthreads();  // the previous tile's dG is consumed (and C2 is written)
    for (int k = g; k < L; k += NG) {
      const size_t o = (size_t)k * NN + px;
      dG[k * DPIX + p] = GSd[o] - GSd0[o];
      const R d = Sd[o] - Sd0[o];
      ds2 = fma(d, d, ds2);
    }
    __syncthreads();
    R acc[ROWS];
#pragma unroll
    for (int j = 0; j < ROWS; j++) acc[j] = 0;
    for (int k = 0; k < L; k++) {
      const R d = dG[k * DPIX + p];
      const R* c = C2 + ((size_t)k * NG + g) * ROWS;
#pragma unroll
      for (int j = 0; j < ROWS; j += 4) {
        R c4[4];
        ld4(c + j, c4);
#pragma unroll
        for (int i = 0; i < 4; i++) acc[j + i] = fma(c4[i], d, acc[j + i]);
      }
    }
#pragma unroll
    for (int j = 0; j < ROWS; j++) {
      const int l = g + j * NG;
      if (l < L) {
        const size_t o = (size_t)l * NN + px;
        const R a = ((b[o] - GP[o]) - pre[o]) - acc[j];
        pre[o] = a;
        bad |= !isfinite(a);
      }
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

size_t dual_cubes() { return 3; }  // pre (then acc), S W_nu and Gamma_S W_nu snapshots

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
cudaError_t dual_spectral(mf_plan* p, cudaStream_t s) {
  R* base = (R*)p->dual;
  const size_t V = p->cube;
  const int N = p->N, L = p->L, NN = N * N;
  R *pre = base, *Sd0 = base + V, *GSd0 = base + 2 * V;
  constexpr int NG = DNT / DPIX;
  const unsigned gs = capped_grid((size_t)NN / DPIX);
  cudaError_t e;
  if (L <= 8 * NG) {  // up to 8 bands per warp (L <= 64)
    const size_t sm = sizeof(R) * ((size_t)L * NG * 8 + (size_t)L * DPIX);
    if ((e = cudaFuncSetAttribute(k_dual_spec<R, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm))) return e;
    k_dual_spec<R, 8><<<gs, DNT, sm, s>>>((const R*)p->b, (const R*)p->GP, pre, (const R*)p->Sd, Sd0,
                                          (const R*)p->GSd, GSd0, (const R*)p->dctC, NN, L, p->partials);
  } else if constexpr (sizeof(R) == 4) {  // L <= 128 (FP64 plans take at most 64 bands)
    const size_t sm = sizeof(R) * ((size_t)L * NG * 16 + (size_t)L * DPIX);
    if ((e = cudaFuncSetAttribute(k_dual_spec<R, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)))
      return e;
    k_dual_spec<R, 16><<<gs, DNT, sm, s>>>((const R*)p->b, (const R*)p->GP, pre, (const R*)p->Sd, Sd0,
                                           (const R*)p->GSd, GSd0, (const R*)p->dctC, NN, L, p->partials);
  } else {
    return cudaErrorInvalidValue;
  }
  if ((e = cudaGetLastError())) return e;
  return launch_finalize(p->partials, (int)gs, p->sums, 1, s);
}

template <class R>
R* dual_acc(mf_plan* p) {
  return (R*)p->dual;
}

template <class R>
cudaError_t dual_norm(mf_plan* p, cudaStream_t s) {
  const size_t V = p->cube;
  const unsigned gn = capped_grid((V + DNT - 1) / DNT);
  k_dual_norm<R><<<gn, DNT, 0, s>>>((const R*)p->dual, V, p->partials);
  cudaError_t e = cudaGetLastError();
  if (e) return e;
  return launch_finalize(p->partials, (int)gn, p->sums, 1, s);
}

template cudaError_t dual_snapshot<float>(mf_plan*, cudaStream_t);
template cudaError_t dual_snapshot<double>(mf_plan*, cudaStream_t);
template cudaError_t dual_spectral<float>(mf_plan*, cudaStream_t);
template cudaError_t dual_spectral<double>(mf_plan*, cudaStream_t);
template float* dual_acc<float>(mf_plan*);
template double* dual_acc<double>(mf_plan*);
template cudaError_t dual_norm<float>(mf_plan*, cudaStream_t);
template cudaError_t dual_norm<double>(mf_plan*, cudaStream_t);

}  // namespace mf
