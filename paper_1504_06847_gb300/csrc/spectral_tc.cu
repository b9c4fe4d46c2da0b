// Precision form of the spectral step (steps II, IV, V, VI; Algorithm 1):
// the same arithmetic as spectral.cu, with the two DCT contractions of an
// iteration (X W_nu and (Gamma_S + rho_S S) W_nu^T, each a (pixels x L).(L x L)
// product) on the tcgen05 tensor cores.  Operands are split into two BF16
// terms, a = a_hi + a_lo, and each product is a_hi b_hi + a_hi b_lo + a_lo b_hi
// accumulated in FP32 in tensor memory (the a_lo b_lo term, ~2^-16 relative,
// is dropped).
//
// One CTA = 128 pixels = the M dimension of the MMA; after tcgen05.ld each
// thread holds a part of one pixel's spectrum for the pointwise updates (warps
// w, w + 4, ... read the same tensor-memory lanes, 32 (w mod 4) onwards).
// Operand layout in shared memory: no swizzle, K-major core matrices of
// 8 rows x 16 bytes; element (r, k) of an R x K operand sits at byte
// (r / 8) SBO + (k / 8) LBO + (r % 8) 16 + (k % 8) 2 with LBO = 128 and
// SBO = (K / 8) 128.  Every wait on the MMA completion is bounded: on expiry
// the CTA records an error word, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstring>

#include "mf_internal.cuh"
#include "reduce.cuh"

namespace mf {

namespace {

constexpr int TC_M = 128;       // pixels per CTA (MMA M)
// Threads per pixel: four (each on a quarter of the spectral axis) when a
// quarter is a whole number of 8-column tensor-memory loads, else two.
template <int LP> struct TcCfg {
  static constexpr int NPART = ((LP / 4) % 8 == 0) ? 4 : 2;
  static constexpr int NT = TC_M * NPART;  // threads per CTA
};
constexpr int TC_TMEM_COLS = 64;
constexpr long long TC_WAIT_CYCLES = 4000000000LL;  // ~2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t smem_desc(const void* p, uint32_t lbo, uint32_t sbo) {
  const uint32_t a = smem_u32(p);
  uint64_t d = (uint64_t)((a >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= 1ull << 46;  // descriptor version for tcgen05
  return d;         // base offset 0, no swizzle
}

// kind::f16 instruction descriptor: D = F32, A = B = BF16, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(mbar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait; false when the limit (in SM clock cycles) expired.
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, long long limit) {
  const long long t0 = clock64();
  while (!mbar_try_wait(mbar, parity)) {
    if (clock64() - t0 > limit) return false;
  }
  return true;
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r0, r1, r2, r3, r4, r5, r6, r7;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3), "=r"(r4), "=r"(r5), "=r"(r6), "=r"(r7)
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
  v[0] = __uint_as_float(r0);
  v[1] = __uint_as_float(r1);
  v[2] = __uint_as_float(r2);
  v[3] = __uint_as_float(r3);
  v[4] = __uint_as_float(r4);
  v[5] = __uint_as_float(r5);
  v[6] = __uint_as_float(r6);
  v[7] = __uint_as_float(r7);
}

__device__ __forceinline__ uint32_t bf16_bits(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }

// Splits 8 floats into hi and lo BF16 rows of 16 bytes each.
__device__ __forceinline__ void split8(const float* v, uint4& hi, uint4& lo) {
  uint32_t h[8], l[8];
#pragma unroll
  for (int t = 0; t < 8; t++) {
    const __nv_bfloat16 hb = __float2bfloat16_rn(v[t]);
    h[t] = __bfloat16_as_ushort(hb);
    l[t] = bf16_bits(v[t] - __bfloat162float(hb));
  }
  hi = make_uint4(h[0] | (h[1] << 16), h[2] | (h[3] << 16), h[4] | (h[5] << 16), h[6] | (h[7] << 16));
  lo = make_uint4(l[0] | (l[1] << 16), l[2] | (l[3] << 16), l[4] | (l[5] << 16), l[6] | (l[7] << 16));
}

__device__ __forceinline__ float soft_tc(float t, float tau) {
  const float a = fabsf(t) - tau;
  return a > 0.f ? copysignf(a, t) : 0.f;
}

// Issues the 3-term split product D = A_hi B_hi + A_hi B_lo + A_lo B_hi over K = LP.
template <int LP>
__device__ __forceinline__ void issue_split_gemm(uint32_t tmem, const uint16_t* Ahi, const uint16_t* Alo,
                                                 const uint16_t* Bhi, const uint16_t* Blo) {
  constexpr uint32_t LBO = 128, SBO = (LP / 8) * 128;
  constexpr uint32_t idesc = idesc_bf16(TC_M, LP);
#pragma unroll
  for (int term = 0; term < 3; term++) {
    const uint16_t* A = term == 2 ? Alo : Ahi;
    const uint16_t* B = term == 1 ? Blo : Bhi;
#pragma unroll
    for (int s = 0; s < LP / 16; s++) {
      // one K-step covers 16 elements = two core matrices along K
      const uint64_t ad = smem_desc(reinterpret_cast<const char*>(A) + s * 2 * LBO, LBO, SBO);
      const uint64_t bd = smem_desc(reinterpret_cast<const char*>(B) + s * 2 * LBO, LBO, SBO);
      mma_bf16(tmem, ad, bd, idesc, (term > 0 || s > 0) ? 1u : 0u);
    }
  }
}

// byte offset of the 8-element row segment (r, k0..k0+7) in an R x K operand
template <int K>
__device__ __forceinline__ uint32_t seg_off(int r, int k0) {
  return (uint32_t)((r >> 3) * ((K / 8) * 128) + (k0 >> 3) * 128 + (r & 7) * 16);
}

template <int LP, int RESID>
__global__ void __launch_bounds__(TcCfg<LP>::NT, 2) k_spectral_tc(const float* __restrict__ X, float* __restrict__ GP,
                                                           float* __restrict__ Sd, float* __restrict__ GV,
                                                           float* __restrict__ GSd, float* __restrict__ b,
                                                           const uint16_t* __restrict__ bmats, int NN, int L,
                                                           IterScalars<float> sc, double* __restrict__ partials,
                                                           int* __restrict__ err, long long stall_cycles) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  uint16_t* B1hi = reinterpret_cast<uint16_t*>(smem_raw);  // C as (N = k) x (K = l)
  uint16_t* B1lo = B1hi + LP * LP;
  uint16_t* B2hi = B1lo + LP * LP;  // C^T as (N = l) x (K = k)
  uint16_t* B2lo = B2hi + LP * LP;
  uint16_t* Ahi = B2lo + LP * LP;   // TC_M x LP operand: X, then U
  uint16_t* Alo = Ahi + TC_M * LP;
  float* Xs = reinterpret_cast<float*>(Alo + TC_M * LP);  // [LP][TC_M]
  uint64_t* mbar = reinterpret_cast<uint64_t*>(Xs + LP * TC_M);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);

  const int tid = threadIdx.x, warp = tid >> 5;
  const int row = tid & (TC_M - 1);     // pixel within the tile = tensor-memory lane
  constexpr int NT = TcCfg<LP>::NT;
  const int half = tid / TC_M;          // which part of the bands / frequencies
  constexpr int HL = LP / TcCfg<LP>::NPART;  // bands or frequencies per thread (a multiple of 8)
  const int p = blockIdx.x * TC_M + row;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(TC_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // this pixel's half spectrum: FP32 copy and the split A operand
  {
    float v[HL];
#pragma unroll
    for (int t = 0; t < HL; t++) {
      const int l = half * HL + t;
      v[t] = l < L ? X[(size_t)l * NN + p] : 0.f;
    }
    // L2 prefetch of the tile's rows of S, Gamma_V, Gamma_S (read after the first
    // product) and Gamma_P (after the second): one 128-byte line per warp-row
    // segment, so the later phases find them in L2 instead of waiting on HBM.
    {
      const size_t p0 = (size_t)blockIdx.x * TC_M;
      for (int e = tid; e < 4 * L * (TC_M / 32); e += NT) {
        const int seg = e % (TC_M / 32), rest = e / (TC_M / 32);
        const int l = rest % L, a = rest / L;
        const float* base = a == 0 ? Sd : a == 1 ? GV : a == 2 ? GSd : GP;
        asm volatile("prefetch.global.L2 [%0];" ::"l"(base + (size_t)l * NN + p0 + 32 * seg));
      }
    }
    {
      // the DCT operands (L2-resident, shared by every CTA)
      const uint4* src = reinterpret_cast<const uint4*>(bmats);
      uint4* dst = reinterpret_cast<uint4*>(B1hi);
      for (int e = tid; e < 4 * LP * LP / 8; e += NT) dst[e] = src[e];
    }
#pragma unroll
    for (int c0 = 0; c0 < HL; c0 += 8) {
      const int l0 = half * HL + c0;
#pragma unroll
      for (int t = 0; t < 8; t++) Xs[(l0 + t) * TC_M + row] = v[c0 + t];
      uint4 hi, lo;
      split8(v + c0, hi, lo);
      *reinterpret_cast<uint4*>(reinterpret_cast<char*>(Ahi) + seg_off<LP>(row, l0)) = hi;
      *reinterpret_cast<uint4*>(reinterpret_cast<char*>(Alo) + seg_off<LP>(row, l0)) = lo;
    }
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t trow = tmem + ((uint32_t)(32 * (warp & 3)) << 16);

  // x^ = X W_nu.  With stall_cycles > 0 (a test of the timeout path) CTA 0
  // issues neither the product nor its commit, so nothing is in flight when
  // its wait of stall_cycles cycles runs out.
  const bool stalled = stall_cycles > 0 && blockIdx.x == 0;
  const long long limit = stalled ? stall_cycles : TC_WAIT_CYCLES;
  if (tid == 0 && !stalled) {
    issue_split_gemm<LP>(tmem, Ahi, Alo, B1hi, B1lo);
    mma_commit(mbar);
  }
  bool ok = mbar_wait(mbar, 0, limit);
  tc_fence_after();

  // residual terms of this thread's voxels in FP32, folded into the FP64
  // partial rows once (FP64 arithmetic per voxel is slow)
  float r_dgv = 0.f, r_dgs = 0.f, r_l1 = 0.f, r_dgp = 0.f, r_x2 = 0.f, r_xmin = 3.0e38f;
  bool r_bad = false;

  if (ok) {
    // DCT-domain part of steps IV, V, VI; U = Gamma_S + rho_S S becomes the next A operand
#pragma unroll
    for (int k0 = half * HL; k0 < (half + 1) * HL; k0 += 8) {
      float xh[8], u[8];
      tmem_ld8(trow + k0, xh);
#pragma unroll
      for (int t = 0; t < 8; t++) {
        const int k = k0 + t;
        u[t] = 0.f;
        if (k < L) {
          const size_t o = (size_t)k * NN + p;
          const float s = Sd[o], gv = GV[o], gs = GSd[o];
          const float v = soft_tc(s - gv * sc.inv_rho_V, sc.tau_V);
          const float sn = (gv + sc.rho_V * v - gs + sc.rho_S * xh[t]) * sc.inv_VS;
          const float gvn = gv + sc.rho_V * (v - sn);
          const float gsn = gs + sc.rho_S * (sn - xh[t]);
          Sd[o] = sn;
          GV[o] = gvn;
          GSd[o] = gsn;
          u[t] = gsn + sc.rho_S * sn;
          if (RESID) {
            const float dv = gvn - gv, ds = gsn - gs;
            r_dgv = fmaf(dv, dv, r_dgv);
            r_dgs = fmaf(ds, ds, r_dgs);
            r_l1 += fabsf(xh[t]);
            r_bad |= !isfinite(gvn) || !isfinite(gsn);
          }
        }
      }
      uint4 hi, lo;
      split8(u, hi, lo);
      *reinterpret_cast<uint4*>(reinterpret_cast<char*>(Ahi) + seg_off<LP>(row, k0)) = hi;
      *reinterpret_cast<uint4*>(reinterpret_cast<char*>(Alo) + seg_off<LP>(row, k0)) = lo;
    }
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

  // (Gamma_S + rho_S S) = U W_nu^T
  if (ok && tid == 0) {
    issue_split_gemm<LP>(tmem, Ahi, Alo, B2hi, B2lo);
    mma_commit(mbar);
  }
  if (ok) ok = mbar_wait(mbar, 1, limit);
  tc_fence_after();

  if (ok) {
    // pixel domain: step II, Gamma_P, and b
#pragma unroll
    for (int l0 = half * HL; l0 < (half + 1) * HL; l0 += 8) {
      float bs[8];
      tmem_ld8(trow + l0, bs);
#pragma unroll
      for (int t = 0; t < 8; t++) {
        const int l = l0 + t;
        if (l < L) {
          const size_t o = (size_t)l * NN + p;
          const float x = Xs[l * TC_M + row];
          const float gp = GP[o];
          const float pt = x - gp * sc.inv_rho_P;
          const float pp = pt > 0.f ? pt : 0.f;
          const float gpn = gp + sc.rho_P * (pp - x);
          GP[o] = gpn;
          b[o] = gpn + sc.rho_P * pp + bs[t];
          if (RESID) {
            const float d = gpn - gp;
            r_dgp = fmaf(d, d, r_dgp);
            r_x2 = fmaf(x, x, r_x2);
            r_xmin = fminf(r_xmin, x);
            r_bad |= !isfinite(x) || !isfinite(gpn);
          }
        }
      }
    }
  } else if (tid == 0) {
    atomicExch(err, 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS));
  if (RESID) {
    float q[Q_COUNT];
#pragma unroll
    for (int i = 0; i < Q_COUNT; i++) q[i] = 0.f;
    q[Q_DGV] = r_dgv;
    q[Q_DGS] = r_dgs;
    q[Q_L1NU] = r_l1;
    q[Q_DGP] = r_dgp;
    q[Q_X2] = r_x2;
    q[Q_XMIN] = r_xmin;  // 3e38 (no voxel) becomes the FP64 sentinel in the reduction
    q[Q_NONFIN] = r_bad ? 1.f : 0.f;
    block_reduce_write<NT>(q, partials + (size_t)blockIdx.x * MF_NQ);
  }
}

template <int LP>
cudaError_t spectral_tc_lp(const float* X, float* GP, float* Sd, float* GV, float* GSd, float* b,
                           const uint16_t* bmats, int N, int L, IterScalars<float> sc, double* partials, int resid,
                           int* err, long long stall, cudaStream_t s) {
  const int NN = N * N;
  const size_t sm = 4 * LP * LP * 2 + 2 * TC_M * LP * 2 + LP * TC_M * 4 + 16;
  const int blocks = NN / TC_M;
  cudaError_t e;
  if (resid) {
    e = cudaFuncSetAttribute(k_spectral_tc<LP, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_spectral_tc<LP, 1><<<blocks, TcCfg<LP>::NT, sm, s>>>(X, GP, Sd, GV, GSd, b, bmats, NN, L, sc, partials, err,
                                                           stall);
  } else {
    e = cudaFuncSetAttribute(k_spectral_tc<LP, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_spectral_tc<LP, 0><<<blocks, TcCfg<LP>::NT, sm, s>>>(X, GP, Sd, GV, GSd, b, bmats, NN, L, sc, partials, err,
                                                           stall);
  }
  return cudaGetLastError();
}

uint16_t host_bf16(double x) {
  // round to nearest even through FP32
  float f = (float)x;
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

double host_bf16_value(uint16_t h) {
  uint32_t u = (uint32_t)h << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return (double)f;
}

}  // namespace

int spectral_tc_lp_of(int L) { return L <= 16 ? 16 : L <= 32 ? 32 : L <= 48 ? 48 : L <= 64 ? 64 : 0; }

size_t spectral_tc_operand_elems(int L) {
  const int LP = spectral_tc_lp_of(L);
  return (size_t)4 * LP * LP;
}

void spectral_tc_build_operands(int L, uint16_t* out) {
  const int LP = spectral_tc_lp_of(L);
  const size_t n = (size_t)LP * LP;
  for (size_t i = 0; i < 4 * n; i++) out[i] = 0;
  auto off = [&](int r, int k) {  // element index of (r, k) in the core-matrix layout
    return (size_t)((r / 8) * (LP / 8) * 64 + (k / 8) * 64 + (r % 8) * 8 + (k % 8));
  };
  for (int k = 0; k < L; k++) {
    const double ak = k == 0 ? std::sqrt(1.0 / L) : std::sqrt(2.0 / L);
    for (int l = 0; l < L; l++) {
      const double c = ak * std::cos(M_PI * (2.0 * l + 1.0) * k / (2.0 * L));
      const uint16_t hi = host_bf16(c);
      const uint16_t lo = host_bf16(c - host_bf16_value(hi));
      out[0 * n + off(k, l)] = hi;  // B1: N = k, K = l
      out[1 * n + off(k, l)] = lo;
      out[2 * n + off(l, k)] = hi;  // B2: N = l, K = k
      out[3 * n + off(l, k)] = lo;
    }
  }
}

cudaError_t launch_spectral_tc(const float* X, float* GP, float* Sd, float* GV, float* GSd, float* b,
                               const uint16_t* bmats, int N, int L, IterScalars<float> sc, double* partials,
                               int resid, int* err, long long stall, cudaStream_t s) {
  switch (spectral_tc_lp_of(L)) {
    case 16: return spectral_tc_lp<16>(X, GP, Sd, GV, GSd, b, bmats, N, L, sc, partials, resid, err, stall, s);
    case 32: return spectral_tc_lp<32>(X, GP, Sd, GV, GSd, b, bmats, N, L, sc, partials, resid, err, stall, s);
    case 48: return spectral_tc_lp<48>(X, GP, Sd, GV, GSd, b, bmats, N, L, sc, partials, resid, err, stall, s);
    case 64: return spectral_tc_lp<64>(X, GP, Sd, GV, GSd, b, bmats, N, L, sc, partials, resid, err, stall, s);
    default: return cudaErrorInvalidValue;
  }
}

int spectral_tc_blocks(int N) { return N * N / TC_M; }

}  // namespace mf
