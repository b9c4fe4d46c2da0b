// Per-block FP64 reduction of the residual quantities (see the Q_* slots).
#pragma once

#include "mf_internal.cuh"

namespace mf {

// The neutral value of the min slot in a kernel's per-thread sums (FP32
// values >= 3e38 become the FP64 sentinel 1e300 in the reduction).
template <class R> struct NoMin;
template <> struct NoMin<float> { static constexpr float v = 3.0e38f; };
template <> struct NoMin<double> { static constexpr double v = 1.0e300; };

// Reduces the Q_COUNT per-thread values over the CTA in a fixed order and
// writes one MF_NQ-wide row of partials (thread count NT, multiple of 32).
template <int NT>
__device__ __forceinline__ void block_reduce_write(double* q, double* out) {
  __shared__ double red[NT / 32][Q_COUNT];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < Q_COUNT; i++) {
    double v = q[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double u = __shfl_down_sync(0xffffffffu, v, o);
      v = (i == Q_XMIN) ? fmin(v, u) : v + u;
    }
    if (lane == 0) red[wid][i] = v;
  }
  __syncthreads();
  if (threadIdx.x < Q_COUNT) {
    const int i = threadIdx.x;
    double v = red[0][i];
    for (int w = 1; w < NT / 32; w++) v = (i == Q_XMIN) ? fmin(v, red[w][i]) : v + red[w][i];
    out[i] = v;
  }
  if (threadIdx.x >= Q_COUNT && threadIdx.x < MF_NQ) out[threadIdx.x] = 0.0;
}

// Same for per-thread values in FP32 (the FP32 kernels' per-thread sums): the
// warp stage runs in FP32 (32-bit shuffles and adds; FP64 arithmetic is slow on
// this GPU), the stage across warps and everything after it in FP64.
template <int NT>
__device__ __forceinline__ void block_reduce_write(const float* q, double* out) {
  __shared__ double red[NT / 32][Q_COUNT];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < Q_COUNT; i++) {
    float v = q[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float u = __shfl_down_sync(0xffffffffu, v, o);
      v = (i == Q_XMIN) ? fminf(v, u) : v + u;
    }
    if (lane == 0) red[wid][i] = (i == Q_XMIN && !(v < 3.0e38f)) ? 1e300 : (double)v;
  }
  __syncthreads();
  if (threadIdx.x < Q_COUNT) {
    const int i = threadIdx.x;
    double v = red[0][i];
    for (int w = 1; w < NT / 32; w++) v = (i == Q_XMIN) ? fmin(v, red[w][i]) : v + red[w][i];
    out[i] = v;
  }
  if (threadIdx.x >= Q_COUNT && threadIdx.x < MF_NQ) out[threadIdx.x] = 0.0;
}

}  // namespace mf
