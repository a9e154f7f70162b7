// devutil.cuh -- small device helpers shared by the solver's kernels.
#pragma once
#include <cuda_runtime.h>
#include "gabp_internal.cuh"

namespace gabp {

// IEEE division, kept out of line so that the common path of rcp64 does not
// carry its instructions.
static __device__ __noinline__ double rcp64_slow(double d) { return 1.0 / d; }

// Reciprocal of a double by one step of Chebyshev's third-order iteration for 1/d:
// with e = 1 - d y, y <- y (1 + e + e^2) = y + y (e + e^2).  If y = (1 - eps)/d, then
// e = eps and the step gives (1 - eps^3)/d: the relative error is cubed (Newton's
// y + y e would only square it).  The seed is the single-precision hardware
// approximation (PTX rcp.approx.ftz.f32) of d rounded toward zero to 20 mantissa
// bits, relative error below 2^-19, so one step leaves ~2^-57 plus the final
// rounding: three FMAs on the (narrow) FP64 pipe instead of the four of two Newton
// steps.  The float operand and the double seed are assembled from the IEEE-754
// fields with integer operations, which keeps the conversions off the FP64 pipe.
// Exponents outside [-120, 120] (and 0, subnormals, inf, NaN) take the IEEE division.
__device__ __forceinline__ double rcp64(double d) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(d);
  const unsigned hi = (unsigned)(u >> 32);
  const int e = (int)((hi >> 20) & 0x7ffu) - 1023;
  const unsigned fb = (hi & 0x80000000u) | ((unsigned)(e + 127) << 23) | ((hi & 0xfffffu) << 3);
  float yf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(__uint_as_float(fb)));
  const unsigned yb = __float_as_uint(yf);
  const int ey = (int)((yb >> 23) & 0xffu) - 127;
  const unsigned yhi = (yb & 0x80000000u) | ((unsigned)(ey + 1023) << 20) | ((yb >> 3) & 0xfffffu);
  double y = __hiloint2double((int)yhi, (int)((yb & 7u) << 29));
  const double r = fma(-d, y, 1.0);  // e
  y = fma(y, fma(r, r, r), y);       // y (1 + e + e^2)
  if (e < -120 || e > 120) y = rcp64_slow(d);
  return y;
}

// d == +0 or -0, tested on the bit pattern.  The two 32-bit halves come out of an
// inline move so the test stays on the integer pipe: written on the 64-bit pattern
// in C, it is recognised as d == 0.0 and becomes an FP64 compare, one more
// instruction per message on the FP64 pipe that bounds the FP64 rounds.
__device__ __forceinline__ bool is_zero64(double d) {
  unsigned lo, hi;
  asm("mov.b64 {%0, %1}, %2;" : "=r"(lo), "=r"(hi) : "d"(d));
  return ((hi << 1) | lo) == 0u;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// max that keeps a NaN from either side (fmax drops it): a NaN change or
// residual must never read as "small".
template <typename T>
__device__ __forceinline__ T nan_max(T a, T b) {
  return (a > b || a != a) ? a : b;
}

// |now - prev| / |now| with 0 for an unchanged value (an explicitly stored zero
// coupling keeps a zero message: 0/0 must not read as a NaN change).
__device__ __forceinline__ float rel_change(float now, float prev) {
  const float d = fabsf(now - prev);
  return d == 0.f ? 0.f : d / fabsf(now);
}

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = nan_max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Sum over the L lanes of a sub-warp (L a power of two dividing 32); every lane
// of the warp must call it.
template <int L, typename T>
__device__ __forceinline__ T sub_sum(T v) {
#pragma unroll
  for (int o = L / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, L);
  return v;
}

// Block-wide sum of NV doubles over NT threads.  Result valid in thread 0.
template <int NV, int NT>
__device__ __forceinline__ void block_sum_nt(double (&v)[NV]) {
  __shared__ double sh[NV][NT / 32];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    double s = warp_sum(v[j]);
    if (l == 0) sh[j][w] = s;
  }
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      double s = l < NT / 32 ? sh[j][l] : 0.0;
      v[j] = warp_sum(s);
    }
  }
  __syncthreads();
}

// Block-wide max of NV doubles over NT threads.  Result valid in thread 0.
template <int NV, int NT>
__device__ __forceinline__ void block_max_nt(double (&v)[NV]) {
  __shared__ double sh[NV][NT / 32];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    double s = warp_max(v[j]);
    if (l == 0) sh[j][w] = s;
  }
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      double s = l < NT / 32 ? sh[j][l] : -1.0;
      v[j] = warp_max(s);
    }
  }
  __syncthreads();
}

// Block-wide sum of NV doubles (kBlock threads).  Result valid in thread 0.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
  __shared__ double sh[NV][kBlock / 32];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    double s = warp_sum(v[j]);
    if (l == 0) sh[j][w] = s;
  }
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      double s = l < kBlock / 32 ? sh[j][l] : 0.0;
      v[j] = warp_sum(s);
    }
  }
  __syncthreads();
}

// Block-wide max of NV doubles.  Result valid in thread 0.
template <int NV>
__device__ __forceinline__ void block_max(double (&v)[NV]) {
  __shared__ double sh[NV][kBlock / 32];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    double s = warp_max(v[j]);
    if (l == 0) sh[j][w] = s;
  }
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      double s = l < kBlock / 32 ? sh[j][l] : -1.0;
      v[j] = warp_max(s);
    }
  }
  __syncthreads();
}

// Publish this block's NV partial values (thread 0 holds them) into
// partials[j * gridDim.x + blockIdx.x] and find out whether this block is the
// last of the grid to finish.  In the last block, tot[] (valid in thread 0)
// receives the sums over all blocks, taken in block order (deterministic).
// modes[j] = 0 sums, 1 takes the max.
template <int NV>
__device__ __forceinline__ bool last_block_reduce(double (&v)[NV], const int (&modes)[NV], double *partials,
                                                  unsigned int *arrive, double (&tot)[NV]) {
  __shared__ bool s_last;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) partials[j * gridDim.x + blockIdx.x] = v[j];
    __threadfence();
    unsigned int prev = atomicAdd(arrive, 1u);
    s_last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  double acc[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) acc[j] = modes[j] ? -1.0 : 0.0;
  for (int bI = threadIdx.x; bI < (int)gridDim.x; bI += kBlock) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      double p = __ldcg(partials + j * gridDim.x + bI);
      acc[j] = modes[j] ? nan_max(acc[j], p) : acc[j] + p;
    }
  }
  // deterministic: each thread's stripe is fixed; the block tree is fixed
  double s[NV], m[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) { s[j] = modes[j] ? 0.0 : acc[j]; m[j] = modes[j] ? acc[j] : -1.0; }
  block_sum<NV>(s);
  block_max<NV>(m);
#pragma unroll
  for (int j = 0; j < NV; ++j) tot[j] = modes[j] ? m[j] : s[j];
  return true;
}

}  // namespace gabp
