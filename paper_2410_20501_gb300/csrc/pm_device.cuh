// Device helpers shared by the CUDA translation units of libpmgb.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pmgb {

// Per-axis TSC weights (§3.4, W_TSC) of a particle whose offset from its cell
// centre is d (in cells, -1/2 <= d < 1/2), towards the cells o = -1, 0, +1,
// i.e. W_TSC at separations d + 1, d and d - 1.
__device__ __forceinline__ void tsc_weights(float d, float w[3]) {
  float a = 0.5f - d, b = 0.5f + d;
  w[0] = 0.5f * a * a;
  w[1] = 0.75f - d * d;
  w[2] = 0.5f * b * b;
}

// Offset of a uint32 fixed-point coordinate from the centre of its cell
// (n = 2^log2n cells per side), in cells.
__device__ __forceinline__ float cell_offset(uint32_t x, int log2n) {
  uint32_t f = x << log2n;  // position within the cell in units of 2^-32 cells
  return (float)(int32_t)(f - 0x80000000u) * 2.3283064365386963e-10f;  // * 2^-32
}

// Error-free transformation a + b = s + e (Knuth's TwoSum).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bp = s - a;
  e = (a - (s - bp)) + (b - bp);
}

// Compensated warp sum; the result is valid in lane 0, as a double.
__device__ __forceinline__ double warp_sum_comp(float v) {
  float s = v, c = 0.0f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    float os = __shfl_down_sync(0xffffffffu, s, o);
    float oc = __shfl_down_sync(0xffffffffu, c, o);
    float t, e;
    two_sum(s, os, t, e);
    s = t;
    c = c + oc + e;
  }
  return (double)s + (double)c;
}

// Kahan accumulation of one term.
__device__ __forceinline__ void kahan_add(float& sum, float& comp, float x) {
  float y = x - comp;
  float t = sum + y;
  comp = (t - sum) - y;
  sum = t;
}

// Block reduction of per-thread (sum, comp) pairs into float64, written by
// thread 0 to out[0].  All threads of the block must call it; blockDim.x is a
// multiple of 32 and at most 1024.
__device__ __forceinline__ void block_sum_to(double* out, float sum, float comp, double* scratch32) {
  double w = warp_sum_comp(sum - comp);
  if ((threadIdx.x & 31) == 0) scratch32[threadIdx.x >> 5] = w;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += scratch32[i];
    *out = t;
  }
  __syncthreads();
}

}  // namespace pmgb
