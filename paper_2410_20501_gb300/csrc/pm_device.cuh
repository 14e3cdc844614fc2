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

// Sum over the block of per-thread compensated pairs (sum, comp), returned to
// every thread as the same float pair (hi, lo): warp shuffles with error-free
// additions, then warp 0 over the per-warp pairs, whose result thread 0
// publishes in scratch[32] (so every thread takes the same decision from it).
// All threads call it; scratch holds 33 pairs.
__device__ __forceinline__ float2 block_pair_sum(float sum, float comp, float2* scratch) {
  float s = sum - comp, c = 0.0f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float os = __shfl_down_sync(0xffffffffu, s, o), oc = __shfl_down_sync(0xffffffffu, c, o);
    float t, e;
    two_sum(s, os, t, e);
    s = t;
    c = c + oc + e;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) scratch[warp] = make_float2(s, c);
  __syncthreads();
  if (warp == 0) {
    float2 v = lane < nw ? scratch[lane] : make_float2(0.0f, 0.0f);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float os = __shfl_down_sync(0xffffffffu, v.x, o), oc = __shfl_down_sync(0xffffffffu, v.y, o);
      float t, e;
      two_sum(v.x, os, t, e);
      v.x = t;
      v.y = v.y + oc + e;
    }
    if (lane == 0) scratch[32] = v;
  }
  __syncthreads();
  return scratch[32];
}

// Flat indices (32-bit: n <= 1024) of a cell's six periodic face neighbours in
// the order x+, x-, y+, y-, z+, z-, for c = (i n + j) n + k.
__device__ __forceinline__ void nb_index(uint32_t c, uint32_t i, uint32_t j, uint32_t k, int log2n,
                                         uint32_t idx[6]) {
  const uint32_t m = (1u << log2n) - 1, n = 1u << log2n, n2 = n << log2n;
  idx[0] = i == m ? c - m * n2 : c + n2;
  idx[1] = i == 0 ? c + m * n2 : c - n2;
  idx[2] = j == m ? c - m * n : c + n;
  idx[3] = j == 0 ? c + m * n : c - n;
  idx[4] = k == m ? c - m : c + 1;
  idx[5] = k == 0 ? c + m : c - 1;
}

// The 32 values of u that the 8 children of coarse cell (I, J, K) and their
// face neighbours touch on the fine grid (n = 2^log2n), z pairs as float2:
//   core[a][b][t]: x = 2I + a, y = 2J + b, z = 2K - 1 + t (t = 0..3)
//   xf[0|1][b][c]: x = 2I - 1 | 2I + 2, y = 2J + b, z = 2K + c
//   yf[a][0|1][c]: x = 2I + a, y = 2J - 1 | 2J + 2, z = 2K + c
// The 6 neighbours of child (a, b, c) in the order x+, x-, y+, y-, z+, z- then
// come from child_nb().
__device__ __forceinline__ void load_children_block(const float* __restrict__ u, int I, int J, int K, int log2n,
                                                    float core[2][2][4], float xf[2][2][2], float yf[2][2][2]) {
  const int m = (1 << log2n) - 1;
  auto at = [&](int x, int y, int z) -> uint32_t {   // offset inside one box (below 2^30)
    return ((uint32_t)(x & m) << (2 * log2n)) | ((uint32_t)(y & m) << log2n) | (uint32_t)(z & m);
  };
  const int x0 = 2 * I, y0 = 2 * J, z0 = 2 * K;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const float2 c2 = __ldg(reinterpret_cast<const float2*>(u + at(x0 + a, y0 + b, z0)));
      core[a][b][0] = __ldg(u + at(x0 + a, y0 + b, z0 - 1));
      core[a][b][1] = c2.x;
      core[a][b][2] = c2.y;
      core[a][b][3] = __ldg(u + at(x0 + a, y0 + b, z0 + 2));
    }
#pragma unroll
  for (int side = 0; side < 2; ++side)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const float2 v = __ldg(reinterpret_cast<const float2*>(u + at(side ? x0 + 2 : x0 - 1, y0 + b, z0)));
      xf[side][b][0] = v.x;
      xf[side][b][1] = v.y;
    }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const float2 v = __ldg(reinterpret_cast<const float2*>(u + at(x0 + a, side ? y0 + 2 : y0 - 1, z0)));
      yf[a][side][0] = v.x;
      yf[a][side][1] = v.y;
    }
}

__device__ __forceinline__ void child_nb(const float core[2][2][4], const float xf[2][2][2], const float yf[2][2][2],
                                         int a, int b, int c, float nb[6]) {
  nb[0] = a ? xf[1][b][c] : core[1][b][c + 1];
  nb[1] = a ? core[0][b][c + 1] : xf[0][b][c];
  nb[2] = b ? yf[a][1][c] : core[a][1][c + 1];
  nb[3] = b ? core[a][0][c + 1] : yf[a][0][c];
  nb[4] = core[a][b][c + 2];
  nb[5] = core[a][b][c];
}

}  // namespace pmgb
