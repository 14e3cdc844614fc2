// Force from the potential and its interpolation to the particles:
//  - g = -grad(Phi) with the central stencils of Table 1, where for f(R)
//    Phi = phi + alpha (2 eps + eps^2), alpha = -(c~^2/2) fbar, i.e. the
//    force F = F_N + (c~^2/2) grad f~_R of §3.10 (the constant background part
//    of f~_R = fbar (1 + eps)^2 has no gradient);
//  - inverse TSC (§3.4) at the cell-sorted particles, optionally fused with
//    the kick v += a dt_kick and the drift x += v dt_drift on uint32
//    fixed-point positions (exact periodic wrap).
#include "pm_device.cuh"
#include "pm_internal.cuh"

namespace pmgb {

namespace {

__device__ __forceinline__ int64_t idx3(int i, int j, int k, int log2n) {
  return ((int64_t)i << (2 * log2n)) | ((int64_t)j << log2n) | k;
}

// phi + alpha (u^(n+1) - 1), u = 1 + eps: the combined potential up to a
// constant (alpha = -(c~^2/2) fbar; n = nh, 1 or 2).
template <bool FR>
__device__ __forceinline__ float pot(const float* __restrict__ phi, const float* __restrict__ eps, float alpha,
                                     int64_t c, int nh) {
  float v = __ldg(phi + c);
  if (FR) {
    const float e = __ldg(eps + c);
    v = fmaf(alpha, nh == 2 ? e * fmaf(e, 3.0f + e, 3.0f) : e * (2.0f + e), v);
  }
  return v;
}

// Table 1 coefficients c_1..c_3 of the antisymmetric central derivative
// (1/h) sum_k c_k (u_{i+k} - u_{i-k}).
template <int ORDER> struct Stencil;
template <> struct Stencil<3> { static constexpr int R = 1; __device__ static float c(int k) { return 0.5f; } };
template <> struct Stencil<5> {
  static constexpr int R = 2;
  __device__ static float c(int k) { return k == 1 ? 2.0f / 3.0f : -1.0f / 12.0f; }
};
template <> struct Stencil<7> {
  static constexpr int R = 3;
  __device__ static float c(int k) { return k == 1 ? 0.75f : (k == 2 ? -0.15f : 1.0f / 60.0f); }
};

template <int ORDER, bool FR>
__global__ void k_gradient(const float* __restrict__ phi, const float* __restrict__ eps, float alpha,
                           float* __restrict__ g, int log2n, float inv_h, int nh) {
  const int m = (1 << log2n) - 1;
  const int64_t total = (int64_t)1 << (3 * log2n);
  phi += (int64_t)blockIdx.z * total;          // the box of a batched launch
  if (FR) eps += (int64_t)blockIdx.z * total;
  g += (int64_t)blockIdx.z * 3 * total;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < total;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(c & m), j = (int)((c >> log2n) & m), i = (int)(c >> (2 * log2n));
    float gx = 0.0f, gy = 0.0f, gz = 0.0f;
#pragma unroll
    for (int q = Stencil<ORDER>::R; q >= 1; --q) {
      const float w = Stencil<ORDER>::c(q);
      gx = fmaf(w, pot<FR>(phi, eps, alpha, idx3((i + q) & m, j, k, log2n), nh) -
                       pot<FR>(phi, eps, alpha, idx3((i - q) & m, j, k, log2n), nh), gx);
      gy = fmaf(w, pot<FR>(phi, eps, alpha, idx3(i, (j + q) & m, k, log2n), nh) -
                       pot<FR>(phi, eps, alpha, idx3(i, (j - q) & m, k, log2n), nh), gy);
      gz = fmaf(w, pot<FR>(phi, eps, alpha, idx3(i, j, (k + q) & m, log2n), nh) -
                       pot<FR>(phi, eps, alpha, idx3(i, j, (k - q) & m, log2n), nh), gz);
    }
    const int64_t N = total;
    g[c] = -gx * inv_h;
    g[N + c] = -gy * inv_h;
    g[2 * N + c] = -gz * inv_h;
  }
}

// Streaming gradient for n >= 64: a CTA owns a 16 x 64 (y, z) column and a
// chunk of x planes, keeps the 2R + 1 planes of Phi (with a halo of R in y and
// z) that the stencil needs in shared memory, so every Phi value is read from
// HBM once (plus halos).  Same arithmetic order as k_gradient.  VEC4 writes
// g interleaved as float4 (gx, gy, gz, 0) for the interpolation.
constexpr int GTY = 16, GTZ = 64, GNT = 256;

template <int ORDER, bool FR, bool VEC4>
__global__ void __launch_bounds__(GNT) k_gradient_stream(const float* __restrict__ phi,
                                                        const float* __restrict__ eps, float alpha,
                                                        float* __restrict__ g, int log2n, float inv_h,
                                                        int chunk, int nitems, int nh) {
  constexpr int R = Stencil<ORDER>::R, W = 2 * R + 1, EY = GTY + 2 * R, EZ = GTZ + 2 * R, PL = EY * EZ;
  extern __shared__ float P[];   // [W][EY][EZ]
  const int n = 1 << log2n, m = n - 1;
  const int tiles_z = n / GTZ, tiles = (n / GTY) * tiles_z;
  const int64_t N = (int64_t)1 << (3 * log2n);
  const int tid = threadIdx.x;
  phi += (int64_t)blockIdx.z * N;              // the box of a batched launch
  if (FR) eps += (int64_t)blockIdx.z * N;
  g += (int64_t)blockIdx.z * (VEC4 ? 4 : 3) * N;
  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
    const int tile = item % tiles, xc = item / tiles;
    const int y0 = (tile / tiles_z) * GTY, z0 = (tile % tiles_z) * GTZ;
    const int x0 = xc * chunk, x1 = x0 + chunk;
    for (int t = x0 - R; t < x1 + R; ++t) {
      float* Pt = P + (((t % W) + W) % W) * PL;
      const int64_t pb = (int64_t)(t & m) << (2 * log2n);
      for (int e = tid; e < PL; e += GNT) {
        const int ly = e / EZ, lz = e - ly * EZ;
        Pt[e] = pot<FR>(phi, eps, alpha, pb | ((int64_t)((y0 - R + ly) & m) << log2n) | ((z0 - R + lz) & m), nh);
      }
      __syncthreads();
      const int xo = t - R;
      if (xo >= x0) {
        const float* Pc = P + (((xo % W) + W) % W) * PL;
        for (int e = tid; e < GTY * GTZ; e += GNT) {
          const int ly = e / GTZ, lz = e - ly * GTZ;
          const int c = (ly + R) * EZ + lz + R;
          float gx = 0.0f, gy = 0.0f, gz = 0.0f;
#pragma unroll
          for (int q = R; q >= 1; --q) {
            const float w = Stencil<ORDER>::c(q);
            const float* Pp = P + ((((xo + q) % W) + W) % W) * PL;
            const float* Pm = P + ((((xo - q) % W) + W) % W) * PL;
            gx = fmaf(w, Pp[c] - Pm[c], gx);
            gy = fmaf(w, Pc[c + q * EZ] - Pc[c - q * EZ], gy);
            gz = fmaf(w, Pc[c + q] - Pc[c - q], gz);
          }
          const int64_t cell = ((int64_t)xo << (2 * log2n)) | ((int64_t)(y0 + ly) << log2n) | (z0 + lz);
          if (VEC4) {
            reinterpret_cast<float4*>(g)[cell] = make_float4(-gx * inv_h, -gy * inv_h, -gz * inv_h, 0.0f);
          } else {
            g[cell] = -gx * inv_h;
            g[N + cell] = -gy * inv_h;
            g[2 * N + cell] = -gz * inv_h;
          }
        }
      }
      __syncthreads();
    }
  }
}

// Inverse TSC; mode 1 also kicks and drifts.  Particles are read in cell
// order (Xs, Vs) and written in the same order (Xo, Vo).
template <bool VEC4, bool MAXES>
__global__ void __launch_bounds__(256) k_interp_kdk(const float* __restrict__ g, const uint32_t* __restrict__ Xs,
                                                    const float* __restrict__ Vs,
                                                    const uint32_t* __restrict__ ids_in, int64_t np, int log2n,
                                                    float* __restrict__ acc, uint32_t* __restrict__ Xo,
                                                    float* __restrict__ Vo, uint32_t* __restrict__ ids_out,
                                                    float dt_kick, float drift_scale, int mode, int64_t np_box,
                                                    const float* __restrict__ dtk_box,
                                                    const float* __restrict__ dtd_box,
                                                    float2* __restrict__ blockmax) {
  const int m = (1 << log2n) - 1, sh = 32 - log2n;
  const int64_t N = (int64_t)1 << (3 * log2n);
  // the box of a batched launch: its grid and its particles p0 .. p0 + np_box
  // (np stays the plane stride of the particle arrays)
  const int64_t p0 = (int64_t)blockIdx.z * np_box, p1 = p0 + np_box;
  g += (int64_t)blockIdx.z * (VEC4 ? 4 : 3) * N;
  if (dtk_box) dt_kick = __ldg(dtk_box + blockIdx.z);
  if (dtd_box) drift_scale = __ldg(dtd_box + blockIdx.z) * 4294967296.0f;
  float amax = 0.0f, vmax = 0.0f;   // largest |a| and |v after the kick| of this thread
  for (int64_t p = p0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < p1;
       p += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t x = __ldg(Xs + p), y = __ldg(Xs + np + p), z = __ldg(Xs + 2 * np + p);
    float wx[3], wy[3], wz[3];
    tsc_weights(cell_offset(x, log2n), wx);
    tsc_weights(cell_offset(y, log2n), wy);
    tsc_weights(cell_offset(z, log2n), wz);
    const int ix = (int)(x >> sh), iy = (int)(y >> sh), iz = (int)(z >> sh);
    float ax = 0.0f, ay = 0.0f, az = 0.0f;
#pragma unroll
    for (int ox = 0; ox < 3; ++ox) {
      const int ci = (ix + ox - 1) & m;
#pragma unroll
      for (int oy = 0; oy < 3; ++oy) {
        const int cj = (iy + oy - 1) & m;
        const float wxy = wx[ox] * wy[oy];
#pragma unroll
        for (int oz = 0; oz < 3; ++oz) {
          const int64_t c = idx3(ci, cj, (iz + oz - 1) & m, log2n);
          const float w = wxy * wz[oz];
          if (VEC4) {
            const float4 v = __ldg(reinterpret_cast<const float4*>(g) + c);
            ax = fmaf(w, v.x, ax);
            ay = fmaf(w, v.y, ay);
            az = fmaf(w, v.z, az);
          } else {
            ax = fmaf(w, __ldg(g + c), ax);
            ay = fmaf(w, __ldg(g + N + c), ay);
            az = fmaf(w, __ldg(g + 2 * N + c), az);
          }
        }
      }
    }
    if (acc) {
      acc[p] = ax;
      acc[np + p] = ay;
      acc[2 * np + p] = az;
    }
    if (MAXES) amax = fmaxf(amax, sqrtf(fmaf(ax, ax, fmaf(ay, ay, az * az))));
    if (mode == 1) {
      const float vx = fmaf(ax, dt_kick, __ldg(Vs + p));
      const float vy = fmaf(ay, dt_kick, __ldg(Vs + np + p));
      const float vz = fmaf(az, dt_kick, __ldg(Vs + 2 * np + p));
      Vo[p] = vx;
      Vo[np + p] = vy;
      Vo[2 * np + p] = vz;
      if (MAXES) vmax = fmaxf(vmax, sqrtf(fmaf(vx, vx, fmaf(vy, vy, vz * vz))));
      Xo[p] = x + (uint32_t)__float2int_rn(vx * drift_scale);
      Xo[np + p] = y + (uint32_t)__float2int_rn(vy * drift_scale);
      Xo[2 * np + p] = z + (uint32_t)__float2int_rn(vz * drift_scale);
      if (ids_out) ids_out[p] = __ldg(ids_in + p);
    }
  }
  if (MAXES) {   // block maxima (non-negative floats order like their bit patterns)
    __shared__ unsigned wa[8], wv[8];
    const unsigned ua = __reduce_max_sync(0xffffffffu, __float_as_uint(amax));
    const unsigned uv = __reduce_max_sync(0xffffffffu, __float_as_uint(vmax));
    if ((threadIdx.x & 31) == 0) {
      wa[threadIdx.x >> 5] = ua;
      wv[threadIdx.x >> 5] = uv;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned ma = 0, mv = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        ma = max(ma, wa[w]);
        mv = max(mv, wv[w]);
      }
      blockmax[(int64_t)blockIdx.z * gridDim.x + blockIdx.x] = make_float2(__uint_as_float(ma), __uint_as_float(mv));
    }
  }
}

// Force and inverse TSC + kick-drift-kick in one pass for cell-sorted
// particles (n >= 32): a CTA owns a IT_Y x IT_Z column of cells and a chunk
// of x planes and walks the planes in order.  The force planes around plane
// x (with a one-cell halo in y and z) are computed in shared memory from the
// potential (the gradient of k_gradient, same arithmetic), so the force field
// never goes through HBM; the particles of the column's cells on plane x are
// IT_Y contiguous runs of the sorted arrays (one per row), which the threads
// take in flat order.  Every particle then reads its 27 x 3 force values
// from shared memory at fixed offsets from its cell, in the same order and
// with the same operations as k_interp_kdk (bitwise the same result).
constexpr int IT_Y = 16, IT_Z = 32, IE_Y = IT_Y + 2, IE_Z = IT_Z + 2, I_PL = IE_Y * IE_Z, I_THREADS = 256;
// Warp 0: the runs of the column's rows on plane q (start of each row's
// particles, flat prefix of the run lengths).
__device__ __forceinline__ void column_runs(const uint32_t* __restrict__ cellstart, int q, int y0, int z0,
                                            int log2n, uint32_t* start, uint32_t* pre) {
  const int tid = threadIdx.x;
  if (tid >= 32) return;
  const int m = (1 << log2n) - 1, j = tid & (IT_Y - 1);
  const int64_t row = ((int64_t)(q & m) << (2 * log2n)) | ((int64_t)(y0 + j) << log2n);
  const uint32_t v = __ldg(cellstart + row + z0 + (tid < IT_Y ? 0 : IT_Z));
  const uint32_t end = __shfl_down_sync(0xffffffffu, v, IT_Y);
  uint32_t incl = tid < IT_Y ? end - v : 0u;
#pragma unroll
  for (int o = 1; o < IT_Y; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (j >= o) incl += y;
  }
  if (tid < IT_Y) {
    start[j] = v;
    pre[j + 1] = incl;
    if (j == 0) pre[0] = 0;
  }
}

// Inverse TSC (+ kick and drift) of the particles of one plane of a column,
// force planes x-1, x, x+1 at S[0..2] (each [3][IE_Y][IE_Z]).
template <bool MAXES>
__device__ __forceinline__ void column_particles(const float2* const S2[3], const float* const Sz[3],
                                                 const uint32_t* st, const uint32_t* pre,
                                                 int y0, int z0, const uint32_t* __restrict__ Xs,
                                                 const float* __restrict__ Vs, const uint32_t* __restrict__ ids_in,
                                                 int64_t np, int log2n, float* __restrict__ acc,
                                                 uint32_t* __restrict__ Xo, float* __restrict__ Vo,
                                                 uint32_t* __restrict__ ids_out, float dt_kick, float drift_scale,
                                                 int mode, float& amax, float& vmax) {
  const int sh = 32 - log2n;
  const uint32_t total = pre[IT_Y];
  for (uint32_t i = threadIdx.x; i < total; i += I_THREADS) {
    int j = 0;   // the run holding flat index i
#pragma unroll
    for (int b = IT_Y / 2; b > 0; b >>= 1)
      if (pre[j + b] <= i) j += b;
    const int64_t p = (int64_t)st[j] + (i - pre[j]);
    const uint32_t x = __ldg(Xs + p), y = __ldg(Xs + np + p), z = __ldg(Xs + 2 * np + p);
    // velocities in flight while the force is summed
    float v0x = 0.0f, v0y = 0.0f, v0z = 0.0f;
    if (mode == 1) {
      v0x = __ldg(Vs + p);
      v0y = __ldg(Vs + np + p);
      v0z = __ldg(Vs + 2 * np + p);
    }
    float wx[3], wy[3], wz[3];
    tsc_weights(cell_offset(x, log2n), wx);
    tsc_weights(cell_offset(y, log2n), wy);
    tsc_weights(cell_offset(z, log2n), wz);
    const int c = ((int)(y >> sh) - y0 + 1) * IE_Z + ((int)(z >> sh) - z0 + 1);
    float ax = 0.0f, ay = 0.0f, az = 0.0f;
#pragma unroll
    for (int ox = 0; ox < 3; ++ox) {
#pragma unroll
      for (int oy = 0; oy < 3; ++oy) {
        const float wxy = wx[ox] * wy[oy];
        const float2* r2 = S2[ox] + c + (oy - 1) * IE_Z;
        const float* rz = Sz[ox] + c + (oy - 1) * IE_Z;
#pragma unroll
        for (int oz = 0; oz < 3; ++oz) {
          const float w = wxy * wz[oz];
          const float2 fxy = r2[oz - 1];
          ax = fmaf(w, fxy.x, ax);
          ay = fmaf(w, fxy.y, ay);
          az = fmaf(w, rz[oz - 1], az);
        }
      }
    }
    if (acc) {
      acc[p] = ax;
      acc[np + p] = ay;
      acc[2 * np + p] = az;
    }
    if (MAXES) amax = fmaxf(amax, sqrtf(fmaf(ax, ax, fmaf(ay, ay, az * az))));
    if (mode == 1) {
      const float vx = fmaf(ax, dt_kick, v0x);
      const float vy = fmaf(ay, dt_kick, v0y);
      const float vz = fmaf(az, dt_kick, v0z);
      Vo[p] = vx;
      Vo[np + p] = vy;
      Vo[2 * np + p] = vz;
      if (MAXES) vmax = fmaxf(vmax, sqrtf(fmaf(vx, vx, fmaf(vy, vy, vz * vz))));
      Xo[p] = x + (uint32_t)__float2int_rn(vx * drift_scale);
      Xo[np + p] = y + (uint32_t)__float2int_rn(vy * drift_scale);
      Xo[2 * np + p] = z + (uint32_t)__float2int_rn(vz * drift_scale);
      if (ids_out) ids_out[p] = __ldg(ids_in + p);
    }
  }
}

// Block maxima of |a| and |v| (non-negative floats order like their bit
// patterns), one float2 per block.
__device__ __forceinline__ void block_maxima(float amax, float vmax, float2* __restrict__ blockmax) {
  __shared__ unsigned wa[I_THREADS / 32], wv[I_THREADS / 32];
  const int tid = threadIdx.x;
  const unsigned ua = __reduce_max_sync(0xffffffffu, __float_as_uint(amax));
  const unsigned uv = __reduce_max_sync(0xffffffffu, __float_as_uint(vmax));
  if ((tid & 31) == 0) {
    wa[tid >> 5] = ua;
    wv[tid >> 5] = uv;
  }
  __syncthreads();
  if (tid == 0) {
    unsigned ma = 0, mv = 0;
    for (int w = 0; w < I_THREADS / 32; ++w) {
      ma = max(ma, wa[w]);
      mv = max(mv, wv[w]);
    }
    blockmax[(int64_t)blockIdx.z * gridDim.x + blockIdx.x] = make_float2(__uint_as_float(ma), __uint_as_float(mv));
  }
}

// The force planes from the potential in shared memory, then the particles.
// Per plane step u: the potential plane u (with a halo of R + 1 in y and z;
// loaded into registers one step ahead, combined with eps for f(R)) goes to a
// ring of 2R + 2 slots; after the step's one barrier the force plane u - R
// (with a one-cell halo) is computed into a ring of 4 slots while the
// particles of plane u - R - 2 are interpolated from the three force planes
// computed in the steps before.
template <int ORDER, bool FR, bool MAXES>
__global__ void __launch_bounds__(I_THREADS) k_force_interp_stream(
    const float* __restrict__ phi, const float* __restrict__ eps, float alpha, int nh, float inv_h,
    const uint32_t* __restrict__ cellstart, const uint32_t* __restrict__ Xs, const float* __restrict__ Vs,
    const uint32_t* __restrict__ ids_in, int64_t np, int log2n, int chunk, int nitems, float* __restrict__ acc,
    uint32_t* __restrict__ Xo, float* __restrict__ Vo, uint32_t* __restrict__ ids_out, float dt_kick,
    float drift_scale, int mode, const float* __restrict__ dtk_box, const float* __restrict__ dtd_box,
    float2* __restrict__ blockmax) {
  constexpr int R = Stencil<ORDER>::R, H = R + 1, PEY = IT_Y + 2 * H, PEZ = IT_Z + 2 * H, PPL = PEY * PEZ,
                PS = 2 * R + 2, PL_T = (PPL + I_THREADS - 1) / I_THREADS;
  extern __shared__ float fsm[];
  float2* Gxy = reinterpret_cast<float2*>(fsm);   // [4][IE_Y][IE_Z] (g_x, g_y)
  float* Gz = fsm + 4 * 2 * I_PL;                  // [4][IE_Y][IE_Z] g_z
  float* Ps = fsm + 4 * 3 * I_PL;                  // [PS][PEY][PEZ]
  __shared__ uint32_t s_start[2][IT_Y], s_pre[2][IT_Y + 1];
  const int n = 1 << log2n, m = n - 1;
  const int64_t N = (int64_t)1 << (3 * log2n);
  phi += (int64_t)blockIdx.z * N;   // the box of a batched launch
  if (FR) eps += (int64_t)blockIdx.z * N;
  cellstart += (int64_t)blockIdx.z * N;
  if (dtk_box) dt_kick = __ldg(dtk_box + blockIdx.z);
  if (dtd_box) drift_scale = __ldg(dtd_box + blockIdx.z) * 4294967296.0f;
  const int tiles_z = n / IT_Z, tiles = (n / IT_Y) * tiles_z;
  const int tid = threadIdx.x;
  float amax = 0.0f, vmax = 0.0f;
  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
    const int tile = item % tiles, xc = item / tiles;
    const int y0 = (tile / tiles_z) * IT_Y, z0 = (tile % tiles_z) * IT_Z;
    const int x0 = xc * chunk, x1 = x0 + chunk;
    // raw potential (and eps) of plane q at this thread's positions
    float rp[PL_T], re[PL_T];
    auto fetch = [&](int q) {
      const int64_t pb = (int64_t)(q & m) << (2 * log2n);
#pragma unroll
      for (int k = 0; k < PL_T; ++k) {
        const int e = tid + k * I_THREADS;
        if (e < PPL) {
          const int ly = e / PEZ, lz = e - ly * PEZ;
          const int64_t c = pb | ((int64_t)((y0 - H + ly) & m) << log2n) | ((z0 - H + lz) & m);
          rp[k] = __ldg(phi + c);
          if (FR) re[k] = __ldg(eps + c);
        }
      }
    };
    auto store = [&](int q) {
      float* P = Ps + (((q % PS) + PS) % PS) * PPL;
#pragma unroll
      for (int k = 0; k < PL_T; ++k) {
        const int e = tid + k * I_THREADS;
        if (e < PPL) {
          float v = rp[k];
          if (FR) {
            const float ev = re[k];
            v = fmaf(alpha, nh == 2 ? ev * fmaf(ev, 3.0f + ev, 3.0f) : ev * (2.0f + ev), v);
          }
          P[e] = v;
        }
      }
    };
    // step u: potential plane u stored, force plane u - R computed, particles
    // of plane u - R - 2 interpolated (their force planes were computed in
    // the three steps before): one barrier per step
    const int u0 = x0 - 1 - R, ulast = x1 + R + 1;
    fetch(u0);
    for (int u = u0; u <= ulast; ++u) {
      if (u <= x1 + R) store(u);
      if (u < x1 + R) fetch(u + 1);
      __syncthreads();
      const int qg = u - R;
      if (qg >= x0 - 1 && qg <= x1) {
        float2* G2 = Gxy + (qg & 3) * I_PL;
        float* G1 = Gz + (qg & 3) * I_PL;
        const float* Pc = Ps + (((qg % PS) + PS) % PS) * PPL;
        for (int e = tid; e < I_PL; e += I_THREADS) {
          const int ly = e / IE_Z, lz = e - ly * IE_Z;
          const int c = (ly + R) * PEZ + lz + R;   // potential position of force cell (ly - 1, lz - 1)
          float gx = 0.0f, gy = 0.0f, gz = 0.0f;
#pragma unroll
          for (int q = R; q >= 1; --q) {
            const float w = Stencil<ORDER>::c(q);
            const float* Pp = Ps + ((((qg + q) % PS) + PS) % PS) * PPL;
            const float* Pm = Ps + ((((qg - q) % PS) + PS) % PS) * PPL;
            gx = fmaf(w, Pp[c] - Pm[c], gx);
            gy = fmaf(w, Pc[c + q * PEZ] - Pc[c - q * PEZ], gy);
            gz = fmaf(w, Pc[c + q] - Pc[c - q], gz);
          }
          G2[e] = make_float2(-gx * inv_h, -gy * inv_h);
          G1[e] = -gz * inv_h;
        }
      }
      const int t = qg - 2;   // particle plane of this step
      if (t + 1 >= x0 && t + 1 < x1)
        column_runs(cellstart, t + 1, y0, z0, log2n, s_start[(t + 1) & 1], s_pre[(t + 1) & 1]);
      if (t >= x0 && t < x1) {
        const float2* S2[3];
        const float* Sz[3];
#pragma unroll
        for (int ox = 0; ox < 3; ++ox) {
          S2[ox] = Gxy + ((t + ox - 1) & 3) * I_PL;
          Sz[ox] = Gz + ((t + ox - 1) & 3) * I_PL;
        }
        column_particles<MAXES>(S2, Sz, s_start[t & 1], s_pre[t & 1], y0, z0, Xs, Vs, ids_in, np, log2n, acc, Xo, Vo,
                                ids_out, dt_kick, drift_scale, mode, amax, vmax);
      }
    }
    __syncthreads();   // the rings and run buffers are reused by the next item
  }
  if (MAXES) block_maxima(amax, vmax, blockmax);
}

template <int ORDER>
constexpr size_t force_interp_smem() {
  return sizeof(float) * (4 * 3 * I_PL + (2 * Stencil<ORDER>::R + 2) * (IT_Y + 2 * Stencil<ORDER>::R + 2) *
                                             (IT_Z + 2 * Stencil<ORDER>::R + 2));
}

// Largest |v| of the velocity planes V [3][np]: one float2 (0, max) per block
// (float bits of non-negative values order like unsigned integers).
__global__ void __launch_bounds__(256) k_speed_max(const float* __restrict__ V, int64_t np,
                                                   float2* __restrict__ blockmax) {
  __shared__ unsigned wv[8];
  unsigned mv = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x) {
    const float vx = __ldg(V + i), vy = __ldg(V + np + i), vz = __ldg(V + 2 * np + i);
    mv = max(mv, __float_as_uint(sqrtf(vx * vx + vy * vy + vz * vz)));
  }
  mv = __reduce_max_sync(0xffffffffu, mv);
  if ((threadIdx.x & 31) == 0) wv[threadIdx.x >> 5] = mv;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 0; w < 8; ++w) mv = max(mv, wv[w]);
    blockmax[blockIdx.x] = make_float2(0.0f, __uint_as_float(mv));
  }
}

// Maximum over count float2 pairs, per component, into out[0], out[1]
// (float64); one block.
__global__ void __launch_bounds__(1024) k_max_pairs(const float2* __restrict__ v, int64_t count,
                                                    double* __restrict__ out) {
  __shared__ unsigned wa[32], wv[32];
  unsigned ma = 0, mv = 0;
  for (int64_t i = threadIdx.x; i < count; i += blockDim.x) {
    const float2 x = v[i];
    ma = max(ma, __float_as_uint(x.x));
    mv = max(mv, __float_as_uint(x.y));
  }
  ma = __reduce_max_sync(0xffffffffu, ma);
  mv = __reduce_max_sync(0xffffffffu, mv);
  if ((threadIdx.x & 31) == 0) {
    wa[threadIdx.x >> 5] = ma;
    wv[threadIdx.x >> 5] = mv;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      ma = max(ma, wa[w]);
      mv = max(mv, wv[w]);
    }
    out[0] = __uint_as_float(ma);
    out[1] = __uint_as_float(mv);
  }
}

template <int ORDER>
pm_status launch_grad(const float* phi, const float* eps, float alpha, float* g, int n, bool vec4, cudaStream_t s,
                      int B, int nh) {
  const int64_t N = (int64_t)n * n * n;
  const double bytes = ((eps ? 8.0 : 4.0) * N + (vec4 ? 16.0 : 12.0) * N) * B;
  if (n >= 64) {
    constexpr int R = Stencil<ORDER>::R;
    constexpr size_t smem = sizeof(float) * (2 * R + 1) * (GTY + 2 * R) * (GTZ + 2 * R);
    const int tiles = (n / GTY) * (n / GTZ);
    int chunk = n;
    while (chunk > 16 && (int64_t)tiles * (n / chunk) < 8 * 152) chunk >>= 1;
    const int nitems = tiles * (n / chunk);
    unsigned gx = (unsigned)(nitems < 152 * 4 ? nitems : 152 * 4);
    if (B > 1) gx = (unsigned)nitems;   // the boxes fill the GPU: one item per CTA
    const dim3 grid(gx, 1, (unsigned)B);
#define PM_GRAD_STREAM(FRB, V4)                                                                                    \
  PM_LAUNCH(K_GRADIENT, bytes, (k_gradient_stream<ORDER, FRB, V4>), grid, GNT, smem, s, phi, eps, alpha, g, ilog2(n), \
            (float)n, chunk, nitems, nh)
    if (eps) {
      if (vec4) PM_GRAD_STREAM(true, true); else PM_GRAD_STREAM(true, false);
    } else {
      if (vec4) PM_GRAD_STREAM(false, true); else PM_GRAD_STREAM(false, false);
    }
#undef PM_GRAD_STREAM
    return launch_status();
  }
  if (vec4) return PM_EINVAL;
  const dim3 grid(grid_for(N, 256), 1, (unsigned)B);
  if (eps)
    PM_LAUNCH(K_GRADIENT, bytes, (k_gradient<ORDER, true>), grid, 256, 0, s, phi, eps, alpha, g, ilog2(n), (float)n,
              nh);
  else
    PM_LAUNCH(K_GRADIENT, bytes, (k_gradient<ORDER, false>), grid, 256, 0, s, phi, eps, alpha, g, ilog2(n), (float)n,
              nh);
  return launch_status();
}

}  // namespace

pm_status gradient_launch(const float* phi, const float* eps, float alpha, float* g, int n, int order, bool vec4,
                          cudaStream_t s, int batch, int nh) {
  if (order == 3) return launch_grad<3>(phi, eps, alpha, g, n, vec4, s, batch, nh);
  if (order == 5) return launch_grad<5>(phi, eps, alpha, g, n, vec4, s, batch, nh);
  if (order == 7) return launch_grad<7>(phi, eps, alpha, g, n, vec4, s, batch, nh);
  return PM_EINVAL;
}

template <int ORDER>
pm_status launch_force_interp(const float* phi, const float* eps, float alpha, int nh, const uint32_t* cellstart,
                              const uint32_t* Xs, const float* Vs, const uint32_t* ids_in, int64_t np, int n,
                              float* acc, uint32_t* Xo, float* Vo, uint32_t* ids_out, float dt_kick,
                              float drift_scale, int mode, cudaStream_t s, const Batch& bt, float2* blockmax,
                              int64_t* nblocks) {
  constexpr size_t smem = force_interp_smem<ORDER>();
  PM_TRY(smem_attr(k_force_interp_stream<ORDER, false, false>, smem));
  PM_TRY(smem_attr(k_force_interp_stream<ORDER, false, true>, smem));
  PM_TRY(smem_attr(k_force_interp_stream<ORDER, true, false>, smem));
  PM_TRY(smem_attr(k_force_interp_stream<ORDER, true, true>, smem));
  const int tiles = (n / IT_Y) * (n / IT_Z);
  int chunk = n;
  while (chunk > 16 && (int64_t)tiles * (n / chunk) * bt.B < 16 * 152) chunk >>= 1;
  if (bt.B > 1) {   // batches: the x chunk is tuned (each particle's force is chunk-independent)
    int cand[3], nc = 0;
    for (int c = 16; c <= 64 && c <= n; c *= 2) cand[nc++] = c;
    chunk = tune_begin(TUNE_FORCE_CHUNK, n, bt.B, cand, nc, chunk, s);
  }
  const int nitems = tiles * (n / chunk);
  const dim3 grid((unsigned)nitems, 1, (unsigned)bt.B);
  *nblocks = (int64_t)grid.x * grid.z;
  const double N = (double)n * n * n * bt.B;
  const double bytes = (eps ? 8.0 : 4.0) * N + np * (12.0 + (mode ? 36.0 : 0.0) + (acc ? 12.0 : 0.0) +
                                                      (ids_out ? 8.0 : 0.0));
#define PM_FI(FRB, MX)                                                                                          \
  PM_LAUNCH(K_INTERP, bytes, (k_force_interp_stream<ORDER, FRB, MX>), grid, I_THREADS, smem, s, phi, eps, alpha, nh, \
            (float)n, cellstart, Xs, Vs, ids_in, np, ilog2(n), chunk, nitems, acc, Xo, Vo, ids_out, dt_kick,       \
            drift_scale, mode, bt.dt_kick, bt.dt_drift, blockmax)
  if (eps) {
    if (blockmax) PM_FI(true, true); else PM_FI(true, false);
  } else {
    if (blockmax) PM_FI(false, true); else PM_FI(false, false);
  }
#undef PM_FI
  if (bt.B > 1) tune_end(s);
  return launch_status();
}

pm_status max_speed_launch(const float* V, int64_t np, float2* blockmax, double* max_out, cudaStream_t s) {
  const unsigned nb = grid_for(np, 256, 152 * 16);
  PM_LAUNCH(K_REDUCE, 12.0 * np, k_speed_max, nb, 256, 0, s, V, np, blockmax);
  PM_LAUNCH(K_REDUCE, 8.0 * nb, k_max_pairs, 1, 1024, 0, s, blockmax, (int64_t)nb, max_out);
  return launch_status();
}

pm_status force_interp_launch(const float* phi, const float* eps, float alpha, int nh, int order,
                              const uint32_t* cellstart, const uint32_t* Xs, const float* Vs, const uint32_t* ids_in,
                              int64_t np, int n, float* acc, uint32_t* Xo, float* Vo, uint32_t* ids_out,
                              float dt_kick, float dt_drift, int mode, cudaStream_t s, const Batch& bt,
                              float2* blockmax, double* max_out) {
  if (np == 0) return PM_OK;
  if (n < 32 || !cellstart) return PM_EINVAL;
  const float drift_scale = (float)((double)dt_drift * 4294967296.0);
  if (!max_out) blockmax = nullptr;
  int64_t nblocks = 0;
  pm_status r = PM_EINVAL;
  if (order == 3)
    r = launch_force_interp<3>(phi, eps, alpha, nh, cellstart, Xs, Vs, ids_in, np, n, acc, Xo, Vo, ids_out, dt_kick,
                               drift_scale, mode, s, bt, blockmax, &nblocks);
  else if (order == 5)
    r = launch_force_interp<5>(phi, eps, alpha, nh, cellstart, Xs, Vs, ids_in, np, n, acc, Xo, Vo, ids_out, dt_kick,
                               drift_scale, mode, s, bt, blockmax, &nblocks);
  else if (order == 7)
    r = launch_force_interp<7>(phi, eps, alpha, nh, cellstart, Xs, Vs, ids_in, np, n, acc, Xo, Vo, ids_out, dt_kick,
                               drift_scale, mode, s, bt, blockmax, &nblocks);
  if (r != PM_OK) return r;
  if (blockmax) PM_LAUNCH(K_REDUCE, 8.0 * nblocks, k_max_pairs, 1, 1024, 0, s, blockmax, nblocks, max_out);
  return launch_status();
}

pm_status interp_launch(const float* g, const uint32_t* Xs, const float* Vs, const uint32_t* ids_in, int64_t np,
                        int n, float* acc, uint32_t* Xo, float* Vo, uint32_t* ids_out, float dt_kick,
                        float dt_drift, int mode, bool vec4, cudaStream_t s, const Batch& bt,
                        float2* blockmax, double* max_out) {
  if (np == 0) return PM_OK;
  const float drift_scale = (float)((double)dt_drift * 4294967296.0);
  const double bytes = (vec4 ? 16.0 : 12.0) * n * n * (double)n * bt.B +
                       np * (12.0 + (mode ? 36.0 : 0.0) + (acc ? 12.0 : 0.0) + (ids_out ? 8.0 : 0.0));
  const int64_t np_box = bt.B > 1 ? bt.np_box : np;
  const dim3 grid(grid_for(np_box, 256), 1, (unsigned)bt.B);
  if (!max_out) blockmax = nullptr;
#define PM_INTERP(V4, MX)                                                                                       \
  PM_LAUNCH(K_INTERP, bytes, (k_interp_kdk<V4, MX>), grid, 256, 0, s, g, Xs, Vs, ids_in, np, ilog2(n), acc, Xo, Vo, \
            ids_out, dt_kick, drift_scale, mode, np_box, bt.dt_kick, bt.dt_drift, blockmax)
  if (vec4) {
    if (blockmax) PM_INTERP(true, true); else PM_INTERP(true, false);
  } else {
    if (blockmax) PM_INTERP(false, true); else PM_INTERP(false, false);
  }
#undef PM_INTERP
  if (blockmax) {
    const int64_t nb = (int64_t)grid.x * grid.z;
    PM_LAUNCH(K_REDUCE, 8.0 * nb, k_max_pairs, 1, 1024, 0, s, blockmax, nb, max_out);
  }
  return launch_status();
}

}  // namespace pmgb
