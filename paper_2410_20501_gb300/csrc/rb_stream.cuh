// Streaming red-black smoother: S full red-black sweeps (S = 1 or 2) of a
// level in one pass over HBM.
//
// A CTA owns a TY x TZ column of (y, z) cells and a chunk of x planes.  It
// streams the planes through a rolling window in shared memory: when plane t
// arrives, stage s = 1 .. 2S updates the cells of colour (s - 1) & 1 (red
// first) of plane t - s; stage s works on the column plus a halo of 2S - s
// cells in y and z, so the last stage covers exactly the column, whose plane
// t - 2S is then final and written out.  Running the stages in the order
// 1, 2, ..., 2S within a time step gives every update exactly the neighbour
// values of the plain colour-by-colour sweeps (stage s reads plane t - s - 1
// before stage s + 1 updates it), so the result is bitwise identical to
// 2S colour passes of the unfused kernels.  Reads come from `uin` and writes
// go to `uout` (ping-pong), so neighbouring CTAs never see each other's new
// values.  The update rule is a functor: linear SOR (Poisson) or the f(R)
// cubic.
#pragma once

#include "pm_internal.cuh"

namespace pmgb {

constexpr int kStreamTY = 16;
constexpr int kStreamTZ = 64;
constexpr int kStreamThreads = 256;

template <int S>
struct StreamGeom {
  static constexpr int H = 2 * S;                  // halo of the loaded planes
  static constexpr int EY = kStreamTY + 2 * H;
  static constexpr int EZ = kStreamTZ + 2 * H;
  static constexpr int W = 2 * S + 2;              // u planes held
  static constexpr int WF = 2 * S;                 // source planes held
  static constexpr size_t smem_bytes = sizeof(float) * (size_t)(W + WF) * EY * EZ;
};

__device__ __forceinline__ int pmod(int a, int b) { int r = a % b; return r < 0 ? r + b : r; }

// Update functors: (old value, 6 neighbours in the order x+, x-, y+, y-, z+,
// z-, source value, sweep index, stage-is-first-of-sweep-0 flags) -> new value.
struct PoissonUpdate {
  float h2;
  float omega[2];
  float gscale;     // warm-start rescale applied to never-updated values
  // Explicit rounding intrinsics (no contraction) so that the fused and the
  // colour-by-colour kernels produce bitwise identical updates.
  __device__ __forceinline__ float operator()(float old, const float nb[6], float fv, int sweep,
                                              bool nb_old, bool own_old) const {
    float s = __fadd_rn(nb[0], nb[1]);
    s = __fadd_rn(s, nb[2]);
    s = __fadd_rn(s, nb[3]);
    s = __fadd_rn(s, nb[4]);
    s = __fadd_rn(s, nb[5]);
    if (nb_old) s = __fmul_rn(gscale, s);
    const float ugs = __fmul_rn(__fsub_rn(s, __fmul_rn(h2, fv)), 1.0f / 6.0f);
    const float w = omega[sweep];
    if (w == 1.0f) return ugs;
    const float o = own_old ? __fmul_rn(gscale, old) : old;
    return __fadd_rn(__fmul_rn(w, ugs), __fmul_rn(1.0f - w, o));
  }
};

template <int S, class Upd>
__global__ void __launch_bounds__(kStreamThreads) k_rb_stream(const float* __restrict__ uin,
                                                             float* __restrict__ uout, Src f, int log2n,
                                                             int chunk, int nitems, int zero_guess, Upd upd) {
  using G = StreamGeom<S>;
  constexpr int TY = kStreamTY, TZ = kStreamTZ, H = G::H, EY = G::EY, EZ = G::EZ, W = G::W, WF = G::WF;
  constexpr int PL = EY * EZ;
  extern __shared__ float sm[];
  float* U = sm;               // [W][EY][EZ]
  float* F = sm + W * PL;      // [WF][EY][EZ]
  const int n = 1 << log2n, m = n - 1;
  const int tiles_z = n / TZ, tiles_y = n / TY;
  const int tiles = tiles_z * tiles_y;
  const float mean = f.mean ? (float)*f.mean : 0.0f;
  const int tid = threadIdx.x;

  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
    const int tile = item % tiles, xc = item / tiles;
    const int y0 = (tile / tiles_z) * TY, z0 = (tile % tiles_z) * TZ;
    const int x0 = xc * chunk, x1 = x0 + chunk;
    for (int t = x0 - H; t < x1 + H; ++t) {
      // plane t of u (halo H) and plane t - 1 of the source (halo H - 1)
      {
        const int slot = pmod(t, W), pt = t & m;
        float* Up = U + slot * PL;
        for (int e = tid; e < PL; e += kStreamThreads) {
          const int ly = e / EZ, lz = e - ly * EZ;
          const int gy = (y0 - H + ly) & m, gz = (z0 - H + lz) & m;
          Up[e] = zero_guess ? 0.0f : __ldg(uin + (((int64_t)pt << (2 * log2n)) | ((int64_t)gy << log2n) | gz));
        }
        const int pf = t - 1, fslot = pmod(pf, WF), pft = pf & m;
        float* Fp = F + fslot * PL;
        for (int e = tid; e < PL; e += kStreamThreads) {
          const int ly = e / EZ, lz = e - ly * EZ;
          if (ly == 0 || ly == EY - 1 || lz == 0 || lz == EZ - 1) continue;
          const int gy = (y0 - H + ly) & m, gz = (z0 - H + lz) & m;
          Fp[e] = f.s * (__ldg(f.p + (((int64_t)pft << (2 * log2n)) | ((int64_t)gy << log2n) | gz)) - mean);
        }
      }
      __syncthreads();
#pragma unroll
      for (int s = 1; s <= 2 * S; ++s) {
        const int p = t - s;
        if (p >= x0 - H + s) {
          const int hs = 2 * S - s, colour = (s - 1) & 1, sweep = (s - 1) >> 1;
          const bool nb_old = (s == 1), own_old = (s <= 2);
          const int rows = TY + 2 * hs, half = (TZ + 2 * hs) >> 1;
          float* Up = U + pmod(p, W) * PL;
          const float* Um = U + pmod(p - 1, W) * PL;
          const float* Upp = U + pmod(p + 1, W) * PL;
          const float* Fp = F + pmod(p, WF) * PL;
          for (int idx = tid; idx < rows * half; idx += kStreamThreads) {
            const int r = idx / half, kk = idx - r * half;
            const int ly = H - hs + r, lz0 = H - hs;
            const int gy = y0 - hs + r, gz0 = z0 - hs;
            const int off = (colour + p + gy + gz0) & 1;
            const int c = ly * EZ + lz0 + 2 * kk + off;
            float nb[6];
            nb[0] = Upp[c];
            nb[1] = Um[c];
            nb[2] = Up[c + EZ];
            nb[3] = Up[c - EZ];
            nb[4] = Up[c + 1];
            nb[5] = Up[c - 1];
            Up[c] = upd(Up[c], nb, Fp[c], sweep, nb_old, own_old);
          }
        }
        __syncthreads();
      }
      const int po = t - 2 * S;
      if (po >= x0 && po < x1) {
        const float* Uo = U + pmod(po, W) * PL;
        const int64_t pbase = (int64_t)(po & m) << (2 * log2n);
        for (int e = tid; e < TY * TZ; e += kStreamThreads) {
          const int ly = e / TZ, lz = e - ly * TZ;
          uout[pbase | ((int64_t)(y0 + ly) << log2n) | (z0 + lz)] = Uo[(ly + H) * EZ + lz + H];
        }
      }
    }
    __syncthreads();
  }
}

// Work decomposition for a level of size n: chunk of x planes and item count.
inline void stream_plan(int n, int* chunk, int* nitems) {
  const int tiles = (n / kStreamTZ) * (n / kStreamTY);
  int c = n;
  while (c > 32 && (int64_t)tiles * (n / c) < 4 * 152) c >>= 1;
  *chunk = c;
  *nitems = tiles * (n / c);
}

inline bool stream_ok(int n) { return n >= 128; }

}  // namespace pmgb
