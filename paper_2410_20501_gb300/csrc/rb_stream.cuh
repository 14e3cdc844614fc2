// Streaming red-black smoother: S full red-black sweeps (S = 1 or 2) of a
// level in one pass over HBM.
//
// A CTA owns a TY x TZ column of (y, z) cells and a chunk of x planes.  It
// streams the planes through a rolling window in shared memory: when plane t
// arrives, stage s = 1 .. 2S updates the cells of colour (s - 1) & 1 (red
// first) of plane t - s; stage s covers the column plus a halo of 2S - s
// cells in y and z, so after the last stage plane t - 2S is final on the
// column and is written out.  Running the stages in the order 1, 2, ..., 2S
// within a time step hands every update exactly the neighbour values of the
// plain colour-by-colour sweeps (stage s reads plane t - s - 1 before stage
// s + 1 updates it), so the result is bitwise identical to 2S colour passes
// of the unfused kernels.  Reads come from `uin`, writes go to `uout`
// (ping-pong), so neighbouring CTAs never see each other's new values.
//
// Shared memory keeps every row split by colour (red cells of a row
// contiguous, then black), so the six neighbours of four consecutive
// same-colour cells come in 16-byte loads: the y, x neighbours sit at the same
// split index in the other colour's row, the two z neighbours at index kk + o
// and kk + o - 1 where o is the row's parity.  The next plane is fetched into
// registers while the current plane's stages run.  The update rule is a
// functor: linear SOR (Poisson) or the f(R) cubic.
#pragma once

#include "pm_internal.cuh"

namespace pmgb {

constexpr int kStreamTY = 16;
constexpr int kStreamTZ = 64;
constexpr int kStreamThreads = 192;

template <int S>
struct StreamGeom {
  static constexpr int H = 2 * S;                    // halo of the loaded planes
  static constexpr int EY = kStreamTY + 2 * H;       // rows per plane
  static constexpr int EZ = kStreamTZ + 2 * H;       // cells per row
  static constexpr int HALF = EZ / 2;                // loaded cells of one colour per row
  static constexpr int HALF4 = (HALF + 3) / 4 * 4;   // rounded up to whole float4 groups; the extra
                                                     // slots lie outside every stage's valid region
  static constexpr int PAD = 4;                      // padding in front of / behind each colour row
  static constexpr int RW = PAD + HALF4 + PAD;       // stored floats per colour row
  static constexpr int PL = 2 * EY * RW;             // floats per plane (both colours)
  static constexpr int W = 2 * S + 2;                // u planes held
  static constexpr int WF = 2 * S;                   // source planes held
  static constexpr int GROUPS = HALF4 / 4;           // float4 groups per colour row
  static constexpr int PAIRS = EY * HALF;            // float2 pairs per natural plane
  static constexpr int PER_T = (PAIRS + kStreamThreads - 1) / kStreamThreads;
  static constexpr size_t smem_bytes = sizeof(float) * (size_t)(W + WF) * PL;
};

__device__ __forceinline__ int pmod(int a, int b) { int r = a % b; return r < 0 ? r + b : r; }

// Update functors: (old value, 6 neighbours in the order x+, x-, y+, y-, z+,
// z-, source value, sweep index, neighbours-never-updated, own-never-updated)
// -> new value.
struct PoissonUpdate {
  float h2;
  float omega[2];
  float gscale;     // warm-start rescale applied to never-updated values
  const float* gbox = nullptr;   // per-box gscale of a batched launch (replaces gscale)
  __device__ __forceinline__ PoissonUpdate box(int b) const {
    PoissonUpdate u = *this;
    if (gbox) u.gscale = __ldg(gbox + b);
    return u;
  }
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
  constexpr int TY = kStreamTY, TZ = kStreamTZ, H = G::H, EY = G::EY, EZ = G::EZ, RW = G::RW;
  constexpr int PL = G::PL, W = G::W, WF = G::WF, NT = kStreamThreads;
  constexpr int PAIRS = G::PAIRS, PER_T = G::PER_T, ROWP = EZ / 2;
  extern __shared__ float4 sm4[];
  float* sm = reinterpret_cast<float*>(sm4);
  float* U = sm;                 // [W][2 colours][EY][RW]
  float* F = sm + W * PL;        // [WF][2 colours][EY][RW]
  const int n = 1 << log2n, m = n - 1;
  const int tiles_z = n / TZ, tiles = (n / TY) * tiles_z;
  const float mean = f.mean ? (float)*f.mean : 0.0f;
  const int tid = threadIdx.x;
  // colour row c of row ly in a plane: base + (c * EY + ly) * RW + PAD
  auto row = [&](float* plane, int c, int ly) -> float* { return plane + (c * EY + ly) * RW + G::PAD; };

  for (int i = tid; i < (W + WF) * PL; i += NT) sm[i] = 0.0f;   // paddings stay 0
  __syncthreads();

  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
    const int tile = item % tiles, xc = item / tiles;
    const int y0 = (tile / tiles_z) * TY, z0 = (tile % tiles_z) * TZ;
    const int x0 = xc * chunk, x1 = x0 + chunk;
    float2 pu[PER_T], pf[PER_T];

    // fetch plane t of u and plane t - 1 of the source into registers
    auto fetch = [&](int t) {
      const int64_t pt = (int64_t)(t & m) << (2 * log2n), pft = (int64_t)((t - 1) & m) << (2 * log2n);
#pragma unroll
      for (int q = 0; q < PER_T; ++q) {
        const int e = tid + q * NT;
        if (e < PAIRS) {
          const int ly = e / ROWP, kp = e - ly * ROWP;
          const int64_t off = ((int64_t)((y0 - H + ly) & m) << log2n) | ((z0 - H + 2 * kp) & m);
          pu[q] = zero_guess ? make_float2(0.0f, 0.0f) : __ldg(reinterpret_cast<const float2*>(uin + (pt | off)));
          const float2 fr = __ldg(reinterpret_cast<const float2*>(f.p + (pft | off)));
          pf[q] = make_float2(f.s * (fr.x - mean), f.s * (fr.y - mean));
        }
      }
    };
    // store the fetched pairs, split by colour: the pair (z, z+1) holds one
    // cell of each colour; colour of z is (plane + y + z) & 1
    auto store = [&](int t) {
      float* Up = U + pmod(t, W) * PL;
      float* Fp = F + pmod(t - 1, WF) * PL;
#pragma unroll
      for (int q = 0; q < PER_T; ++q) {
        const int e = tid + q * NT;
        if (e < PAIRS) {
          const int ly = e / ROWP, kp = e - ly * ROWP;
          const int gy = y0 - H + ly;
          const int cz = (t + gy) & 1;           // colour of the even cell z = z0 - H + 2 kp (z0 - H even)
          row(Up, cz, ly)[kp] = pu[q].x;
          row(Up, cz ^ 1, ly)[kp] = pu[q].y;
          const int cf = (t - 1 + gy) & 1;
          row(Fp, cf, ly)[kp] = pf[q].x;
          row(Fp, cf ^ 1, ly)[kp] = pf[q].y;
        }
      }
    };

    fetch(x0 - H);
    for (int t = x0 - H; t < x1 + H; ++t) {
      store(t);
      __syncthreads();
      if (t + 1 < x1 + H) fetch(t + 1);   // in flight while the stages run
#pragma unroll
      for (int s = 1; s <= 2 * S; ++s) {
        const int p = t - s;
        if (p >= x0 - H + s) {
          const int hs = 2 * S - s, colour = (s - 1) & 1, sweep = (s - 1) >> 1;
          const bool nb_old = (s == 1), own_old = (s <= 2);
          const int rows = TY + 2 * hs, r0 = H - hs;
          float* Up = U + pmod(p, W) * PL;
          const float* Um = U + pmod(p - 1, W) * PL;
          const float* Upp = U + pmod(p + 1, W) * PL;
          const float* Fp = F + pmod(p, WF) * PL;
          for (int w = tid; w < rows * G::GROUPS; w += NT) {
            const int r = w / G::GROUPS, kk0 = (w - r * G::GROUPS) * 4;
            const int ly = r0 + r, gy = y0 - H + ly;
            const int o = (p + gy + colour) & 1;   // target cells at z = 2 kk + o (local)
            float* tgt = row(Up, colour, ly);
            const float* oth = row(Up, colour ^ 1, ly);
            const float4 own = *reinterpret_cast<const float4*>(tgt + kk0);
            const float4 fv = *reinterpret_cast<const float4*>(row(const_cast<float*>(Fp), colour, ly) + kk0);
            const float4 xp = *reinterpret_cast<const float4*>(row(const_cast<float*>(Upp), colour ^ 1, ly) + kk0);
            const float4 xm = *reinterpret_cast<const float4*>(row(const_cast<float*>(Um), colour ^ 1, ly) + kk0);
            const float4 yp = *reinterpret_cast<const float4*>(row(Up, colour ^ 1, ly + 1) + kk0);
            const float4 ym = *reinterpret_cast<const float4*>(row(Up, colour ^ 1, ly - 1) + kk0);
            const float4 zc = *reinterpret_cast<const float4*>(oth + kk0);
            const float zx = o ? oth[kk0 + 4] : oth[kk0 - 1];
            const float ov[4] = {own.x, own.y, own.z, own.w};
            const float fa[4] = {fv.x, fv.y, fv.z, fv.w};
            const float xpa[4] = {xp.x, xp.y, xp.z, xp.w}, xma[4] = {xm.x, xm.y, xm.z, xm.w};
            const float ypa[4] = {yp.x, yp.y, yp.z, yp.w}, yma[4] = {ym.x, ym.y, ym.z, ym.w};
            const float za[4] = {zc.x, zc.y, zc.z, zc.w};
            float res[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              // z neighbours: other colour at kk + o (z + 1) and kk + o - 1 (z - 1)
              const float zplus = o ? (i < 3 ? za[i + 1] : zx) : za[i];
              const float zminus = o ? za[i] : (i > 0 ? za[i - 1] : zx);
              const float nb[6] = {xpa[i], xma[i], ypa[i], yma[i], zplus, zminus};
              res[i] = upd(ov[i], nb, fa[i], sweep, nb_old, own_old);
            }
            *reinterpret_cast<float4*>(tgt + kk0) = make_float4(res[0], res[1], res[2], res[3]);
          }
        }
        __syncthreads();
      }
      const int po = t - 2 * S;
      if (po >= x0 && po < x1) {
        const float* Uo = U + pmod(po, W) * PL;
        const int64_t pbase = (int64_t)(po & m) << (2 * log2n);
        for (int e = tid; e < TY * (TZ / 2); e += NT) {
          const int ly = e / (TZ / 2), kp = e - ly * (TZ / 2);
          const int gy = y0 + ly;
          const int cz = (po + gy) & 1;          // colour of the even cell z = z0 + 2 kp
          const int lrow = ly + H, lk = kp + H / 2;
          const float2 v = make_float2(row(const_cast<float*>(Uo), cz, lrow)[lk],
                                       row(const_cast<float*>(Uo), cz ^ 1, lrow)[lk]);
          *reinterpret_cast<float2*>(uout + (pbase | ((int64_t)gy << log2n) | (z0 + 2 * kp))) = v;
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
