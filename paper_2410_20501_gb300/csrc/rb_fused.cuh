// One full red-black sweep of a level in one pass over HBM.
//
// A CTA owns a 32 x 32 column of (y, z) cells and a chunk of x planes and
// marches along x.  At step t it updates the red cells of plane t on the
// column plus a one-cell ring around it, from the old values of planes
// t - 1, t, t + 1 (red cells only have black neighbours, and no black cell
// has moved yet), and the black cells of plane t - 2 on the column, from the
// new red values of planes t - 3, t - 2, t - 1 computed in earlier steps (all
// in shared memory: the ring supplies the in-plane neighbours owned by the
// next columns).  Every update therefore sees exactly the neighbour values of the
// plain red pass followed by the black pass, and with the same update functor
// the result is bitwise that of the two colour passes.  Old values come from
// `uin`, the result goes to `uout` (ping-pong), so neighbouring CTAs never
// see each other's new values.  Each cell's old value and source are read
// from HBM once and its new value written once: 12 bytes per cell and sweep.
//
// Shared memory holds rings of 8 planes of old values (rows y0-2 .. y0+33,
// columns z0-4 .. z0+35, stored as float4) and 4 planes of new red values
// (same layout); with these depths one barrier per plane suffices.  Old
// values and sources are fetched into registers two planes ahead.  Threads 0..511 own the red-black pair (z = 2kp, 2kp + 1) of row
// y = tid / 16 (one red update and one black update per plane); threads
// 512..575 update the 64 red cells of the ring (rows y0-1 and y0+32,
// columns z0-1 and z0+32).
#pragma once

#include "pm_internal.cuh"

namespace pmgb {

constexpr int kFusedT = 32;                        // tile edge (y and z)
constexpr int kFusedThreads = 16 * kFusedT + 64;   // 512 pair owners + 64 ring cells
constexpr int kFusedER = kFusedT + 4;              // stored rows: y0-2 .. y0+33
constexpr int kFusedEC = kFusedT + 8;              // stored columns: z0-4 .. z0+35
constexpr int kFusedPL = kFusedER * kFusedEC;      // floats per stored plane
constexpr int kFusedRingOld = 8;   // old values: planes t - 7 .. t + 1 (a store may run ahead of
                                   // the previous step's readers: no barrier between them)
constexpr int kFusedRing = 4;      // new red values: planes t - 3 .. t
constexpr size_t kFusedSmem = sizeof(float) * (kFusedRingOld + kFusedRing) * kFusedPL;
constexpr int kFusedLoads = kFusedER * (kFusedEC / 4);   // float4 loads per plane (360)
static_assert(kFusedLoads <= kFusedThreads, "one float4 per thread per plane");

// Update functor interface: upd(old, nb[6] (x+, x-, y+, y-, z+, z-), source,
// sweep index (0 here), neighbours-never-updated, own-never-updated).  MINB:
// resident CTAs per SM the register allocation is sized for.  LAG: planes
// between the red and the black update of a step (1 or 2, below).
template <class Upd, int MINB, int LAG>
__global__ void __launch_bounds__(kFusedThreads, MINB) k_rb_fused(const float* __restrict__ uin,
                                                               float* __restrict__ uout, Src f, int log2n, int chunk,
                                                               int zero, int first, Upd upd) {
  constexpr int T = kFusedT, EC = kFusedEC, PL = kFusedPL, R = kFusedRing, RO = kFusedRingOld;
  extern __shared__ float4 fsm4[];
  float* Old = reinterpret_cast<float*>(fsm4);   // [RO][ER][EC]
  float* Red = Old + RO * PL;                    // [R][ER][EC]
  const int n = 1 << log2n, m = n - 1;
  const int tiles_z = n / T, tiles = (n / T) * tiles_z;
  const int item = blockIdx.x;
  {   // the box of a batched launch
    const int64_t off = (int64_t)blockIdx.z << (3 * log2n);
    uin += off;
    uout += off;
    f = box_src(f, (int64_t)1 << (3 * log2n));
    upd = upd.box(blockIdx.z);
  }
  const int tile = item % tiles, xc = item / tiles;
  const int y0 = (tile / tiles_z) * T, z0 = (tile % tiles_z) * T;
  const int x0 = xc * chunk, x1 = x0 + chunk;
  const float mean = f.mean ? (float)*f.mean : 0.0f;
  const int tid = threadIdx.x;
  const bool nb_old_red = first != 0, own_old = first != 0;
  // stored position of local (y, z): row y + 2, column z + 4

  // plane loads: thread tid < 360 moves one float4 (row lr, column group lc)
  const int lr = tid / (EC / 4), lc4 = tid - lr * (EC / 4);
  const bool loader = tid < kFusedLoads;
  const int64_t goff = loader ? (((int64_t)((y0 - 2 + lr) & m) << log2n) | ((z0 - 4 + 4 * lc4) & m)) : 0;
  auto fetch = [&](int t) -> float4 {
    return __ldg(reinterpret_cast<const float4*>(uin + (((int64_t)(t & m) << (2 * log2n)) | goff)));
  };
  auto store = [&](int t, float4 v) {
    *reinterpret_cast<float4*>(Old + (t & (RO - 1)) * PL + lr * EC + 4 * lc4) = v;
  };

  if (zero) {
    for (int i = tid; i < RO * PL; i += kFusedThreads) Old[i] = 0.0f;
  } else if (loader) {
    store(x0 - 2, fetch(x0 - 2));
    store(x0 - 1, fetch(x0 - 1));
  }
  // old values of planes t + 1 and t + 2 in flight (two planes ahead)
  float4 pre0 = make_float4(0.0f, 0.0f, 0.0f, 0.0f), pre1 = pre0;
  if (!zero && loader) {
    pre0 = fetch(x0);
    pre1 = fetch(x0 + 1);
  }

  // pair owners: row py, pair kp; ring workers: task h
  const bool owner = tid < 16 * T;
  const int py = tid >> 4, kp = tid & 15, h = tid - 16 * T;
  // the red cell (local y, z) this thread updates on plane t
  auto red_cell = [&](int t, int& y, int& z) {
    if (owner) {
      y = py;
      z = 2 * kp + ((t + y0 + y) & 1);
    } else if (h < 32) {                       // rows y0 - 1 and y0 + 32
      y = h < 16 ? -1 : T;
      z = 2 * (h & 15) + ((t + y0 + y) & 1);
    } else {                                   // columns z0 - 1 and z0 + 32
      z = h < 48 ? -1 : T;
      y = 2 * (h & 15) + ((t + y0 + z0 + z) & 1);
    }
  };
  // source values of plane t, fetched one step ahead: owners read their pair
  // (red and black cell), ring workers their red cell
  auto fetch_f = [&](int t) -> float2 {
    const int64_t gplane = (int64_t)(t & m) << (2 * log2n);
    if (owner)
      return __ldg(reinterpret_cast<const float2*>(f.p + (gplane | ((int64_t)((y0 + py) & m) << log2n) |
                                                         (z0 + 2 * kp))));
    int y, z;
    red_cell(t, y, z);
    return make_float2(__ldg(f.p + (gplane | ((int64_t)((y0 + y) & m) << log2n) | ((z0 + z) & m))), 0.0f);
  };
  float2 f0 = fetch_f(x0 - 1), f1 = fetch_f(x0);   // sources of planes t and t + 1

  // One plane step t: store the old values of plane t + 1, a barrier, then
  // the red cells of plane t and the black cells of plane p = t - LAG, whose
  // red neighbours on planes p - 1 .. p + 1 are complete: with LAG = 2 they
  // were all computed in earlier steps (one barrier per step); with LAG = 1
  // plane t is among them and a second barrier separates the two updates.
  // The prefetch registers alternate between even and odd steps (no register
  // copies, which would wait for the loads in flight): pa holds plane t + 1
  // and is refilled with plane t + 3, fa the sources of plane t, refilled
  // with plane t + 2; fb_t receives the black source of plane t, fb_p holds
  // that of plane p (the same register as fb_t when LAG = 2).
  auto black = [&](int p, float fbp) {
    if (!(owner && p >= x0 && p < x1)) return;
    const float* Op = Old + (p & (RO - 1)) * PL;
    const float* Rp = Red + (p & (R - 1)) * PL;      // new red values, planes p - 1, p, p + 1
    const float* Rm = Red + ((p - 1) & (R - 1)) * PL;
    const float* Rq = Red + ((p + 1) & (R - 1)) * PL;
    const int y = py;
    const int o = (p + y0 + y) & 1;                  // red cell of the pair at z = 2 kp + o
    const int qr = (y + 2) * EC + 2 * kp + 4;        // first cell of the pair
    const int q = qr + 1 - o;                        // black cell
    const float nb[6] = {Rq[q], Rm[q], Rp[q + EC], Rp[q - EC], Rp[q + 1], Rp[q - 1]};
    const float vb = upd(Op[q], nb, fbp, 0, false, own_old);
    const float vr = Rp[qr + o];
    const float2 out = o ? make_float2(vb, vr) : make_float2(vr, vb);
    *reinterpret_cast<float2*>(uout + (((int64_t)(p & m) << (2 * log2n)) | ((int64_t)((y0 + y) & m) << log2n) |
                                       (z0 + 2 * kp))) = out;
  };
  auto red = [&](int t, float2 f_t, float& fb_t) {
    if (t > x1) return;
    const float* Om = Old + ((t - 1) & (RO - 1)) * PL;   // old values, planes t - 1, t, t + 1
    const float* O0 = Old + (t & (RO - 1)) * PL;
    const float* Oq = Old + ((t + 1) & (RO - 1)) * PL;
    int y, z;
    red_cell(t, y, z);
    const int q = (y + 2) * EC + z + 4;
    const float nb[6] = {Oq[q], Om[q], O0[q + EC], O0[q - EC], O0[q + 1], O0[q - 1]};
    float fv;
    if (owner) {
      const bool red_first = ((t + y0 + y) & 1) == 0;
      fv = f.s * ((red_first ? f_t.x : f_t.y) - mean);
      fb_t = f.s * ((red_first ? f_t.y : f_t.x) - mean);
    } else {
      fv = f.s * (f_t.x - mean);
    }
    Red[(t & (R - 1)) * PL + q] = upd(O0[q], nb, fv, 0, nb_old_red, own_old);
  };
  auto step = [&](int t, float4& pa, float2& fa, float& fb_t, float& fb_p) {
    if (!zero && loader && t + 1 <= x1 + 1) {
      store(t + 1, pa);
      if (t + 3 <= x1 + 1) pa = fetch(t + 3);
    }
    const float2 f_t = fa;
    if (t + 2 <= x1) fa = fetch_f(t + 2);
    __syncthreads();
    if constexpr (LAG == 2) {
      black(t - 2, fb_p);       // fb_p is fb_t: read before red() replaces it
      red(t, f_t, fb_t);
    } else {
      red(t, f_t, fb_t);
      __syncthreads();
      black(t - 1, fb_p);
    }
  };
  float fb0 = 0.0f, fb1 = 0.0f;
  for (int t = x0 - 1; t <= x1 + LAG - 1; t += 2) {
    step(t, pre0, f0, fb0, LAG == 2 ? fb0 : fb1);
    if (t + 1 <= x1 + LAG - 1) step(t + 1, pre1, f1, fb1, LAG == 2 ? fb1 : fb0);
  }
}

// Work decomposition: x chunk for a level of size n (n >= 128): enough CTAs
// for about eight waves of two resident CTAs per SM (the tail wave is then a
// small part of the sweep), chunks of at least 16 planes (each chunk
// recomputes two red planes at its ends).
inline int fused_chunk(int n) {
  const int tiles = (n / kFusedT) * (n / kFusedT);
  int c = n;
  while (c > 16 && (int64_t)tiles * (n / c) < 8 * 2 * 152) c >>= 1;
  return c;
}

// Levels the fused kernel takes: n >= 128, or n = 64 in a batch of at least 8
// boxes (enough CTAs to fill the GPU).
inline bool fused_ok(int n, int B = 1) { return n >= 128 || (n >= 64 && B >= 8); }

// float4 plane loads, float2 source loads and pair stores need 16- and 8-byte
// aligned level arrays (workspace levels always are; caller arrays may not be).
inline bool fused_aligned(const float* u, const float* alt, const float* f) {
  return (((uintptr_t)u | (uintptr_t)alt) & 15) == 0 && ((uintptr_t)f & 7) == 0;
}

}  // namespace pmgb
