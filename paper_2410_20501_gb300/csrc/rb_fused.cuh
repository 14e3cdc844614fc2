// One full red-black sweep of a level in one pass over HBM.
//
// A CTA owns a 32 x 32 column of (y, z) cells and a chunk of x planes and
// marches along x.  At step t it updates the red cells of plane t on the
// column plus a one-cell ring around it, from the old values of planes
// t - 1, t, t + 1 (red cells only have black neighbours, and no black cell
// has moved yet), and the black cells of plane t - 2 on the column, from the
// new red values of planes t - 3, t - 2, t - 1 computed in earlier steps (all
// in shared memory: the ring supplies the in-plane neighbours owned by the
// next columns).  Every update therefore sees exactly the neighbour values of
// the plain red pass followed by the black pass, in the functor's order x+,
// x-, y+, y-, z+, z-, and with the same update functor the result is bitwise
// that of the two colour passes.  Old values come from `uin`, the result goes
// to `uout` (ping-pong), so neighbouring CTAs never see each other's new
// values.  Each cell's old value and source are read from HBM once and its
// new value written once: 12 bytes per cell and sweep.
//
// Shared memory holds rings of 8 planes of old values (rows y0-2 .. y0+33,
// columns z0-4 .. z0+35) and 4 planes of new red values (same layout); with
// these depths one barrier per plane suffices.  The old-value planes arrive
// by per-thread asynchronous copies (cp.async, 16 bytes each) issued three
// planes ahead, so no registers hold them in flight; the sources are fetched
// into registers two planes ahead.
//
// 320 threads: threads 0..255 each own a run of four consecutive z cells of
// one row (two red and two black cells on every plane), threads 256..319
// update the 64 red cells of the ring (rows y0-1 and y0+32, columns z0-1 and
// z0+32).  A run's neighbours come in 16-byte shared-memory loads (x+, x-,
// y+, y- and its own row) plus one scalar for the z neighbour outside the
// run, and its result leaves in one 16-byte store.  Warp w owns the rows
// (w / 2) * 8 + (w & 1) + {0, 2, 4, 6}, all of one parity, so which cells of
// a run are red is the same for the whole warp.
#pragma once

#include "pm_internal.cuh"

namespace pmgb {

constexpr int kFusedT = 32;                        // tile edge (y and z)
constexpr int kFusedER = kFusedT + 4;              // stored rows: y0-2 .. y0+33
constexpr int kFusedEC = kFusedT + 8;              // stored columns: z0-4 .. z0+35
constexpr int kFusedPL = kFusedER * kFusedEC;      // floats per stored plane
constexpr int kFusedRingOld = 8;   // old values: planes t - 3 .. t + 3 (copies run three planes
                                   // ahead while warps finishing step t - 1 still read plane t - 3)
constexpr int kFusedRing = 4;      // new red values: planes t - 3 .. t
constexpr size_t kFusedSmem = sizeof(float) * (kFusedRingOld + kFusedRing) * kFusedPL;
constexpr int kFusedLoads = kFusedER * (kFusedEC / 4);   // float4 loads per plane (360)

// Work decomposition: x chunk for a level of size n (n >= 128): enough CTAs
// for about eight waves of two CTAs per SM (the tail wave is then a small
// part of the sweep), chunks of at least 16 planes (each chunk recomputes two
// red planes at its ends).
inline int fused_chunk(int n) {
  const int tiles = (n / kFusedT) * (n / kFusedT);
  int c = n;
  while (c > 16 && (int64_t)tiles * (n / c) < 8 * 2 * 152) c >>= 1;
  return c;
}

// Levels the fused kernel takes: n >= 128, or n = 64 in a batch of at least 8
// boxes (enough CTAs to fill the GPU).
inline bool fused_ok(int n, int B = 1) { return n >= 128 || (n >= 64 && B >= 8); }

// float4 plane, source and run loads and stores need 16-byte aligned level
// arrays (workspace levels always are; caller arrays are checked on entry).
inline bool fused_aligned(const float* u, const float* alt, const float* f) {
  return (((uintptr_t)u | (uintptr_t)alt | (uintptr_t)f) & 15) == 0;
}

}  // namespace pmgb

namespace pmgb {

constexpr int kQuadRuns = 8 * kFusedT;                 // 256 run owners
constexpr int kQuadThreads = kQuadRuns + 64;           // + 64 ring cells
constexpr int kQuadExtra = kFusedLoads - kQuadThreads; // plane loads taken by a second thread set
static_assert(kQuadExtra > 0 && kQuadExtra <= kQuadThreads, "two float4 plane loads per thread at most");

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit_group() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_group2() { asm volatile("cp.async.wait_group 2;\n" ::: "memory"); }

// Update functor interface: upd(old, nb[6] (x+, x-, y+, y-, z+, z-), source,
// sweep index (0 here), neighbours-never-updated, own-never-updated).  first:
// this is the first sweep of the level in the cycle (values never updated
// yet take the functor's warm-start factor); zero: the level's values are
// taken as 0 (nothing is loaded).  MINB: resident CTAs per SM the register
// allocation is sized for.
template <class Upd, int MINB>
__global__ void __launch_bounds__(kQuadThreads, MINB) k_rb_fused4(const float* __restrict__ uin,
                                                                 float* __restrict__ uout, Src f, int log2n,
                                                                 int chunk, int zero, int first, Upd upd) {
  constexpr int T = kFusedT, EC = kFusedEC, PL = kFusedPL, R = kFusedRing, RO = kFusedRingOld;
  extern __shared__ float4 fsm4[];
  float* Old = reinterpret_cast<float*>(fsm4);   // [RO][ER][EC]
  float* Red = Old + RO * PL;                    // [R][ER][EC]
  const uint32_t n = 1u << log2n, m = n - 1;
  const uint32_t tiles_z = n / T, tiles = (n / T) * tiles_z;
  const uint32_t item = blockIdx.x;
  {   // the box of a batched launch
    const int64_t off = (int64_t)blockIdx.z << (3 * log2n);
    uin += off;
    uout += off;
    f = box_src(f, (int64_t)1 << (3 * log2n));
    upd = upd.box(blockIdx.z);
  }
  const uint32_t tile = item % tiles, xc = item / tiles;
  const uint32_t y0 = (tile / tiles_z) * T, z0 = (tile % tiles_z) * T;
  const int x0 = (int)(xc * chunk), x1 = x0 + chunk;
  const float mean = f.mean ? (float)*f.mean : 0.0f;
  const int tid = threadIdx.x;
  const int sh2 = 2 * log2n;
  // offsets inside one box are below 2^30 (n <= 1024): 32-bit arithmetic
  auto plane = [&](int t) -> uint32_t { return ((uint32_t)t & m) << sh2; };

  // plane loads: float4 number tid, and tid + kQuadExtra for the last
  // kQuadExtra threads (rows y0-2 .. y0+33, columns z0-4 .. z0+35)
  const bool two = tid >= kQuadThreads - kQuadExtra;
  auto goff = [&](int idx) -> uint32_t {
    const int lr = idx / (EC / 4), lc4 = idx - lr * (EC / 4);
    return (((y0 - 2 + lr) & m) << log2n) | ((z0 - 4 + 4 * lc4) & m);
  };
  auto soff = [&](int idx) -> int {
    const int lr = idx / (EC / 4), lc4 = idx - lr * (EC / 4);
    return lr * EC + 4 * lc4;
  };
  const uint32_t g1 = goff(tid), g2 = two ? goff(tid + kQuadExtra) : 0u;
  const int s1 = soff(tid), s2 = two ? soff(tid + kQuadExtra) : 0;
  auto issue = [&](int t) {   // asynchronous copy of old plane t into its ring slot
    const uint32_t pt = plane(t);
    float* sp = Old + (t & (RO - 1)) * PL;
    cp_async16(sp + s1, uin + (pt | g1));
    if (two) cp_async16(sp + s2, uin + (pt | g2));
  };

  if (zero) {
    for (int i = tid; i < RO * PL; i += kQuadThreads) Old[i] = 0.0f;
  } else {
    for (int t = x0 - 2; t <= x0 + 1; ++t) {
      if (t <= x1 + 1) issue(t);
      cp_async_commit_group();
    }
  }

  // run owners: row qy, first column qz (local); ring workers: task h
  const bool run = tid < kQuadRuns;
  const int lane = tid & 31, warp = tid >> 5;
  const int qy = (warp >> 1) * 8 + 2 * (lane >> 3) + (warp & 1), qz = 4 * (lane & 7);
  const int qs = (qy + 2) * EC + qz + 4;                        // stored position of the run
  const uint32_t ro = (((y0 + qy) & m) << log2n) | (z0 + qz);   // its offset inside a plane
  const int h = tid - kQuadRuns;
  // the red ring cell (local y, z) of worker h on plane t
  auto ring_cell = [&](int t, int& y, int& z) {
    if (h < 32) {                              // rows y0 - 1 and y0 + 32
      y = h < 16 ? -1 : T;
      z = 2 * (h & 15) + ((t + y0 + y) & 1);
    } else {                                   // columns z0 - 1 and z0 + 32
      z = h < 48 ? -1 : T;
      y = 2 * (h & 15) + ((t + y0 + z0 + z) & 1);
    }
  };
  // sources of plane t: a run's four cells, a ring worker's red cell
  auto fetch_f = [&](int t) -> float4 {
    if (run) return __ldg(reinterpret_cast<const float4*>(f.p + (plane(t) | ro)));
    int y, z;
    ring_cell(t, y, z);
    return make_float4(__ldg(f.p + (plane(t) | (((y0 + y) & m) << log2n) | ((z0 + z) & m))), 0.0f, 0.0f, 0.0f);
  };
  auto src = [&](float v) { return f.s * (v - mean); };
  const bool own_old = first != 0;
  auto upd_red = [&](float old, const float nb[6], float fv) -> float {
    return upd(old, nb, fv, 0, own_old, own_old);   // red neighbours are old values too
  };
  auto upd_black = [&](float old, const float nb[6], float fv) -> float {
    return upd(old, nb, fv, 0, false, own_old);     // black neighbours are new red values
  };

  // black cells of plane p on the run, from the new red values of planes
  // p - 1 .. p + 1; fb: the raw sources of the two black cells
  auto black = [&](int p, float2 fb) {
    if (!(run && p >= x0 && p < x1)) return;
    const float* Rp = Red + (p & (R - 1)) * PL + qs;
    const float4 A = *reinterpret_cast<const float4*>(Red + ((p + 1) & (R - 1)) * PL + qs);
    const float4 B = *reinterpret_cast<const float4*>(Red + ((p - 1) & (R - 1)) * PL + qs);
    const float4 C = *reinterpret_cast<const float4*>(Rp + EC);
    const float4 D = *reinterpret_cast<const float4*>(Rp - EC);
    const float4 E = *reinterpret_cast<const float4*>(Rp);
    const float4 O = *reinterpret_cast<const float4*>(Old + (p & (RO - 1)) * PL + qs);
    float4 out;
    if (((p + y0 + qy) & 1) == 0) {            // black cells z + 1, z + 3
      const float nb1[6] = {A.y, B.y, C.y, D.y, E.z, E.x};
      const float nb3[6] = {A.w, B.w, C.w, D.w, Rp[4], E.z};
      out = make_float4(E.x, upd_black(O.y, nb1, src(fb.x)), E.z,
                        upd_black(O.w, nb3, src(fb.y)));
    } else {                                   // black cells z, z + 2
      const float nb0[6] = {A.x, B.x, C.x, D.x, E.y, Rp[-1]};
      const float nb2[6] = {A.z, B.z, C.z, D.z, E.w, E.y};
      out = make_float4(upd_black(O.x, nb0, src(fb.x)), E.y,
                        upd_black(O.z, nb2, src(fb.y)), E.w);
    }
    *reinterpret_cast<float4*>(uout + (plane(p) | ro)) = out;
  };
  // red cells of plane t (run or ring cell) from the old values of planes
  // t - 1 .. t + 1; fb receives the raw sources of the run's black cells
  auto red = [&](int t, float4 F, float2& fb) {
    if (t > x1) return;
    const float* Om = Old + ((t - 1) & (RO - 1)) * PL;
    const float* O0 = Old + (t & (RO - 1)) * PL;
    const float* Oq = Old + ((t + 1) & (RO - 1)) * PL;
    float* Rt = Red + (t & (R - 1)) * PL;
    if (run) {
      const float4 A = *reinterpret_cast<const float4*>(Oq + qs);
      const float4 B = *reinterpret_cast<const float4*>(Om + qs);
      const float4 C = *reinterpret_cast<const float4*>(O0 + qs + EC);
      const float4 D = *reinterpret_cast<const float4*>(O0 + qs - EC);
      const float4 E = *reinterpret_cast<const float4*>(O0 + qs);
      float4 out;
      if (((t + y0 + qy) & 1) == 0) {          // red cells z, z + 2
        const float nb0[6] = {A.x, B.x, C.x, D.x, E.y, O0[qs - 1]};
        const float nb2[6] = {A.z, B.z, C.z, D.z, E.w, E.y};
        out = make_float4(upd_red(E.x, nb0, src(F.x)), E.y,
                          upd_red(E.z, nb2, src(F.z)), E.w);
        fb = make_float2(F.y, F.w);
      } else {                                 // red cells z + 1, z + 3
        const float nb1[6] = {A.y, B.y, C.y, D.y, E.z, E.x};
        const float nb3[6] = {A.w, B.w, C.w, D.w, O0[qs + 4], E.z};
        out = make_float4(E.x, upd_red(E.y, nb1, src(F.y)), E.z,
                          upd_red(E.w, nb3, src(F.w)));
        fb = make_float2(F.x, F.z);
      }
      *reinterpret_cast<float4*>(Rt + qs) = out;
    } else {
      int y, z;
      ring_cell(t, y, z);
      const int q = (y + 2) * EC + z + 4;
      const float nb[6] = {Oq[q], Om[q], O0[q + EC], O0[q - EC], O0[q + 1], O0[q - 1]};
      Rt[q] = upd_red(O0[q], nb, src(F.x));
    }
  };
  // One plane step t: the old plane t + 3 is put in flight, plane t + 1 has
  // landed (at most the two newest copy groups pending), a barrier, then the
  // black cells of plane t - 2 (their red neighbours on planes t - 3 .. t - 1
  // were computed in earlier steps) and the red cells of plane t.
  auto step = [&](int t, float4& Fa, float2& fb) {
    if (!zero) {
      if (t + 3 <= x1 + 1) issue(t + 3);
      cp_async_commit_group();
      cp_async_wait_group2();
    }
    const float4 F_t = Fa;
    if (t + 2 <= x1) Fa = fetch_f(t + 2);
    __syncthreads();
    black(t - 2, fb);   // fb holds plane t - 2's black sources: read before red() replaces it
    red(t, F_t, fb);
  };
  float4 F0 = fetch_f(x0 - 1), F1 = fetch_f(x0);
  float2 fb0 = make_float2(0.0f, 0.0f), fb1 = fb0;
  for (int t = x0 - 1; t <= x1 + 1; t += 2) {
    step(t, F0, fb0);
    if (t + 1 <= x1 + 1) step(t + 1, F1, fb1);
  }
}

}  // namespace pmgb
