// TSC mass assignment (§3.4) as a deterministic gather over cell-sorted
// particles, and fixed-order float64 grid reductions.
//
// The "moments" of a source cell are the 27 sums m[o] = sum_p W_x W_y W_z of
// its particles' TSC weight products, one per neighbour o = -1..1 per axis:
// what the cell sends to each of its 27 destination cells.  Every kernel here
// forms them in a fixed order and every destination cell adds the ones that
// point at it in a fixed order: no atomics, the density is bitwise
// reproducible.
//
// n >= 32: the streaming kernel k_deposit_stream walks the x planes of a
// column of cells (cells of up to kWalkRun particles weighed there, larger
// ones summed beforehand by k_group_moments, k_medium_moments and
// k_crowded_moments into the moment buffer).  n < 32: k_deposit<T>, one CTA
// per T^3 tile: one thread per source cell of the tile plus a one-cell halo
// walks the cell's particles into moments in shared memory, then every
// destination cell sums its 27.
#include "pm_device.cuh"
#include "pm_internal.cuh"

namespace pmgb {

namespace {

template <int T>
__global__ void __launch_bounds__(T * T * T) k_deposit(const uint32_t* __restrict__ Xs, int64_t np,
                                                       const uint32_t* __restrict__ cellstart, int n,
                                                       int log2n, const float* __restrict__ vals, float scale,
                                                       float* __restrict__ rho, double* __restrict__ partial) {
  constexpr int E = T + 2, S = E * E * E, NT = T * T * T;
  extern __shared__ float M[];  // [27][S]
  __shared__ double wsum[NT / 32];
  const int tiles = n / T;
  const int b = blockIdx.x;
  const int bz = b % tiles, by = (b / tiles) % tiles, bx = b / (tiles * tiles);
  const int tid = threadIdx.x;
  const int mask = n - 1;

  for (int s = tid; s < S; s += NT) {
    const int sx = s / (E * E), sy = (s / E) % E, sz = s % E;
    const uint32_t cx = (bx * T + sx - 1) & mask, cy = (by * T + sy - 1) & mask,
                   cz = (bz * T + sz - 1) & mask;
    const uint32_t c = (((cx << log2n) | cy) << log2n) | cz;
    const uint32_t beg = __ldg(cellstart + c), end = __ldg(cellstart + c + 1);
    float m[27];
#pragma unroll
    for (int o = 0; o < 27; ++o) m[o] = 0.0f;
    for (uint32_t p = beg; p < end; ++p) {
      float wx[3], wy[3], wz[3];
      tsc_weights(cell_offset(__ldg(Xs + p), log2n), wx);
      tsc_weights(cell_offset(__ldg(Xs + np + p), log2n), wy);
      tsc_weights(cell_offset(__ldg(Xs + 2 * np + p), log2n), wz);
      if (vals) {
        const float v = __ldg(vals + p);
        wx[0] *= v; wx[1] *= v; wx[2] *= v;
      }
#pragma unroll
      for (int ox = 0; ox < 3; ++ox)
#pragma unroll
        for (int oy = 0; oy < 3; ++oy) {
          const float wxy = wx[ox] * wy[oy];
#pragma unroll
          for (int oz = 0; oz < 3; ++oz) m[(ox * 3 + oy) * 3 + oz] = fmaf(wxy, wz[oz], m[(ox * 3 + oy) * 3 + oz]);
        }
    }
#pragma unroll
    for (int o = 0; o < 27; ++o) M[o * S + s] = m[o];
  }
  __syncthreads();

  const int tz = tid % T, ty = (tid / T) % T, tx = tid / (T * T);
  float acc = 0.0f;
#pragma unroll
  for (int ox = 0; ox < 3; ++ox)
#pragma unroll
    for (int oy = 0; oy < 3; ++oy)
#pragma unroll
      for (int oz = 0; oz < 3; ++oz)
        acc += M[((ox * 3 + oy) * 3 + oz) * S + ((tx + 2 - ox) * E + (ty + 2 - oy)) * E + (tz + 2 - oz)];
  const float r = acc * scale;
  const int64_t cell = (((int64_t)(bx * T + tx) << log2n | (by * T + ty)) << log2n) | (bz * T + tz);
  rho[cell] = r;

  double ws = warp_sum_comp(r);
  if ((tid & 31) == 0) wsum[tid >> 5] = ws;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < NT / 32; ++w) t += wsum[w];
    partial[b] = t;
  }
}

// Streaming variant for n >= 32: a CTA owns a DTY x DTZ column of
// destination cells and a chunk of x planes; it walks the source planes in
// order.  A source thread owns one (y, z) column of source cells (the column
// plus a one-cell halo in y and z: one per thread) for the whole chunk and
// keeps in registers the partial sums its column sends to the three
// destination planes a source plane reaches (9 (y, z) offsets each): the
// particles of source plane x add their TSC weight products to destination
// planes x - 1, x and x + 1, after which plane x - 1 has everything from this
// column and its 9 sums go to shared memory.  Destination warps (two cells
// per thread, rows ty and ty + DTY / 2) add, in a fixed order, the 9 column
// sums that point at each of their cells and write the density.  The sums
// are double-buffered: sources emit plane x - 1 while the destinations add
// plane x - 2 (one barrier per plane), on different warps.
//
// Particle loads: a source thread copies the first KP particles of its cell
// on the next plane into its own shared-memory slots with asynchronous copies
// (cp.async, 4 bytes each) while it weighs the particles of this plane, so a
// cell with up to KP particles is weighed without waiting on global memory;
// particles beyond KP are loaded in the walk, the next one while the current
// one is weighed.  The slots of a thread are written and read by that thread
// only, so they need no barrier.  The cell starts of plane x + 2 are loaded
// while plane x is processed.  The particles of a cell are weighed in the
// same order (ascending index) either way.
//
// Cells of more than kWalkRun particles are not walked here: eight or sixteen
// lanes, a warp or a block per cell summed their moments beforehand
// (k_group_moments, k_medium_moments, k_crowded_moments), and the cell's
// thread adds the 27 sums, so a source thread weighs at most kWalkRun
// particles per plane.
constexpr int DTY = 16, DTZ = 16, DEY = DTY + 2, DEZ = DTZ + 2, DNT = DTY * DTZ;
constexpr int DPL = DEY * DEZ;                     // source cells of a plane (one per source thread)
constexpr int DSRC_T = (DPL + 31) / 32 * 32;       // source warps
constexpr int DDST_T = DNT / 2;                    // destination threads (two cells each)
constexpr int DTHREADS = DSRC_T + DDST_T;
static_assert(DDST_T % 32 == 0 && DTY % 2 == 0, "whole destination warps, two rows per thread");
// Staged particles per cell and words per particle (x, y, z [, value]).
template <bool VALS> struct DepositStage {
  static constexpr int KP = kWalkRun, NC = VALS ? 4 : 3;
  static constexpr size_t smem = sizeof(float) * (2 * 9 * DPL + 2 * KP * NC * DPL);
};

__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gsrc) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

template <bool VALS>
__global__ void __launch_bounds__(DTHREADS, 2) k_deposit_stream(const uint32_t* __restrict__ Xs, int64_t np,
                                                                const uint32_t* __restrict__ cellstart, int log2n,
                                                                int chunk, int nitems, const float* __restrict__ vals,
                                                                float scale, float* __restrict__ rho,
                                                                double* __restrict__ partial,
                                                                const float* __restrict__ crowd) {
  using G = DepositStage<VALS>;
  constexpr int KP = G::KP, NC = G::NC, PL = DPL;
  extern __shared__ float sm[];
  {   // the box of a batched launch: its cell starts (global particle indices), density, partials
    const int64_t off = (int64_t)blockIdx.z << (3 * log2n);
    cellstart += off;
    rho += off;
    partial += (int64_t)blockIdx.z * nitems;
  }
  float* Col = sm;                                                 // [2][9][PL] column sums
  uint32_t* Slot = reinterpret_cast<uint32_t*>(sm + 2 * 9 * PL);   // [2][KP][NC][PL]
  __shared__ double wsum[DTHREADS / 32];
  const int n = 1 << log2n, mask = n - 1;
  const int tiles_z = n / DTZ, tiles = (n / DTY) * tiles_z;
  const int tid = threadIdx.x;
  const bool src = tid < PL, dst = tid >= DSRC_T;
  const int sly = tid / DEZ, slz = tid - sly * DEZ;            // source column of this thread (if src)
  const int dt = tid - DSRC_T;
  const int ty = dt / DTZ, tz = dt - ty * DTZ;                 // destination cells (ty, tz), (ty + DTY / 2, tz) (if dst)
  // copies the first KP particles [b, min(e, b + KP)) into slot buffer `buf`
  // (none for a cell whose moments are ready in `crowd`)
  auto stage = [&](int buf, uint32_t b, uint32_t e) {
    if (crowd && e - b > kWalkRun) return;
    uint32_t* s0 = Slot + buf * KP * NC * PL + tid;
#pragma unroll
    for (int k = 0; k < KP; ++k) {
      if (b + k < e) {
#pragma unroll
        for (int d = 0; d < 3; ++d) cp_async4(s0 + (k * NC + d) * PL, Xs + d * np + b + k);
        if (VALS) cp_async4(s0 + (k * NC + 3) * PL, vals + b + k);
      }
    }
  };
  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
    const int tile = item % tiles, xc = item / tiles;
    const int y0 = (tile / tiles_z) * DTY, z0 = (tile % tiles_z) * DTZ;
    const int x0 = xc * chunk, x1 = x0 + chunk;
    const uint32_t cy = (uint32_t)((y0 - 1 + sly) & mask), cz = (uint32_t)((z0 - 1 + slz) & mask);
    auto cell_of = [&](int x) -> uint32_t { return ((((uint32_t)(x & mask)) << log2n | cy) << log2n) | cz; };
    float wsum_s = 0.0f, wsum_c = 0.0f;
    // pipeline registers: cell starts of planes xs and xs + 1
    uint32_t b0 = 0, e0 = 0, b1 = 0, e1 = 0;
    if (src) {
      const uint32_t c0 = cell_of(x0 - 1), c1 = cell_of(x0);
      b0 = __ldg(cellstart + c0); e0 = __ldg(cellstart + c0 + 1);
      b1 = __ldg(cellstart + c1); e1 = __ldg(cellstart + c1 + 1);
      stage((x0 - 1) & 1, b0, e0);
      cp_async_commit();
    }
    // one plane step: source plane xs adds to the column sums of destination
    // planes xs - 1 (A), xs (B) and xs + 1 (C, started here), emits A; the
    // destinations add the column sums of plane xs - 2 emitted in the step
    // before.  The caller rotates the roles of the three register arrays.
    auto step = [&](int xs, float (&A)[9], float (&B)[9], float (&C)[9]) {
      float* ColW = Col + (xs & 1) * 9 * PL;
      const float* ColR = Col + ((xs - 1) & 1) * 9 * PL;
      uint32_t b2 = 0, e2 = 0;
      if (src && xs <= x1) {
        if (xs + 1 <= x1) stage((xs + 1) & 1, b1, e1);   // the next plane's particles, in flight
        cp_async_commit();
        if (xs + 2 <= x1) {
          const uint32_t c2 = cell_of(xs + 2);
          b2 = __ldg(cellstart + c2); e2 = __ldg(cellstart + c2 + 1);
        }
        cp_async_wait1();                                  // this plane's particles have arrived
#pragma unroll
        for (int o = 0; o < 9; ++o) C[o] = 0.0f;
        auto weigh = [&](uint32_t px, uint32_t py, uint32_t pz, float v) {
          float wx[3], wy[3], wz[3];
          tsc_weights(cell_offset(px, log2n), wx);
          tsc_weights(cell_offset(py, log2n), wy);
          tsc_weights(cell_offset(pz, log2n), wz);
          if (VALS) {
            wx[0] *= v; wx[1] *= v; wx[2] *= v;
          }
#pragma unroll
          for (int oy = 0; oy < 3; ++oy) {
            const float w0 = wx[0] * wy[oy], w1 = wx[1] * wy[oy], w2 = wx[2] * wy[oy];
#pragma unroll
            for (int oz = 0; oz < 3; ++oz) {
              A[oy * 3 + oz] = fmaf(w0, wz[oz], A[oy * 3 + oz]);
              B[oy * 3 + oz] = fmaf(w1, wz[oz], B[oy * 3 + oz]);
              C[oy * 3 + oz] = fmaf(w2, wz[oz], C[oy * 3 + oz]);
            }
          }
        };
        const uint32_t* s0 = Slot + (xs & 1) * KP * NC * PL + tid;
        const uint32_t cnt = e0 - b0;
        if (crowd && cnt > kWalkRun) {   // its moments were summed already
          const float* mo = crowd + kMomStride * (int64_t)b0;
#pragma unroll
          for (int o = 0; o < 9; ++o) {
            A[o] += __ldg(mo + o);
            B[o] += __ldg(mo + 9 + o);
            C[o] += __ldg(mo + 18 + o);
          }
        } else {
#pragma unroll
          for (int k = 0; k < KP; ++k)
            if ((uint32_t)k < cnt)
              weigh(s0[(k * NC) * PL], s0[(k * NC + 1) * PL], s0[(k * NC + 2) * PL],
                    VALS ? __uint_as_float(s0[(k * NC + 3) * PL]) : 1.0f);
          if (cnt > (uint32_t)KP) {   // the rest from global memory
            uint32_t p = b0 + KP;
            uint32_t px = __ldg(Xs + p), py = __ldg(Xs + np + p), pz = __ldg(Xs + 2 * np + p);
            for (; p < e0; ++p) {
              // the next particle of the cell is loaded while this one is weighed
              uint32_t qx = 0, qy = 0, qz = 0;
              if (p + 1 < e0) { qx = __ldg(Xs + p + 1); qy = __ldg(Xs + np + p + 1); qz = __ldg(Xs + 2 * np + p + 1); }
              weigh(px, py, pz, VALS ? __ldg(vals + p) : 1.0f);
              px = qx;
              py = qy;
              pz = qz;
            }
          }
        }
        // destination plane xs - 1 has all of this column's contributions
#pragma unroll
        for (int o = 0; o < 9; ++o) ColW[o * PL + tid] = A[o];
      }
      const int done = xs - 2;   // the destination plane whose column sums were emitted in the step before
      if (dst && done >= x0 && done < x1) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int ry = ty + h * (DTY / 2);
          float a = 0.0f;
#pragma unroll
          for (int oy = 0; oy < 3; ++oy)
#pragma unroll
            for (int oz = 0; oz < 3; ++oz) a += ColR[(oy * 3 + oz) * PL + (ry + 2 - oy) * DEZ + (tz + 2 - oz)];
          const float r = a * scale;
          rho[((((int64_t)done << log2n) | (y0 + ry)) << log2n) | (z0 + tz)] = r;
          kahan_add(wsum_s, wsum_c, r);
        }
      }
      __syncthreads();
      b0 = b1; e0 = e1; b1 = b2; e1 = e2;
    };
    // column sums of destination planes xs - 1 and xs (the first source plane
    // reaches planes x0 - 2 .. x0; the first two are outside the chunk)
    float R0[9], R1[9], R2[9];
#pragma unroll
    for (int o = 0; o < 9; ++o) {
      R0[o] = 0.0f;
      R1[o] = 0.0f;
    }
    for (int xs = x0 - 1; xs <= x1 + 1; xs += 3) {
      step(xs, R0, R1, R2);
      if (xs + 1 <= x1 + 1) step(xs + 1, R1, R2, R0);
      if (xs + 2 <= x1 + 1) step(xs + 2, R2, R0, R1);
    }
    const double ws = warp_sum_comp(wsum_s - wsum_c);
    if ((tid & 31) == 0) wsum[tid >> 5] = ws;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < DTHREADS / 32; ++w) t += wsum[w];
      partial[item] = t;
    }
    __syncthreads();
  }
}

// The 27 moments of one particle (TSC weight products), added into m.
template <bool VALS>
__device__ __forceinline__ void add_moments(const uint32_t* __restrict__ Xs, int64_t np, uint32_t p, int log2n,
                                            const float* __restrict__ vals, float m[27]) {
  float wx[3], wy[3], wz[3];
  tsc_weights(cell_offset(__ldg(Xs + p), log2n), wx);
  tsc_weights(cell_offset(__ldg(Xs + np + p), log2n), wy);
  tsc_weights(cell_offset(__ldg(Xs + 2 * np + p), log2n), wz);
  if (VALS) {
    const float v = __ldg(vals + p);
    wx[0] *= v; wx[1] *= v; wx[2] *= v;
  }
#pragma unroll
  for (int ox = 0; ox < 3; ++ox)
#pragma unroll
    for (int oy = 0; oy < 3; ++oy) {
      const float wxy = wx[ox] * wy[oy];
#pragma unroll
      for (int oz = 0; oz < 3; ++oz) m[(ox * 3 + oy) * 3 + oz] = fmaf(wxy, wz[oz], m[(ox * 3 + oy) * 3 + oz]);
    }
}

// The 27 moments of each cell of a list of cells holding at most 2G
// particles, G lanes per cell (32 / G cells per warp): the small cells
// (kWalkRun < particles <= kMedRun, the sort's smalls list) with G = 8 and the
// medium ones (kMedRun < particles <= kLongRun, its meds list) with G = 16.
// Lane g of a group weighs the cell's particles g and g + G, then the group
// adds the lanes' sums in a fixed shuffle tree.  The moments go to
// crowd[kMomStride a .. + 26] (a = the cell's first rank).
template <bool VALS, int G>
__global__ void __launch_bounds__(256) k_group_moments(const uint32_t* __restrict__ Xs, int64_t np,
                                                       const uint32_t* __restrict__ cellstart,
                                                       const uint32_t* __restrict__ list, int log2n,
                                                       const float* __restrict__ vals, float* __restrict__ crowd) {
  static_assert(G == 8 || G == 16, "group width");
  constexpr int PERW = 32 / G, NOUT = (27 + G - 1) / G;
  const uint32_t ncells = list[0];
  const uint32_t lane = threadIdx.x & 31, g = lane & (G - 1);
  const uint32_t groups = gridDim.x * 8 * PERW;
  // the groups of a warp take consecutive list entries; a warp with no entry
  // left stops as a whole (the shuffles below need every lane)
  for (uint32_t q0 = (blockIdx.x * 8 + (threadIdx.x >> 5)) * PERW; q0 < ncells; q0 += groups) {
    const uint32_t q = q0 + lane / G;
    uint32_t a = 0, b = 0;
    if (q < ncells) {
      const uint32_t c = list[1 + q];
      a = cellstart[c];
      b = cellstart[c + 1];
    }
    float m[27];
#pragma unroll
    for (int o = 0; o < 27; ++o) m[o] = 0.0f;
    if (a + g < b) add_moments<VALS>(Xs, np, a + g, log2n, vals, m);
    if (a + g + G < b) add_moments<VALS>(Xs, np, a + g + G, log2n, vals, m);
#pragma unroll
    for (int o = 0; o < 27; ++o) {
#pragma unroll
      for (int d = G / 2; d > 0; d >>= 1) m[o] += __shfl_down_sync(0xffffffffu, m[o], d, G);
    }
    // lane 0 of the group holds the sums; lane g writes moments g, g + G, ...
    float out[NOUT];
#pragma unroll
    for (int k = 0; k < NOUT; ++k) out[k] = 0.0f;
#pragma unroll
    for (int o = 0; o < 27; ++o) {
      const float v = __shfl_sync(0xffffffffu, m[o], 0, G);
      if (g == (uint32_t)(o % G)) out[o / G] = v;
    }
    if (q < ncells) {
#pragma unroll
      for (int k = 0; k < NOUT; ++k)
        if (g + G * k < 27) crowd[kMomStride * (int64_t)a + g + G * k] = out[k];
    }
  }
}

// The 27 moments of each crowded cell of at most kWarpRun particles (the
// cell sort's runs list, longer runs skipped), one warp per cell: lane i
// weighs the cell's particles i, i + 32, ... in that order, then the warp adds
// the lanes' sums in a fixed shuffle tree.  The moments go to
// crowd[kMomStride a .. + 26] (a = the cell's first rank).
template <bool VALS>
__global__ void __launch_bounds__(256) k_medium_moments(const uint32_t* __restrict__ Xs, int64_t np,
                                                        const uint32_t* __restrict__ cellstart,
                                                        const uint32_t* __restrict__ runs, int log2n,
                                                        const float* __restrict__ vals, float* __restrict__ crowd) {
  const uint32_t ntot = runs[0];
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t warps = gridDim.x * 8;
  for (uint32_t q = blockIdx.x * 8 + (threadIdx.x >> 5); q < ntot; q += warps) {
    const uint32_t c = runs[1 + q];
    const uint32_t a = cellstart[c], b = cellstart[c + 1];
    if (b - a > kWarpRun) continue;   // the same for the whole warp: a block's cell
    float m[27];
#pragma unroll
    for (int o = 0; o < 27; ++o) m[o] = 0.0f;
    for (uint32_t p = a + lane; p < b; p += 32) add_moments<VALS>(Xs, np, p, log2n, vals, m);
#pragma unroll
    for (int o = 0; o < 27; ++o) {
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) m[o] += __shfl_down_sync(0xffffffffu, m[o], d);
    }
    // lane 0 holds the sums; lanes 0..26 write one each
    float out = 0.0f;
#pragma unroll
    for (int o = 0; o < 27; ++o) {
      const float v = __shfl_sync(0xffffffffu, m[o], 0);
      if (lane == (uint32_t)o) out = v;
    }
    if (lane < 27) crowd[kMomStride * (int64_t)a + lane] = out;
  }
}

// The 27 moments of each crowded cell of more than kWarpRun particles (the
// cell sort's bigs list), one block per cell: thread t weighs particles
// a + t, a + t + CT, ... of the cell in that order, then the block adds the
// per-thread sums in a fixed tree (warp shuffles, then the warps in order), so
// the result does not depend on scheduling.  The moments go to
// crowd[kMomStride a .. + 26], as for medium cells.
constexpr int CT = 256;
template <bool VALS>
__global__ void __launch_bounds__(CT) k_crowded_moments(const uint32_t* __restrict__ Xs, int64_t np,
                                                        const uint32_t* __restrict__ cellstart,
                                                        const uint32_t* __restrict__ bigs, int log2n,
                                                        const float* __restrict__ vals, float* __restrict__ crowd) {
  __shared__ float part[CT / 32][27];
  const uint32_t nruns = bigs[0];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint32_t q = blockIdx.x; q < nruns; q += gridDim.x) {
    const uint32_t c = bigs[1 + q];
    const uint32_t a = cellstart[c], b = cellstart[c + 1];
    float m[27];
#pragma unroll
    for (int o = 0; o < 27; ++o) m[o] = 0.0f;
    for (uint32_t p = a + threadIdx.x; p < b; p += CT) add_moments<VALS>(Xs, np, p, log2n, vals, m);
#pragma unroll
    for (int o = 0; o < 27; ++o) {
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) m[o] += __shfl_down_sync(0xffffffffu, m[o], d);
      if (lane == 0) part[warp][o] = m[o];
    }
    __syncthreads();
    if (threadIdx.x < 27) {
      float t = 0.0f;
#pragma unroll
      for (int w = 0; w < CT / 32; ++w) t += part[w][threadIdx.x];
      crowd[kMomStride * (int64_t)a + threadIdx.x] = t;
    }
    __syncthreads();
  }
}

inline void deposit_stream_plan(int n, int* chunk, int* nitems) {
  const int tiles = (n / DTY) * (n / DTZ);
  int c = n;
  while (c > 16 && (int64_t)tiles * (n / c) < 8 * 152) c >>= 1;
  *chunk = c;
  *nitems = tiles * (n / c);
}

// Sum of a float32 array: per-block float64 partials (fixed order).
__global__ void __launch_bounds__(256) k_sum_partials(const float* __restrict__ f, int64_t count,
                                                      double* __restrict__ partial) {
  __shared__ double wsum[8];
  float v = 0.0f, c = 0.0f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    float y = __ldg(f + i) - c;   // Kahan
    float t = v + y;
    c = (t - v) - y;
    v = t;
  }
  double ws = warp_sum_comp(v - c);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = ws;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += wsum[w];
    partial[blockIdx.x] = t;
  }
}

// out[k] = scale * sum_i partial[k * stride + i], i < count, for k < nout
// (one block, fixed order: strided per-thread sums then a tree).
__global__ void __launch_bounds__(1024) k_reduce_partials(const double* __restrict__ partial,
                                                          int64_t count, int64_t stride, int nout,
                                                          double scale, double* __restrict__ out) {
  __shared__ double red[1024];
  for (int k = blockIdx.x; k < nout; k += gridDim.x) {   // one output per block (fixed order within it)
    double t = 0.0;
    for (int64_t i = threadIdx.x; i < count; i += blockDim.x) t += partial[k * stride + i];
    red[threadIdx.x] = t;
    __syncthreads();
    for (int o = 512; o > 0; o >>= 1) {
      if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[k] = red[0] * scale;
    __syncthreads();
  }
}

template <int T>
pm_status launch_deposit(const uint32_t* Xs, int64_t np, const uint32_t* cellstart, int n, const float* vals,
                         float scale, float* rho, double* partials, double* mean_out, cudaStream_t s) {
  constexpr int E = T + 2;
  constexpr size_t smem = sizeof(float) * 27 * E * E * E;
  PM_TRY(smem_attr(k_deposit<T>, smem));
  const int tiles = n / T;
  const int64_t nblocks = (int64_t)tiles * tiles * tiles;
  PM_LAUNCH(K_DEPOSIT, (vals ? 16.0 : 12.0) * np + 8.0 * n * n * (double)n + 4.0, k_deposit<T>, (unsigned)nblocks,
            T * T * T, smem, s, Xs, np, cellstart, n, ilog2(n), vals, scale, rho, partials);
  PM_LAUNCH(K_REDUCE, 8.0 * nblocks, k_reduce_partials, 1, 1024, 0, s, partials, nblocks, (int64_t)0, 1,
            1.0 / ((double)n * n * n), mean_out);
  return launch_status();
}

}  // namespace

int deposit_items(int n) {
  int chunk, nitems;
  deposit_stream_plan(n, &chunk, &nitems);
  return nitems;
}

int64_t reduce_partials_capacity(int n, int64_t np) {
  int64_t t = (int64_t)n / 4;
  int64_t c = t * t * t;               // deposit blocks with 4^3 tiles (upper bound)
  const int64_t b = np / 256 + 1;      // interpolation blocks (one float2 of maxima each)
  if (b > c) c = b;
  return c > 152 * 64 ? c : 152 * 64;
}

pm_status deposit_sorted(const uint32_t* Xs, int64_t np, const uint32_t* cellstart, int n,
                         float* rho, double* partials, double* mean_out, cudaStream_t s, const Crowded& cr) {
  const float scale = np > 0 ? (float)((double)n * n * n / (double)np) : 0.0f;
  return deposit_sorted_values(Xs, np, cellstart, n, nullptr, scale, rho, partials, mean_out, s, cr);
}

namespace {
// Moments of the crowded cells into cr.moments (a no-op launch when there are
// none); the caller's streaming deposit then reads them.
pm_status crowded_moments(const uint32_t* Xs, int64_t np, const uint32_t* cellstart, int n, const float* vals,
                          const Crowded& cr, cudaStream_t s) {
  if (!cr.runs || np == 0) return PM_OK;
  const int l2 = ilog2(n);
  if (vals) {
    PM_LAUNCH(K_DEPOSIT, 0.0, (k_group_moments<true, 8>), 8 * 152, 256, 0, s, Xs, np, cellstart, cr.smalls, l2, vals,
              cr.moments);
    PM_LAUNCH(K_DEPOSIT, 0.0, (k_group_moments<true, 16>), 8 * 152, 256, 0, s, Xs, np, cellstart, cr.meds, l2, vals,
              cr.moments);
    PM_LAUNCH(K_DEPOSIT, 0.0, k_medium_moments<true>, 8 * 152, 256, 0, s, Xs, np, cellstart, cr.runs, l2, vals,
              cr.moments);
    PM_LAUNCH(K_DEPOSIT, 0.0, k_crowded_moments<true>, 4 * 152, CT, 0, s, Xs, np, cellstart, cr.bigs, l2, vals,
              cr.moments);
  } else {
    PM_LAUNCH(K_DEPOSIT, 0.0, (k_group_moments<false, 8>), 8 * 152, 256, 0, s, Xs, np, cellstart, cr.smalls, l2,
              vals, cr.moments);
    PM_LAUNCH(K_DEPOSIT, 0.0, (k_group_moments<false, 16>), 8 * 152, 256, 0, s, Xs, np, cellstart, cr.meds, l2, vals,
              cr.moments);
    PM_LAUNCH(K_DEPOSIT, 0.0, k_medium_moments<false>, 8 * 152, 256, 0, s, Xs, np, cellstart, cr.runs, l2, vals,
              cr.moments);
    PM_LAUNCH(K_DEPOSIT, 0.0, k_crowded_moments<false>, 4 * 152, CT, 0, s, Xs, np, cellstart, cr.bigs, l2, vals,
              cr.moments);
  }
  return PM_OK;
}
}  // namespace

pm_status deposit_sorted_values(const uint32_t* Xs, int64_t np, const uint32_t* cellstart, int n, const float* vals,
                                float scale, float* rho, double* partials, double* mean_out, cudaStream_t s,
                                const Crowded& cr) {
  if (n >= 32) {
    PM_TRY(crowded_moments(Xs, np, cellstart, n, vals, cr, s));
    const float* crowd = cr.runs && np > 0 ? cr.moments : nullptr;
    int chunk, nitems;
    deposit_stream_plan(n, &chunk, &nitems);
    const unsigned grid = (unsigned)nitems;   // one item per CTA, two 512-thread CTAs per SM
    const double bytes = (vals ? 16.0 : 12.0) * np + 8.0 * n * n * (double)n + 4.0;
    if (vals) {
      PM_TRY(smem_attr(k_deposit_stream<true>, DepositStage<true>::smem));
      PM_LAUNCH(K_DEPOSIT, bytes, k_deposit_stream<true>, grid, DTHREADS, DepositStage<true>::smem, s, Xs, np,
                cellstart, ilog2(n), chunk, nitems, vals, scale, rho, partials, crowd);
    } else {
      PM_TRY(smem_attr(k_deposit_stream<false>, DepositStage<false>::smem));
      PM_LAUNCH(K_DEPOSIT, bytes, k_deposit_stream<false>, grid, DTHREADS, DepositStage<false>::smem, s, Xs, np,
                cellstart, ilog2(n), chunk, nitems, vals, scale, rho, partials, crowd);
    }
    PM_LAUNCH(K_REDUCE, 8.0 * nitems, k_reduce_partials, 1, 1024, 0, s, partials, (int64_t)nitems, (int64_t)0, 1,
              1.0 / ((double)n * n * n), mean_out);
    return launch_status();
  }
  if (n >= 8) return launch_deposit<8>(Xs, np, cellstart, n, vals, scale, rho, partials, mean_out, s);
  return launch_deposit<4>(Xs, np, cellstart, n, vals, scale, rho, partials, mean_out, s);
}

pm_status deposit_sorted_batch(const uint32_t* Xs, int64_t np_box, int B, const uint32_t* cellstart, int n,
                               float* rho, double* partials, double* mean_out, cudaStream_t s, const Crowded& cr) {
  if (n < 32 || B < 1) return PM_EINVAL;
  PM_TRY(crowded_moments(Xs, np_box * B, cellstart, n, nullptr, cr, s));
  PM_TRY(smem_attr(k_deposit_stream<false>, DepositStage<false>::smem));
  int chunk, nitems;
  deposit_stream_plan(n, &chunk, &nitems);
  const float scale = np_box > 0 ? (float)((double)n * n * n / (double)np_box) : 0.0f;
  // one item per CTA: B x nitems CTAs balance over the SMs (two resident each)
  const int gx = nitems;
  const int64_t np = np_box * B;
  PM_LAUNCH(K_DEPOSIT, 12.0 * np + 8.0 * n * n * (double)n * B + 4.0, k_deposit_stream<false>, dim3(gx, 1, B),
            DTHREADS, DepositStage<false>::smem, s, Xs, np, cellstart, ilog2(n), chunk, nitems, (const float*)nullptr, scale, rho,
            partials, cr.runs && np > 0 ? (const float*)cr.moments : nullptr);
  PM_LAUNCH(K_REDUCE, 8.0 * nitems * B, k_reduce_partials, B, 1024, 0, s, partials, (int64_t)nitems,
            (int64_t)nitems, B, 1.0 / ((double)n * n * n), mean_out);
  return launch_status();
}

pm_status grid_mean(const float* f, int64_t count, double* partials, double* mean_out,
                    cudaStream_t s) {
  const unsigned nb = grid_for(count, 256, 152 * 8);
  PM_LAUNCH(K_REDUCE, 4.0 * count, k_sum_partials, nb, 256, 0, s, f, count, partials);
  PM_LAUNCH(K_REDUCE, 8.0 * nb, k_reduce_partials, 1, 1024, 0, s, partials, (int64_t)nb, (int64_t)0, 1,
            1.0 / (double)count, mean_out);
  return launch_status();
}

pm_status reduce_partials(const double* partials, int64_t count, int64_t stride, int nout,
                          double scale, double* out, cudaStream_t s) {
  PM_LAUNCH(K_REDUCE, 8.0 * count * nout, k_reduce_partials, nout, 1024, 0, s, partials, count, stride, nout, scale,
            out);
  return launch_status();
}

}  // namespace pmgb
