// Cell keys, stable LSD radix sort, cell start offsets and the particle
// permutation: the cell ordering that replaces PySCo's periodic Morton
// reordering (§3.2, Appendix E) and that the deterministic TSC gather needs.
//
// The radix sort is stable by construction: each tile ranks its keys with
// warp-level __match_any_sync in (warp, round, lane) order, which is the input
// order, so ties keep their input order and the permutation is bit-exact.
#include "pm_internal.cuh"

namespace pmgb {

namespace {

constexpr int RT = 256;             // threads per radix block
constexpr int RI = 16;              // keys per thread
constexpr int RTILE = RT * RI;      // keys per tile
constexpr int RWARPS = RT / 32;
constexpr int RMAXBINS = 512;       // at most 9 bits per digit

constexpr int SCAN_T = 1024;
constexpr int SCAN_CHUNK = 4 * SCAN_T;

// key = (i n + j) n + k of the cell holding each particle; with np_box > 0
// (a batch of boxes) prefixed by the box, i / np_box.
template <bool BOX>
__global__ void k_cell_keys(const uint32_t* __restrict__ X, int64_t np, int log2n, int64_t np_box,
                            uint32_t* __restrict__ keys) {
  const int sh = 32 - log2n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t ix = __ldg(X + i) >> sh;
    uint32_t iy = __ldg(X + np + i) >> sh;
    uint32_t iz = __ldg(X + 2 * np + i) >> sh;
    uint32_t key = (((ix << log2n) | iy) << log2n) | iz;
    if (BOX) key |= (uint32_t)(i / np_box) << (3 * log2n);
    keys[i] = key;
  }
}

// Per-tile digit histogram, written digit-major: counts[d * ntiles + tile].
// Each thread counts RI consecutive keys and adds runs of equal digits with
// one shared atomic (cell-ordered input has long runs in the high digits).
__global__ void __launch_bounds__(RT) k_radix_up(const uint32_t* __restrict__ keys, int64_t np,
                                                 int shift, int rbits,
                                                 uint32_t* __restrict__ counts, int64_t ntiles) {
  __shared__ uint32_t hist[RMAXBINS];
  const int R = 1 << rbits;
  for (int d = threadIdx.x; d < R; d += RT) hist[d] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * RTILE + (int64_t)threadIdx.x * RI;
  uint32_t k[RI];
  if (base + RI <= np) {
    const uint4* v = reinterpret_cast<const uint4*>(keys + base);
#pragma unroll
    for (int q = 0; q < RI / 4; ++q) {
      const uint4 t = __ldg(v + q);
      k[4 * q] = t.x; k[4 * q + 1] = t.y; k[4 * q + 2] = t.z; k[4 * q + 3] = t.w;
    }
  } else {
#pragma unroll
    for (int r = 0; r < RI; ++r) k[r] = base + r < np ? __ldg(keys + base + r) : 0xffffffffu;
  }
  uint32_t cur = 0xffffffffu, run = 0;
#pragma unroll
  for (int r = 0; r < RI; ++r) {
    if (base + r >= np) break;
    const uint32_t d = (k[r] >> shift) & (R - 1);
    if (d != cur) {
      if (run) atomicAdd(&hist[cur], run);
      cur = d;
      run = 0;
    }
    ++run;
  }
  if (run) atomicAdd(&hist[cur], run);
  __syncthreads();
  for (int d = threadIdx.x; d < R; d += RT) counts[(int64_t)d * ntiles + blockIdx.x] = hist[d];
}

// ---- exclusive scan of a uint32 array (three kernels) ----
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* warp_tot,
                                                         uint32_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int nw = blockDim.x >> 5;
    uint32_t t = lane < nw ? warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < nw) warp_tot[lane] = t;
    if (lane == nw - 1) *total = t;
  }
  __syncthreads();
  uint32_t before = warp ? warp_tot[warp - 1] : 0;
  uint32_t r = before + x - v;
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_reduce(const uint32_t* __restrict__ a, int64_t len,
                                                        uint32_t* __restrict__ sums) {
  __shared__ uint32_t wt[32];
  __shared__ uint32_t tot;
  const int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK + (int64_t)threadIdx.x * 4;
  uint32_t v = 0;
  for (int k = 0; k < 4; ++k)
    if (base + k < len) v += a[base + k];
  block_exclusive_scan(v, wt, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_sums(uint32_t* __restrict__ sums, int64_t nsums) {
  __shared__ uint32_t wt[32];
  __shared__ uint32_t tot;
  uint32_t carry = 0;
  for (int64_t base = 0; base < nsums; base += SCAN_T) {
    int64_t i = base + threadIdx.x;
    uint32_t v = i < nsums ? sums[i] : 0;
    uint32_t e = block_exclusive_scan(v, wt, &tot);
    if (i < nsums) sums[i] = carry + e;
    carry += tot;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(SCAN_T) k_scan_apply(uint32_t* __restrict__ a, int64_t len,
                                                       const uint32_t* __restrict__ sums) {
  __shared__ uint32_t wt[32];
  __shared__ uint32_t tot;
  const int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK + (int64_t)threadIdx.x * 4;
  uint32_t v[4], s = 0;
  for (int k = 0; k < 4; ++k) {
    v[k] = base + k < len ? a[base + k] : 0;
    s += v[k];
  }
  uint32_t e = block_exclusive_scan(s, wt, &tot) + sums[blockIdx.x];
  for (int k = 0; k < 4; ++k) {
    if (base + k < len) a[base + k] = e;
    e += v[k];
  }
}

// Stable scatter of one digit pass.  offsets[d * ntiles + tile] is the global
// rank of the first key of digit d in this tile.
__global__ void __launch_bounds__(RT) k_radix_down(const uint32_t* __restrict__ keys_in,
                                                   const uint32_t* __restrict__ vals_in,
                                                   int64_t np, int shift, int rbits,
                                                   const uint32_t* __restrict__ offsets,
                                                   int64_t ntiles,
                                                   uint32_t* __restrict__ keys_out,
                                                   uint32_t* __restrict__ vals_out) {
  extern __shared__ uint32_t smem[];
  uint32_t* whist = smem;                          // [RWARPS][RMAXBINS]
  uint32_t* tprefix = whist + RWARPS * RMAXBINS;   // [RMAXBINS]
  uint32_t* goff = tprefix + RMAXBINS;             // [RMAXBINS]
  uint32_t* skeys = goff + RMAXBINS;               // [RTILE]
  uint32_t* svals = skeys + RTILE;                 // [RTILE]
  __shared__ uint32_t wt[32];
  __shared__ uint32_t tot;

  const int R = 1 << rbits;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < RWARPS * RMAXBINS; i += RT) whist[i] = 0;
  __syncthreads();

  const int64_t base = (int64_t)blockIdx.x * RTILE;
  const int64_t wbase = base + (int64_t)warp * (RI * 32);
  const uint32_t lt = (1u << lane) - 1u;
  uint32_t k[RI], v[RI], rk[RI];
  // issue every load of the tile before the ranking rounds
#pragma unroll
  for (int r = 0; r < RI; ++r) {
    const int64_t i = wbase + r * 32 + lane;
    k[r] = i < np ? __ldg(keys_in + i) : 0u;
  }
#pragma unroll
  for (int r = 0; r < RI; ++r) {
    const int64_t i = wbase + r * 32 + lane;
    v[r] = i < np ? (vals_in ? __ldg(vals_in + i) : (uint32_t)i) : 0u;
  }
#pragma unroll
  for (int r = 0; r < RI; ++r) {
    int64_t i = wbase + r * 32 + lane;
    bool valid = i < np;
    uint32_t key = k[r];
    uint32_t d = valid ? ((key >> shift) & (R - 1)) : (uint32_t)R;
    uint32_t peers = __match_any_sync(0xffffffffu, d);
    int leader = __ffs(peers) - 1;
    uint32_t b = (valid && lane == leader) ? whist[warp * RMAXBINS + d] : 0u;
    b = __shfl_sync(0xffffffffu, b, leader);
    __syncwarp();
    if (valid && lane == leader) whist[warp * RMAXBINS + d] = b + __popc(peers);
    __syncwarp();
    rk[r] = valid ? b + __popc(peers & lt) : 0xffffffffu;
  }
  __syncthreads();
  for (int d = tid; d < RMAXBINS; d += RT) {
    uint32_t run = 0;
    if (d < R) {
      for (int w = 0; w < RWARPS; ++w) {
        uint32_t t = whist[w * RMAXBINS + d];
        whist[w * RMAXBINS + d] = run;
        run += t;
      }
      goff[d] = offsets[(int64_t)d * ntiles + blockIdx.x];
    }
    tprefix[d] = run;
  }
  __syncthreads();
  // exclusive scan of tprefix[0..511], two digits per thread
  {
    uint32_t a0 = tprefix[2 * tid], a1 = tprefix[2 * tid + 1];
    uint32_t e = block_exclusive_scan(a0 + a1, wt, &tot);
    tprefix[2 * tid] = e;
    tprefix[2 * tid + 1] = e + a0;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < RI; ++r) {
    if (rk[r] != 0xffffffffu) {
      uint32_t d = (k[r] >> shift) & (R - 1);
      uint32_t lp = tprefix[d] + whist[warp * RMAXBINS + d] + rk[r];
      skeys[lp] = k[r];
      svals[lp] = v[r];
    }
  }
  __syncthreads();
  const int64_t rem = np - base;
  const int tile_n = rem < RTILE ? (int)rem : RTILE;
  for (int i = tid; i < tile_n; i += RT) {
    uint32_t key = skeys[i];
    uint32_t d = (key >> shift) & (R - 1);
    uint32_t pos = goff[d] + (uint32_t)(i - (int)tprefix[d]);
    keys_out[pos] = key;
    vals_out[pos] = svals[i];
  }
}

constexpr size_t kDownSmem = sizeof(uint32_t) * (RWARPS * RMAXBINS + 2 * RMAXBINS + 2 * RTILE);

// cellstart[c] = first rank whose key is >= c; cellstart[ncells] = np.
__global__ void k_cellstart(const uint32_t* __restrict__ skeys, int64_t np, uint32_t ncells,
                            uint32_t* __restrict__ cellstart) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= np;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t lo = i == 0 ? 0u : skeys[i - 1] + 1u;
    uint32_t hi = i == np ? ncells : skeys[i];
    for (uint32_t c = lo; c <= hi && c <= ncells; ++c) cellstart[c] = (uint32_t)i;
  }
}

__global__ void k_permute(const uint32_t* __restrict__ perm, int64_t np,
                          const uint32_t* __restrict__ X, const float* __restrict__ V,
                          const uint32_t* __restrict__ id, uint32_t* __restrict__ Xs,
                          float* __restrict__ Vs, uint32_t* __restrict__ ids) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < np;
       j += (int64_t)gridDim.x * blockDim.x) {
    uint32_t p = __ldg(perm + j);
#pragma unroll
    for (int d = 0; d < 3; ++d) Xs[d * np + j] = __ldg(X + d * np + p);
    if (V) {
#pragma unroll
      for (int d = 0; d < 3; ++d) Vs[d * np + j] = __ldg(V + d * np + p);
    }
    if (id) ids[j] = __ldg(id + p);
  }
}

pm_status scan_u32(uint32_t* a, int64_t len, uint32_t* sums, cudaStream_t s) {
  int64_t nb = (len + SCAN_CHUNK - 1) / SCAN_CHUNK;
  if (nb == 0) return PM_OK;
  PM_LAUNCH(K_SORT_SCAN, 4.0 * len, k_scan_reduce, (unsigned)nb, SCAN_T, 0, s, a, len, sums);
  PM_LAUNCH(K_SORT_SCAN, 8.0 * nb, k_scan_sums, 1, SCAN_T, 0, s, sums, nb);
  PM_LAUNCH(K_SORT_SCAN, 8.0 * len, k_scan_apply, (unsigned)nb, SCAN_T, 0, s, a, len, sums);
  return PM_OK;
}

}  // namespace

int64_t radix_tiles(int64_t np) { return (np + RTILE - 1) / RTILE; }

int64_t radix_scan_blocks(int64_t np) {
  return (radix_tiles(np) * RMAXBINS + SCAN_CHUNK - 1) / SCAN_CHUNK + 1;
}

pm_status sort_particles(const uint32_t* X, int64_t np, int n, Workspace& w, cudaStream_t s,
                         uint32_t** perm_out, uint32_t** skeys_out, const Batch& bt) {
  static bool attr_done = false;
  if (!attr_done) {
    PM_TRY(cuda_status(cudaFuncSetAttribute(k_radix_down, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)kDownSmem)));
    attr_done = true;
  }
  const int log2n = ilog2(n);
  *perm_out = w.vals_a;
  *skeys_out = w.keys_a;
  if (np == 0) return PM_OK;
  const int64_t np_box = bt.B > 1 ? bt.np_box : 0;
  if (np_box > 0)
    PM_LAUNCH(K_KEYS, 16.0 * np, k_cell_keys<true>, grid_for(np, 256), 256, 0, s, X, np, log2n, np_box, w.keys_a);
  else
    PM_LAUNCH(K_KEYS, 16.0 * np, k_cell_keys<false>, grid_for(np, 256), 256, 0, s, X, np, log2n, np_box, w.keys_a);
  const int keybits = 3 * log2n + (bt.B > 1 ? ilog2(2 * bt.B - 1) : 0);   // + ceil(log2 B) box bits
  const int passes = (keybits + 8) / 9;
  const int bpp = (keybits + passes - 1) / passes;
  const int64_t ntiles = radix_tiles(np);
  uint32_t *kin = w.keys_a, *vin = nullptr;
  for (int p = 0; p < passes; ++p) {
    const int shift = p * bpp;
    const int rb = (keybits - shift) < bpp ? (keybits - shift) : bpp;
    const int64_t len = ((int64_t)1 << rb) * ntiles;
    uint32_t* kout = (kin == w.keys_a) ? w.keys_b : w.keys_a;
    uint32_t* vout = (vin == w.vals_b) ? w.vals_a : w.vals_b;
    PM_LAUNCH(K_SORT_UP, 4.0 * np, k_radix_up, (unsigned)ntiles, RT, 0, s, kin, np, shift, rb, w.counts, ntiles);
    PM_TRY(scan_u32(w.counts, len, w.scan_blocks, s));
    PM_LAUNCH(K_SORT_DOWN, (vin ? 16.0 : 12.0) * np, k_radix_down, (unsigned)ntiles, RT, kDownSmem, s, kin, vin, np, shift, rb,
              w.counts, ntiles, kout, vout);
    kin = kout;
    vin = vout;
  }
  *perm_out = vin;
  *skeys_out = kin;
  return launch_status();
}

pm_status build_cellstart(const uint32_t* skeys, int64_t np, int n, uint32_t* cellstart,
                          cudaStream_t s, int batch) {
  const uint32_t ncells = (uint32_t)((int64_t)n * n * n * batch);
  PM_LAUNCH(K_CELLSTART, 4.0 * np + 4.0 * (ncells + 1.0), k_cellstart, grid_for(np + 1, 256), 256, 0, s, skeys, np, ncells, cellstart);
  return launch_status();
}

pm_status permute_particles(const uint32_t* perm, int64_t np, const uint32_t* X, const float* V,
                            const uint32_t* id, uint32_t* Xs, float* Vs, uint32_t* ids,
                            cudaStream_t s) {
  if (np == 0) return PM_OK;
  PM_LAUNCH(K_PERMUTE, (28.0 + (V ? 24.0 : 0.0) + (id ? 8.0 : 0.0)) * np, k_permute, grid_for(np, 256), 256, 0, s, perm, np, X, V, id, Xs, Vs, ids);
  return launch_status();
}

}  // namespace pmgb
