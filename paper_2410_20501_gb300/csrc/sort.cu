// Cell keys, the stable counting sort by cell, cell start offsets and the
// particle permutation: the cell ordering that replaces PySCo's periodic
// Morton reordering (§3.2, Appendix E) and that the deterministic TSC gather
// needs.
//
// With about one particle per cell the cell index itself is the natural
// bucket: one pass counts the particles of each cell with atomics into the
// cell-start array, keeping each particle's rank among its cell's particles
// (the value its atomic returned); an in-place exclusive scan turns the counts
// into cell starts; one pass writes each particle to its cell's start plus its
// rank.  The atomics leave the order of equal keys to the hardware, so a last
// pass restores the stable order (ascending input index) inside every cell:
// one thread per cell for short runs, one warp per cell for medium and
// crowded runs up to kWarpRun particles, one block per cell (bitonic chunks
// in shared memory, then merges) for longer ones.  The permutation is therefore
// bit-exact and deterministic, equal to a stable sort by key.
//
// The step writes particles back in cell order, so the input of the next
// step is nearly sorted: the counts and scatters then touch neighbouring
// words and the per-cell runs are already in order.
#include "pm_internal.cuh"

namespace pmgb {

namespace {

constexpr int SCAN_T = 1024;
constexpr int SCAN_V = 16;                  // values per thread of the scan passes
constexpr int SCAN_CHUNK = SCAN_V * SCAN_T;
constexpr int KT = 256;             // threads of the key, scatter and order kernels
constexpr int CI = 4;               // particles per thread of the counting kernel
constexpr uint32_t SHORT_RUN = kLongRun;  // runs up to this length are ordered by one thread or warp
constexpr int WT = 256;             // threads of the warp-per-run kernel
constexpr int LT = 256;             // threads of a long-run block
constexpr int LCH = 4096;           // elements sorted in shared memory at once
constexpr int LONG_BLOCKS = 8 * 152;


// key = (i n + j) n + k of the cell holding each particle; with np_box > 0
// (a batch of boxes) prefixed by the box, i / np_box.  Counts the particles of
// each cell into cnt[key] (zeroed) and stores kr[i] = (key, rank of i among
// its cell's particles).  A thread takes CI particles, KT apart (coalesced),
// with their loads and atomics all in flight together; a run of equal keys
// in adjacent lanes takes one atomic (its head's) and ranks in lane order.
template <bool BOX>
__global__ void __launch_bounds__(KT) k_cell_count(const uint32_t* __restrict__ X, int64_t np, int log2n,
                                                   int64_t np_box, uint2* __restrict__ kr,
                                                   uint32_t* __restrict__ cnt) {
  const int64_t i0 = blockIdx.x * (int64_t)(KT * CI) + threadIdx.x;
  const int sh = 32 - log2n;
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t upto = (2u << lane) - 1u;       // lanes 0 .. lane
  uint32_t key[CI], r[CI], start[CI];
#pragma unroll
  for (int k = 0; k < CI; ++k) {
    const int64_t i = i0 + k * KT;
    key[k] = 0xffffffffu;
    if (i < np) {
      const uint32_t ix = __ldg(X + i) >> sh;
      const uint32_t iy = __ldg(X + np + i) >> sh;
      const uint32_t iz = __ldg(X + 2 * np + i) >> sh;
      key[k] = (((ix << log2n) | iy) << log2n) | iz;
      if (BOX) key[k] |= (uint32_t)(i / np_box) << (3 * log2n);
    }
  }
#pragma unroll
  for (int k = 0; k < CI; ++k) {
    const uint32_t prev = __shfl_up_sync(0xffffffffu, key[k], 1);
    const uint32_t heads = __ballot_sync(0xffffffffu, lane == 0 || key[k] != prev);
    start[k] = 31 - __clz(heads & upto);
    const uint32_t after = heads & ~upto;
    const uint32_t end = after ? (uint32_t)__ffs(after) - 1 : 32u;
    r[k] = 0;
    if (key[k] != 0xffffffffu && start[k] == lane) r[k] = atomicAdd(cnt + key[k], end - lane);
  }
#pragma unroll
  for (int k = 0; k < CI; ++k) {
    const uint32_t base = __shfl_sync(0xffffffffu, r[k], start[k]);
    const int64_t i = i0 + k * KT;
    if (i < np) kr[i] = make_uint2(key[k], base + lane - start[k]);
  }
}

// perm[cellstart[key] + rank] = i; a thread takes CI particles, KT apart, with
// their loads in flight together.
__global__ void __launch_bounds__(KT) k_cell_scatter(const uint2* __restrict__ kr, int64_t np,
                                                     const uint32_t* __restrict__ cellstart,
                                                     uint32_t* __restrict__ perm) {
  const int64_t i0 = blockIdx.x * (int64_t)(KT * CI) + threadIdx.x;
  uint2 t[CI];
  uint32_t base[CI];
#pragma unroll
  for (int k = 0; k < CI; ++k) t[k] = i0 + k * KT < np ? __ldg(kr + i0 + k * KT) : make_uint2(0u, 0u);
#pragma unroll
  for (int k = 0; k < CI; ++k) base[k] = i0 + k * KT < np ? __ldg(cellstart + t[k].x) : 0u;
#pragma unroll
  for (int k = 0; k < CI; ++k)
    if (i0 + k * KT < np) perm[base[k] + t[k].y] = (uint32_t)(i0 + k * KT);
}

// Stable order inside each cell: the ranks of cell c, cellstart[c] ..
// cellstart[c+1]-1, in ascending particle index.  A thread takes OC
// consecutive cells (16-byte loads of their starts).  Runs of at most
// kWalkRun are insertion-sorted here; runs of at most kMedRun are listed in
// smalls[1 ..] (for k_cell_order_med<16> and the deposit), runs of at most
// SHORT_RUN in meds[1 ..] for k_cell_order_med<32>, longer ones in runs[1 ..] for
// k_cell_order_warp and, if longer than kWarpRun, in bigs[1 ..] for
// k_cell_order_long as well (list[0] counts the entries, zeroed).  A block
// reserves the room for its entries of each list with one atomic (the lists'
// counters are shared by the whole grid), its warps and lanes in order after
// it; a block without entries skips the reservation and its second barrier.
constexpr int OC = 8;
__device__ __forceinline__ uint32_t cell_lists(uint32_t m) {   // bit L: the run goes to list L
  return (m > kWalkRun && m <= kMedRun ? 1u : 0u) | (m > kMedRun && m <= SHORT_RUN ? 2u : 0u) |
         (m > SHORT_RUN ? 4u : 0u) | (m > kWarpRun ? 8u : 0u);
}
__global__ void __launch_bounds__(KT) k_cell_order(const uint32_t* __restrict__ cellstart, int64_t ncells,
                                                   uint32_t* __restrict__ perm, uint32_t* __restrict__ smalls,
                                                   uint32_t* __restrict__ meds, uint32_t* __restrict__ runs,
                                                   uint32_t* __restrict__ bigs) {
  __shared__ uint32_t wtot[4][KT / 32];
  __shared__ uint32_t lbase[4];
  const int64_t c0 = (blockIdx.x * (int64_t)KT + threadIdx.x) * OC;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t st[OC + 1];
#pragma unroll
  for (int k = 0; k <= OC; ++k) st[k] = 0u;
  if (c0 < ncells) {   // ncells is a multiple of OC
#pragma unroll
    for (int k = 0; k < OC; k += 4) {
      const uint4 v = __ldg(reinterpret_cast<const uint4*>(cellstart + c0 + k));
      st[k] = v.x; st[k + 1] = v.y; st[k + 2] = v.z; st[k + 3] = v.w;
    }
    st[OC] = __ldg(cellstart + c0 + OC);
  }
  // entries of this lane per list, their exclusive prefix over the warp
  uint32_t cnt[4] = {0u, 0u, 0u, 0u}, pre[4];
#pragma unroll
  for (int k = 0; k < OC; ++k) {
    const uint32_t f = cell_lists(st[k + 1] - st[k]);
#pragma unroll
    for (int L = 0; L < 4; ++L) cnt[L] += (f >> L) & 1u;
  }
#pragma unroll
  for (int L = 0; L < 4; ++L) {
    uint32_t x = cnt[L];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= (uint32_t)o) x += y;
    }
    pre[L] = x - cnt[L];
    if (lane == 31) wtot[L][warp] = x;
  }
  const bool any = __syncthreads_or((cnt[0] | cnt[1] | cnt[2] | cnt[3]) != 0u);
  if (any && threadIdx.x < 4) {   // one thread per list: the warps' offsets, the block's room
    const int L = threadIdx.x;
    uint32_t run = 0;
    for (int w = 0; w < KT / 32; ++w) {
      const uint32_t t = wtot[L][w];
      wtot[L][w] = run;
      run += t;
    }
    uint32_t* list = L == 0 ? smalls : L == 1 ? meds : L == 2 ? runs : bigs;
    lbase[L] = run ? atomicAdd(list, run) : 0u;
  }
  // the short runs are ordered while the room is reserved
#pragma unroll
  for (int k = 0; k < OC; ++k) {
    const uint32_t a = st[k], b = st[k + 1];
    if (b - a < 2 || b - a > kWalkRun) continue;   // larger runs: k_cell_order_med
    for (uint32_t p = a + 1; p < b; ++p) {
      const uint32_t v = perm[p];
      uint32_t q = p;
      for (; q > a; --q) {
        const uint32_t u = perm[q - 1];
        if (u < v) break;
        perm[q] = u;
      }
      if (q != p) perm[q] = v;
    }
  }
  if (!any) return;   // the same for the whole block
  __syncthreads();
  uint32_t pos[4];
#pragma unroll
  for (int L = 0; L < 4; ++L) pos[L] = 1u + lbase[L] + wtot[L][warp] + pre[L];
#pragma unroll
  for (int k = 0; k < OC; ++k) {
    const uint32_t c = (uint32_t)(c0 + k);
    const uint32_t f = cell_lists(st[k + 1] - st[k]);
    if (f & 1u) smalls[pos[0]++] = c;
    if (f & 2u) meds[pos[1]++] = c;
    if (f & 4u) runs[pos[2]++] = c;
    if (f & 8u) bigs[pos[3]++] = c;
  }
}

// The runs of a list whose cells hold at most G particles, G lanes per run
// (32 / G runs per warp): lane i of a group holds the run's i-th particle
// index and moves it to its rank among the run's (distinct) indices, counted
// over the group by shuffles.  G = 16 for the small runs (kWalkRun + 1 ..
// kMedRun particles), G = 32 for the medium ones (kMedRun + 1 .. SHORT_RUN).
template <int G>
__global__ void __launch_bounds__(KT) k_cell_order_med(const uint32_t* __restrict__ cellstart,
                                                       const uint32_t* __restrict__ list,
                                                       uint32_t* __restrict__ perm) {
  constexpr int PERW = 32 / G;
  const uint32_t nlist = list[0];
  const uint32_t lane = threadIdx.x & 31, g = lane & (G - 1);
  const uint32_t groups = gridDim.x * (KT / 32) * PERW;
  // the groups of a warp take consecutive list entries; a warp with no entry
  // left stops as a whole (the shuffles need every lane)
  for (uint32_t q0 = (blockIdx.x * (KT / 32) + (threadIdx.x >> 5)) * PERW; q0 < nlist; q0 += groups) {
    const uint32_t q = q0 + lane / G;
    uint32_t a = 0, m = 0;
    if (q < nlist) {
      const uint32_t c = list[1 + q];
      a = cellstart[c];
      m = cellstart[c + 1] - a;
    }
    const uint32_t v = g < m ? perm[a + g] : 0xffffffffu;
    uint32_t rank = 0;
    for (uint32_t k = 0; k < (uint32_t)G; ++k) rank += __shfl_sync(0xffffffffu, v, k, G) < v;
    __syncwarp();
    if (g < m) perm[a + rank] = v;
  }
}

// Ranks of the R * 32 elements a lane may hold of a run of m distinct values
// in buf (the warp's shared-memory copy): each lane counts, for each of its
// elements buf[lane + 32 k], the run's smaller values and stores the element
// at that rank of seg.
template <int R>
__device__ __forceinline__ void warp_rank_sort(const uint32_t* buf, uint32_t m, uint32_t lane, uint32_t* seg) {
  uint32_t v[R], r[R];
#pragma unroll
  for (int k = 0; k < R; ++k) {
    v[k] = lane + 32 * k < m ? buf[lane + 32 * k] : 0xffffffffu;
    r[k] = 0;
  }
  for (uint32_t j = 0; j < m; ++j) {
    const uint32_t u = buf[j];   // the same word for every lane: one broadcast read
#pragma unroll
    for (int k = 0; k < R; ++k) r[k] += u < v[k];
  }
#pragma unroll
  for (int k = 0; k < R; ++k)
    if (lane + 32 * k < m) seg[r[k]] = v[k];
}

// The crowded runs listed by k_cell_order of at most kWarpRun particles, one
// warp each (many runs in flight per SM): the run is copied to the warp's
// shared-memory buffer and every element moved to its rank.  Longer runs are
// skipped here (k_cell_order_long orders them).
__global__ void __launch_bounds__(WT) k_cell_order_warp(const uint32_t* __restrict__ cellstart,
                                                        const uint32_t* __restrict__ runs,
                                                        uint32_t* __restrict__ perm) {
  __shared__ uint32_t sbuf[WT / 32][kWarpRun];
  const uint32_t nruns = runs[0];
  const uint32_t lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  uint32_t* buf = sbuf[wib];
  const uint32_t warps = gridDim.x * (WT / 32);
  for (uint32_t q = blockIdx.x * (WT / 32) + wib; q < nruns; q += warps) {
    const uint32_t c = runs[1 + q];
    const uint32_t a = cellstart[c], m = cellstart[c + 1] - a;
    if (m > kWarpRun) continue;   // the same for the whole warp
    uint32_t* seg = perm + a;
    for (uint32_t t = lane; t < m; t += 32) buf[t] = seg[t];
    __syncwarp();
    if (m <= 64) warp_rank_sort<2>(buf, m, lane, seg);
    else if (m <= 128) warp_rank_sort<4>(buf, m, lane, seg);
    else warp_rank_sort<8>(buf, m, lane, seg);
    __syncwarp();   // the buffer is reused by the warp's next run
  }
}

// Ascending bitonic sort of s[0 .. p2) (p2 a power of two) by the block.
__device__ void block_bitonic(uint32_t* s, int p2) {
  for (int k = 2; k <= p2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < (p2 >> 1); t += LT) {
        const int i = 2 * t - (t & (j - 1)), l = i + j;
        const uint32_t x = s[i], y = s[l];
        if ((x > y) == ((i & k) == 0)) {
          s[i] = y;
          s[l] = x;
        }
      }
      __syncthreads();
    }
  }
}

// out[0 .. la+lb) = merge of the ascending runs A[0 .. la) and B[0 .. lb),
// split evenly over the block's threads along the merge path.
__device__ void block_merge(const uint32_t* A, int64_t la, const uint32_t* B, int64_t lb, uint32_t* out) {
  const int64_t L = la + lb;
  const int64_t d0 = L * threadIdx.x / LT, d1 = L * (threadIdx.x + 1) / LT;
  int64_t lo = d0 > lb ? d0 - lb : 0, hi = d0 < la ? d0 : la;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (A[mid] < B[d0 - 1 - mid]) lo = mid + 1;
    else hi = mid;
  }
  int64_t ia = lo, ib = d0 - lo;
  for (int64_t d = d0; d < d1; ++d) {
    const bool take_a = ib >= lb || (ia < la && A[ia] < B[ib]);
    out[d] = take_a ? A[ia++] : B[ib++];
  }
}

// The runs longer than kWarpRun (k_cell_order's bigs list), one block each:
// LCH-element chunks sorted in shared memory, then pairwise merges between
// the run and the same ranks of `scratch`.  Runs already in order are left as
// they are.
__global__ void __launch_bounds__(LT) k_cell_order_long(const uint32_t* __restrict__ cellstart,
                                                        const uint32_t* __restrict__ runs,
                                                        uint32_t* __restrict__ perm,
                                                        uint32_t* __restrict__ scratch) {
  __shared__ uint32_t sv[LCH];
  const uint32_t nruns = runs[0];
  for (uint32_t q = blockIdx.x; q < nruns; q += gridDim.x) {
    const uint32_t c = runs[1 + q];
    const uint32_t a = cellstart[c];
    const int64_t m = (int64_t)cellstart[c + 1] - a;
    uint32_t* seg = perm + a;
    int unsorted = 0;
    for (int64_t t = threadIdx.x; t + 1 < m; t += LT) unsorted |= seg[t] > seg[t + 1];
    if (!__syncthreads_or(unsorted)) continue;
    for (int64_t c0 = 0; c0 < m; c0 += LCH) {
      const int len = (int)(m - c0 < LCH ? m - c0 : LCH);
      int p2 = 1;
      while (p2 < len) p2 <<= 1;
      for (int t = threadIdx.x; t < p2; t += LT) sv[t] = t < len ? seg[c0 + t] : 0xffffffffu;
      __syncthreads();
      block_bitonic(sv, p2);
      for (int t = threadIdx.x; t < len; t += LT) seg[c0 + t] = sv[t];
      __syncthreads();
    }
    uint32_t* in = seg;
    uint32_t* out = scratch + a;
    for (int64_t w = LCH; w < m; w *= 2) {
      for (int64_t lo = 0; lo < m; lo += 2 * w) {
        const int64_t la = m - lo < w ? m - lo : w;
        const int64_t rest = m - lo - la;
        block_merge(in + lo, la, in + lo + la, rest < w ? rest : w, out + lo);
      }
      __syncthreads();
      uint32_t* t = in;
      in = out;
      out = t;
    }
    if (in != seg) {
      for (int64_t t = threadIdx.x; t < m; t += LT) seg[t] = in[t];
    }
    __syncthreads();
  }
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

// A thread's SCAN_V consecutive values (four 16-byte loads in flight where
// the array is aligned and the run is whole; plain loads at the tail).
__device__ __forceinline__ void scan_load(const uint32_t* __restrict__ a, int64_t len, int64_t base,
                                          uint32_t v[SCAN_V]) {
  if (base + SCAN_V <= len && ((uintptr_t)a & 15) == 0) {
#pragma unroll
    for (int q = 0; q < SCAN_V / 4; ++q) {
      const uint4 t = __ldg(reinterpret_cast<const uint4*>(a + base) + q);
      v[4 * q] = t.x; v[4 * q + 1] = t.y; v[4 * q + 2] = t.z; v[4 * q + 3] = t.w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < SCAN_V; ++k) v[k] = base + k < len ? a[base + k] : 0u;
  }
}

__global__ void __launch_bounds__(SCAN_T) k_scan_reduce(const uint32_t* __restrict__ a, int64_t len,
                                                        uint32_t* __restrict__ sums) {
  __shared__ uint32_t wt[32];
  __shared__ uint32_t tot;
  const int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK + (int64_t)threadIdx.x * SCAN_V;
  uint32_t v[SCAN_V], t = 0;
  scan_load(a, len, base, v);
#pragma unroll
  for (int k = 0; k < SCAN_V; ++k) t += v[k];
  block_exclusive_scan(t, wt, &tot);
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
  const int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK + (int64_t)threadIdx.x * SCAN_V;
  uint32_t v[SCAN_V], t = 0;
  scan_load(a, len, base, v);
#pragma unroll
  for (int k = 0; k < SCAN_V; ++k) t += v[k];
  uint32_t e = block_exclusive_scan(t, wt, &tot) + sums[blockIdx.x];
  if (base + SCAN_V <= len && ((uintptr_t)a & 15) == 0) {
#pragma unroll
    for (int q = 0; q < SCAN_V / 4; ++q) {
      uint4 o;
      o.x = e; e += v[4 * q];
      o.y = e; e += v[4 * q + 1];
      o.z = e; e += v[4 * q + 2];
      o.w = e; e += v[4 * q + 3];
      reinterpret_cast<uint4*>(a + base)[q] = o;
    }
  } else {
#pragma unroll
    for (int k = 0; k < SCAN_V; ++k) {
      if (base + k < len) a[base + k] = e;
      e += v[k];
    }
  }
}

// Xs[d][j] = X[d][perm[j]] (and V, ids likewise): four particles per thread,
// PT apart (coalesced), their permutation entries and then their gathers all
// in flight together.
constexpr int PT = 256, PK = 4;
__global__ void __launch_bounds__(PT) k_permute(const uint32_t* __restrict__ perm, int64_t np,
                                                const uint32_t* __restrict__ X, const float* __restrict__ V,
                                                const uint32_t* __restrict__ id, uint32_t* __restrict__ Xs,
                                                float* __restrict__ Vs, uint32_t* __restrict__ ids) {
  const int64_t j0 = (int64_t)blockIdx.x * (PT * PK) + threadIdx.x;
  uint32_t p[PK];
#pragma unroll
  for (int k = 0; k < PK; ++k) p[k] = j0 + k * PT < np ? __ldg(perm + j0 + k * PT) : 0u;
  if (X) {
    uint32_t x[PK][3];
#pragma unroll
    for (int k = 0; k < PK; ++k)
#pragma unroll
      for (int d = 0; d < 3; ++d) x[k][d] = j0 + k * PT < np ? __ldg(X + d * np + p[k]) : 0u;
#pragma unroll
    for (int k = 0; k < PK; ++k)
      if (j0 + k * PT < np) {
#pragma unroll
        for (int d = 0; d < 3; ++d) Xs[d * np + j0 + k * PT] = x[k][d];
      }
  }
  if (V) {
    float v[PK][3];
#pragma unroll
    for (int k = 0; k < PK; ++k)
#pragma unroll
      for (int d = 0; d < 3; ++d) v[k][d] = j0 + k * PT < np ? __ldg(V + d * np + p[k]) : 0.0f;
#pragma unroll
    for (int k = 0; k < PK; ++k)
      if (j0 + k * PT < np) {
#pragma unroll
        for (int d = 0; d < 3; ++d) Vs[d * np + j0 + k * PT] = v[k][d];
      }
  }
  if (id) {
#pragma unroll
    for (int k = 0; k < PK; ++k)
      if (j0 + k * PT < np) ids[j0 + k * PT] = __ldg(id + p[k]);
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

int64_t sort_scan_blocks(int64_t ncells) { return (ncells + 1 + SCAN_CHUNK - 1) / SCAN_CHUNK + 1; }

int64_t sort_runs_capacity(int64_t np) { return np / (SHORT_RUN + 1) + 2; }
int64_t sort_meds_capacity(int64_t np) { return np / (kMedRun + 1) + 2; }
int64_t sort_bigs_capacity(int64_t np) { return np / (kWarpRun + 1) + 2; }
int64_t sort_smalls_capacity(int64_t np) { return np / (kWalkRun + 1) + 2; }

pm_status sort_cells(const uint32_t* X, int64_t np, int n, Workspace& w, cudaStream_t s, uint32_t* cellstart,
                     uint32_t** perm_out, const Batch& bt) {
  const int log2n = ilog2(n);
  const int64_t ncells = (int64_t)n * n * n * bt.B;
  *perm_out = w.perm;
  PM_TRY(cuda_status(cudaMemsetAsync(cellstart, 0, (size_t)(ncells + 1) * 4, s)));
  PM_TRY(cuda_status(cudaMemsetAsync(w.runs, 0, 4, s)));   // no crowded or medium cells yet
  PM_TRY(cuda_status(cudaMemsetAsync(w.meds, 0, 4, s)));
  PM_TRY(cuda_status(cudaMemsetAsync(w.bigs, 0, 4, s)));
  PM_TRY(cuda_status(cudaMemsetAsync(w.smalls, 0, 4, s)));
  if (np == 0) return PM_OK;
  const int64_t np_box = bt.B > 1 ? bt.np_box : 0;
  const unsigned gc = grid_for(np, KT * CI);
  if (np_box > 0)
    PM_LAUNCH(K_KEYS, 28.0 * np, k_cell_count<true>, gc, KT, 0, s, X, np, log2n, np_box, w.keyrank, cellstart);
  else
    PM_LAUNCH(K_KEYS, 28.0 * np, k_cell_count<false>, gc, KT, 0, s, X, np, log2n, np_box, w.keyrank, cellstart);
  PM_TRY(scan_u32(cellstart, ncells + 1, w.scan_blocks, s));
  PM_LAUNCH(K_SCATTER, 16.0 * np, k_cell_scatter, gc, KT, 0, s, w.keyrank, np, cellstart, w.perm);
  PM_LAUNCH(K_ORDER, 4.0 * ncells + 8.0 * np, k_cell_order, grid_for(ncells / OC, KT), KT, 0, s, cellstart, ncells,
            w.perm, w.smalls, w.meds, w.runs, w.bigs);
  PM_LAUNCH(K_ORDER, 0.0, k_cell_order_med<16>, 8 * 152, KT, 0, s, cellstart, w.smalls, w.perm);
  PM_LAUNCH(K_ORDER, 0.0, k_cell_order_med<32>, 8 * 152, KT, 0, s, cellstart, w.meds, w.perm);
  PM_LAUNCH(K_ORDER, 0.0, k_cell_order_warp, 8 * 152, WT, 0, s, cellstart, w.runs, w.perm);
  PM_LAUNCH(K_ORDER, 0.0, k_cell_order_long, LONG_BLOCKS, LT, 0, s, cellstart, w.bigs, w.perm,
            reinterpret_cast<uint32_t*>(w.keyrank));
  return launch_status();
}

pm_status permute_particles(const uint32_t* perm, int64_t np, const uint32_t* X, const float* V,
                            const uint32_t* id, uint32_t* Xs, float* Vs, uint32_t* ids,
                            cudaStream_t s) {
  if (np == 0) return PM_OK;
  PM_LAUNCH(K_PERMUTE, (4.0 + (X ? 24.0 : 0.0) + (V ? 24.0 : 0.0) + (id ? 8.0 : 0.0)) * np, k_permute,
            grid_for(np, PT * PK), PT, 0, s, perm, np, X, V, id, Xs, Vs, ids);
  return launch_status();
}

}  // namespace pmgb
