// Linear multigrid for the periodic 7-point Poisson problem (§3.5, §3.6.1):
// red-black SOR smoothing (Eq. jacobi_sweep_laplacian with over-relaxation),
// residual + 8-child-average restriction, 27/9/3/1 prolongation and
// correction, a single-CTA coarsest-level solve, V-cycles.
//
// Precision: smoothing and transfers in float32.  The finest-level residual is
// formed as sum_nb (u_nb - u) with every difference and partial sum kept
// exactly (TwoSum), so the float32-stored iterate is tested against f with
// float64-class accuracy; norms are accumulated in float64.
#include <math.h>

#include "pm_device.cuh"
#include "pm_internal.cuh"
#include "rb_fused.cuh"
#include "rb_stream.cuh"

namespace pmgb {

namespace {

constexpr float kSixth = 1.0f / 6.0f;

__device__ __forceinline__ float load_mean(const Src& f) { return f.mean ? (float)*f.mean : 0.0f; }
__device__ __forceinline__ float src_at(const Src& f, int64_t i, float mean) {
  return f.s * (__ldg(f.p + i) - mean);
}

// Offset of cell (i, j, k) inside one box (n <= 1024: below 2^30).
__device__ __forceinline__ uint32_t idx3(int i, int j, int k, int log2n) {
  return ((uint32_t)i << (2 * log2n)) | ((uint32_t)j << log2n) | (uint32_t)k;
}

// sum_nb (u_nb - u) with TwoSum on every difference and partial sum: S + E.
__device__ __forceinline__ void lap_diff_comp(float uc, const float nb[6], float& S, float& E) {
  float s, e, t;
  two_sum(nb[0], -uc, S, E);
#pragma unroll
  for (int q = 1; q < 6; ++q) {
    two_sum(nb[q], -uc, s, e);
    two_sum(S, s, S, t);
    E += t + e;
  }
}

__device__ __forceinline__ void load_nb(const float* __restrict__ u, int i, int j, int k, int log2n,
                                        float nb[6]) {
  const int m = (1 << log2n) - 1;
  nb[0] = __ldg(u + idx3((i + 1) & m, j, k, log2n));
  nb[1] = __ldg(u + idx3((i - 1) & m, j, k, log2n));
  nb[2] = __ldg(u + idx3(i, (j + 1) & m, k, log2n));
  nb[3] = __ldg(u + idx3(i, (j - 1) & m, k, log2n));
  nb[4] = __ldg(u + idx3(i, j, (k + 1) & m, log2n));
  nb[5] = __ldg(u + idx3(i, j, (k - 1) & m, log2n));
}

// u = -h^2 f / 6 (Eq. multigrid_initial_guess).
__global__ void k_jacobi_guess(float* __restrict__ u, Src f, int64_t count, float h2) {
  u += (int64_t)blockIdx.z * count;
  f = box_src(f, count);
  const float mean = load_mean(f);
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < count;
       c += (int64_t)gridDim.x * blockDim.x)
    u[c] = -h2 * src_at(f, c, mean) * kSixth;
}

// u *= a (per box: ab[box] if ab is set).
__global__ void k_scale(float* __restrict__ u, int64_t count, float a, const float* __restrict__ ab) {
  u += (int64_t)blockIdx.z * count;
  if (ab) a = __ldg(ab + blockIdx.z);
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < count;
       c += (int64_t)gridDim.x * blockDim.x)
    u[c] *= a;
}

// One colour of a red-black SOR sweep (the update rule is PoissonUpdate,
// shared with the streaming smoother).  zero: the values of this level are
// taken as 0 (the coarse-level error starts from zero): the red pass reads
// nothing, the black pass ignores its own old value.
__global__ void k_rb_sweep(float* __restrict__ u, Src f, int log2n, int colour, PoissonUpdate upd,
                           int nb_old, int own_old, int zero) {
  const int m = (1 << log2n) - 1, half = log2n - 1;
  u += (int64_t)blockIdx.z << (3 * log2n);
  f = box_src(f, (int64_t)1 << (3 * log2n));
  upd = upd.box(blockIdx.z);
  const float mean = load_mean(f);
  const int64_t total = (int64_t)1 << (3 * log2n - 1);
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    const int kk = (int)(t & ((1 << half) - 1));
    const int64_t rest = t >> half;
    const int j = (int)(rest & m), i = (int)(rest >> log2n);
    const int k = 2 * kk + ((colour + i + j) & 1);
    const int64_t c = idx3(i, j, k, log2n);
    float nb[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    float old = 0.0f;
    if (!(zero && colour == 0)) {
      nb[0] = u[idx3((i + 1) & m, j, k, log2n)];
      nb[1] = u[idx3((i - 1) & m, j, k, log2n)];
      nb[2] = u[idx3(i, (j + 1) & m, k, log2n)];
      nb[3] = u[idx3(i, (j - 1) & m, k, log2n)];
      nb[4] = u[idx3(i, j, (k + 1) & m, log2n)];
      nb[5] = u[idx3(i, j, (k - 1) & m, log2n)];
    }
    if (!zero) old = u[c];
    u[c] = upd(old, nb, src_at(f, c, mean), 0, nb_old != 0, own_old != 0);
  }
}

// Coarse right-hand side fc = R(f - L u): residual of the 8 children,
// averaged.  Summed over the 2x2x2 block the Laplacian fluxes through the 12
// inner faces cancel pairwise, so  h^2 sum_c L u_c  is the sum of
// (u_nb - u_c) over the 24 outer faces only.  With COMP the differences are
// exact (TwoSum) and summed with compensation, as is the sum of the sources,
// and the one cancelling subtraction is a single rounding (fused
// multiply-add).
template <bool COMP>
__global__ void k_resid_restrict(const float* __restrict__ u, Src f, int log2n, float inv_h2,
                                 float* __restrict__ fc) {
  const int lc = log2n - 1, mc = (1 << lc) - 1;
  u += (int64_t)blockIdx.z << (3 * log2n);
  f = box_src(f, (int64_t)1 << (3 * log2n));
  fc += (int64_t)blockIdx.z << (3 * lc);
  const float mean = load_mean(f);
  const int64_t total = (int64_t)1 << (3 * lc);
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    const int K = (int)(t & mc), J = (int)((t >> lc) & mc), I = (int)(t >> (2 * lc));
    float core[2][2][4], xf[2][2][2], yf[2][2][2];
    load_children_block(u, I, J, K, log2n, core, xf, yf);
    float fz[8];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        const float2 fr = __ldg(reinterpret_cast<const float2*>(f.p + idx3(2 * I + a, 2 * J + b, 2 * K, log2n)));
        fz[(a * 2 + b) * 2] = f.s * (fr.x - mean);
        fz[(a * 2 + b) * 2 + 1] = f.s * (fr.y - mean);
      }
    // outer faces (neighbour, child): x-, x+ for each (b, c); y-, y+ for each
    // (a, c); z-, z+ for each (a, b)
    float nbv[24], chv[24];
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int side = 0; side < 2; ++side) {
          const int q = (b * 2 + c) * 2 + side;
          nbv[q] = xf[side][b][c];
          chv[q] = core[side][b][c + 1];
          nbv[8 + q] = yf[b][side][c];          // here b plays a (x offset)
          chv[8 + q] = core[b][side][c + 1];
          nbv[16 + q] = core[b][c][side ? 3 : 0];   // here (b, c) play (a, b)
          chv[16 + q] = core[b][c][side ? 2 : 1];
        }
    float d;
    if (COMP) {
      float S, E, sq, eq, tq;
      two_sum(nbv[0], -chv[0], S, E);
#pragma unroll
      for (int q = 1; q < 24; ++q) {
        two_sum(nbv[q], -chv[q], sq, eq);
        two_sum(S, sq, S, tq);
        E += tq + eq;
      }
      float F = fz[0], Fe = 0.0f;
#pragma unroll
      for (int q = 1; q < 8; ++q) {
        two_sum(F, fz[q], F, tq);
        Fe += tq;
      }
      d = fmaf(-inv_h2, S, F) + (Fe - inv_h2 * E);
    } else {
      float L[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
      for (int q = 0; q < 24; ++q) L[q & 3] += nbv[q] - chv[q];
      const float F = ((fz[0] + fz[1]) + (fz[2] + fz[3])) + ((fz[4] + fz[5]) + (fz[6] + fz[7]));
      d = fmaf(-inv_h2, (L[0] + L[1]) + (L[2] + L[3]), F);
    }
    fc[t] = 0.125f * d;
  }
}

// Residual norm^2 and source norm^2 partials (finest level, compensated
// residual): partial[blockIdx] and partial[gridDim + blockIdx].
__global__ void __launch_bounds__(256) k_resid_norm(const float* __restrict__ u, Src f, int log2n,
                                                    float inv_h2, double* __restrict__ partial) {
  __shared__ double scratch[32];
  const float mean = load_mean(f);
  const int m = (1 << log2n) - 1;
  const int64_t total = (int64_t)1 << (3 * log2n);
  float sd = 0.0f, cd = 0.0f, sf = 0.0f, cf = 0.0f;
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < total; c += gridDim.x * blockDim.x) {
    const int k = (int)(c & m), j = (int)((c >> log2n) & m), i = (int)(c >> (2 * log2n));
    float nb[6];
    load_nb(u, i, j, k, log2n, nb);
    const float uc = __ldg(u + c), fv = src_at(f, c, mean);
    float S, E;
    lap_diff_comp(uc, nb, S, E);
    const float d = fmaf(-inv_h2, S, fv) - inv_h2 * E;
    kahan_add(sd, cd, d * d);
    kahan_add(sf, cf, fv * fv);
  }
  block_sum_to(partial + blockIdx.x, sd, cd, scratch);
  block_sum_to(partial + gridDim.x + blockIdx.x, sf, cf, scratch);
}

// Block sum of per-thread float64 values, written by thread 0 to *out (a
// fixed order: shuffles, then the warps in order).
__device__ __forceinline__ void block_sum_f64(double* out, double v, double* scratch32) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) scratch32[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += scratch32[i];
    *out = t;
  }
  __syncthreads();
}

// Residual of a float64 iterate in float64: r = (f - <f>) - (L(u) - 6u)/h^2,
// with L(u) - 6u as the neighbour sum minus 6u (the float64 pipe bounds this
// kernel on GB300, so it spends 12 float64 operations per cell; the six
// differences u_nb - u would take five more).  r is stored rounded to float32
// (the source of the correction solve); the squares of r and of f - <f> are
// summed per block in float64.
__global__ void __launch_bounds__(256) k_resid_f64(const double* __restrict__ u, const float* __restrict__ f,
                                                   const double* __restrict__ fmean, int log2n, double inv_h2,
                                                   float* __restrict__ r, double* __restrict__ partial) {
  __shared__ double scratch[32];
  const double mean = *fmean;
  const int m = (1 << log2n) - 1;
  const int64_t total = (int64_t)1 << (3 * log2n);
  double sr = 0.0, sf = 0.0;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < total; c += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(c & m), j = (int)((c >> log2n) & m), i = (int)(c >> (2 * log2n));
    const double uc = u[c];
    const double nsum = ((u[idx3((i + 1) & m, j, k, log2n)] + u[idx3((i - 1) & m, j, k, log2n)]) +
                         (u[idx3(i, (j + 1) & m, k, log2n)] + u[idx3(i, (j - 1) & m, k, log2n)])) +
                        (u[idx3(i, j, (k + 1) & m, log2n)] + u[idx3(i, j, (k - 1) & m, log2n)]);
    const double L = fma(-6.0, uc, nsum);
    const double fv = (double)__ldg(f + c) - mean;
    const double d = fma(-inv_h2, L, fv);
    r[c] = (float)d;
    sr = fma(d, d, sr);
    sf = fma(fv, fv, sf);
  }
  block_sum_f64(partial + blockIdx.x, sr, scratch);
  block_sum_f64(partial + gridDim.x + blockIdx.x, sf, scratch);
}

// u += e (float64 iterate, float32 correction).
__global__ void k_add_correction_f64(double* __restrict__ u, const float* __restrict__ e, int64_t count) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < count; c += (int64_t)gridDim.x * blockDim.x)
    u[c] += (double)__ldg(e + c);
}

// u += P(uc - uc2): cell-centred trilinear prolongation, weights 27/9/3/1 over
// 64 (§3.6.1); uc2 may be NULL.  One thread per two coarse cells along z
// (K = 2G, 2G + 1): it reads their 3x3x4 coarse neighbourhood once (a float2
// and two scalars per coarse row) and corrects their 16 children (runs of
// four along z as float4).  Per child the interpolation runs z, then y, then
// x, parent (weight 3/4) before neighbour (1/4), in fused multiply-adds.
__global__ void k_prolong_correct(float* __restrict__ u, const float* __restrict__ uc,
                                  const float* __restrict__ uc2, int log2n) {
  const int lc = log2n - 1, mc = (1 << lc) - 1;
  const int64_t total = (int64_t)1 << (3 * lc);
  u += (int64_t)blockIdx.z << (3 * log2n);
  uc += (int64_t)blockIdx.z * total;
  if (uc2) uc2 += (int64_t)blockIdx.z * total;
  const int hz = lc - 1;   // log2 of the pairs per coarse row
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < (total >> 1); t += gridDim.x * blockDim.x) {
    const int K = 2 * (int)(t & ((1 << hz) - 1));
    const int64_t row = t >> hz;
    const int J = (int)(row & mc), I = (int)(row >> lc);
    float c[3][3][4];   // [x][y][z]: x, y = I-1 .. I+1, J-1 .. J+1; z = K-1 .. K+2
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const int64_t base = idx3((I + a - 1) & mc, (J + b - 1) & mc, 0, lc);
        const float2 mid = __ldg(reinterpret_cast<const float2*>(uc + base + K));
        float v[4] = {__ldg(uc + base + ((K - 1) & mc)), mid.x, mid.y, __ldg(uc + base + ((K + 2) & mc))};
        if (uc2) {
          const float2 m2 = __ldg(reinterpret_cast<const float2*>(uc2 + base + K));
          v[0] -= __ldg(uc2 + base + ((K - 1) & mc));
          v[1] -= m2.x;
          v[2] -= m2.y;
          v[3] -= __ldg(uc2 + base + ((K + 2) & mc));
        }
#pragma unroll
        for (int z = 0; z < 4; ++z) c[a][b][z] = v[z];
      }
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int jn = b ? 2 : 0;
      // z then y contractions: vy[x][q] for the fine z offsets q = 0..3 (coarse
      // cell q / 2 at column q / 2 + 1, child q & 1)
      float vy[3][4];
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int kc = (q >> 1) + 1, kn = (q & 1) ? kc + 1 : kc - 1;
          const float vz0 = fmaf(0.25f, c[a][1][kn], fmaf(0.75f, c[a][1][kc], 0.0f));
          const float vz1 = fmaf(0.25f, c[a][jn][kn], fmaf(0.75f, c[a][jn][kc], 0.0f));
          vy[a][q] = fmaf(0.25f, vz1, fmaf(0.75f, vz0, 0.0f));
        }
#pragma unroll
      for (int ax = 0; ax < 2; ++ax) {
        const int in = ax ? 2 : 0;
        float4* dst = reinterpret_cast<float4*>(u + idx3(2 * I + ax, 2 * J + b, 2 * K, log2n));
        float4 w = *dst;
        w.x += fmaf(0.25f, vy[in][0], fmaf(0.75f, vy[1][0], 0.0f));
        w.y += fmaf(0.25f, vy[in][1], fmaf(0.75f, vy[1][1], 0.0f));
        w.z += fmaf(0.25f, vy[in][2], fmaf(0.75f, vy[1][2], 0.0f));
        w.w += fmaf(0.25f, vy[in][3], fmaf(0.75f, vy[1][3], 0.0f));
        *dst = w;
      }
    }
  }
}

// Coarsest level (n <= 16) in one CTA of 1024 threads: red-black SOR sweeps
// (factor omega) until the residual norm dropped by `drop`, its running
// minimum stalls for 5 sweeps (float32 floor), or `max_sweeps` sweeps.  Thread
// t owns the cell pairs (2P, 2P+1), P = t and t + 1024 (same i, j; k even and
// odd), so each colour pass gives every thread one cell per pair.  The
// residual of a black cell is taken from its own update (its neighbours are
// red and do not move during the black pass).  The red residuals of a sweep
// and the next sweep's red values come from the same neighbour sums (the black
// cells do not move in between): the new red values are held in registers
// until the sweep's norm has decided whether there is a next sweep.
__global__ void __launch_bounds__(1024) k_mg_coarse(float* __restrict__ u, Src f, int log2n, float h2,
                                                    float omega, int max_sweeps, float drop,
                                                    int zero_guess) {
  __shared__ float su[4096], sf[4096];
  __shared__ float2 scratch[33];
  const int n = 1 << log2n, m = n - 1, N = n * n * n, npair = N >> 1;
  u += (int64_t)blockIdx.z * N;   // one CTA per box
  f = box_src(f, N);
  const float mean = load_mean(f);
  const float inv_h2 = 1.0f / h2;
  for (int c = threadIdx.x; c < N; c += blockDim.x) {
    su[c] = zero_guess ? 0.0f : u[c];
    sf[c] = src_at(f, c, mean);
  }
  __syncthreads();
  auto nbsum = [&](int c) -> float {
    const int k = c & m, j = (c >> log2n) & m, i = c >> (2 * log2n);
    return su[(((i + 1) & m) << (2 * log2n)) | (j << log2n) | k] +
           su[(((i - 1) & m) << (2 * log2n)) | (j << log2n) | k] +
           su[(i << (2 * log2n)) | (((j + 1) & m) << log2n) | k] +
           su[(i << (2 * log2n)) | (((j - 1) & m) << log2n) | k] +
           su[(i << (2 * log2n)) | (j << log2n) | ((k + 1) & m)] +
           su[(i << (2 * log2n)) | (j << log2n) | ((k - 1) & m)];
  };
  // the cell of pair P with colour col: k of 2P is even, so its colour is (i + j) & 1
  auto cell_of = [&](int P, int col) -> int {
    const int c0 = P << 1;
    return c0 + ((col ^ ((c0 >> log2n) + (c0 >> (2 * log2n)))) & 1);
  };
  // SOR update of cell c from its neighbour sum
  auto sor = [&](int c, float nb) -> float {
    const float ugs = (nb - h2 * sf[c]) * kSixth;
    return (omega == 1.0f) ? ugs : omega * ugs + (1.0f - omega) * su[c];
  };
  const int P0 = threadIdx.x, P1 = threadIdx.x + blockDim.x;   // npair <= 2048 = 2 x 1024
  float2 r2p;
  {
    float s = 0.0f, cmp = 0.0f;
    for (int c = threadIdx.x; c < N; c += blockDim.x) {
      const float d = sf[c] - (nbsum(c) - 6.0f * su[c]) * inv_h2;
      kahan_add(s, cmp, d * d);
    }
    r2p = block_pair_sum(s, cmp, scratch);
  }
  float best = r2p.x + r2p.y;
  const float target = drop * drop * best;
  int stale = 0;
  if (max_sweeps > 0) {   // the first sweep's red cells
    for (int P = threadIdx.x; P < npair; P += blockDim.x) {
      const int c = cell_of(P, 0);
      su[c] = sor(c, nbsum(c));
    }
    __syncthreads();
  }
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    // here the red cells hold this sweep's values
    float s = 0.0f, cmp = 0.0f;
    for (int P = threadIdx.x; P < npair; P += blockDim.x) {      // black, with its residual
      const int c = cell_of(P, 1);
      const float nb = nbsum(c);
      const float un = sor(c, nb);
      su[c] = un;
      const float d = sf[c] - (nb - 6.0f * un) * inv_h2;
      kahan_add(s, cmp, d * d);
    }
    __syncthreads();
    // red residuals, and the next sweep's red values from the same sums
    float pend0 = 0.0f, pend1 = 0.0f;
    const int c0 = P0 < npair ? cell_of(P0, 0) : 0, c1 = P1 < npair ? cell_of(P1, 0) : 0;
    if (P0 < npair) {
      const float nb = nbsum(c0);
      const float d = sf[c0] - (nb - 6.0f * su[c0]) * inv_h2;
      kahan_add(s, cmp, d * d);
      pend0 = sor(c0, nb);
    }
    if (P1 < npair) {
      const float nb = nbsum(c1);
      const float d = sf[c1] - (nb - 6.0f * su[c1]) * inv_h2;
      kahan_add(s, cmp, d * d);
      pend1 = sor(c1, nb);
    }
    r2p = block_pair_sum(s, cmp, scratch);   // its barriers end every read of this sweep
    const float r = r2p.x + r2p.y;
    if (r <= target) break;
    if (r < 0.998f * best) {   // squared norms: a 0.1% improvement of the norm
      best = r;
      stale = 0;
    } else if (++stale >= 5) {
      break;                  // no progress for 5 sweeps: the float32 floor
    }
    if (sweep + 1 < max_sweeps) {   // the next sweep's red cells
      if (P0 < npair) su[c0] = pend0;
      if (P1 < npair) su[c1] = pend1;
      __syncthreads();
    }
  }
  for (int c = threadIdx.x; c < N; c += blockDim.x) u[c] = su[c];
}

// SOR factor of the coarsest level: the caller's, else Young's optimum
// 2 / (1 + sqrt(1 - mu^2)) for red-black ordering of the periodic 7-point
// Laplacian on n^3 cells, mu = (2 + cos(2 pi / n)) / 3 the largest Jacobi
// eigenvalue below 1 (the constant mode is absent from a zero-mean problem).
float coarse_omega(const mg_params& p, int n) {
  if (p.coarse_omega > 0.0f) return p.coarse_omega;
  const double mu = (2.0 + cos(2.0 * M_PI / n)) / 3.0;
  return (float)(2.0 / (1.0 + sqrt(1.0 - mu * mu)));
}

struct MG {
  int n0;
  const mg_params* p;
  cudaStream_t s;
  float* u[12];     // current iterate of each level
  float* alt[12];   // ping-pong partner for the streaming smoother (or NULL)
  Src f[12];
  bool first_cycle;
  float gscale;
  int B = 1;                    // boxes of a batched solve (blockIdx.z of every launch)
  const float* gbox = nullptr;  // per-box warm-start factors (batched MG_GUESS_SCALED)
  dim3 grid(unsigned gx) const { return dim3(gx, 1, (unsigned)B); }
};

pm_status stream_attributes() {
  PM_TRY(smem_attr(k_rb_stream<2, PoissonUpdate>, StreamGeom<2>::smem_bytes));
  PM_TRY(smem_attr(k_rb_stream<1, PoissonUpdate>, StreamGeom<1>::smem_bytes));
  PM_TRY(smem_attr(k_rb_fused4<PoissonUpdate, 3>, kFusedSmem));
  return PM_OK;
}

// `count` smoothing sweeps on level l with SOR factors w[0..count-1].
// zero: the level's values start at 0; scale (sbox: per box): warm-start
// factor applied to the values present before the first sweep.
pm_status smooth(MG& g, int l, int count, const float* w, bool zero, float scale, const float* sbox = nullptr) {
  const int n = g.n0 >> l, log2n = ilog2(n);
  const float h2 = 1.0f / ((float)n * (float)n);
  const int64_t N = (int64_t)n * n * n;
  int done = 0;
  if (g.p->smoother == 0 && stream_ok(n) && g.alt[l] && g.B == 1) {
    int chunk, nitems;
    stream_plan(n, &chunk, &nitems);
    while (done < count) {
      const int S = (count - done) >= 2 ? 2 : 1;
      PoissonUpdate upd{h2, {w[done], S == 2 ? w[done + 1] : 1.0f}, done == 0 ? scale : 1.0f};
      const int z = (done == 0 && zero) ? 1 : 0;
      const unsigned grid = (unsigned)(nitems < 152 * 2 ? nitems : 152 * 2);   // 2 CTAs/SM (shared memory)
      if (S == 2)
        PM_LAUNCH(l == 0 ? K_MG_SMOOTH0 : K_MG_SMOOTH, (z ? 20.0 : 24.0) * N, (k_rb_stream<2, PoissonUpdate>), grid, kStreamThreads,
                  StreamGeom<2>::smem_bytes, g.s, g.u[l], g.alt[l], g.f[l], log2n, chunk, nitems, z, upd);
      else
        PM_LAUNCH(l == 0 ? K_MG_SMOOTH0 : K_MG_SMOOTH, (z ? 8.0 : 12.0) * N, (k_rb_stream<1, PoissonUpdate>), grid, kStreamThreads,
                  StreamGeom<1>::smem_bytes, g.s, g.u[l], g.alt[l], g.f[l], log2n, chunk, nitems, z, upd);
      float* t = g.u[l];
      g.u[l] = g.alt[l];
      g.alt[l] = t;
      done += S;
    }
    return PM_OK;
  }
  // fused sweeps (one pass per sweep) or colour passes (two per sweep), bitwise
  // the same result; on 64^3 levels of a batch the form is tuned, and the
  // fused sweep's x chunk is tuned on every batched level
  const bool fused_valid = g.p->smoother == 2 && n >= 64 && g.alt[l] && fused_aligned(g.u[l], g.alt[l], g.f[l].p);
  bool fused = fused_valid && fused_ok(n, g.B);
  const bool tune_form = fused_valid && g.B > 1 && n < 128;
  if (tune_form) {
    static const int forms[2] = {0, 1};
    fused = tune_begin(TUNE_MG_SMOOTHER, n, g.B, forms, 2, fused ? 1 : 0, g.s) == 1;
  }
  const bool form_timed = tune_form && tune_active();
  if (fused) {
    for (; done < count; ++done) {
      int chunk = fused_chunk(n);
      const bool tune_chunk = g.B > 1 && !form_timed;   // one timing at a time
      if (tune_chunk) {
        int cand[3], nc = 0;
        for (int c = 16; c <= 64 && c <= n; c *= 2) cand[nc++] = c;
        chunk = tune_begin(TUNE_MG_FUSED_CHUNK, n, g.B, cand, nc, chunk, g.s);
      }
      const unsigned grid = (unsigned)((n / kFusedT) * (n / kFusedT) * (n / chunk));
      PoissonUpdate upd{h2, {w[done], 1.0f}, done == 0 ? scale : 1.0f, done == 0 ? sbox : nullptr};
      const int z = (done == 0 && zero) ? 1 : 0;
      PM_LAUNCH(l == 0 ? K_MG_SMOOTH0 : K_MG_SMOOTH, (z ? 8.0 : 12.0) * N * g.B, (k_rb_fused4<PoissonUpdate, 3>),
                g.grid(grid), kQuadThreads, kFusedSmem, g.s, g.u[l], g.alt[l], g.f[l], log2n, chunk, z,
                done == 0 ? 1 : 0, upd);
      if (tune_chunk) tune_end(g.s);
      float* t = g.u[l];
      g.u[l] = g.alt[l];
      g.alt[l] = t;
    }
  } else {
    const unsigned grid = grid_for(N / 2, 256);
    for (; done < count; ++done) {
      PoissonUpdate upd{h2, {w[done], 1.0f}, done == 0 ? scale : 1.0f, done == 0 ? sbox : nullptr};
      const int z = (done == 0 && zero) ? 1 : 0;
      const int first = done == 0 ? 1 : 0;
      PM_LAUNCH(l == 0 ? K_MG_SMOOTH0 : K_MG_SMOOTH, (z ? 4.0 : 6.0) * N * g.B, k_rb_sweep, g.grid(grid), 256, 0,
                g.s, g.u[l], g.f[l], log2n, 0, upd, first, first, z);
      PM_LAUNCH(l == 0 ? K_MG_SMOOTH0 : K_MG_SMOOTH, (z ? 4.0 : 6.0) * N * g.B, k_rb_sweep, g.grid(grid), 256, 0,
                g.s, g.u[l], g.f[l], log2n, 1, upd, 0, first, z);
    }
  }
  if (form_timed) tune_end(g.s);
  return PM_OK;
}

pm_status v_cycle(MG& g, int l, bool zero_guess) {
  const int n = g.n0 >> l, log2n = ilog2(n);
  const mg_params& p = *g.p;
  const float h2 = 1.0f / ((float)n * (float)n);
  const bool scaled = (l == 0 && g.first_cycle && (g.gbox || g.gscale != 1.0f));
  const float* sbox = scaled ? g.gbox : nullptr;
  if (n <= p.coarsest || n <= 4) {
    float* u = g.u[l];
    if (!zero_guess && scaled) {
      const int64_t N = (int64_t)n * n * n;
      PM_LAUNCH(K_MG_GUESS, 8.0 * N * g.B, k_scale, g.grid(grid_for(N, 256)), 256, 0, g.s, u, N, g.gscale, sbox);
    }
    PM_LAUNCH(K_MG_COARSE, 12.0 * n * n * n * g.B, k_mg_coarse, g.grid(1), 1024, 0, g.s, u, g.f[l], log2n, h2,
              coarse_omega(p, n), p.coarse_max_sweeps, p.coarse_drop, zero_guess ? 1 : 0);
    return PM_OK;
  }
  float w[64];
  if (p.npre == 0) {
    const int64_t N = (int64_t)n * n * n;
    if (zero_guess) PM_TRY(cuda_status(cudaMemsetAsync(g.u[l], 0, N * g.B * sizeof(float), g.s)));
    else if (scaled)
      PM_LAUNCH(K_MG_GUESS, 8.0 * N * g.B, k_scale, g.grid(grid_for(N, 256)), 256, 0, g.s, g.u[l], N, g.gscale, sbox);
  } else {
    for (int si = 0; si < p.npre; ++si) w[si] = si == 0 ? 1.0f : p.omega;
    PM_TRY(smooth(g, l, p.npre, w, zero_guess, scaled ? g.gscale : 1.0f, sbox));
  }
  const int64_t nc = ((int64_t)n * n * n) / 8;
  const unsigned grid = grid_for(nc, 256);
  if (l == 0)
    PM_LAUNCH(K_MG_RESTRICT, 68.0 * nc * g.B, k_resid_restrict<true>, g.grid(grid), 256, 0, g.s, g.u[l], g.f[l],
              log2n, (float)n * (float)n, const_cast<float*>(g.f[l + 1].p));
  else
    PM_LAUNCH(K_MG_RESTRICT, 68.0 * nc * g.B, k_resid_restrict<false>, g.grid(grid), 256, 0, g.s, g.u[l], g.f[l],
              log2n, (float)n * (float)n, const_cast<float*>(g.f[l + 1].p));
  PM_TRY(v_cycle(g, l + 1, true));
  PM_LAUNCH(K_MG_PROLONG, 68.0 * nc * g.B, k_prolong_correct, g.grid(grid_for(nc / 2, 256)), 256, 0, g.s, g.u[l],
            g.u[l + 1], (const float*)nullptr, log2n);
  if (p.npost > 0) {
    for (int si = 0; si < p.npost; ++si) w[si] = si == p.npost - 1 ? 1.0f : p.omega;
    PM_TRY(smooth(g, l, p.npost, w, false, 1.0f));
  }
  return PM_OK;
}

}  // namespace

pm_status prolong_correct_launch(float* u, const float* uc, const float* uc2, int n_fine, int cls,
                                 cudaStream_t s, int B) {
  const int64_t N = (int64_t)n_fine * n_fine * n_fine;
  PM_LAUNCH(cls, (8.0 * N + (uc2 ? 1.0 : 0.5) * N) * B, k_prolong_correct, dim3(grid_for(N / 16, 256), 1, (unsigned)B),
            256, 0, s, u, uc, uc2, ilog2(n_fine));
  return PM_OK;
}

pm_status fetch_scalars(const double* dev, double* host, int count, cudaStream_t s) {
  static double* pinned = nullptr;
  if (!pinned) PM_TRY(cuda_status(cudaHostAlloc((void**)&pinned, 64 * sizeof(double), cudaHostAllocPortable)));
  PM_TRY(cuda_status(cudaMemcpyAsync(pinned, dev, count * sizeof(double), cudaMemcpyDeviceToHost, s)));
  PM_TRY(cuda_status(cudaStreamSynchronize(s)));
  for (int i = 0; i < count; ++i) host[i] = pinned[i];
  return PM_OK;
}

pm_status mg_solve_batch_src(Src f, float* phi, int n, int B, const mg_params& prm, const float* gbox, Workspace& w,
                         cudaStream_t s) {
  if (B < 1 || prm.fixed_cycles < 1) return PM_EINVAL;
  MG g;
  g.n0 = n;
  g.p = &prm;
  g.s = s;
  g.B = B;
  g.u[0] = phi;
  g.f[0] = f;
  for (int l = 0; l < 12; ++l) {
    if (l > 0) {
      g.u[l] = w.mg_u[l];
      g.f[l] = Src{w.mg_f[l], 1.0f, nullptr};
    }
    g.alt[l] = w.mg_alt[l];
  }
  PM_TRY(stream_attributes());
  g.first_cycle = true;
  g.gscale = 1.0f;
  g.gbox = prm.first_guess == MG_GUESS_SCALED ? gbox : nullptr;
  const int64_t N = (int64_t)n * n * n;
  const float h2 = 1.0f / ((float)n * (float)n);
  if (prm.first_guess == MG_GUESS_JACOBI)
    PM_LAUNCH(K_MG_GUESS, 8.0 * N * B, k_jacobi_guess, g.grid(grid_for(N, 256)), 256, 0, s, phi, f, N, h2);
  for (int c = 0; c < prm.fixed_cycles; ++c) {
    PM_TRY(v_cycle(g, 0, false));
    g.first_cycle = false;
    if (g.u[0] != phi) {   // the iterate ended in the ping-pong partner: bring it home
      PM_TRY(cuda_status(cudaMemcpyAsync(phi, g.u[0], N * B * sizeof(float), cudaMemcpyDeviceToDevice, s)));
      g.alt[0] = g.u[0];
      g.u[0] = phi;
    }
  }
  return launch_status();
}

pm_status mg_solve_src(Src f, float* phi, int n, const mg_params& prm, mg_stats* st, Workspace& w,
                       cudaStream_t s) {
  MG g;
  g.n0 = n;
  g.p = &prm;
  g.s = s;
  g.u[0] = phi;
  g.f[0] = f;
  for (int l = 0; l < 12; ++l) {
    if (l > 0) {
      g.u[l] = w.mg_u[l];
      g.f[l] = Src{w.mg_f[l], 1.0f, nullptr};
    }
    g.alt[l] = w.mg_alt[l];
  }
  PM_TRY(stream_attributes());
  g.first_cycle = true;
  g.gscale = prm.first_guess == MG_GUESS_SCALED ? prm.guess_scale : 1.0f;
  const int64_t N = (int64_t)n * n * n;
  const float h2 = 1.0f / ((float)n * (float)n);
  if (prm.first_guess == MG_GUESS_JACOBI)
    PM_LAUNCH(K_MG_GUESS, 8.0 * N, k_jacobi_guess, grid_for(N, 256), 256, 0, s, phi, f, N, h2);
  mg_stats local{PM_OK, 0, -1.0, -1.0, -1.0};
  auto cycle = [&]() -> pm_status {
    PM_TRY(v_cycle(g, 0, false));
    g.first_cycle = false;
    if (g.u[0] != phi) {   // the iterate ended in the ping-pong partner: bring it home
      PM_TRY(cuda_status(cudaMemcpyAsync(phi, g.u[0], N * sizeof(float), cudaMemcpyDeviceToDevice, s)));
      g.alt[0] = g.u[0];
      g.u[0] = phi;
    }
    return PM_OK;
  };
  if (prm.fixed_cycles > 0) {
    for (int c = 0; c < prm.fixed_cycles; ++c) PM_TRY(cycle());
    local.cycles = prm.fixed_cycles;
    if (st) *st = local;
    return launch_status();
  }
  const int log2n = ilog2(n);
  const unsigned nb = grid_for(N, 256, 152 * 8);
  double prev = -1.0;
  pm_status status = PM_ENOCONV;
  for (int c = 0; c < prm.max_cycles; ++c) {
    PM_TRY(cycle());
    local.cycles = c + 1;
    PM_LAUNCH(K_MG_NORM, 8.0 * N, k_resid_norm, nb, 256, 0, s, phi, f, log2n, (float)n * (float)n, w.partials);
    PM_TRY(reduce_partials(w.partials, nb, nb, 2, 1.0, w.scalars + 4, s));
    double h[2];
    PM_TRY(fetch_scalars(w.scalars + 4, h, 2, s));
    const double res = sqrt(h[0]), nf = sqrt(h[1]);
    local.res = res;
    local.norm_f = nf;
    if (!isfinite(res)) { status = PM_ENAN; break; }
    if (res <= prm.tol * nf) { status = PM_OK; break; }
    // a cycle that gained less than 1/stall ends the solve only near the
    // float32 floor of the stored iterate (residual below 1e-3 of the source)
    if (prev > 0.0 && prm.stall > 0.0 && res > prm.stall * prev && res <= 1e-3 * nf) { status = PM_OK; break; }
    prev = res;
  }
  local.status = status;
  if (st) *st = local;
  PM_TRY(launch_status());
  return status;
}

pm_status mg_solve_refine_src(const float* f, const double* fmean, double* phi, int n, int outer,
                              const mg_params& prm, mg_stats* st, Workspace& w, cudaStream_t s) {
  const int64_t N = (int64_t)n * n * n;
  const int log2n = ilog2(n);
  const unsigned nb = grid_for(N, 256, 152 * 8);
  const double inv_h2 = (double)n * (double)n;
  mg_params cp = prm;
  cp.first_guess = MG_GUESS_INPUT;   // the correction starts from zero
  mg_stats local{PM_OK, 0, -1.0, -1.0, -1.0};
  // float64 residual of the current iterate into w.ref_r; its norm and ||f - <f>||
  auto residual = [&](double* res, double* nf) -> pm_status {
    PM_LAUNCH(K_MG_NORM, 16.0 * N, k_resid_f64, nb, 256, 0, s, phi, f, fmean, log2n, inv_h2, w.ref_r, w.partials);
    PM_TRY(reduce_partials(w.partials, nb, nb, 2, 1.0, w.scalars + 20, s));
    double h[2];
    PM_TRY(fetch_scalars(w.scalars + 20, h, 2, s));
    *res = sqrt(h[0]);
    *nf = sqrt(h[1]);
    return PM_OK;
  };
  pm_status status = PM_OK;
  for (int it = 0; it <= outer; ++it) {
    double res, nf;
    PM_TRY(residual(&res, &nf));
    if (it == 0) local.res0 = res;
    local.res = res;
    local.norm_f = nf;
    if (!isfinite(res)) { status = PM_ENAN; break; }
    if (it == outer || res == 0.0) break;
    // correction: (L(e) - 6e)/h^2 = r - <r>, float32 multigrid from e = 0
    PM_TRY(grid_mean(w.ref_r, N, w.partials, w.scalars + 22, s));
    PM_TRY(cuda_status(cudaMemsetAsync(w.ref_e, 0, N * sizeof(float), s)));
    mg_stats cst;
    const pm_status r = mg_solve_src(Src{w.ref_r, 1.0f, w.scalars + 22, nullptr}, w.ref_e, n, cp, &cst, w, s);
    if (r != PM_OK && r != PM_ENOCONV) return r;
    local.cycles += cst.cycles;
    PM_LAUNCH(K_MISC, 20.0 * N, k_add_correction_f64, grid_for(N, 256), 256, 0, s, phi, w.ref_e, N);
  }
  local.status = status;
  if (st) *st = local;
  PM_TRY(launch_status());
  return status;
}

}  // namespace pmgb
