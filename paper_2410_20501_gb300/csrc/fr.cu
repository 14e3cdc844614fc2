// Hu-Sawicki f(R) scalaron (n = 1 and n = 2) by non-linear FAS multigrid
// (§3.6.2, §3.10).  The kernels are templates on the exponent NH; the text
// below is for n = 1, and n = 2 follows the same pattern with u^3:
//   N_h(eps) = (fbar/h^2) sum_nb (eps_nb - eps)(3 + 3 eps_nb + 3 eps + eps_nb^2
//              + eps_nb eps + eps^2) + kappa eps/(1 + eps),
//   eps^4 + 4 eps^3 + 6 eps^2 + c1 eps + c0 = 0, c1 = 3 + beta (b - kappa) - T/6,
//   c0 = beta b - T/6, T = sum_nb eps_nb (3 + 3 eps_nb + eps_nb^2)
// (u^4 + p u + q = 0, the quartic of §3.10, with u = 1 + eps).
//
// Unknown: eps = u - 1 with u = (f~_R / fbar)^(1/2).  Discrete operator
//   N_h(eps) = (fbar/h^2) sum_nb (eps_nb - eps)(2 + eps_nb + eps) + kappa eps/(1 + eps)
// (= (fbar/h^2)(L(u^2) - 6u^2) - kappa (1/u - 1) written in differences, so the
// O(1) background cancels analytically), equation N_h(eps) = b.
// Gauss-Seidel: with the neighbours fixed, u solves the depressed cubic
// u^3 + p u + q = 0 of Eq. fr_depressed_equation; in eps it reads
//   eps^3 + 3 eps^2 + c1 eps + c0 = 0,
//   c1 = 2 + beta (b - kappa) - S/6,  c0 = beta b - S/6,
//   S = sum_nb eps_nb (2 + eps_nb),   beta = h^2 / (6 fbar),  q = beta kappa < 0,
// whose unique root eps > -1 is found in float32 by safeguarded Newton (the
// paper evaluates the closed-form root in float64, which the eps form makes
// unnecessary: no term of size 1 is ever subtracted).
#include <math.h>

#include "pm_device.cuh"
#include "pm_internal.cuh"
#include "rb_fused.cuh"
#include "rb_stream.cuh"

namespace pmgb {

namespace {

__device__ __forceinline__ float load_mean(const Src& f) { return f.mean ? (float)*f.mean : 0.0f; }
__device__ __forceinline__ float src_at(const Src& f, int64_t i, float mean) {
  return f.s * (__ldg(f.p + i) - mean);
}
// Offset of cell (i, j, k) inside one box (n <= 1024: below 2^30).
__device__ __forceinline__ uint32_t idx3(int i, int j, int k, int log2n) {
  return ((uint32_t)i << (2 * log2n)) | ((uint32_t)j << log2n) | (uint32_t)k;
}

// Root eps > -1 of g(e) = e^3 + 3e^2 + c1 e + c0 (g(-1) = q < 0, g convex on
// e > -1, so the root is unique).  One Halley step from the current value
// reaches float32 resolution in a warm sweep (the value moved little since
// the last one); otherwise up to two plain Newton steps from the Halley
// point, then Newton inside a shrinking bracket [lo, hi]; when a step leaves
// the bracket (or g' <= 0) the upper end is set from the bound
// u* <= sqrt(max(-p, 0)) + (-q)^(1/3), p = c1 - 3, and the step falls back to
// bisection.  Stops when g is at its float32 rounding level or the step is
// below 2e-7 relative.
// g(e) of the cell equation in eps = u - 1 (NH = 1: cubic, NH = 2: quartic),
// its derivative, half its second and a sixth of its third derivative, the
// float32 rounding level of its evaluation, and an upper bound of the root
// (from u* <= sqrt(max(-p, 0)) + (-q)^(1/3) for the cubic,
// u* <= max(1, (|p| + |q|)^(1/3)) for the quartic).
template <int NH> struct CellPoly;
template <> struct CellPoly<1> {
  __device__ static float g(float e, float c1, float c0) { return ((e + 3.0f) * e + c1) * e + c0; }
  __device__ static float gp(float e, float c1) { return (3.0f * e + 6.0f) * e + c1; }
  __device__ static float half_gpp(float e) { return 3.0f * e + 3.0f; }
  __device__ static float sixth_gppp(float) { return 1.0f; }
  __device__ static float noise(float e, float c1, float c0) {
    const float e2 = e * e;
    return 1.5e-7f * (fabsf(c0) + fabsf(c1 * e) + 3.0f * e2 + fabsf(e2 * e));
  }
  __device__ static float upper(float c1, float q, float lo) {
    return fmaxf(sqrtf(fmaxf(3.0f - c1, 0.0f)) + cbrtf(-q) - 1.0f, lo);
  }
};
template <> struct CellPoly<2> {
  __device__ static float g(float e, float c1, float c0) { return (((e + 4.0f) * e + 6.0f) * e + c1) * e + c0; }
  __device__ static float gp(float e, float c1) { return ((4.0f * e + 12.0f) * e + 12.0f) * e + c1; }
  __device__ static float half_gpp(float e) { const float u = e + 1.0f; return 6.0f * u * u; }
  __device__ static float sixth_gppp(float e) { return 4.0f * (e + 1.0f); }
  __device__ static float noise(float e, float c1, float c0) {
    const float e2 = e * e;
    return 1.5e-7f * (fabsf(c0) + fabsf(c1 * e) + 6.0f * e2 + 4.0f * fabsf(e2 * e) + e2 * e2);
  }
  __device__ static float upper(float c1, float q, float lo) {
    return fmaxf(fmaxf(cbrtf(fabsf(c1 - 4.0f) + fabsf(q)), 1.0f) - 1.0f, lo);
  }
};

template <int NH>
__device__ __forceinline__ float fr_root(float e, float c1, float c0, float q) {
  using P = CellPoly<NH>;
  float lo = -1.0f, hi = __int_as_float(0x7f800000);  // +inf until needed
  if (!(e > lo)) e = 0.0f;
  {
    // Halley: e1 = e - g g' / (g'^2 - g g''/2); its remaining error is about
    // C d^3 for a step d, C = (g''/2g')^2 - g'''/(6 g') (Halley's cubic error
    // constant), tested without a division
    const float g0 = P::g(e, c1, c0), gp0 = P::gp(e, c1), hg = P::half_gpp(e);
    const float den = gp0 * gp0 - g0 * hg;
    const float e1 = e - __fdividef(g0 * gp0, den);
    if (gp0 > 0.0f && den > 0.0f && e1 > lo) {
      const float d = e1 - e;
      if (fabsf(hg * hg - P::sixth_gppp(e) * gp0) * fabsf(d * d * d) <= (1e-7f * fabsf(e1) + 1e-20f) * (gp0 * gp0))
        return e1;
      e = e1;   // not yet at resolution: the Newton steps start from here
    }
  }
  {
    // one or two plain Newton steps;
    // accepted when the remaining error is at float32 resolution and the root
    // is admissible.  Newton's error after a step of length d is about K d^2,
    // K = g''/(2 g')
    const float g0 = P::g(e, c1, c0), gp0 = P::gp(e, c1);
    const float e1 = e - __fdividef(g0, gp0);
    {
      const float d0 = e1 - e;
      if (gp0 > 0.0f && e1 > lo && d0 * d0 * P::half_gpp(e) <= (1e-7f * fabsf(e1) + 1e-20f) * gp0) return e1;
    }
    const float g1 = P::g(e1, c1, c0), gp1 = P::gp(e1, c1);
    const float e2 = e1 - __fdividef(g1, gp1);
    // the same test for the second step, d = e2 - e1
    const float d = e2 - e1;
    if (gp0 > 0.0f && gp1 > 0.0f && e2 > lo && d * d * P::half_gpp(e1) <= (1e-7f * fabsf(e2) + 1e-20f) * gp1)
      return e2;
    if (gp1 > 0.0f && e2 > lo) e = e2;   // continue from the better point
  }
  for (int it = 0; it < 30; ++it) {
    const float g = P::g(e, c1, c0);
    const float gp = P::gp(e, c1);
    if (g > 0.0f) hi = fminf(hi, e);
    else if (g < 0.0f) lo = fmaxf(lo, e);
    else return e;
    if (fabsf(g) <= P::noise(e, c1, c0)) return e;
    float en = gp > 0.0f ? e - __fdividef(g, gp) : lo;
    if (!(en > lo && en < hi)) {
      if (isinf(hi)) hi = P::upper(c1, q, lo);
      en = 0.5f * (lo + hi);
    }
    if (fabsf(en - e) <= 2e-7f * fabsf(en) + 1e-12f) return en;
    e = en;
  }
  return e;
}

__device__ __forceinline__ void load_nb(const float* u, int i, int j, int k, int log2n, float nb[6]) {
  const int m = (1 << log2n) - 1;
  nb[0] = u[idx3((i + 1) & m, j, k, log2n)];
  nb[1] = u[idx3((i - 1) & m, j, k, log2n)];
  nb[2] = u[idx3(i, (j + 1) & m, k, log2n)];
  nb[3] = u[idx3(i, (j - 1) & m, k, log2n)];
  nb[4] = u[idx3(i, j, (k + 1) & m, log2n)];
  nb[5] = u[idx3(i, j, (k - 1) & m, log2n)];
}

// N_h(eps) at one cell: (fbar/h^2) sum_nb (u_nb^(n+1) - u^(n+1)) written in
// differences, plus kappa eps/(1 + eps).
template <int NH>
__device__ __forceinline__ float fr_op(float ec, const float nb[6], float alpha, float kappa) {
  float L = 0.0f;
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    if (NH == 1) {
      L = fmaf(nb[q] - ec, 2.0f + nb[q] + ec, L);
    } else {   // u_nb^3 - u^3 = (e_nb - e)(3 + 3 (e_nb + e) + e_nb^2 + e_nb e + e^2)
      const float s = nb[q] + ec;
      L = fmaf(nb[q] - ec, fmaf(3.0f, s, 3.0f) + fmaf(nb[q], s, ec * ec), L);
    }
  }
  return alpha * L + kappa * ec / (1.0f + ec);
}

template <int NH>
__device__ __forceinline__ float fr_update(float ec, const float nb[6], float bv, float beta, float kappa,
                                           float q) {
  float S = 0.0f;
#pragma unroll
  for (int t = 0; t < 6; ++t)
    S = NH == 1 ? fmaf(nb[t], 2.0f + nb[t], S) : fmaf(nb[t], fmaf(nb[t], 3.0f + nb[t], 3.0f), S);
  const float S6 = S * (1.0f / 6.0f);
  const float c1 = (NH == 1 ? 2.0f : 3.0f) + beta * (bv - kappa) - S6;
  const float c0 = beta * bv - S6;
  return fr_root<NH>(ec, c1, c0, q);
}

template <int NH>
__global__ void __launch_bounds__(256) k_fr_sweep(float* __restrict__ e, Src b, int log2n, int colour, float beta,
                                                  float kappa, float q) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (1u << (3 * log2n - 1))) return;
  {   // the box of a batched launch
    const int64_t N = (int64_t)1 << (3 * log2n);
    e += (int64_t)blockIdx.z * N;
    b = box_src(b, N);
  }
  const uint32_t m = (1u << log2n) - 1;
  const uint32_t kk = t & ((1u << (log2n - 1)) - 1), row = t >> (log2n - 1);
  const uint32_t j = row & m, i = row >> log2n;
  const uint32_t k = 2 * kk + ((colour + i + j) & 1);
  const uint32_t c = (row << log2n) | k;
  uint32_t qi[6];
  nb_index(c, i, j, k, log2n, qi);
  float nb[6];
#pragma unroll
  for (int r = 0; r < 6; ++r) nb[r] = e[qi[r]];
  const float bv = b.s * (__ldg(b.p + c) - load_mean(b));
  e[c] = fr_update<NH>(e[c], nb, bv, beta, kappa, q);
}

// The non-linear flux of N_h through one face, (u_nb^(n+1) - u^(n+1)) in
// eps differences; it changes sign with the face's orientation.
template <int NH>
__device__ __forceinline__ float fr_flux(float enb, float ec) {
  if (NH == 1) return (enb - ec) * (2.0f + enb + ec);
  const float s = enb + ec;
  return (enb - ec) * (fmaf(3.0f, s, 3.0f) + fmaf(enb, s, ec * ec));
}

// eH = rH = R eps, bH = R(b - N_h eps).  Summed over the 2x2x2 block the
// fluxes through the 12 inner faces cancel pairwise, so only the 24 outer
// faces enter the restricted operator.  BOXES: a batched launch (box =
// blockIdx.z); the single-box form keeps its own register allocation.
template <int NH, bool BOXES>
__global__ void k_fr_restrict(const float* __restrict__ e, Src b, int log2n, float alpha, float kappa,
                              float* __restrict__ eH, float* __restrict__ rH, float* __restrict__ bH) {
  const int lc = log2n - 1, mc = (1 << lc) - 1;
  const int64_t total = (int64_t)1 << (3 * lc);
  if (BOXES) {   // the box of a batched launch
    e += (int64_t)blockIdx.z << (3 * log2n);
    b = box_src(b, (int64_t)1 << (3 * log2n));
    const int64_t offc = (int64_t)blockIdx.z * total;
    eH += offc;
    rH += offc;
    bH += offc;
  }
  const float mean = load_mean(b);
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    const int K = (int)(t & mc), J = (int)((t >> lc) & mc), I = (int)(t >> (2 * lc));
    float core[2][2][4], xf[2][2][2], yf[2][2][2];
    load_children_block(e, I, J, K, log2n, core, xf, yf);
    float se = 0.0f, sb = 0.0f, sk = 0.0f;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int bb = 0; bb < 2; ++bb) {
        const float2 br = __ldg(reinterpret_cast<const float2*>(b.p + idx3(2 * I + a, 2 * J + bb, 2 * K, log2n)));
        sb += b.s * (br.x - mean) + b.s * (br.y - mean);
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
          const float ec = core[a][bb][cc + 1];
          se += ec;
          sk += ec / (1.0f + ec);
        }
      }
    float L[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int side = 0; side < 2; ++side) {
          L[0] += fr_flux<NH>(xf[side][p][c], core[side][p][c + 1]);       // x faces of children (side, p, c)
          L[1] += fr_flux<NH>(yf[p][side][c], core[p][side][c + 1]);       // y faces of children (p, side, c)
          L[2] += fr_flux<NH>(core[p][c][side ? 3 : 0], core[p][c][side ? 2 : 1]);   // z faces of (p, c, side)
        }
    const float ops = fmaf(alpha, (L[0] + L[1]) + L[2], kappa * sk);
    eH[t] = 0.125f * se;
    rH[t] = 0.125f * se;
    bH[t] = 0.125f * (sb - ops);
  }
}

// bH += N_H(eH).  A thread takes four consecutive z cells of a row (n >= 4):
// the rows at x +- 1, y +- 1 and its own in 16-byte loads, plus the two z
// neighbours beyond the run; each cell sees its neighbours in the order
// x+, x-, y+, y-, z+, z- as everywhere else.
template <int NH>
__global__ void k_fr_coarse_op(const float* __restrict__ eH, float* __restrict__ bH, int log2n, float alpha,
                               float kappa) {
  const uint32_t m = (1u << log2n) - 1;
  const uint32_t quads = 1u << (3 * log2n - 2);
  {   // the box of a batched launch
    const int64_t off = (int64_t)blockIdx.z << (3 * log2n);
    eH += off;
    bH += off;
  }
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < quads; t += gridDim.x * blockDim.x) {
    const uint32_t c0 = t << 2;
    const uint32_t k0 = c0 & m, j = (c0 >> log2n) & m, i = c0 >> (2 * log2n);
    auto rowp = [&](uint32_t ii, uint32_t jj) -> const float* {
      return eH + (((ii & m) << (2 * log2n)) | ((jj & m) << log2n));
    };
    const float* rc = rowp(i, j);
    const float4 C = __ldg(reinterpret_cast<const float4*>(rc + k0));
    const float4 XP = __ldg(reinterpret_cast<const float4*>(rowp(i + 1, j) + k0));
    const float4 XM = __ldg(reinterpret_cast<const float4*>(rowp(i - 1, j) + k0));
    const float4 YP = __ldg(reinterpret_cast<const float4*>(rowp(i, j + 1) + k0));
    const float4 YM = __ldg(reinterpret_cast<const float4*>(rowp(i, j - 1) + k0));
    const float zl = __ldg(rc + ((k0 - 1) & m)), zr = __ldg(rc + ((k0 + 4) & m));
    float4* bp = reinterpret_cast<float4*>(bH + c0);
    float4 B = *bp;
    const float e[4] = {C.x, C.y, C.z, C.w}, xp[4] = {XP.x, XP.y, XP.z, XP.w}, xm[4] = {XM.x, XM.y, XM.z, XM.w},
                yp[4] = {YP.x, YP.y, YP.z, YP.w}, ym[4] = {YM.x, YM.y, YM.z, YM.w};
    float r[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float nb[6] = {xp[q], xm[q], yp[q], ym[q], q < 3 ? e[q + 1] : zr, q > 0 ? e[q - 1] : zl};
      r[q] = fr_op<NH>(e[q], nb, alpha, kappa);
    }
    B.x += r[0];
    B.y += r[1];
    B.z += r[2];
    B.w += r[3];
    *bp = B;
  }
}

template <int NH>
__global__ void __launch_bounds__(256) k_fr_norm(const float* __restrict__ e, Src b, int log2n, float alpha,
                                                 float kappa, double* __restrict__ partial) {
  __shared__ double scratch[32];
  const float mean = load_mean(b);
  const int m = (1 << log2n) - 1;
  const int64_t total = (int64_t)1 << (3 * log2n);
  float sd = 0.0f, cd = 0.0f, sb = 0.0f, cb = 0.0f;
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < total; c += gridDim.x * blockDim.x) {
    const int k = (int)(c & m), j = (int)((c >> log2n) & m), i = (int)(c >> (2 * log2n));
    float nb[6];
    load_nb(e, i, j, k, log2n, nb);
    const float bv = src_at(b, c, mean);
    const float d = bv - fr_op<NH>(e[c], nb, alpha, kappa);
    kahan_add(sd, cd, d * d);
    kahan_add(sb, cb, bv * bv);
  }
  block_sum_to(partial + blockIdx.x, sd, cd, scratch);
  block_sum_to(partial + gridDim.x + blockIdx.x, sb, cb, scratch);
}

// Coarsest level (n <= 16) in one CTA: non-linear sweeps until the residual
// dropped by `drop`, its running minimum stalls for 5 sweeps (float32 floor), or
// `max_sweeps` sweeps.
template <int NH>
__global__ void __launch_bounds__(1024) k_fr_coarse(float* __restrict__ e, Src b, int log2n, float alpha,
                                                    float beta, float kappa, float q, int max_sweeps,
                                                    float drop) {
  __shared__ float se[4096], sbv[4096];
  __shared__ float2 scratch[33];
  const int n = 1 << log2n, m = n - 1, N = n * n * n;
  e += (int64_t)blockIdx.z * N;   // one CTA per box of a batched launch
  b = box_src(b, N);
  const float mean = load_mean(b);
  for (int c = threadIdx.x; c < N; c += blockDim.x) {
    se[c] = e[c];
    sbv[c] = src_at(b, c, mean);
  }
  __syncthreads();
  auto nbs = [&](int c, float nb[6]) {
    const int k = c & m, j = (c >> log2n) & m, i = c >> (2 * log2n);
    nb[0] = se[(((i + 1) & m) << (2 * log2n)) | (j << log2n) | k];
    nb[1] = se[(((i - 1) & m) << (2 * log2n)) | (j << log2n) | k];
    nb[2] = se[(i << (2 * log2n)) | (((j + 1) & m) << log2n) | k];
    nb[3] = se[(i << (2 * log2n)) | (((j - 1) & m) << log2n) | k];
    nb[4] = se[(i << (2 * log2n)) | (j << log2n) | ((k + 1) & m)];
    nb[5] = se[(i << (2 * log2n)) | (j << log2n) | ((k - 1) & m)];
  };
  // squared residual norm: per-thread compensated sums, then a compensated
  // float pair over the block, the same in every thread
  auto norm2 = [&]() -> float {
    float s = 0.0f, cmp = 0.0f;
    for (int c = threadIdx.x; c < N; c += blockDim.x) {
      float nb[6];
      nbs(c, nb);
      const float d = sbv[c] - fr_op<NH>(se[c], nb, alpha, kappa);
      kahan_add(s, cmp, d * d);
    }
    const float2 r = block_pair_sum(s, cmp, scratch);
    return r.x + r.y;
  };
  float best = norm2();
  const float target = drop * drop * best;
  int stale = 0;
  // the cell of pair P (cells 2P, 2P + 1: same i, j) with colour col: k of
  // 2P is even, so its colour is (i + j) & 1; every thread gets one cell of a
  // pair per colour pass (the cells of one colour are independent)
  auto cell_of = [&](int P, int col) -> int {
    const int c0 = P << 1;
    return c0 + ((col ^ ((c0 >> log2n) + (c0 >> (2 * log2n)))) & 1);
  };
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    for (int colour = 0; colour < 2; ++colour) {
      for (int P = threadIdx.x; P < (N >> 1); P += blockDim.x) {
        const int c = cell_of(P, colour);
        float nb[6];
        nbs(c, nb);
        se[c] = fr_update<NH>(se[c], nb, sbv[c], beta, kappa, q);
      }
      __syncthreads();
    }
    const float r = norm2();
    if (r <= target) break;
    if (r < 0.998f * best) {   // squared norms: a 0.1% improvement of the norm
      best = r;
      stale = 0;
    } else if (++stale >= 5) {
      break;                  // no progress for 5 sweeps: the float32 floor
    }
  }
  for (int c = threadIdx.x; c < N; c += blockDim.x) e[c] = se[c];
}

// The non-linear Gauss-Seidel update as a functor for the streaming smoother.
template <int NH>
struct FRUpdate {
  float beta, kappa, q;
  __device__ __forceinline__ FRUpdate box(int) const { return *this; }
  __device__ __forceinline__ float operator()(float old, const float nb[6], float bv, int, bool, bool) const {
    return fr_update<NH>(old, nb, bv, beta, kappa, q);
  }
};

struct FR {
  int n0;
  const fr_params* p;
  cudaStream_t s;
  float* e[12];
  float* alt[12];   // ping-pong partner for the streaming smoother (or NULL)
  float* r[12];
  Src b[12];
  double fbar, kappa;
  int nh;           // Hu-Sawicki exponent (1 or 2)
  int B = 1;        // boxes of a batched solve (blockIdx.z of every launch)
  dim3 grid(unsigned gx) const { return dim3(gx, 1, (unsigned)B); }
};

// Runs the statement with the compile-time exponent NH of f.
#define FR_NH(f, ...)                      \
  do {                                     \
    if ((f).nh == 2) {                     \
      constexpr int NH = 2;                \
      __VA_ARGS__;                         \
    } else {                               \
      constexpr int NH = 1;                \
      __VA_ARGS__;                         \
    }                                      \
  } while (0)

struct LevelConst {
  int n, log2n;
  float alpha, beta, kappa, q;
};

LevelConst level_const(const FR& f, int l) {
  LevelConst c;
  c.n = f.n0 >> l;
  c.log2n = ilog2(c.n);
  const double h = 1.0 / c.n, h2 = h * h;
  c.alpha = (float)(f.fbar / h2);
  c.beta = (float)(h2 / (6.0 * f.fbar));
  c.kappa = (float)f.kappa;
  c.q = (float)(h2 * f.kappa / (6.0 * f.fbar));
  return c;
}

// Resident CTAs per SM that the four-cell fused f(R) sweep's registers are
// sized for.
constexpr int kFrRunsMinBlocks = 3;

template <int NH>
pm_status stream_attributes_nh() {
  PM_TRY(smem_attr(k_rb_stream<2, FRUpdate<NH>>, StreamGeom<2>::smem_bytes));
  PM_TRY(smem_attr(k_rb_stream<1, FRUpdate<NH>>, StreamGeom<1>::smem_bytes));
  PM_TRY(smem_attr(k_rb_fused4<FRUpdate<NH>, kFrRunsMinBlocks>, kFusedSmem));
  return PM_OK;
}

pm_status stream_attributes(int nh) { return nh == 2 ? stream_attributes_nh<2>() : stream_attributes_nh<1>(); }

template <int NH>
pm_status fr_smooth_nh(FR& f, int l, int count) {
  using FRUpdate = ::pmgb::FRUpdate<NH>;
  const LevelConst c = level_const(f, l);
  const double N = (double)c.n * c.n * c.n * f.B;
  if (f.p->smoother == 0 && stream_ok(c.n) && f.alt[l] && f.B == 1) {
    int chunk, nitems;
    stream_plan(c.n, &chunk, &nitems);
    const unsigned grid = (unsigned)(nitems < 152 * 2 ? nitems : 152 * 2);   // 2 CTAs/SM (shared memory)
    const FRUpdate upd{c.beta, c.kappa, c.q};
    for (int done = 0; done < count;) {
      const int S = (count - done) >= 2 ? 2 : 1;
      if (S == 2)
        PM_LAUNCH(l == 0 ? K_FR_SMOOTH0 : K_FR_SMOOTH, 24.0 * N, (k_rb_stream<2, FRUpdate>), grid, kStreamThreads, StreamGeom<2>::smem_bytes,
                  f.s, f.e[l], f.alt[l], f.b[l], c.log2n, chunk, nitems, 0, upd);
      else
        PM_LAUNCH(l == 0 ? K_FR_SMOOTH0 : K_FR_SMOOTH, 12.0 * N, (k_rb_stream<1, FRUpdate>), grid, kStreamThreads, StreamGeom<1>::smem_bytes,
                  f.s, f.e[l], f.alt[l], f.b[l], c.log2n, chunk, nitems, 0, upd);
      float* t = f.e[l];
      f.e[l] = f.alt[l];
      f.alt[l] = t;
      done += S;
    }
    return PM_OK;
  }
  // a box of a batch takes the kernels it would take alone (fused_ok of one
  // box), so every box evolves bitwise as in a batch of one
  if (f.p->smoother == 2 && fused_ok(c.n) && f.alt[l] && fused_aligned(f.e[l], f.alt[l], f.b[l].p)) {
    const int chunk = fused_chunk(c.n);
    const dim3 grid = f.grid((unsigned)((c.n / kFusedT) * (c.n / kFusedT) * (c.n / chunk)));
    const FRUpdate upd{c.beta, c.kappa, c.q};
    for (int it = 0; it < count; ++it) {
      PM_LAUNCH(l == 0 ? K_FR_SMOOTH0 : K_FR_SMOOTH, 12.0 * N, (k_rb_fused4<FRUpdate, kFrRunsMinBlocks>), grid,
                kQuadThreads, kFusedSmem, f.s, f.e[l], f.alt[l], f.b[l], c.log2n, chunk, 0, 0, upd);
      float* t = f.e[l];
      f.e[l] = f.alt[l];
      f.alt[l] = t;
    }
    return PM_OK;
  }
  const dim3 grid = f.grid(grid_for(((int64_t)c.n * c.n * c.n) / 2, 256));
  for (int it = 0; it < count; ++it)
    for (int colour = 0; colour < 2; ++colour)
      PM_LAUNCH(l == 0 ? K_FR_SMOOTH0 : K_FR_SMOOTH, 6.0 * N, k_fr_sweep<NH>, grid, 256, 0, f.s, f.e[l], f.b[l],
                c.log2n, colour, c.beta, c.kappa, c.q);
  return PM_OK;
}

pm_status fr_smooth(FR& f, int l, int count) {
  return f.nh == 2 ? fr_smooth_nh<2>(f, l, count) : fr_smooth_nh<1>(f, l, count);
}

bool is_coarsest(const FR& f, int l) {
  const int n = f.n0 >> l;
  return n <= f.p->coarsest || n <= 4;
}

pm_status fr_coarse(FR& f, int l) {
  const LevelConst c = level_const(f, l);
  FR_NH(f, PM_LAUNCH(K_FR_COARSE, 12.0 * c.n * c.n * (double)c.n * f.B, k_fr_coarse<NH>, f.grid(1), 1024, 0, f.s,
                     f.e[l], f.b[l],
                     c.log2n, c.alpha, c.beta, c.kappa, c.q, f.p->coarse_max_sweeps, f.p->coarse_drop));
  return PM_OK;
}

// Pre-smooth level l, then build the FAS coarse problem on level l + 1.
pm_status fr_to_coarse(FR& f, int l) {
  PM_TRY(fr_smooth(f, l, f.p->npre));
  const LevelConst c = level_const(f, l), cH = level_const(f, l + 1);
  const int64_t nc = (int64_t)cH.n * cH.n * cH.n;
  if (f.B == 1)
    FR_NH(f, PM_LAUNCH(K_FR_RESTRICT, 76.0 * nc, (k_fr_restrict<NH, false>), grid_for(nc, 256), 256, 0, f.s, f.e[l],
                       f.b[l], c.log2n, c.alpha, c.kappa, f.e[l + 1], f.r[l + 1], const_cast<float*>(f.b[l + 1].p)));
  else
    FR_NH(f, PM_LAUNCH(K_FR_RESTRICT, 76.0 * nc * f.B, (k_fr_restrict<NH, true>), f.grid(grid_for(nc, 256)), 256, 0,
                       f.s, f.e[l], f.b[l], c.log2n, c.alpha, c.kappa, f.e[l + 1], f.r[l + 1],
                       const_cast<float*>(f.b[l + 1].p)));
  FR_NH(f, PM_LAUNCH(K_FR_COARSEOP, 12.0 * nc * f.B, k_fr_coarse_op<NH>, f.grid(grid_for(nc / 4, 256)), 256, 0, f.s,
                     f.e[l + 1], const_cast<float*>(f.b[l + 1].p), cH.log2n, cH.alpha, cH.kappa));
  return PM_OK;
}

pm_status fr_v(FR& f, int l) {
  if (is_coarsest(f, l)) return fr_coarse(f, l);
  PM_TRY(fr_to_coarse(f, l));
  PM_TRY(fr_v(f, l + 1));
  PM_TRY(prolong_correct_launch(f.e[l], f.e[l + 1], f.r[l + 1], f.n0 >> l, K_FR_PROLONG, f.s, f.B));
  return fr_smooth(f, l, f.p->npost);
}

pm_status fr_f(FR& f, int l) {
  if (is_coarsest(f, l)) return fr_coarse(f, l);
  PM_TRY(fr_to_coarse(f, l));
  PM_TRY(fr_f(f, l + 1));
  PM_TRY(prolong_correct_launch(f.e[l], f.e[l + 1], f.r[l + 1], f.n0 >> l, K_FR_PROLONG, f.s, f.B));
  return fr_v(f, l);
}

}  // namespace

void fr_background(const fr_params& p, double* fbar, double* kappa, double* c2) {
  const double a = p.a;
  const double Rbar = 3.0 * p.Om * (1.0 / (a * a * a) + 4.0 * p.OL / p.Om);
  const double Rbar0 = 3.0 * p.Om * (1.0 + 4.0 * p.OL / p.Om);
  const double ratio = Rbar0 / Rbar;
  *fbar = a * a * p.fR0 * (p.nhs == 2 ? ratio * ratio * ratio : ratio * ratio);   // (R0/R)^(n+1)
  const double ct = 299792.458 / (100.0 * p.boxsize);
  *c2 = ct * ct;
  *kappa = a * a * a * a * Rbar / (3.0 * *c2);
}

pm_status fr_solve_src(Src b, float* eps, int n, const fr_params& prm, mg_stats* st, Workspace& w,
                       cudaStream_t s, int B) {
  FR f;
  f.n0 = n;
  f.B = B;
  f.p = &prm;
  f.s = s;
  f.e[0] = eps;
  f.r[0] = nullptr;
  f.b[0] = b;
  for (int l = 0; l < 12; ++l) {
    if (l > 0) {
      f.e[l] = w.fr_e[l];
      f.r[l] = w.fr_r[l];
      f.b[l] = Src{w.fr_b[l], 1.0f, nullptr};
    }
    f.alt[l] = w.fr_alt[l];
  }
  f.nh = prm.nhs == 2 ? 2 : 1;
  PM_TRY(stream_attributes(f.nh));
  double c2;
  fr_background(prm, &f.fbar, &f.kappa, &c2);
  mg_stats local{PM_OK, 0, -1.0, -1.0, -1.0};
  const int64_t N0 = (int64_t)n * n * n * B;
  auto one = [&]() -> pm_status {
    PM_TRY(prm.cycle == 1 ? fr_f(f, 0) : fr_v(f, 0));
    if (f.e[0] != eps) {   // the iterate ended in the ping-pong partner: bring it home
      PM_TRY(cuda_status(cudaMemcpyAsync(eps, f.e[0], N0 * sizeof(float), cudaMemcpyDeviceToDevice, s)));
      f.alt[0] = f.e[0];
      f.e[0] = eps;
    }
    return PM_OK;
  };
  if (prm.tol <= 0.0 || B > 1) {
    for (int c = 0; c < prm.cycles; ++c) PM_TRY(one());
    local.cycles = prm.cycles;
    if (st) *st = local;
    return launch_status();
  }
  const LevelConst c0 = level_const(f, 0);
  const int64_t N = (int64_t)n * n * n;
  const unsigned nb = grid_for(N, 256, 152 * 8);
  pm_status status = PM_ENOCONV;
  for (int c = 0; c < prm.max_cycles; ++c) {
    PM_TRY(one());
    local.cycles = c + 1;
    FR_NH(f, PM_LAUNCH(K_FR_NORM, 8.0 * N, k_fr_norm<NH>, nb, 256, 0, s, eps, b, c0.log2n, c0.alpha, c0.kappa,
                       w.partials));
    PM_TRY(reduce_partials(w.partials, nb, nb, 2, 1.0, w.scalars + 8, s));
    double h[2];
    PM_TRY(fetch_scalars(w.scalars + 8, h, 2, s));
    local.res = sqrt(h[0]);
    local.norm_f = sqrt(h[1]);
    if (!isfinite(local.res)) { status = PM_ENAN; break; }
    if (local.res <= prm.tol * local.norm_f) { status = PM_OK; break; }
  }
  local.status = status;
  if (st) *st = local;
  PM_TRY(launch_status());
  return status;
}

}  // namespace pmgb
