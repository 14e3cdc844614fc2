// Adjoint (reverse-mode) kernels of the Newtonian PM step (§3.4-§3.7 forward
// operators, transposed):
//  - gradient: g = -G phi with the antisymmetric Table 1 stencil, so the
//    cotangent is phi_bar = G g_bar summed over axes (G^T = -G);
//  - Poisson: phi = A^+ s (rho - <rho>) with the self-adjoint 7-point
//    Laplacian, so rho_bar = s A^+ phi_bar (the same multigrid solve);
//  - inverse TSC a_p = sum_c W_pc g_c: g_bar = sum_p W_pc a_bar_p (a TSC
//    deposit of a_bar) and x_bar_p += n sum_c dW_pc (g_c . a_bar_p);
//  - TSC deposit rho_c = (n^3/N) sum_p W_pc: x_bar_p += (n^3/N) n sum_c dW_pc rho_bar_c;
//  - kick-drift: v' = v + a dt_kick, x' = x + v' dt_drift.
// dW is the derivative of the product of per-axis TSC weights with respect to
// the particle's offset along one axis (W_TSC is C1, so it is continuous).
#include "pm_device.cuh"
#include "pm_internal.cuh"

namespace pmgb {

namespace {

__device__ __forceinline__ void tsc_dweights(float d, float w[3]) {
  w[0] = d - 0.5f;          // d/dd of (1/2)(1/2 - d)^2
  w[1] = -2.0f * d;         // d/dd of 3/4 - d^2
  w[2] = 0.5f + d;          // d/dd of (1/2)(1/2 + d)^2
}

// a_bar = dt_kick (v_bar' + dt_drift x_bar'), the cotangent reaching the
// acceleration through the kick (x' = x + dt_drift v').
__global__ void k_adj_accel(const float* __restrict__ xbar_out, const float* __restrict__ vbar_out, int64_t np,
                            float dt_kick, float dt_drift, float* __restrict__ abar) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 3 * np;
       i += (int64_t)gridDim.x * blockDim.x)
    abar[i] = dt_kick * fmaf(dt_drift, __ldg(xbar_out + i), __ldg(vbar_out + i));
}

template <int ORDER> struct DStencil;
template <> struct DStencil<3> { static constexpr int R = 1; __device__ static float c(int) { return 0.5f; } };
template <> struct DStencil<5> {
  static constexpr int R = 2;
  __device__ static float c(int k) { return k == 1 ? 2.0f / 3.0f : -1.0f / 12.0f; }
};
template <> struct DStencil<7> {
  static constexpr int R = 3;
  __device__ static float c(int k) { return k == 1 ? 0.75f : (k == 2 ? -0.15f : 1.0f / 60.0f); }
};

// phi_bar = sum_d (1/h) sum_q c_q (g_bar_d(+q) - g_bar_d(-q)).
template <int ORDER>
__global__ void k_divergence(const float* __restrict__ gbar, float* __restrict__ phibar, int log2n, float inv_h) {
  const int64_t N = (int64_t)1 << (3 * log2n);
  const int m = (1 << log2n) - 1;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < N; c += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(c & m), j = (int)((c >> log2n) & m), i = (int)(c >> (2 * log2n));
    auto at = [&](int x, int y, int z) -> int64_t {
      return ((int64_t)(x & m) << (2 * log2n)) | ((int64_t)(y & m) << log2n) | (z & m);
    };
    float sx = 0.0f, sy = 0.0f, sz = 0.0f;
#pragma unroll
    for (int q = DStencil<ORDER>::R; q >= 1; --q) {
      const float w = DStencil<ORDER>::c(q);
      sx = fmaf(w, __ldg(gbar + at(i + q, j, k)) - __ldg(gbar + at(i - q, j, k)), sx);
      sy = fmaf(w, __ldg(gbar + N + at(i, j + q, k)) - __ldg(gbar + N + at(i, j - q, k)), sy);
      sz = fmaf(w, __ldg(gbar + 2 * N + at(i, j, k + q)) - __ldg(gbar + 2 * N + at(i, j, k - q)), sz);
    }
    phibar[c] = (sx + sy + sz) * inv_h;
  }
}

// Position (and velocity) cotangents of particle p (in the order of X):
//   x_bar = x_bar' + n [ J a_bar + s_rho R ],  J_de = sum_c d_d W g_e,c,
//   R_d = sum_c d_d W psi_c,   v_bar = v_bar' + dt_drift x_bar'.
// Any of g/abar, psi, xbar_out/vbar_out may be NULL (term absent).  With perm
// the results go to position perm[p] (back to the step's input order).
__global__ void __launch_bounds__(256) k_pos_grad(const uint32_t* __restrict__ X, int64_t np, int log2n,
                                                  const float* __restrict__ g, const float* __restrict__ abar,
                                                  const float* __restrict__ psi, float s_rho,
                                                  const float* __restrict__ xbar_out,
                                                  const float* __restrict__ vbar_out, float dt_drift,
                                                  const uint32_t* __restrict__ perm, float* __restrict__ xbar_in,
                                                  float* __restrict__ vbar_in) {
  const int m = (1 << log2n) - 1, sh = 32 - log2n;
  const int64_t N = (int64_t)1 << (3 * log2n);
  const float nf = (float)(1 << log2n);
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np;
       p += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t x = __ldg(X + p), y = __ldg(X + np + p), z = __ldg(X + 2 * np + p);
    float w[3][3], dw[3][3];
    const float dx = cell_offset(x, log2n), dy = cell_offset(y, log2n), dz = cell_offset(z, log2n);
    tsc_weights(dx, w[0]); tsc_weights(dy, w[1]); tsc_weights(dz, w[2]);
    tsc_dweights(dx, dw[0]); tsc_dweights(dy, dw[1]); tsc_dweights(dz, dw[2]);
    const int ix = (int)(x >> sh), iy = (int)(y >> sh), iz = (int)(z >> sh);
    float J[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
    float R[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int ox = 0; ox < 3; ++ox) {
      const int ci = (ix + ox - 1) & m;
#pragma unroll
      for (int oy = 0; oy < 3; ++oy) {
        const int cj = (iy + oy - 1) & m;
#pragma unroll
        for (int oz = 0; oz < 3; ++oz) {
          const int64_t c = ((int64_t)ci << (2 * log2n)) | ((int64_t)cj << log2n) | ((iz + oz - 1) & m);
          const float dwx = dw[0][ox] * w[1][oy] * w[2][oz];
          const float dwy = w[0][ox] * dw[1][oy] * w[2][oz];
          const float dwz = w[0][ox] * w[1][oy] * dw[2][oz];
          if (g) {
            const float g0 = __ldg(g + c), g1 = __ldg(g + N + c), g2 = __ldg(g + 2 * N + c);
            J[0][0] = fmaf(dwx, g0, J[0][0]); J[0][1] = fmaf(dwx, g1, J[0][1]); J[0][2] = fmaf(dwx, g2, J[0][2]);
            J[1][0] = fmaf(dwy, g0, J[1][0]); J[1][1] = fmaf(dwy, g1, J[1][1]); J[1][2] = fmaf(dwy, g2, J[1][2]);
            J[2][0] = fmaf(dwz, g0, J[2][0]); J[2][1] = fmaf(dwz, g1, J[2][1]); J[2][2] = fmaf(dwz, g2, J[2][2]);
          }
          if (psi) {
            const float r = __ldg(psi + c);
            R[0] = fmaf(dwx, r, R[0]); R[1] = fmaf(dwy, r, R[1]); R[2] = fmaf(dwz, r, R[2]);
          }
        }
      }
    }
    float a[3] = {0.f, 0.f, 0.f};
    if (abar) { a[0] = __ldg(abar + p); a[1] = __ldg(abar + np + p); a[2] = __ldg(abar + 2 * np + p); }
    const int64_t dst = perm ? (int64_t)__ldg(perm + p) : p;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const float xo = xbar_out ? __ldg(xbar_out + d * np + p) : 0.0f;
      const float term = J[d][0] * a[0] + J[d][1] * a[1] + J[d][2] * a[2] + s_rho * R[d];
      xbar_in[d * np + dst] = fmaf(nf, term, xo);
      if (vbar_in) {
        const float vo = vbar_out ? __ldg(vbar_out + d * np + p) : 0.0f;
        vbar_in[d * np + dst] = fmaf(dt_drift, xo, vo);
      }
    }
  }
}

template <int ORDER>
void launch_div(const float* gbar, float* phibar, int n, cudaStream_t s) {
  const int64_t N = (int64_t)n * n * n;
  PM_LAUNCH(K_ADJOINT, 16.0 * N, k_divergence<ORDER>, grid_for(N, 256), 256, 0, s, gbar, phibar, ilog2(n), (float)n);
}

}  // namespace

pm_status divergence_launch(const float* gbar, float* phibar, int n, int order, cudaStream_t s) {
  if (order == 3) launch_div<3>(gbar, phibar, n, s);
  else if (order == 5) launch_div<5>(gbar, phibar, n, s);
  else if (order == 7) launch_div<7>(gbar, phibar, n, s);
  else return PM_EINVAL;
  return launch_status();
}

pm_status adj_accel_launch(const float* xbar_out, const float* vbar_out, int64_t np, float dt_kick, float dt_drift,
                           float* abar, cudaStream_t s) {
  if (np == 0) return PM_OK;
  PM_LAUNCH(K_ADJOINT, 36.0 * np, k_adj_accel, grid_for(3 * np, 256), 256, 0, s, xbar_out, vbar_out, np, dt_kick,
            dt_drift, abar);
  return launch_status();
}

pm_status pos_grad_launch(const uint32_t* X, int64_t np, int n, const float* g, const float* abar, const float* psi,
                          float s_rho, const float* xbar_out, const float* vbar_out, float dt_drift,
                          const uint32_t* perm, float* xbar_in, float* vbar_in, cudaStream_t s) {
  if (np == 0) return PM_OK;
  const double N = (double)n * n * n;
  const double bytes = (g ? 12.0 * N : 0.0) + (psi ? 4.0 * N : 0.0) +
                       np * (12.0 + (abar ? 12.0 : 0.0) + (perm ? 4.0 : 0.0) + (xbar_out ? 12.0 : 0.0) +
                             (vbar_out ? 12.0 : 0.0) + 12.0 + (vbar_in ? 12.0 : 0.0));
  PM_LAUNCH(K_ADJOINT, bytes, k_pos_grad, grid_for(np, 256), 256, 0, s, X, np, ilog2(n), g, abar, psi, s_rho,
            xbar_out, vbar_out, dt_drift, perm, xbar_in, vbar_in);
  return launch_status();
}

}  // namespace pmgb
