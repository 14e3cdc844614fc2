// Poisson solve by 3-D FFT (§3.7): FFT_7pt (the Fourier symbol of the 7-point
// Laplacian, -(4/h^2) sum_d sin^2(pi m_d / n), no mass-assignment
// compensation) and FFT (-1 / (k^2 W_TSC(k)^2), W_TSC = prod_d sinc(pi m_d / n)^3).
//
// phi = scale * IFFT[ G(k) FFT[rho] ] with G(0) = 0 (which also removes the
// mean of rho).  The transforms are hand-written: a shared-memory Stockham
// FFT (radix 8, then 4 or 2; a thread holds 8 points per stage), twiddles from
// a float2 table built in float64 on the host.  Passes over HBM, with the
// half-spectrum C[x][y][kz], kz = 0 .. n/2, stored as float2 rows of n/2 + 1:
//   z: real rows -> n/2-point complex FFT of the even/odd pairs -> n/2 + 1
//      outputs (R2C);
//   y: forward FFT of the columns;
//   x: forward FFT of the columns, multiply by scale G and the transforms'
//      normalisation 2 / n^3, inverse FFT;
//   y: inverse FFT;  z: inverse C2R, real rows out.
// Each pass reads and writes the grid once (about 40 B per cell in all).
#include <math.h>
#include <mutex>
#include <vector>

#include "pm_device.cuh"
#include "pm_internal.cuh"

namespace pmgb {

namespace {

// Twiddle tables: the table of length L (a power of two, 2..1024) occupies
// g_tw[L .. 2L): g_tw[L + j] = exp(-2 pi i j / L).
__device__ float2 g_tw[2048];
constexpr int kMaxDev = 64;
bool g_tw_ready[kMaxDev];
std::mutex g_tw_mu;

pm_status twiddles_ready() {
  int dev = 0;
  PM_TRY(cuda_status(cudaGetDevice(&dev)));
  if (dev < 0 || dev >= kMaxDev) return PM_EINVAL;
  std::lock_guard<std::mutex> lock(g_tw_mu);
  if (g_tw_ready[dev]) return PM_OK;
  std::vector<float2> h(2048, make_float2(0.0f, 0.0f));
  for (int L = 2; L <= 1024; L *= 2)
    for (int j = 0; j < L; ++j) {
      const double a = -2.0 * M_PI * j / L;
      h[L + j] = make_float2((float)cos(a), (float)sin(a));
    }
  PM_TRY(cuda_status(cudaMemcpyToSymbol(g_tw, h.data(), h.size() * sizeof(float2))));
  g_tw_ready[dev] = true;
  return PM_OK;
}

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// multiply by -i (forward) or +i (inverse)
template <bool INV> __device__ __forceinline__ float2 mul_mi(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

template <bool INV> __device__ __forceinline__ void dft2(float2& a, float2& b) {
  const float2 t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

template <bool INV> __device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
  const float2 t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), t3 = mul_mi<INV>(csub(a1, a3));
  a0 = cadd(t0, t2);
  a2 = csub(t0, t2);
  a1 = cadd(t1, t3);
  a3 = csub(t1, t3);
}

// 8-point DFT in place (v[0..7] in natural order in and out).
template <bool INV> __device__ __forceinline__ void dft8(float2 v[8]) {
  float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<INV>(e0, e1, e2, e3);
  dft4<INV>(o0, o1, o2, o3);
  const float r = 0.70710678118654752f;
  // w8^k o_k, w8 = exp(-+ 2 pi i / 8)
  const float2 w1 = INV ? make_float2(r, r) : make_float2(r, -r);
  const float2 p1 = cmul(o1, w1);
  const float2 p2 = mul_mi<INV>(o2);
  const float2 w3 = INV ? make_float2(-r, r) : make_float2(-r, -r);
  const float2 p3 = cmul(o3, w3);
  v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
  v[1] = cadd(e1, p1); v[5] = csub(e1, p1);
  v[2] = cadd(e2, p2); v[6] = csub(e2, p2);
  v[3] = cadd(e3, p3); v[7] = csub(e3, p3);
}

template <int R, bool INV> __device__ __forceinline__ void dft_r(float2* v) {
  if constexpr (R == 8) dft8<INV>(v);
  else if constexpr (R == 4) dft4<INV>(v[0], v[1], v[2], v[3]);
  else dft2<INV>(v[0], v[1]);
}

// One Stockham stage of radix R on a line of L points at a (stride-1), done
// by the L/8 threads of the line (thread t): 8/R butterflies per thread.
template <int L, int R, bool INV>
__device__ __forceinline__ void stockham_stage(float2* a, int t, int Ns) {
  constexpr int PER = 8 / R, Q = L / R;
  float2 v[8];
  int base[PER];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int j = t + q * (L / 8);
    const int k = j & (Ns - 1);                  // Ns is a power of two
    base[q] = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) v[q * R + r] = a[j + r * Q];
    if (Ns > 1) {
      const int step = L / (Ns * R);
#pragma unroll
      for (int r = 1; r < R; ++r) {
        float2 w = g_tw[L + r * k * step];
        if (INV) w = cconj(w);
        v[q * R + r] = cmul(v[q * R + r], w);
      }
    }
    dft_r<R, INV>(v + q * R);
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < PER; ++q)
#pragma unroll
    for (int r = 0; r < R; ++r) a[base[q] + r * Ns] = v[q * R + r];
  __syncthreads();
}

// In-place FFT of the line at a (L points, unnormalised), by its L/8
// threads; all threads of the block must call it (it synchronises).
template <int L, bool INV>
__device__ __forceinline__ void fft_line(float2* a, int t) {
  constexpr int LOG = (L >= 1024) ? 10 : (L >= 512) ? 9 : (L >= 256) ? 8 : (L >= 128) ? 7 : (L >= 64) ? 6 :
                      (L >= 32) ? 5 : (L >= 16) ? 4 : 3;
  constexpr int S8 = LOG / 3, REM = LOG % 3;
  int Ns = 1;
#pragma unroll
  for (int s = 0; s < S8; ++s) {
    stockham_stage<L, 8, INV>(a, t, Ns);
    Ns *= 8;
  }
  if constexpr (REM == 2) stockham_stage<L, 4, INV>(a, t, Ns);
  if constexpr (REM == 1) stockham_stage<L, 2, INV>(a, t, Ns);
}

// Lines per block: 4096 points per block (32 KB of shared memory), capped
// by the number of lines available.
template <int L> __host__ __device__ constexpr int lines_per_block() { return 4096 / L < 1 ? 1 : 4096 / L; }

// ---- z pass: real rows of n = 2M values <-> n/2 + 1 complex ----
// Forward: Z_m = x_2m + i x_2m+1, Z = FFT_M(Z), X[k] = E + w_n^k O with
// E = (Z_k + conj Z_{M-k}) / 2, O = -i (Z_k - conj Z_{M-k}) / 2, k = 0..M.
// The input's mean (float64, device) is subtracted first when given: the
// k = 0 mode is dropped anyway, and without its large value the rounding of
// the transforms stays relative to the fluctuations.
template <int M>
__global__ void __launch_bounds__(lines_per_block<M>() * (M / 8)) k_fft_z_r2c(const float* __restrict__ in,
                                                                              const double* __restrict__ mean,
                                                                              float2* __restrict__ out,
                                                                              int64_t rows) {
  constexpr int LB = lines_per_block<M>(), TPL = M / 8, LP = M + 1, H = M + 1, n = 2 * M;
  __shared__ float2 s[LB * LP];
  const int64_t row0 = (int64_t)blockIdx.x * LB;
  const int nl = (int)((rows - row0) < LB ? (rows - row0) : LB);
  const float mu = mean ? (float)*mean : 0.0f;
  for (int e = threadIdx.x; e < nl * M; e += blockDim.x) {
    const int l = e / M, m = e - l * M;
    const float2 v = __ldg(reinterpret_cast<const float2*>(in + (row0 + l) * n) + m);
    s[l * LP + m] = make_float2(v.x - mu, v.y - mu);
  }
  __syncthreads();
  const int line = threadIdx.x / TPL, t = threadIdx.x - line * TPL;
  fft_line<M, false>(s + line * LP, t);
  for (int e = threadIdx.x; e < nl * H; e += blockDim.x) {
    const int l = e / H, k = e - l * H;
    const float2 zk = s[l * LP + (k == M ? 0 : k)];
    const float2 zc = cconj(s[l * LP + (k == 0 ? 0 : M - k)]);
    const float2 E = make_float2(0.5f * (zk.x + zc.x), 0.5f * (zk.y + zc.y));
    const float2 D = csub(zk, zc);
    const float2 O = make_float2(0.5f * D.y, -0.5f * D.x);        // -i D / 2
    out[(row0 + l) * H + k] = cadd(E, cmul(g_tw[n + k], O));      // k <= M < n
  }
}

// Inverse: Z_k = E + i O, E = (X_k + conj X_{M-k}) / 2,
// O = (X_k - conj X_{M-k}) w_n^{-k} / 2; z = IFFT_M(Z); x_2m = Re, x_2m+1 = Im.
template <int M>
__global__ void __launch_bounds__(lines_per_block<M>() * (M / 8)) k_fft_z_c2r(const float2* __restrict__ in,
                                                                              float* __restrict__ out,
                                                                              int64_t rows) {
  constexpr int LB = lines_per_block<M>(), TPL = M / 8, LP = M + 1, H = M + 1, n = 2 * M;
  __shared__ float2 s[LB * LP];
  const int64_t row0 = (int64_t)blockIdx.x * LB;
  const int nl = (int)((rows - row0) < LB ? (rows - row0) : LB);
  for (int e = threadIdx.x; e < nl * H; e += blockDim.x) {
    const int l = e / H, k = e - l * H;
    s[l * LP + k] = __ldg(in + (row0 + l) * H + k);
  }
  __syncthreads();
  float2 z[(LB * M + lines_per_block<M>() * (M / 8) - 1) / (lines_per_block<M>() * (M / 8))];
  int cnt = 0;
  for (int e = threadIdx.x; e < nl * M; e += blockDim.x, ++cnt) {
    const int l = e / M, k = e - l * M;
    const float2 xk = s[l * LP + k], xc = cconj(s[l * LP + M - k]);
    const float2 E = make_float2(0.5f * (xk.x + xc.x), 0.5f * (xk.y + xc.y));
    const float2 D = make_float2(0.5f * (xk.x - xc.x), 0.5f * (xk.y - xc.y));
    const float2 O = cmul(D, cconj(g_tw[n + k]));
    z[cnt] = make_float2(E.x - O.y, E.y + O.x);                   // E + i O
  }
  __syncthreads();
  cnt = 0;
  for (int e = threadIdx.x; e < nl * M; e += blockDim.x, ++cnt) {
    const int l = e / M, k = e - l * M;
    s[l * LP + k] = z[cnt];
  }
  __syncthreads();
  const int line = threadIdx.x / TPL, t = threadIdx.x - line * TPL;
  fft_line<M, true>(s + line * LP, t);
  for (int e = threadIdx.x; e < nl * M; e += blockDim.x) {
    const int l = e / M, m = e - l * M;
    reinterpret_cast<float2*>(out + (row0 + l) * n)[m] = s[l * LP + m];
  }
}

// ---- column passes on C[x][y][kz] (rows of H = n/2 + 1) ----
// A block takes TW consecutive kz columns of one x (AXIS 1: lines along y) or
// one y (AXIS 0: lines along x); for AXIS 0 with SOLVE the block multiplies by
// scale G(k) (times the normalisation) between the forward and the inverse
// transform.
// Spectral multiplier applied on the x pass (kz = kz0 + line, kx index i,
// ky index `other`; m = index for index < n/2, else index - n; k = 2 pi m):
//   GREEN7   -scale / ((4/h^2) sum_d sin^2(pi m_d / n))      (FFT_7pt)
//   GREENTSC -scale / (k^2 W_TSC^2), W_TSC = prod_d sinc(pi m_d / n)^3   (FFT)
//   AMPLAP   -scale amp(kx, ky, kz) / k^2   (first-order LPT potential)
//   INVLAP   -scale / k^2
//   DERIV    scale i k_d1
//   HESS     -scale k_d1 k_d2
// All are 0 at k = 0; the LPT kinds (AMPLAP .. HESS) also on every Nyquist
// plane (|m_d| = n/2 on any axis).
enum MultKind { GREEN7 = 1, GREENTSC = 2, AMPLAP = 3, INVLAP = 4, DERIV = 5, HESS = 6 };
struct Mult {
  int kind;
  int d1, d2;            // axes of DERIV / HESS (0 = x, 1 = y, 2 = z)
  float scale;           // includes the 2 / n^3 of an inverse transform
  const float* amp;      // AMPLAP: [n][n][n/2 + 1]
};

// Column-pass modes: forward or inverse transform in place; FWDMUL: forward,
// then multiply (x pass, in place); MULINV: multiply the lines read from `in`,
// inverse, write `out` (x pass); SOLVE: forward, multiply, inverse (x pass).
enum ColMode { FWD = 0, INVT = 1, FWDMUL = 2, MULINV = 3, SOLVE = 4 };

template <int L, int AXIS, int MODE>
__global__ void __launch_bounds__(lines_per_block<L>() * (L / 8)) k_fft_cols(const float2* in, float2* out,
                                                                             int ntiles, Mult mu) {
  constexpr bool MUL = MODE == FWDMUL || MODE == MULINV || MODE == SOLVE;
  constexpr int TW = lines_per_block<L>(), TPL = L / 8, LP = L + 1, n = L, H = n / 2 + 1;
  __shared__ float2 s[TW * LP];
  __shared__ float ta[MUL ? n : 1], tb[MUL ? n : 1];
  const int tile = blockIdx.x % ntiles, other = blockIdx.x / ntiles;   // other: x (AXIS 1) or y (AXIS 0)
  const int kz0 = tile * TW;
  const int tw = (H - kz0) < TW ? (H - kz0) : TW;
  const int64_t stride = AXIS == 1 ? H : (int64_t)n * H;
  const int64_t base = (AXIS == 1 ? (int64_t)other * n * H : (int64_t)other * H) + kz0;
  for (int e = threadIdx.x; e < tw * L; e += blockDim.x) {
    const int i = e / tw, l = e - i * tw;
    s[l * LP + i] = in[base + i * stride + l];
  }
  if (MUL) {
    // per-axis tables: GREEN7: sin^2(pi m/n); GREENTSC: k^2 and sinc^6;
    // LPT kinds: k (0 on the Nyquist index, which also flags it in tb)
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const int m = i < n / 2 ? i : i - n;
      const float sp = sinpif((float)m / (float)n);
      if (mu.kind == GREEN7) {
        ta[i] = sp * sp;
      } else if (mu.kind == GREENTSC) {
        ta[i] = 39.47841760435743f * (float)m * (float)m;
        const float sc = m == 0 ? 1.0f : sp / (3.14159265358979f * (float)m / (float)n);
        const float s2 = sc * sc;
        tb[i] = s2 * s2 * s2;
      } else {
        const bool nyq = 2 * i == n;
        ta[i] = nyq ? 0.0f : 6.283185307179586f * (float)m;
        tb[i] = nyq ? 1.0f : 0.0f;
      }
    }
  }
  __syncthreads();
  const int line = threadIdx.x / TPL, t = threadIdx.x - line * TPL;
  if (MODE == FWD || MODE == FWDMUL || MODE == SOLVE) fft_line<L, false>(s + line * LP, t);
  if (MODE == INVT) fft_line<L, true>(s + line * LP, t);
  if (MUL) {
    for (int e = threadIdx.x; e < tw * L; e += blockDim.x) {
      const int l = e / L, i = e - l * L;          // kx index i, kz = kz0 + l
      const int kz = kz0 + l;
      float2& v = s[l * LP + i];
      const int ix[3] = {i, other, kz};
      if (mu.kind == GREEN7) {
        const float lam = ta[i] + ta[other] + ta[kz];
        const float g = lam > 0.0f ? -mu.scale / (4.0f * (float)n * (float)n * lam) : 0.0f;
        v = make_float2(v.x * g, v.y * g);
      } else if (mu.kind == GREENTSC) {
        const float k2 = ta[i] + ta[other] + ta[kz];
        const float g = k2 > 0.0f ? -mu.scale / (k2 * tb[i] * tb[other] * tb[kz]) : 0.0f;
        v = make_float2(v.x * g, v.y * g);
      } else {
        const bool zero = tb[i] + tb[other] + tb[kz] > 0.0f || (i == 0 && other == 0 && kz == 0);
        if (zero) {
          v = make_float2(0.0f, 0.0f);
        } else if (mu.kind == DERIV) {
          const float k = mu.scale * ta[ix[mu.d1]];
          v = make_float2(-k * v.y, k * v.x);                 // i k v
        } else {
          float g;
          if (mu.kind == HESS) {
            g = -mu.scale * ta[ix[mu.d1]] * ta[ix[mu.d2]];
          } else {
            const float k2 = ta[i] * ta[i] + ta[other] * ta[other] + ta[kz] * ta[kz];
            g = -mu.scale / k2;
            if (mu.kind == AMPLAP) g *= __ldg(mu.amp + ((int64_t)i * n + other) * H + kz);
          }
          v = make_float2(v.x * g, v.y * g);
        }
      }
    }
    __syncthreads();
    if (MODE == MULINV || MODE == SOLVE) fft_line<L, true>(s + line * LP, t);
  }
  for (int e = threadIdx.x; e < tw * L; e += blockDim.x) {
    const int i = e / tw, l = e - i * tw;
    out[base + i * stride + l] = s[l * LP + i];
  }
}

// Launch geometry of the transforms of an n^3 grid.
template <int N>
struct FftPlan {
  static constexpr int M = N / 2, H = M + 1, LBz = lines_per_block<M>(), LBc = lines_per_block<N>();
  static constexpr int64_t rows = (int64_t)N * N;
  static constexpr double cells = (double)N * N * N, spec = (double)N * N * H * 8.0;
  static unsigned zblocks() { return (unsigned)((rows + LBz - 1) / LBz); }
  static int ntiles() { return (H + LBc - 1) / LBc; }
  static unsigned cblocks() { return (unsigned)(ntiles() * N); }
};

// spec = M(k) FFT[real]  (unnormalised forward transform, then the multiplier)
template <int N>
pm_status fft_forward_mul(const float* real, const double* mean, float2* spec, const Mult& mu, cudaStream_t s) {
  using P = FftPlan<N>;
  PM_LAUNCH(K_FFT, 4.0 * P::cells + P::spec, k_fft_z_r2c<P::M>, P::zblocks(), P::LBz * (P::M / 8), 0, s, real, mean,
            spec, P::rows);
  PM_LAUNCH(K_FFT, 2.0 * P::spec, (k_fft_cols<N, 1, FWD>), P::cblocks(), P::LBc * (N / 8), 0, s, spec, spec,
            P::ntiles(), mu);
  PM_LAUNCH(K_FFT, 2.0 * P::spec, (k_fft_cols<N, 0, FWDMUL>), P::cblocks(), P::LBc * (N / 8), 0, s, spec, spec,
            P::ntiles(), mu);
  return launch_status();
}

// real = IFFT[M(k) spec]  (spec is read only; tmp receives the intermediate
// spectrum; mu.scale carries the 2 / n^3 normalisation)
template <int N>
pm_status fft_mul_inverse(const float2* spec, float2* tmp, float* real, const Mult& mu, cudaStream_t s) {
  using P = FftPlan<N>;
  PM_LAUNCH(K_FFT, 2.0 * P::spec, (k_fft_cols<N, 0, MULINV>), P::cblocks(), P::LBc * (N / 8), 0, s, spec, tmp,
            P::ntiles(), mu);
  PM_LAUNCH(K_FFT, 2.0 * P::spec, (k_fft_cols<N, 1, INVT>), P::cblocks(), P::LBc * (N / 8), 0, s, tmp, tmp,
            P::ntiles(), mu);
  PM_LAUNCH(K_FFT, P::spec + 4.0 * P::cells, k_fft_z_c2r<P::M>, P::zblocks(), P::LBz * (P::M / 8), 0, s, tmp, real,
            P::rows);
  return launch_status();
}

template <int N>
pm_status launch_fft_poisson(const float* rho, const double* mean, float* phi, float2* C, int kind, double scale,
                             cudaStream_t s) {
  using P = FftPlan<N>;
  // the y and x transform pairs scale by n each, the z pair by n/2 (the
  // inverse runs an n/2-point transform of the packed pairs): divide by n^3/2
  const Mult mu{kind == 1 ? GREEN7 : GREENTSC, 0, 0, (float)(2.0 * scale / P::cells), nullptr};
  PM_LAUNCH(K_FFT, 4.0 * P::cells + P::spec, k_fft_z_r2c<P::M>, P::zblocks(), P::LBz * (P::M / 8), 0, s, rho, mean,
            C, P::rows);
  PM_LAUNCH(K_FFT, 2.0 * P::spec, (k_fft_cols<N, 1, FWD>), P::cblocks(), P::LBc * (N / 8), 0, s, C, C, P::ntiles(),
            mu);
  PM_LAUNCH(K_FFT, 2.0 * P::spec, (k_fft_cols<N, 0, SOLVE>), P::cblocks(), P::LBc * (N / 8), 0, s, C, C,
            P::ntiles(), mu);
  PM_LAUNCH(K_FFT, 2.0 * P::spec, (k_fft_cols<N, 1, INVT>), P::cblocks(), P::LBc * (N / 8), 0, s, C, C,
            P::ntiles(), mu);
  PM_LAUNCH(K_FFT, P::spec + 4.0 * P::cells, k_fft_z_c2r<P::M>, P::zblocks(), P::LBz * (P::M / 8), 0, s, C, phi,
            P::rows);
  return launch_status();
}

// S = phi_xx phi_yy + phi_xx phi_zz + phi_yy phi_zz (H: the three diagonal
// second derivatives, planes of N), then S -= T^2 for each mixed derivative T.
__global__ void k_lpt_diag(const float* __restrict__ H, float* __restrict__ S, int64_t N) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < N; c += (int64_t)gridDim.x * blockDim.x) {
    const float a = H[c], b = H[N + c], d = H[2 * N + c];
    S[c] = fmaf(a, b, fmaf(a, d, b * d));
  }
}

__global__ void k_lpt_sub_sq(const float* __restrict__ T, float* __restrict__ S, int64_t N) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < N; c += (int64_t)gridDim.x * blockDim.x)
    S[c] = fmaf(-T[c], T[c], S[c]);
}

// Particle p on cell centre q_p (lattice order): component d of
// X = q + d1 Psi1 + e2 Psi2 (fixed point: the displacement rounded to units
// of 2^-32 of the box and added to the exact centre, modulo 2^32) and
// V = v1 Psi1 + v2 Psi2.  V holds Psi1_d on entry; psi2 may be NULL (1LPT).
__global__ void k_lpt_combine(const float* __restrict__ psi2, float* __restrict__ V, uint32_t* __restrict__ X,
                              int d, int log2n, float d1, float e2, float v1, float v2) {
  const int64_t N = (int64_t)1 << (3 * log2n);
  const int m = (1 << log2n) - 1;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x) {
    const int cell = (int)((p >> ((2 - d) * log2n)) & m);                 // i, j or k of the particle
    const uint32_t q = (uint32_t)(2 * cell + 1) << (31 - log2n);          // (cell + 1/2)/n in units of 2^-32
    const float p1 = V[p], p2 = psi2 ? psi2[p] : 0.0f;
    const float disp = fmaf(d1, p1, e2 * p2);
    X[p] = q + (uint32_t)__float2int_rn(disp * 4294967296.0f);
    V[p] = fmaf(v1, p1, v2 * p2);
  }
}

template <int N>
pm_status launch_lpt2(const float* noise, const float* amp, float d1, float e2, float v1, float v2, uint32_t* X,
                      float* V, float2* A, float2* B, float* R, cudaStream_t s) {
  using P = FftPlan<N>;
  const int64_t NC = (int64_t)N * N * N;
  const float inv = (float)(2.0 / P::cells);
  float *H = R, *S = R + 3 * NC, *T = R + 4 * NC;
  const unsigned g = grid_for(NC, 256);
  PM_TRY(fft_forward_mul<N>(noise, nullptr, A, Mult{AMPLAP, 0, 0, 1.0f, amp}, s));       // phi1
  for (int d = 0; d < 3; ++d)                                                             // Psi1 = -grad phi1
    PM_TRY(fft_mul_inverse<N>(A, B, V + d * NC, Mult{DERIV, d, 0, -inv, nullptr}, s));
  const bool second = e2 != 0.0f || v2 != 0.0f;
  if (second) {
    for (int d = 0; d < 3; ++d)
      PM_TRY(fft_mul_inverse<N>(A, B, H + d * NC, Mult{HESS, d, d, inv, nullptr}, s));
    PM_LAUNCH(K_MISC, 16.0 * NC, k_lpt_diag, g, 256, 0, s, H, S, NC);
    const int pairs[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    for (const auto& pr : pairs) {
      PM_TRY(fft_mul_inverse<N>(A, B, T, Mult{HESS, pr[0], pr[1], inv, nullptr}, s));
      PM_LAUNCH(K_MISC, 12.0 * NC, k_lpt_sub_sq, g, 256, 0, s, T, S, NC);
    }
    PM_TRY(fft_forward_mul<N>(S, nullptr, A, Mult{INVLAP, 0, 0, 1.0f, nullptr}, s));      // phi2
  }
  for (int d = 0; d < 3; ++d) {
    if (second) PM_TRY(fft_mul_inverse<N>(A, B, T, Mult{DERIV, d, 0, inv, nullptr}, s));  // Psi2 = grad phi2
    PM_LAUNCH(K_MISC, 20.0 * NC, k_lpt_combine, g, 256, 0, s, second ? T : nullptr, V + d * NC, X + d * NC, d,
              ilog2(N), d1, e2, v1, v2);
  }
  return launch_status();
}

}  // namespace

pm_status lpt2_launch(const float* noise, const float* amp, int n, double d1, double e2, double v1, double v2,
                      uint32_t* X, float* V, float2* A, float2* B, float* R, cudaStream_t s) {
  PM_TRY(twiddles_ready());
  const float f[4] = {(float)d1, (float)e2, (float)v1, (float)v2};
  switch (n) {
    case 16: return launch_lpt2<16>(noise, amp, f[0], f[1], f[2], f[3], X, V, A, B, R, s);
    case 32: return launch_lpt2<32>(noise, amp, f[0], f[1], f[2], f[3], X, V, A, B, R, s);
    case 64: return launch_lpt2<64>(noise, amp, f[0], f[1], f[2], f[3], X, V, A, B, R, s);
    case 128: return launch_lpt2<128>(noise, amp, f[0], f[1], f[2], f[3], X, V, A, B, R, s);
    case 256: return launch_lpt2<256>(noise, amp, f[0], f[1], f[2], f[3], X, V, A, B, R, s);
    case 512: return launch_lpt2<512>(noise, amp, f[0], f[1], f[2], f[3], X, V, A, B, R, s);
    case 1024: return launch_lpt2<1024>(noise, amp, f[0], f[1], f[2], f[3], X, V, A, B, R, s);
    default: return PM_EINVAL;
  }
}

pm_status fft_poisson_launch(const float* rho, const double* mean, float* phi, float2* C, int n, int kind,
                             double scale, cudaStream_t s) {
  PM_TRY(twiddles_ready());
  switch (n) {
    case 16: return launch_fft_poisson<16>(rho, mean, phi, C, kind, scale, s);
    case 32: return launch_fft_poisson<32>(rho, mean, phi, C, kind, scale, s);
    case 64: return launch_fft_poisson<64>(rho, mean, phi, C, kind, scale, s);
    case 128: return launch_fft_poisson<128>(rho, mean, phi, C, kind, scale, s);
    case 256: return launch_fft_poisson<256>(rho, mean, phi, C, kind, scale, s);
    case 512: return launch_fft_poisson<512>(rho, mean, phi, C, kind, scale, s);
    case 1024: return launch_fft_poisson<1024>(rho, mean, phi, C, kind, scale, s);
    default: return PM_EINVAL;
  }
}

}  // namespace pmgb
