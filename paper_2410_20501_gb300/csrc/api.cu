// C ABI of libpmgb: argument checks, workspace layout, the step pipeline,
// host-side cosmology utilities and launch instrumentation.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>
#include <utility>
#include <vector>

#include "pm_internal.cuh"

namespace pmgb {

const char* const kKernelClassNames[K_NCLASS] = {
    "cell_count",  "cell_scan",     "cell_scatter", "cell_order",     "permute",
    "tsc_deposit", "reduce",        "mg_guess",    "mg_smooth_l0",    "mg_smooth",   "mg_restrict",
    "mg_prolong",  "mg_coarse",     "mg_norm",     "fr_smooth_l0",    "fr_smooth",   "fr_restrict",
    "fr_coarse_op", "fr_prolong",
    "fr_coarse",   "fr_norm",       "gradient",    "interp_kdk",      "adjoint",     "fft",
    "misc"};

namespace {

uint64_t g_launches = 0;
char g_last_error[256] = "";

struct TimingPool {
  bool on = false;
  std::vector<cudaEvent_t> start, stop;
  std::vector<int> cls;
  std::vector<double> bytes;
  size_t used = 0;
};
TimingPool g_timing;
constexpr size_t kTimingCap = 1 << 15;

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

void launch_begin(int cls, double bytes, cudaStream_t s) {
  ++g_launches;
  if (g_timing.on && g_timing.used < g_timing.start.size()) {
    g_timing.cls[g_timing.used] = cls;
    g_timing.bytes[g_timing.used] = bytes;
    cudaEventRecord(g_timing.start[g_timing.used], s);
  }
}

void launch_end(int cls, cudaStream_t s) {
  if (g_timing.on && g_timing.used < g_timing.start.size()) {
    (void)cls;
    cudaEventRecord(g_timing.stop[g_timing.used], s);
    ++g_timing.used;
  }
}

pm_status smem_attr_fn(const void* fn, size_t bytes) {
  static std::mutex mu;
  static std::vector<std::pair<int, const void*>> done;   // (device, kernel) pairs already raised
  int dev = 0;
  PM_TRY(cuda_status(cudaGetDevice(&dev)));
  std::lock_guard<std::mutex> lock(mu);
  for (const auto& d : done)
    if (d.first == dev && d.second == fn) return PM_OK;
  PM_TRY(cuda_status(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes)));
  done.emplace_back(dev, fn);
  return PM_OK;
}

pm_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return PM_OK;
  strncpy(g_last_error, cudaGetErrorString(e), sizeof(g_last_error) - 1);
  return PM_ECUDA;
}

size_t layout_workspace(Workspace* w, void* base, int n, int64_t np, uint32_t flags, int batch) {
  Workspace tmp;
  if (!w) w = &tmp;
  memset(w, 0, sizeof(*w));
  const bool step = flags & PM_WS_STEP;
  const bool sort = step || (flags & PM_WS_SORT);
  const bool mg = step || (flags & (PM_WS_MG | PM_WS_REFINE));
  const bool fr = (step && batch == 1) || (flags & PM_WS_FR);   // batched steps are Newtonian
  const int64_t N = (int64_t)n * n * n * batch;                  // cells of all boxes
  size_t off = 0;
  char* b = (char*)base;
  auto take = [&](size_t bytes) -> char* {
    off = align256(off);
    char* p = b ? b + off : nullptr;
    off += bytes;
    return p;
  };
  if (sort) {
    const size_t kb = (size_t)np * 4;
    w->keyrank = (uint2*)take(2 * kb);
    w->perm = (uint32_t*)take(kb);
    w->runs = (uint32_t*)take((size_t)sort_runs_capacity(np) * 4);
    w->meds = (uint32_t*)take((size_t)sort_meds_capacity(np) * 4);
    w->bigs = (uint32_t*)take((size_t)sort_bigs_capacity(np) * 4);
    w->smalls = (uint32_t*)take((size_t)sort_smalls_capacity(np) * 4);
    w->moments = (float*)take((size_t)np * kMomStride * 4);
    w->scan_blocks = (uint32_t*)take((size_t)sort_scan_blocks(N) * 4);
    w->cellstart = (uint32_t*)take((size_t)(N + 1) * 4);
    w->Xs = (uint32_t*)take(3 * kb);
  }
  if (step) {
    w->Vs = (float*)take((size_t)np * 12);
    if (flags & PM_WS_IDS) w->ids = (uint32_t*)take((size_t)np * 4);
    w->rho = (float*)take((size_t)N * 4);
    w->g = (float*)take((size_t)N * 16);   // three planes, or float4 per cell
  }
  if (flags & PM_WS_ADJ) {
    w->adj_abar = (float*)take((size_t)np * 12);
    w->adj_phi = (float*)take((size_t)N * 4);
    w->adj_psi = (float*)take((size_t)N * 4);
    w->adj_gbar = (float*)take((size_t)N * 12);
  }
  if (flags & PM_WS_FFT) w->spec = (float2*)take((size_t)n * n * (n / 2 + 1) * 8 * batch);
  if (flags & PM_WS_LPT) {
    w->lpt_a = (float2*)take((size_t)n * n * (n / 2 + 1) * 8);
    w->lpt_b = (float2*)take((size_t)n * n * (n / 2 + 1) * 8);
    w->lpt_r = (float*)take((size_t)N * 4 * 5);
  }
  if (flags & PM_WS_REFINE) {
    w->ref_r = (float*)take((size_t)N * 4);
    w->ref_e = (float*)take((size_t)N * 4);
  }
  w->partials = (double*)take((size_t)2 * reduce_partials_capacity(n, np) * 8 * batch);
  w->scalars = (double*)take(64 * 8);
  w->box_mean = (double*)take((size_t)batch * 8);
  for (int l = 0; l < 12; ++l) {
    const int nl = n >> l;
    if (nl < 4) break;
    const size_t bytes = (size_t)nl * nl * nl * 4 * batch;
    const bool streamed = nl >= 64;   // levels smoothed out of place (fused or streaming sweeps) need a ping-pong partner
    if (mg) {
      if (l > 0) {
        w->mg_u[l] = (float*)take(bytes);
        w->mg_f[l] = (float*)take(bytes);
      }
      if (streamed) w->mg_alt[l] = (float*)take(bytes);
    }
    if (fr) {
      if (l > 0) {
        w->fr_e[l] = (float*)take(bytes);
        w->fr_r[l] = (float*)take(bytes);
        w->fr_b[l] = (float*)take(bytes);
      }
      if (streamed) w->fr_alt[l] = (float*)take(bytes);
    }
  }
  w->base = b;
  w->total = align256(off);
  w->np = np;
  w->n = n;
  w->batch = batch;
  return w->total;
}

}  // namespace pmgb

using namespace pmgb;

namespace {

cudaStream_t as_stream(void* s) { return (cudaStream_t)s; }

// A second stream (and fork / join events) per device for work that runs
// beside the caller's stream inside one call.
struct SideStream {
  cudaStream_t s = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};
SideStream g_side[64];   // the scalaron solve of an f(R) step
SideStream g_copy[64];   // the velocity copies of pm_step_host

// priority: create the stream with the device's highest stream priority
// (its CTAs are scheduled first when both streams have work waiting).
pm_status lib_stream(SideStream* table, SideStream** out, bool priority = false) {
  int dev = 0;
  PM_TRY(cuda_status(cudaGetDevice(&dev)));
  if (dev < 0 || dev >= 64) return PM_EINVAL;
  SideStream& ss = table[dev];
  if (!ss.s) {
    int lowest = 0, highest = 0;
    PM_TRY(cuda_status(cudaDeviceGetStreamPriorityRange(&lowest, &highest)));
    PM_TRY(cuda_status(cudaStreamCreateWithPriority(&ss.s, cudaStreamNonBlocking, priority ? highest : lowest)));
    PM_TRY(cuda_status(cudaEventCreateWithFlags(&ss.fork, cudaEventDisableTiming)));
    PM_TRY(cuda_status(cudaEventCreateWithFlags(&ss.join, cudaEventDisableTiming)));
  }
  *out = &ss;
  return PM_OK;
}

// The scalaron chain is the longer of the step's two solver chains: its
// stream takes the highest priority, so its latency-bound small levels run
// first and the Poisson sweeps fill the rest of the GPU.
pm_status side_stream(SideStream** out) { return lib_stream(g_side, out, true); }

// Offset (in doubles) of the side stream's share of the partials: past the
// 2 x (152 x 8) block sums of a residual norm on the main stream, twice.
constexpr int64_t kSidePartials = 4 * 152 * 8;

bool aligned(const void* p) { return ((uintptr_t)p & 255) == 0; }

// Device arrays of the caller start on 16-byte boundaries (NULL passes: the
// null checks are separate).
bool a16(const void* p) { return ((uintptr_t)p & 15) == 0; }
template <class... P>
bool all_a16(const P*... p) { return (a16(p) && ...); }

pm_status check_ws(Workspace& w, void* ws, size_t ws_bytes, int n, int64_t np, uint32_t flags) {
  const size_t need = layout_workspace(nullptr, nullptr, n, np, flags);
  if (!ws || !aligned(ws)) return PM_EINVAL;
  if (ws_bytes < need) return PM_ENOMEM;
  layout_workspace(&w, ws, n, np, flags);
  return PM_OK;
}

bool valid_np(int64_t np) { return np >= 0 && np < ((int64_t)1 << 31); }

// The cell lists of the workspace's last cell sort and its moment buffer.
Crowded crowded(const Workspace& w) { return Crowded{w.runs, w.meds, w.bigs, w.smalls, w.moments}; }

// 3/2 a Om of the supercomoving Poisson equation (§3.1), times mu(a) =
// 1 + mu0 Omega_L(a)/Omega_L,0 = 1 + mu0 / E(a)^2 for parametrised gravity.
double poisson_scale(const pm_step_params& p) {
  double s = 1.5 * p.a * p.Om;
  if (p.gravity == PM_GRAVITY_PARAM) s *= 1.0 + p.mu0 / (p.Om / (p.a * p.a * p.a) + p.OL);
  return s;
}

bool valid_mg(const mg_params* p) {
  return p && p->npre >= 0 && p->npost >= 0 && p->npre + p->npost > 0 && p->coarsest >= 4 &&
         p->coarsest <= 16 && p->coarse_max_sweeps >= 0 && p->max_cycles >= 1 && p->omega > 0.0f &&
         p->omega < 2.0f && p->first_guess >= MG_GUESS_INPUT && p->first_guess <= MG_GUESS_SCALED &&
         p->smoother >= 0 && p->smoother <= 2 && p->coarse_omega >= 0.0f && p->coarse_omega < 2.0f;
}

bool valid_fr(const fr_params* p) {
  return p && p->a > 0.0 && p->Om > 0.0 && p->fR0 < 0.0 && p->boxsize > 0.0 && p->npre >= 0 && p->npost >= 0 &&
         p->coarsest >= 4 && p->coarsest <= 16 && p->coarse_max_sweeps >= 0 && (p->cycle == 0 || p->cycle == 1) &&
         (p->tol > 0.0 ? p->max_cycles >= 1 : p->cycles >= 0) && p->smoother >= 0 && p->smoother <= 2 &&
         p->nhs >= 0 && p->nhs <= 2;
}

// Adaptive Simpson quadrature of da / (a^3 E(a)).
double integrand(double Om, double OL, double a) { return 1.0 / (a * a * a * sqrt(Om / (a * a * a) + OL)); }

double simpson(double Om, double OL, double a, double b, double fa, double fm, double fb, double whole, double eps,
               int depth) {
  const double m = 0.5 * (a + b), lm = 0.5 * (a + m), rm = 0.5 * (m + b);
  const double flm = integrand(Om, OL, lm), frm = integrand(Om, OL, rm);
  const double left = (m - a) / 6.0 * (fa + 4.0 * flm + fm), right = (b - m) / 6.0 * (fm + 4.0 * frm + fb);
  const double delta = left + right - whole;
  if (depth <= 0 || fabs(delta) <= 15.0 * eps) return left + right + delta / 15.0;
  return simpson(Om, OL, a, m, fa, flm, fm, left, 0.5 * eps, depth - 1) +
         simpson(Om, OL, m, b, fm, frm, fb, right, 0.5 * eps, depth - 1);
}

}  // namespace

extern "C" {

const char* pm_status_string(pm_status s) {
  switch (s) {
    case PM_OK: return "PM_OK";
    case PM_EINVAL: return "PM_EINVAL: invalid argument";
    case PM_ENOMEM: return "PM_ENOMEM: workspace too small";
    case PM_ENOCONV: return "PM_ENOCONV: solver did not converge";
    case PM_ENAN: return "PM_ENAN: non-finite residual";
    case PM_ETIMEOUT: return "PM_ETIMEOUT: device wait timed out";
    case PM_ECUDA: return "PM_ECUDA: CUDA error";
    case PM_EIO: return "PM_EIO: checkpoint file error";
    default: return "unknown status";
  }
}

const char* pm_last_cuda_error(void) { return g_last_error; }
const char* pm_version(void) { return "1.0.0"; }
uint64_t pm_launch_count(void) { return g_launches; }

pm_status pm_workspace_size(int n, int64_t np, uint32_t flags, size_t* bytes) {
  if (!valid_n(n) || !valid_np(np) || !bytes) return PM_EINVAL;
  *bytes = layout_workspace(nullptr, nullptr, n, np, flags);
  return PM_OK;
}

void mg_default_params(mg_params* p) {
  if (!p) return;
  p->npre = 2;
  p->npost = 2;
  p->omega = 1.25f;
  p->coarsest = 16;
  p->coarse_max_sweeps = 200;
  p->coarse_drop = 1e-3f;
  p->max_cycles = 30;
  p->fixed_cycles = 0;
  p->tol = 1e-7;
  p->stall = 0.5;
  p->first_guess = MG_GUESS_INPUT;
  p->guess_scale = 1.0f;
  p->smoother = 2;
  p->coarse_omega = 0.0f;
}

void fr_default_params(fr_params* p) {
  if (!p) return;
  p->a = 1.0;
  p->Om = 0.3;
  p->OL = 0.7;
  p->fR0 = -1e-5;
  p->boxsize = 512.0;
  p->cycle = 1;
  p->npre = 2;
  p->npost = 2;
  p->coarsest = 16;
  p->coarse_max_sweeps = 200;
  p->coarse_drop = 1e-3f;
  p->cycles = 1;
  p->tol = 0.0;
  p->max_cycles = 30;
  p->smoother = 2;
  p->nhs = 1;
}

pm_status pm_sort(const uint32_t* X, int64_t np, int n, uint32_t* perm, uint32_t* cellstart, void* ws,
                  size_t ws_bytes, void* stream) {
  if (!valid_n(n) || !valid_np(np) || (np > 0 && !X) || !all_a16(X, perm, cellstart)) return PM_EINVAL;
  Workspace w;
  PM_TRY(check_ws(w, ws, ws_bytes, n, np, PM_WS_SORT));
  cudaStream_t s = as_stream(stream);
  uint32_t* p;
  PM_TRY(sort_cells(X, np, n, w, s, cellstart ? cellstart : w.cellstart, &p));
  if (perm && np > 0) PM_TRY(cuda_status(cudaMemcpyAsync(perm, p, np * 4, cudaMemcpyDeviceToDevice, s)));
  return launch_status();
}

pm_status pm_deposit(const uint32_t* X, int64_t np, int n, float* rho, void* ws, size_t ws_bytes, void* stream) {
  if (!valid_n(n) || !valid_np(np) || (np > 0 && !X) || !rho || !all_a16(X, rho)) return PM_EINVAL;
  Workspace w;
  PM_TRY(check_ws(w, ws, ws_bytes, n, np, PM_WS_SORT));
  cudaStream_t s = as_stream(stream);
  uint32_t* p;
  PM_TRY(sort_cells(X, np, n, w, s, w.cellstart, &p));
  PM_TRY(permute_particles(p, np, X, nullptr, nullptr, w.Xs, nullptr, nullptr, s));
  PM_TRY(deposit_sorted(w.Xs, np, w.cellstart, n, rho, w.partials, w.scalars, s, crowded(w)));
  return launch_status();
}

pm_status mg_solve(const float* f, float* phi, int n, const mg_params* prm, mg_stats* st, void* ws,
                   size_t ws_bytes, void* stream) {
  if (!valid_n(n) || !f || !phi || !valid_mg(prm) || !all_a16(f, phi)) return PM_EINVAL;
  Workspace w;
  PM_TRY(check_ws(w, ws, ws_bytes, n, 0, PM_WS_MG));
  cudaStream_t s = as_stream(stream);
  PM_TRY(grid_mean(f, (int64_t)n * n * n, w.partials, w.scalars + 1, s));
  return mg_solve_src(Src{f, 1.0f, w.scalars + 1}, phi, n, *prm, st, w, s);
}

pm_status mg_solve_refine(const float* f, double* phi, int n, int outer, const mg_params* prm, mg_stats* st,
                          void* ws, size_t ws_bytes, void* stream) {
  if (!valid_n(n) || !f || !phi || outer < 1 || !valid_mg(prm) || !all_a16(f, phi)) return PM_EINVAL;
  if (prm->first_guess == MG_GUESS_SCALED) return PM_EINVAL;   // phi is float64: nothing to rescale here
  Workspace w;
  PM_TRY(check_ws(w, ws, ws_bytes, n, 0, PM_WS_MG | PM_WS_REFINE));
  cudaStream_t s = as_stream(stream);
  PM_TRY(grid_mean(f, (int64_t)n * n * n, w.partials, w.scalars + 1, s));
  return mg_solve_refine_src(f, w.scalars + 1, phi, n, outer, *prm, st, w, s);
}

pm_status fr_solve(const float* rho, float* eps, int n, const fr_params* prm, mg_stats* st, void* ws,
                   size_t ws_bytes, void* stream) {
  if (!valid_n(n) || !rho || !eps || !valid_fr(prm) || !all_a16(rho, eps)) return PM_EINVAL;
  Workspace w;
  PM_TRY(check_ws(w, ws, ws_bytes, n, 0, PM_WS_FR));
  cudaStream_t s = as_stream(stream);
  PM_TRY(grid_mean(rho, (int64_t)n * n * n, w.partials, w.scalars + 2, s));
  double fbar, kappa, c2;
  fr_background(*prm, &fbar, &kappa, &c2);
  const float sb = (float)(-prm->Om * prm->a / c2);
  return fr_solve_src(Src{rho, sb, w.scalars + 2}, eps, n, *prm, st, w, s);
}

pm_status pm_poisson_fft(const float* rho, float* phi, int n, int kind, double scale, void* ws, size_t ws_bytes,
                         void* stream) {
  if (!valid_n(n) || n < 16 || !rho || !phi || !all_a16(rho, phi)) return PM_EINVAL;
  if (kind != PM_POISSON_FFT7 && kind != PM_POISSON_FFT) return PM_EINVAL;
  Workspace w;
  PM_TRY(check_ws(w, ws, ws_bytes, n, 0, PM_WS_FFT));
  cudaStream_t s = as_stream(stream);
  PM_TRY(grid_mean(rho, (int64_t)n * n * n, w.partials, w.scalars + 3, s));
  return fft_poisson_launch(rho, w.scalars + 3, phi, w.spec, n, kind, scale, s);
}

pm_status pm_lpt2(const float* noise, const float* amp, int n, double d1, double e2, double v1, double v2,
                  uint32_t* X, float* V, void* ws, size_t ws_bytes, void* stream) {
  if (!valid_n(n) || n < 16 || !noise || !amp || !X || !V || !all_a16(noise, amp, X, V)) return PM_EINVAL;
  Workspace w;
  PM_TRY(check_ws(w, ws, ws_bytes, n, 0, PM_WS_LPT));
  return lpt2_launch(noise, amp, n, d1, e2, v1, v2, X, V, w.lpt_a, w.lpt_b, w.lpt_r, as_stream(stream));
}

pm_status pm_gradient(const float* phi, float* g, int n, int order, void* stream) {
  if (!valid_n(n) || !phi || !g || (order != 3 && order != 5 && order != 7) || !all_a16(phi, g)) return PM_EINVAL;
  return gradient_launch(phi, nullptr, 0.0f, g, n, order, false, as_stream(stream));
}

pm_status pm_interp(const float* g, const uint32_t* X, int64_t np, int n, float* acc, void* stream) {
  if (!valid_n(n) || !valid_np(np) || !g || (np > 0 && (!X || !acc)) || !all_a16(g, X, acc)) return PM_EINVAL;
  return interp_launch(g, X, nullptr, nullptr, np, n, acc, nullptr, nullptr, nullptr, 0.0f, 0.0f, 0, false,
                       as_stream(stream));
}

// The step; with V_host, the velocities are copied from that host array on
// the copy stream cp while the positions are sorted and the potentials solved
// (the velocities enter only the force pass, after their own permutation).
// Host-side checks of a step's arguments (nothing is enqueued), with the
// effective f(R) parameters and the workspace carve-up: PM_EINVAL / PM_ENOMEM
// exactly as the step returns them.
pm_status step_args(const pm_state* st_, const pm_step_params* prm, fr_params* frp, Workspace* w) {
  if (!st_ || !prm) return PM_EINVAL;
  const pm_state& S = *st_;
  const int n = S.n;
  const int64_t np = S.np;
  if (!valid_n(n) || !valid_np(np) || (np > 0 && (!S.X || !S.V)) || !S.phi) return PM_EINVAL;
  if (!all_a16(S.X, S.V, S.id, S.phi, S.eps, S.acc)) return PM_EINVAL;
  if (prm->gravity != PM_GRAVITY_NEWTON && prm->gravity != PM_GRAVITY_FR && prm->gravity != PM_GRAVITY_PARAM)
    return PM_EINVAL;
  if (prm->gravity == PM_GRAVITY_FR && !S.eps) return PM_EINVAL;
  if (prm->grad_order != 3 && prm->grad_order != 5 && prm->grad_order != 7) return PM_EINVAL;
  if (!(prm->a > 0.0) || !valid_mg(&prm->mg)) return PM_EINVAL;
  *frp = prm->fr;
  frp->a = prm->a;
  frp->Om = prm->Om;
  frp->OL = prm->OL;
  frp->fR0 = prm->fR0;
  frp->boxsize = prm->boxsize;
  if (prm->gravity == PM_GRAVITY_FR && !valid_fr(frp)) return PM_EINVAL;
  if (prm->poisson != PM_POISSON_MG && prm->poisson != PM_POISSON_FFT7 && prm->poisson != PM_POISSON_FFT)
    return PM_EINVAL;
  if (prm->poisson != PM_POISSON_MG && n < 16) return PM_EINVAL;
  const uint32_t flags = PM_WS_STEP | (S.id ? PM_WS_IDS : 0) | (prm->poisson != PM_POISSON_MG ? PM_WS_FFT : 0);
  return check_ws(*w, S.ws, S.ws_bytes, n, np, flags);
}

pm_status step_impl(pm_state* st_, const pm_step_params* prm, pm_stats* stats, void* stream, const float* V_host,
                    SideStream* cp) {
  fr_params frp;
  Workspace w;
  PM_TRY(step_args(st_, prm, &frp, &w));
  pm_state& S = *st_;
  const int n = S.n;
  const int64_t np = S.np;
  cudaStream_t s = as_stream(stream);
  const int64_t N = (int64_t)n * n * n;
  pm_stats local;
  memset(&local, 0, sizeof(local));

  if (V_host) {
    PM_TRY(cuda_status(cudaEventRecord(cp->fork, s)));
    PM_TRY(cuda_status(cudaStreamWaitEvent(cp->s, cp->fork, 0)));
    PM_TRY(cuda_status(cudaMemcpyAsync(S.V, V_host, (size_t)np * 12, cudaMemcpyHostToDevice, cp->s)));
    PM_TRY(cuda_status(cudaEventRecord(cp->join, cp->s)));
  }
  uint32_t* perm;
  PM_TRY(sort_cells(S.X, np, n, w, s, w.cellstart, &perm));
  PM_TRY(permute_particles(perm, np, S.X, V_host ? nullptr : S.V, S.id, w.Xs, V_host ? nullptr : w.Vs, w.ids, s));
  PM_TRY(deposit_sorted(w.Xs, np, w.cellstart, n, w.rho, w.partials, w.scalars, s, crowded(w)));

  double fbar = 0.0, kappa = 0.0, c2 = 0.0;
  pm_status solve_status = PM_OK;
  // The scalaron (FAS) and the Newtonian potential (multigrid or FFT) both
  // depend on the density only: the scalaron runs on a side stream, forked
  // after the deposit and joined before the force, so the two solvers' many
  // small-level launches overlap.  It reduces its norms in its own part of
  // the partials.
  SideStream* side = nullptr;
  pm_status fr_status = PM_OK;
  if (prm->gravity == PM_GRAVITY_FR) {
    fr_background(frp, &fbar, &kappa, &c2);
    if (!S.have_prev) PM_TRY(cuda_status(cudaMemsetAsync(S.eps, 0, N * sizeof(float), s)));
    const float sb = (float)(-prm->Om * prm->a / c2);
    if (prm->serial) {
      fr_status = fr_solve_src(Src{w.rho, sb, w.scalars}, S.eps, n, frp, &local.fr, w, s);
    } else {
      PM_TRY(side_stream(&side));
      PM_TRY(cuda_status(cudaEventRecord(side->fork, s)));
      PM_TRY(cuda_status(cudaStreamWaitEvent(side->s, side->fork, 0)));
      Workspace wf = w;
      wf.partials = w.partials + kSidePartials;
      fr_status = fr_solve_src(Src{w.rho, sb, w.scalars}, S.eps, n, frp, &local.fr, wf, side->s);
      PM_TRY(cuda_status(cudaEventRecord(side->join, side->s)));
    }
    if (fr_status != PM_OK && fr_status != PM_ENOCONV) {
      if (side) PM_TRY(cuda_status(cudaStreamWaitEvent(s, side->join, 0)));
      return fr_status;
    }
    if (fr_status != PM_OK) solve_status = fr_status;
  }
  mg_params mp = prm->mg;
  mp.first_guess = S.have_prev ? MG_GUESS_SCALED : MG_GUESS_JACOBI;
  mp.guess_scale = (float)prm->phi_rescale;
  if (!S.have_prev) mp.fixed_cycles = 0;   // a cold start always iterates to the tolerance
  pm_status mg_status = PM_OK;
  if (prm->poisson != PM_POISSON_MG) {
    mg_status = fft_poisson_launch(w.rho, w.scalars, S.phi, w.spec, n, prm->poisson, poisson_scale(*prm), s);
  } else {
    mg_status = mg_solve_src(Src{w.rho, (float)poisson_scale(*prm), w.scalars}, S.phi, n, mp, &local.mg, w, s);
  }
  if (side) PM_TRY(cuda_status(cudaStreamWaitEvent(s, side->join, 0)));   // the scalaron is done
  if (mg_status != PM_OK && mg_status != PM_ENOCONV) return mg_status;
  if (mg_status != PM_OK) solve_status = mg_status;
  if (V_host) {   // the velocities have arrived: into cell order
    PM_TRY(cuda_status(cudaStreamWaitEvent(s, cp->join, 0)));
    PM_TRY(permute_particles(perm, np, nullptr, S.V, nullptr, nullptr, w.Vs, nullptr, s));
  }
  const float alpha = (float)(-0.5 * c2 * fbar);
  const float* eps_force = prm->gravity == PM_GRAVITY_FR ? S.eps : nullptr;
  const int nh = frp.nhs == 2 ? 2 : 1;
  double* max_out = prm->report_max ? w.scalars + 24 : nullptr;   // largest |a|, |v| for the time step
  float2* blockmax = reinterpret_cast<float2*>(w.partials);
  if (n >= 32) {   // force computed in shared memory next to the particles
    PM_TRY(force_interp_launch(S.phi, eps_force, alpha, nh, prm->grad_order, w.cellstart, w.Xs, w.Vs, w.ids, np, n,
                               S.acc, S.X, S.V, S.id, (float)prm->dt_kick, (float)prm->dt_drift, 1, s, Batch{},
                               blockmax, max_out));
  } else {
    PM_TRY(gradient_launch(S.phi, eps_force, alpha, w.g, n, prm->grad_order, false, s, 1, nh));
    PM_TRY(interp_launch(w.g, w.Xs, w.Vs, w.ids, np, n, S.acc, S.X, S.V, S.id, (float)prm->dt_kick,
                         (float)prm->dt_drift, 1, false, s, Batch{}, blockmax, max_out));
  }
  if (max_out) {
    double h[2] = {0.0, 0.0};
    if (np > 0) PM_TRY(fetch_scalars(max_out, h, 2, s));
    local.max_acc = h[0];
    local.max_vel = h[1];
  }
  S.have_prev = 1;
  local.status = solve_status;
  if (stats) *stats = local;
  PM_TRY(launch_status());
  return solve_status;
}

pm_status pm_step(pm_state* st_, const pm_step_params* prm, pm_stats* stats, void* stream) {
  return step_impl(st_, prm, stats, stream, nullptr, nullptr);
}

// Positions in on the caller's stream, velocities in on the copy stream
// beside the sort and the solvers; after the force pass, positions out on the
// caller's stream and velocities out on the copy stream (two copy engines).
pm_status pm_step_host(pm_state* st_, const pm_step_params* prm, pm_stats* stats, const uint32_t* X_in,
                       const float* V_in, uint32_t* X_out, float* V_out, void* stream) {
  if (!st_ || !X_in || !V_in || !X_out || !V_out) return PM_EINVAL;
  {   // argument errors before any copy is enqueued
    fr_params frp;
    Workspace w;
    PM_TRY(step_args(st_, prm, &frp, &w));
  }
  cudaStream_t s = as_stream(stream);
  const size_t bytes = (size_t)st_->np * 12;
  SideStream* cp = nullptr;
  PM_TRY(lib_stream(g_copy, &cp));
  PM_TRY(cuda_status(cudaMemcpyAsync(st_->X, X_in, bytes, cudaMemcpyHostToDevice, s)));
  pm_status r = step_impl(st_, prm, stats, stream, V_in, cp);
  if (r != PM_OK && r != PM_ENOCONV) {   // nothing may still read the caller's host arrays
    cudaStreamSynchronize(cp->s);
    cudaStreamSynchronize(s);
    return r;
  }
  PM_TRY(cuda_status(cudaEventRecord(cp->fork, s)));
  PM_TRY(cuda_status(cudaStreamWaitEvent(cp->s, cp->fork, 0)));
  PM_TRY(cuda_status(cudaMemcpyAsync(V_out, st_->V, bytes, cudaMemcpyDeviceToHost, cp->s)));
  PM_TRY(cuda_status(cudaMemcpyAsync(X_out, st_->X, bytes, cudaMemcpyDeviceToHost, s)));
  PM_TRY(cuda_status(cudaEventRecord(cp->join, cp->s)));
  PM_TRY(cuda_status(cudaStreamWaitEvent(s, cp->join, 0)));
  PM_TRY(cuda_status(cudaStreamSynchronize(s)));
  return r;
}

namespace {

const char kCkptMagic[8] = {'P', 'M', 'G', 'B', 'C', 'K', 'P', '1'};
struct CkptHeader {
  char magic[8];
  int32_t n;
  int32_t have_prev;
  int64_t np;
  int32_t has_id, has_eps;
};

// Copies `bytes` between device memory and a file through a host staging
// buffer (dir 0: device -> file, 1: file -> device).
pm_status ckpt_stream(FILE* f, void* dev, size_t bytes, int dir, char* stage, size_t cap) {
  char* d = static_cast<char*>(dev);
  for (size_t off = 0; off < bytes; off += cap) {
    const size_t len = bytes - off < cap ? bytes - off : cap;
    if (dir == 0) {
      PM_TRY(cuda_status(cudaMemcpy(stage, d + off, len, cudaMemcpyDeviceToHost)));
      if (fwrite(stage, 1, len, f) != len) return PM_EIO;
    } else {
      if (fread(stage, 1, len, f) != len) return PM_EIO;
      PM_TRY(cuda_status(cudaMemcpy(d + off, stage, len, cudaMemcpyHostToDevice)));
    }
  }
  return PM_OK;
}

pm_status ckpt_arrays(const pm_state& S, FILE* f, int dir) {
  const size_t cap = (size_t)64 << 20;
  const int64_t N = (int64_t)S.n * S.n * S.n;
  const size_t total = (size_t)S.np * 24 + (S.id ? (size_t)S.np * 4 : 0) + (size_t)N * 4 * (S.eps ? 2 : 1);
  const size_t sz = total < cap ? (total > 0 ? total : 1) : cap;
  char* stage = static_cast<char*>(malloc(sz));
  if (!stage) return PM_EIO;
  pm_status r = ckpt_stream(f, S.X, (size_t)S.np * 12, dir, stage, sz);
  if (r == PM_OK) r = ckpt_stream(f, S.V, (size_t)S.np * 12, dir, stage, sz);
  if (r == PM_OK && S.id) r = ckpt_stream(f, S.id, (size_t)S.np * 4, dir, stage, sz);
  if (r == PM_OK) r = ckpt_stream(f, S.phi, (size_t)N * 4, dir, stage, sz);
  if (r == PM_OK && S.eps) r = ckpt_stream(f, S.eps, (size_t)N * 4, dir, stage, sz);
  free(stage);
  return r;
}

bool ckpt_args(const pm_state* s, const char* path) {
  return s && path && valid_n(s->n) && valid_np(s->np) && (s->np == 0 || (s->X && s->V)) && s->phi;
}

}  // namespace

pm_status pm_state_save(const pm_state* s, const char* path, void* stream) {
  if (!ckpt_args(s, path)) return PM_EINVAL;
  PM_TRY(cuda_status(cudaStreamSynchronize(as_stream(stream))));
  FILE* f = fopen(path, "wb");
  if (!f) return PM_EIO;
  CkptHeader h;
  memset(&h, 0, sizeof(h));
  memcpy(h.magic, kCkptMagic, 8);
  h.n = s->n;
  h.have_prev = s->have_prev;
  h.np = s->np;
  h.has_id = s->id != nullptr;
  h.has_eps = s->eps != nullptr;
  pm_status r = fwrite(&h, sizeof(h), 1, f) == 1 ? PM_OK : PM_EIO;
  if (r == PM_OK) r = ckpt_arrays(*s, f, 0);
  if (fclose(f) != 0 && r == PM_OK) r = PM_EIO;
  return r;
}

pm_status pm_state_load(pm_state* s, const char* path, void* stream) {
  if (!ckpt_args(s, path)) return PM_EINVAL;
  PM_TRY(cuda_status(cudaStreamSynchronize(as_stream(stream))));
  FILE* f = fopen(path, "rb");
  if (!f) return PM_EIO;
  CkptHeader h;
  pm_status r = fread(&h, sizeof(h), 1, f) == 1 ? PM_OK : PM_EIO;
  if (r == PM_OK && (memcmp(h.magic, kCkptMagic, 8) != 0 || h.n != s->n || h.np != s->np ||
                     h.has_id != (s->id != nullptr) || h.has_eps != (s->eps != nullptr)))
    r = PM_EIO;
  if (r == PM_OK) r = ckpt_arrays(*s, f, 1);
  fclose(f);
  if (r == PM_OK) s->have_prev = h.have_prev;
  return r;
}

pm_status pm_deposit_adj(const uint32_t* X, int64_t np, int n, const float* rho_bar, float* dX_bar, void* stream) {
  if (!valid_n(n) || !valid_np(np) || (np > 0 && (!X || !dX_bar)) || !rho_bar || !all_a16(X, rho_bar, dX_bar))
    return PM_EINVAL;
  const float s_rho = np > 0 ? (float)((double)n * n * n / (double)np) : 0.0f;
  return pos_grad_launch(X, np, n, nullptr, nullptr, rho_bar, s_rho, nullptr, nullptr, 0.0f, nullptr, dX_bar,
                         nullptr, as_stream(stream));
}

pm_status pm_interp_adj(const float* g, const uint32_t* X, int64_t np, int n, const float* acc_bar, float* g_bar,
                        float* dX_bar, void* ws, size_t ws_bytes, void* stream) {
  if (!valid_n(n) || !valid_np(np) || !g || !g_bar || (np > 0 && (!X || !acc_bar || !dX_bar))) return PM_EINVAL;
  if (!all_a16(g, X, acc_bar, g_bar, dX_bar)) return PM_EINVAL;
  Workspace w;
  PM_TRY(check_ws(w, ws, ws_bytes, n, np, PM_WS_SORT | PM_WS_ADJ));
  cudaStream_t s = as_stream(stream);
  const int64_t N = (int64_t)n * n * n;
  uint32_t* perm;
  PM_TRY(sort_cells(X, np, n, w, s, w.cellstart, &perm));
  // sorted positions and sorted acc_bar (the three planes permuted like X)
  PM_TRY(permute_particles(perm, np, X, acc_bar, nullptr, w.Xs, w.adj_abar, nullptr, s));
  for (int d = 0; d < 3; ++d)
    PM_TRY(deposit_sorted_values(w.Xs, np, w.cellstart, n, w.adj_abar + d * np, 1.0f, g_bar + d * N, w.partials,
                                 w.scalars + 12, s, crowded(w)));
  return pos_grad_launch(X, np, n, g, acc_bar, nullptr, 0.0f, nullptr, nullptr, 0.0f, nullptr, dX_bar, nullptr, s);
}

pm_status pm_gradient_adj(const float* g_bar, float* phi_bar, int n, int order, void* stream) {
  if (!valid_n(n) || !g_bar || !phi_bar || (order != 3 && order != 5 && order != 7) || !all_a16(g_bar, phi_bar))
    return PM_EINVAL;
  return divergence_launch(g_bar, phi_bar, n, order, as_stream(stream));
}

pm_status mg_solve_adj(const float* phi_bar, float* f_bar, int n, const mg_params* prm, mg_stats* st, void* ws,
                       size_t ws_bytes, void* stream) {
  return mg_solve(phi_bar, f_bar, n, prm, st, ws, ws_bytes, stream);
}

pm_status pm_step_adj(pm_state* st_, const pm_step_params* prm, const float* phi_fwd, const float* X_bar_out,
                      const float* V_bar_out, float* X_bar_in, float* V_bar_in, void* stream) {
  if (!st_ || !prm || !X_bar_out || !V_bar_out || !X_bar_in || !V_bar_in) return PM_EINVAL;
  if (!all_a16(phi_fwd, X_bar_out, V_bar_out, X_bar_in, V_bar_in)) return PM_EINVAL;
  if (!all_a16(st_->X, st_->V, st_->id, st_->phi, st_->eps, st_->acc)) return PM_EINVAL;
  pm_state& S = *st_;
  const int n = S.n;
  const int64_t np = S.np;
  if (!valid_n(n) || !valid_np(np) || (np > 0 && !S.X)) return PM_EINVAL;
  if (prm->gravity != PM_GRAVITY_NEWTON && prm->gravity != PM_GRAVITY_PARAM) return PM_EINVAL;
  if (prm->grad_order != 3 && prm->grad_order != 5 && prm->grad_order != 7) return PM_EINVAL;
  if (!(prm->a > 0.0) || !valid_mg(&prm->mg)) return PM_EINVAL;
  const uint32_t flags = PM_WS_STEP | PM_WS_ADJ | (S.id ? PM_WS_IDS : 0);
  Workspace w;
  PM_TRY(check_ws(w, S.ws, S.ws_bytes, n, np, flags));
  cudaStream_t s = as_stream(stream);
  // the step's sort (cotangent deposits gather in cell order) and, without
  // phi_fwd, its force field recomputed at the input positions
  uint32_t* perm;
  PM_TRY(sort_cells(S.X, np, n, w, s, w.cellstart, &perm));
  PM_TRY(permute_particles(perm, np, S.X, nullptr, nullptr, w.Xs, nullptr, nullptr, s));
  mg_params mp = prm->mg;
  mp.first_guess = MG_GUESS_JACOBI;
  mp.fixed_cycles = 0;
  const float src_scale = (float)poisson_scale(*prm);
  const float* phi = phi_fwd;
  if (!phi) {
    PM_TRY(deposit_sorted(w.Xs, np, w.cellstart, n, w.rho, w.partials, w.scalars, s, crowded(w)));
    pm_status r = mg_solve_src(Src{w.rho, src_scale, w.scalars}, w.adj_phi, n, mp, nullptr, w, s);
    if (r != PM_OK && r != PM_ENOCONV) return r;
    phi = w.adj_phi;
  }
  PM_TRY(gradient_launch(phi, nullptr, 0.0f, w.g, n, prm->grad_order, false, s));
  // reverse sweep
  PM_TRY(adj_accel_launch(X_bar_out, V_bar_out, np, (float)prm->dt_kick, (float)prm->dt_drift, w.adj_abar, s));
  const int64_t N = (int64_t)n * n * n;
  for (int d = 0; d < 3; ++d)
    PM_TRY(deposit_sorted_values(w.Xs, np, w.cellstart, n, w.adj_abar + d * np, 1.0f, w.adj_gbar + d * N,
                                 w.partials, w.scalars + 12, s, crowded(w)));
  PM_TRY(divergence_launch(w.adj_gbar, w.rho, n, prm->grad_order, s));   // phi_bar, in the rho buffer
  PM_TRY(grid_mean(w.rho, N, w.partials, w.scalars + 13, s));
  {
    pm_status r = mg_solve_src(Src{w.rho, 1.0f, w.scalars + 13}, w.adj_psi, n, mp, nullptr, w, s);
    if (r != PM_OK && r != PM_ENOCONV) return r;
  }
  const float s_rho = np > 0 ? (float)((double)src_scale * (double)n * n * n / (double)np) : 0.0f;
  PM_TRY(pos_grad_launch(w.Xs, np, n, w.g, w.adj_abar, w.adj_psi, s_rho, X_bar_out, V_bar_out, (float)prm->dt_drift,
                         perm, X_bar_in, V_bar_in, s));
  return launch_status();
}

bool valid_batch(int n, int B, int64_t np_box) {
  if (!valid_n(n) || n < 32 || B < 1 || np_box < 0) return false;
  if ((int64_t)B * np_box >= ((int64_t)1 << 31)) return false;
  const int bbits = B > 1 ? ilog2(2 * (int64_t)B - 1) : 0;
  return 3 * ilog2(n) + bbits <= 31;   // (box, cell) keys below 2^31: the all-ones key is the sort's sentinel
}

pm_status pm_batch_workspace_size(int n, int B, int64_t np_box, size_t* bytes) {
  if (!valid_batch(n, B, np_box) || !bytes) return PM_EINVAL;
  *bytes = layout_workspace(nullptr, nullptr, n, (int64_t)B * np_box, PM_WS_STEP, B);
  return PM_OK;
}

pm_status pm_step_batch(pm_batch_state* st_, const pm_batch_params* prm, void* stream) {
  if (!st_ || !prm) return PM_EINVAL;
  pm_batch_state& S = *st_;
  const int n = S.n, B = S.B;
  const int64_t np_box = S.np_box, np = (int64_t)B * np_box;
  if (!valid_batch(n, B, np_box) || !S.phi || (np > 0 && (!S.X || !S.V))) return PM_EINVAL;
  if (!prm->src_scale || !prm->dt_kick || !prm->dt_drift || !prm->phi_rescale) return PM_EINVAL;
  if (!all_a16(S.X, S.V, S.phi) || !all_a16(prm->src_scale, prm->dt_kick, prm->dt_drift, prm->phi_rescale))
    return PM_EINVAL;
  if (prm->grad_order != 3 && prm->grad_order != 5 && prm->grad_order != 7) return PM_EINVAL;
  if (!valid_mg(&prm->mg) || prm->mg.fixed_cycles < 1 || prm->cold_cycles < 1) return PM_EINVAL;
  if (!S.ws || !aligned(S.ws)) return PM_EINVAL;
  if (S.ws_bytes < layout_workspace(nullptr, nullptr, n, np, PM_WS_STEP, B)) return PM_ENOMEM;
  Workspace w;
  layout_workspace(&w, S.ws, n, np, PM_WS_STEP, B);
  cudaStream_t s = as_stream(stream);
  Batch bt;
  bt.B = B;
  bt.np_box = np_box;
  bt.dt_kick = prm->dt_kick;
  bt.dt_drift = prm->dt_drift;
  uint32_t* perm;
  PM_TRY(sort_cells(S.X, np, n, w, s, w.cellstart, &perm, bt));
  PM_TRY(permute_particles(perm, np, S.X, S.V, nullptr, w.Xs, w.Vs, nullptr, s));
  PM_TRY(deposit_sorted_batch(w.Xs, np_box, B, w.cellstart, n, w.rho, w.partials, w.box_mean, s, crowded(w)));
  mg_params mp = prm->mg;
  if (mp.smoother == 0) mp.smoother = 2;
  mp.first_guess = S.have_prev ? MG_GUESS_SCALED : MG_GUESS_JACOBI;
  if (!S.have_prev) mp.fixed_cycles = prm->cold_cycles;
  PM_TRY(mg_solve_batch_src(Src{w.rho, 0.0f, w.box_mean, prm->src_scale}, S.phi, n, B, mp, prm->phi_rescale, w, s));
  PM_TRY(force_interp_launch(S.phi, nullptr, 0.0f, 1, prm->grad_order, w.cellstart, w.Xs, w.Vs, nullptr, np, n,
                             nullptr, S.X, S.V, nullptr, 0.0f, 0.0f, 1, s, bt));
  S.have_prev = 1;
  return launch_status();
}

pm_status pm_deposit_batch(const uint32_t* X, int64_t np_box, int n, int B, float* rho, void* ws, size_t ws_bytes,
                           void* stream) {
  const int64_t np = (int64_t)B * np_box;
  if (!valid_batch(n, B, np_box) || (np > 0 && !X) || !rho || !all_a16(X, rho)) return PM_EINVAL;
  if (!ws || !aligned(ws)) return PM_EINVAL;
  if (ws_bytes < layout_workspace(nullptr, nullptr, n, np, PM_WS_STEP, B)) return PM_ENOMEM;
  Workspace w;
  layout_workspace(&w, ws, n, np, PM_WS_STEP, B);
  cudaStream_t s = as_stream(stream);
  Batch bt;
  bt.B = B;
  bt.np_box = np_box;
  uint32_t* perm;
  PM_TRY(sort_cells(X, np, n, w, s, w.cellstart, &perm, bt));
  PM_TRY(permute_particles(perm, np, X, nullptr, nullptr, w.Xs, nullptr, nullptr, s));
  PM_TRY(deposit_sorted_batch(w.Xs, np_box, B, w.cellstart, n, rho, w.partials, w.box_mean, s, crowded(w)));
  return launch_status();
}

pm_status mg_solve_batch(const float* f, float* phi, int n, int B, const mg_params* prm, void* ws, size_t ws_bytes,
                         void* stream) {
  if (!valid_batch(n, B, 0) || !f || !phi || !valid_mg(prm) || prm->fixed_cycles < 1 || !all_a16(f, phi))
    return PM_EINVAL;
  if (prm->first_guess == MG_GUESS_SCALED) return PM_EINVAL;   // a per-box factor is pm_step_batch's business
  if (!ws || !aligned(ws)) return PM_EINVAL;
  if (ws_bytes < layout_workspace(nullptr, nullptr, n, 0, PM_WS_MG, B)) return PM_ENOMEM;
  Workspace w;
  layout_workspace(&w, ws, n, 0, PM_WS_MG, B);
  cudaStream_t s = as_stream(stream);
  const int64_t N = (int64_t)n * n * n;
  for (int b = 0; b < B; ++b) PM_TRY(grid_mean(f + b * N, N, w.partials, w.box_mean + b, s));
  mg_params mp = *prm;
  if (mp.smoother == 0) mp.smoother = 2;
  return mg_solve_batch_src(Src{f, 1.0f, w.box_mean, nullptr}, phi, n, B, mp, nullptr, w, s);
}

pm_status pm_fr_batch_workspace_size(int n, int B, size_t* bytes) {
  if (!valid_batch(n, B, 0) || !bytes) return PM_EINVAL;
  *bytes = layout_workspace(nullptr, nullptr, n, 0, PM_WS_FR, B);
  return PM_OK;
}

pm_status fr_solve_batch(const float* rho, float* eps, int n, int B, const fr_params* prm, void* ws,
                         size_t ws_bytes, void* stream) {
  if (!valid_batch(n, B, 0) || !rho || !eps || !valid_fr(prm) || prm->cycles < 1 || !all_a16(rho, eps))
    return PM_EINVAL;
  if (!ws || !aligned(ws)) return PM_EINVAL;
  if (ws_bytes < layout_workspace(nullptr, nullptr, n, 0, PM_WS_FR, B)) return PM_ENOMEM;
  Workspace w;
  layout_workspace(&w, ws, n, 0, PM_WS_FR, B);
  cudaStream_t s = as_stream(stream);
  const int64_t N = (int64_t)n * n * n;
  for (int b = 0; b < B; ++b) PM_TRY(grid_mean(rho + b * N, N, w.partials, w.box_mean + b, s));
  double fbar, kappa, c2;
  fr_background(*prm, &fbar, &kappa, &c2);
  const float sb = (float)(-prm->Om * prm->a / c2);
  fr_params fp = *prm;
  if (fp.smoother == 0) fp.smoother = 2;   // the two-sweep streaming kernel is single-box
  return fr_solve_src(Src{rho, sb, w.box_mean, nullptr}, eps, n, fp, nullptr, w, s, B);
}

pm_status pm_gradient_batch(const float* phi, float* g, int n, int B, int order, void* stream) {
  if (!valid_n(n) || B < 1 || !phi || !g || (order != 3 && order != 5 && order != 7) || !all_a16(phi, g))
    return PM_EINVAL;
  return gradient_launch(phi, nullptr, 0.0f, g, n, order, false, as_stream(stream), B);
}

pm_status pm_interp_batch(const float* g, const uint32_t* X, int64_t np_box, int n, int B, float* acc,
                          void* stream) {
  const int64_t np = (int64_t)B * np_box;
  if (!valid_n(n) || B < 1 || np_box < 0 || np >= ((int64_t)1 << 31) || !g || (np > 0 && (!X || !acc)) ||
      !all_a16(g, X, acc))
    return PM_EINVAL;
  Batch bt;
  bt.B = B;
  bt.np_box = np_box;
  return interp_launch(g, X, nullptr, nullptr, np, n, acc, nullptr, nullptr, nullptr, 0.0f, 0.0f, 0, false,
                       as_stream(stream), bt);
}

double pm_dt_supercomoving(double Om, double OL, double a0, double a1) {
  if (!(a0 > 0.0) || !(a1 > 0.0)) return NAN;
  if (a0 == a1) return 0.0;
  const double sign = a1 > a0 ? 1.0 : -1.0;
  const double lo = a1 > a0 ? a0 : a1, hi = a1 > a0 ? a1 : a0;
  const double fa = integrand(Om, OL, lo), fb = integrand(Om, OL, hi), fm = integrand(Om, OL, 0.5 * (lo + hi));
  const double whole = (hi - lo) / 6.0 * (fa + 4.0 * fm + fb);
  return sign * simpson(Om, OL, lo, hi, fa, fm, fb, whole, 1e-15 * fabs(whole), 50);
}

pm_status pm_max_speed(const float* V, int64_t np, int n, uint32_t flags, double* max_vel, void* ws,
                       size_t ws_bytes, void* stream) {
  if (!valid_n(n) || !valid_np(np) || (np > 0 && !V) || !max_vel || !all_a16(V)) return PM_EINVAL;
  Workspace w;
  PM_TRY(check_ws(w, ws, ws_bytes, n, np, flags));
  *max_vel = 0.0;
  if (np == 0) return PM_OK;
  cudaStream_t s = as_stream(stream);
  PM_TRY(max_speed_launch(V, np, reinterpret_cast<float2*>(w.partials), w.scalars + 28, s));
  double h[2];
  PM_TRY(fetch_scalars(w.scalars + 28, h, 2, s));
  *max_vel = h[1];
  return PM_OK;
}

pm_status pm_next_timestep(double a, double Om, double OL, int n, double max_acc, double max_vel, double courant,
                           double da_max, double a_end, double* dt, double* a_next) {
  if (!(a > 0.0) || !(a_end > a) || n < 1 || !(max_acc >= 0.0) || !(max_vel >= 0.0) || !(courant > 0.0) ||
      !(da_max > 0.0) || !dt || !a_next)
    return PM_EINVAL;
  const double h = 1.0 / n;
  double lim = pm_dt_supercomoving(Om, OL, a, a * (1.0 + da_max));   // a grows by the fraction da_max
  if (max_acc > 0.0) lim = fmin(lim, sqrt(h / max_acc));            // free fall over one cell
  if (max_vel > 0.0) lim = fmin(lim, h / max_vel);                  // one cell at the largest speed
  const double step = courant * lim;
  const double to_end = pm_dt_supercomoving(Om, OL, a, a_end);
  if (to_end <= step) {
    *dt = to_end;
    *a_next = a_end;
    return PM_OK;
  }
  // t(a) grows monotonically: bisection for the scale factor a step later
  double lo = a, hi = a_end;
  for (int it = 0; it < 200 && hi - lo > 1e-15 * hi; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (pm_dt_supercomoving(Om, OL, a, mid) < step) lo = mid;
    else hi = mid;
  }
  *dt = step;
  *a_next = 0.5 * (lo + hi);
  return PM_OK;
}

double pm_growth_D(double Om, double OL, double a) {
  if (!(a > 0.0)) return NAN;
  // D'' = -gamma D' + beta D in x = ln a (Appendix A), RK4 from the
  // matter-dominated growing mode D = a at a = 1e-5.
  const double x0 = log(1e-5), x1 = log(a);
  const int steps = 20000;
  const double hstep = (x1 - x0) / steps;
  double D = 1e-5, dD = 1e-5;
  auto rhs = [&](double x, double d, double dd, double* o1, double* o2) {
    const double aa = exp(x), a3 = aa * aa * aa;
    const double e2 = Om / a3 + OL;
    const double beta = 1.5 * (Om / a3) / e2, gamma = 0.5 * (1.0 + 3.0 * OL / e2);
    *o1 = dd;
    *o2 = -gamma * dd + beta * d;
  };
  double x = x0;
  for (int i = 0; i < steps; ++i) {
    double k1a, k1b, k2a, k2b, k3a, k3b, k4a, k4b;
    rhs(x, D, dD, &k1a, &k1b);
    rhs(x + 0.5 * hstep, D + 0.5 * hstep * k1a, dD + 0.5 * hstep * k1b, &k2a, &k2b);
    rhs(x + 0.5 * hstep, D + 0.5 * hstep * k2a, dD + 0.5 * hstep * k2b, &k3a, &k3b);
    rhs(x + hstep, D + hstep * k3a, dD + hstep * k3b, &k4a, &k4b);
    D += hstep / 6.0 * (k1a + 2 * k2a + 2 * k3a + k4a);
    dD += hstep / 6.0 * (k1b + 2 * k2b + 2 * k3b + k4b);
    x += hstep;
  }
  return D;
}

pm_status pm_timing_enable(int on) {
  if (on && g_timing.start.empty()) {
    g_timing.start.resize(kTimingCap);
    g_timing.stop.resize(kTimingCap);
    g_timing.cls.resize(kTimingCap);
    g_timing.bytes.resize(kTimingCap);
    for (size_t i = 0; i < kTimingCap; ++i) {
      PM_TRY(cuda_status(cudaEventCreate(&g_timing.start[i])));
      PM_TRY(cuda_status(cudaEventCreate(&g_timing.stop[i])));
    }
  }
  g_timing.on = on != 0;
  g_timing.used = 0;
  return PM_OK;
}

int pm_timing_collect(const char** names, double* ms, int64_t* launches, double* bytes, int cap) {
  if (cudaDeviceSynchronize() != cudaSuccess) return 0;
  double tot[K_NCLASS] = {0}, byt[K_NCLASS] = {0};
  int64_t cnt[K_NCLASS] = {0};
  for (size_t i = 0; i < g_timing.used; ++i) {
    float t = 0.0f;
    if (cudaEventElapsedTime(&t, g_timing.start[i], g_timing.stop[i]) == cudaSuccess) {
      tot[g_timing.cls[i]] += t;
      byt[g_timing.cls[i]] += g_timing.bytes[i];
      cnt[g_timing.cls[i]] += 1;
    }
  }
  int k = 0;
  for (int c = 0; c < K_NCLASS && k < cap; ++c) {
    if (names) names[k] = kKernelClassNames[c];
    if (ms) ms[k] = tot[c];
    if (launches) launches[k] = cnt[c];
    if (bytes) bytes[k] = byt[c];
    ++k;
  }
  return k;
}

}  // extern "C"
