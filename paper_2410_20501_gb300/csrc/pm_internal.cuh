// Internal declarations shared by the CUDA translation units of libpmgb.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pm_api.h"

namespace pmgb {

// Kernel classes for launch counting and CUDA-event timing.
enum KernelClass {
  K_KEYS, K_SORT_SCAN, K_SCATTER, K_ORDER, K_PERMUTE,
  K_DEPOSIT, K_REDUCE,
  K_MG_GUESS, K_MG_SMOOTH0, K_MG_SMOOTH, K_MG_RESTRICT, K_MG_PROLONG, K_MG_COARSE, K_MG_NORM,
  K_FR_SMOOTH0, K_FR_SMOOTH, K_FR_RESTRICT, K_FR_COARSEOP, K_FR_PROLONG, K_FR_COARSE, K_FR_NORM,
  K_GRADIENT, K_INTERP, K_ADJOINT, K_FFT, K_MISC,
  K_NCLASS
};

extern const char* const kKernelClassNames[K_NCLASS];

// Online autotuner of batched launch tiling (tune.cu).  A site calls
// tune_begin before its launch(es) with candidate values that compute bitwise
// the same result, uses the value returned, and calls tune_end after them on
// the same stream; tune_active() says whether this call is being timed.
enum TuneSite { TUNE_FORCE_CHUNK, TUNE_MG_FUSED_CHUNK, TUNE_MG_SMOOTHER };
int tune_begin(int site, int n, int B, const int* cand, int ncand, int dflt, cudaStream_t s);
void tune_end(cudaStream_t s);
bool tune_active();

void launch_begin(int cls, double bytes, cudaStream_t s);
void launch_end(int cls, cudaStream_t s);

// Records a CUDA error string and maps it to PM_ECUDA (PM_OK on cudaSuccess).
pm_status cuda_status(cudaError_t e);
// cudaGetLastError() after a batch of launches.
inline pm_status launch_status() { return cuda_status(cudaGetLastError()); }

// Raises the dynamic shared-memory limit of kernel `fn` to `bytes` on the
// current device.  The attribute belongs to the device that is current when
// it is set, so it is set once per (device, kernel) pair; the record is
// guarded by a mutex.
pm_status smem_attr_fn(const void* fn, size_t bytes);
template <class K>
inline pm_status smem_attr(K* fn, size_t bytes) {
  return smem_attr_fn(reinterpret_cast<const void*>(fn), bytes);
}

// Cells holding more particles than this are "crowded": the cell sort lists
// them (runs[0] = their number, runs[1 ..] = their cells, in no fixed order)
// and orders their particles with a warp each (a block each beyond 256
// particles, listed in bigs as well); the deposit takes their 27 TSC moments
// from a block each.
constexpr uint32_t kLongRun = 32;
// Cells holding more than kMedRun and at most kLongRun particles are
// "medium": listed apart (meds[0] = their number, meds[1 ..] = their cells),
// ordered by a warp each and their moments summed by sixteen lanes each.
constexpr uint32_t kMedRun = 13;
// The deposit's streaming kernel walks the particles of cells holding at most
// kWalkRun of them; the 27 moments of every larger cell are summed beforehand
// (cells of kWalkRun + 1 .. kMedRun particles, the sort's smalls list, by
// eight lanes each) and stored at kMomStride times the cell's
// first rank of a moment buffer of kMomStride floats per particle: a cell of
// more than kWalkRun particles owns at least 30 floats there, room for its
// 27.
constexpr uint32_t kWalkRun = 4;
constexpr int kMomStride = 6;
static_assert(kMomStride * (kWalkRun + 1) >= 27, "room for the moments of the smallest summed cell");
// Crowded cells of at most kWarpRun particles are ordered, and their moments
// summed, by a warp each; longer ones (the sort's bigs list) by a block each.
constexpr uint32_t kWarpRun = 256;

inline int ilog2(int64_t v) { int l = 0; while ((int64_t(1) << (l + 1)) <= v) ++l; return l; }
inline bool valid_n(int n) { return n >= 4 && n <= 1024 && (n & (n - 1)) == 0; }

// Grid size for a grid-stride loop over `count` items with `threads` per
// block.  By default one item per thread: blocks are then scheduled roughly in
// address order, which keeps the neighbouring-plane reuse of the stencil
// kernels inside L2 (a capped grid makes every block jump ahead by the grid's
// span on each iteration and defeats that reuse).  Reductions pass a cap.
inline unsigned grid_for(int64_t count, int threads, int64_t cap = ((int64_t)1 << 30)) {
  int64_t b = (count + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (unsigned)b;
}

// A level-0 source term  s * (p[i] - mean)  with `mean` read from device
// memory (float64), or a plain array (s = 1, mean = NULL).  In a batched
// launch (below) p covers all boxes, mean is per box and sb (if set) holds
// the per-box s.
struct Src {
  const float* p;
  float s;
  const double* mean;
  const float* sb;
};

// Batched launches: B independent boxes stored back to back (grids
// [B][n^3], vector grids [B][3][n^3]; particles [3][B * np_box] with box b's
// particles, in cell order, at b * np_box ...).  Kernels take their box from
// blockIdx.z; with B = 1 every launch is the single-box one.
struct Batch {
  int B = 1;
  int64_t np_box = 0;                   // particles per box
  const float* dt_kick = nullptr;       // per-box kick and drift (device, [B])
  const float* dt_drift = nullptr;
};

#ifdef __CUDACC__
// The source of the box of this block (blockIdx.z) on a level of N cells.
__device__ __forceinline__ Src box_src(const Src& f, int64_t N) {
  const int b = blockIdx.z;
  return Src{f.p + (int64_t)b * N, f.sb ? __ldg(f.sb + b) : f.s, f.mean ? f.mean + b : nullptr, nullptr};
}
#endif

// ------------------------------------------------------------ workspace --
// Byte offsets of every buffer inside the caller's workspace.
struct Workspace {
  char* base;
  size_t total;
  // sort
  uint2* keyrank; uint32_t* perm; uint32_t* runs; uint32_t* meds; uint32_t* bigs; uint32_t* smalls;
  uint32_t* scan_blocks; uint32_t* cellstart;
  float* moments;   // kMomStride floats per particle (the deposit's summed cell moments)
  // particles in cell order
  uint32_t* Xs; float* Vs; uint32_t* ids;
  // grids
  float* rho; float* g;
  // reductions (float64 partials) and device scalars
  double* partials; double* scalars;
  // multigrid pyramids: level l >= 1 arrays (index 0 unused)
  float* mg_u[12]; float* mg_f[12]; float* mg_alt[12];
  float* fr_e[12]; float* fr_r[12]; float* fr_b[12]; float* fr_alt[12];
  // adjoint buffers
  float* adj_abar; float* adj_phi; float* adj_psi; float* adj_gbar;
  double* box_mean;   // per-box mean density of a batch
  float2* spec;       // half spectrum n^2 (n/2 + 1) of the FFT Poisson path
  float2* lpt_a; float2* lpt_b; float* lpt_r;   // LPT: two half spectra, five real grids
  float* ref_r; float* ref_e;                   // refinement: float32 residual and correction
  int64_t np; int n; int batch;
};

// Computes the layout for (n, np, flags) and `batch` boxes of n^3 cells (np
// counts the particles of all boxes); with base == NULL only sizes.
size_t layout_workspace(Workspace* w, void* base, int n, int64_t np, uint32_t flags, int batch = 1);

// Sizes of the scratch pieces.
int64_t sort_scan_blocks(int64_t ncells);
int64_t sort_runs_capacity(int64_t np);
int64_t sort_meds_capacity(int64_t np);
int64_t sort_bigs_capacity(int64_t np);
int64_t sort_smalls_capacity(int64_t np);
int64_t reduce_partials_capacity(int n, int64_t np);
// Work items of the streaming deposit for one box of n^3 cells (n >= 32).
int deposit_items(int n);

// ------------------------------------------------------ stage launchers --
// Stable sort by cell key: *perm_out (in the workspace) lists the particles
// in cell order, ties in input order, and cellstart[c] .. cellstart[c+1]-1 are
// the ranks of cell c (cellstart [ncells + 1], cellstart[ncells] = np).  With
// a batch the key is prefixed by the box (particle index / np_box), so the
// order is by box, then cell, and ncells = B n^3.
pm_status sort_cells(const uint32_t* X, int64_t np, int n, Workspace& w, cudaStream_t s, uint32_t* cellstart,
                     uint32_t** perm_out, const Batch& bt = Batch{});
pm_status permute_particles(const uint32_t* perm, int64_t np, const uint32_t* X, const float* V,
                            const uint32_t* id, uint32_t* Xs, float* Vs, uint32_t* ids,
                            cudaStream_t s);
// The cell lists of the last cell sort (smalls, meds, runs, bigs) and the
// moment buffer (kMomStride floats per particle): the deposit sums the 27
// moments of every cell of more than kWalkRun particles into it, at
// kMomStride times the cell's first rank.  runs == NULL: every cell is walked
// by one thread.
struct Crowded {
  const uint32_t* runs = nullptr;
  const uint32_t* meds = nullptr;
  const uint32_t* bigs = nullptr;
  const uint32_t* smalls = nullptr;
  float* moments = nullptr;
};
// rho = (n^3/np) TSC sum over cell-sorted particles; writes sum(rho)/n^3 to *mean_out.
pm_status deposit_sorted(const uint32_t* Xs, int64_t np, const uint32_t* cellstart, int n,
                         float* rho, double* partials, double* mean_out, cudaStream_t s,
                         const Crowded& cr = Crowded{});
// General form: rho[c] = scale * sum_p vals[p] W(x_p - x_c) (vals may be NULL
// for 1); *mean_out = sum(rho)/n^3.
pm_status deposit_sorted_values(const uint32_t* Xs, int64_t np, const uint32_t* cellstart, int n,
                                const float* vals, float scale, float* rho, double* partials,
                                double* mean_out, cudaStream_t s, const Crowded& cr = Crowded{});
// Batched deposit (n >= 32): box b's density [n^3] from its particles (the
// cell starts cover all boxes); mean_out[b] = box b's mean.
pm_status deposit_sorted_batch(const uint32_t* Xs, int64_t np_box, int B, const uint32_t* cellstart, int n,
                               float* rho, double* partials, double* mean_out, cudaStream_t s,
                               const Crowded& cr = Crowded{});
// out[k] = scale * sum_{i < count} partials[k * stride + i] for k < nout (one block).
pm_status reduce_partials(const double* partials, int64_t count, int64_t stride, int nout,
                          double scale, double* out, cudaStream_t s);
// Mean of a float32 grid into *mean_out (float64, fixed-order reduction).
pm_status grid_mean(const float* f, int64_t count, double* partials, double* mean_out,
                    cudaStream_t s);

pm_status mg_solve_src(Src f, float* phi, int n, const mg_params& prm, mg_stats* st,
                       Workspace& w, cudaStream_t s);
// Mixed-precision iterative refinement: `outer` steps of float64 residual of
// the float64 iterate phi, float32 multigrid correction (prm), float64 update;
// st->res0 / st->res: float64 residual norms before the first and after the
// last step.  Needs the PM_WS_MG | PM_WS_REFINE workspace; fmean: <f> (device).
pm_status mg_solve_refine_src(const float* f, const double* fmean, double* phi, int n, int outer,
                              const mg_params& prm, mg_stats* st, Workspace& w, cudaStream_t s);
// Batched multigrid: fixed cycles only (prm.fixed_cycles > 0); the warm start
// MG_GUESS_SCALED takes the per-box factors gbox [B] (device).
pm_status mg_solve_batch_src(Src f, float* phi, int n, int B, const mg_params& prm, const float* gbox,
                         Workspace& w, cudaStream_t s);
// B > 1: B boxes back to back ([B][n^3]; per-box source scale and mean as in
// Src), prm.cycles fixed cycles each, st unused.
pm_status fr_solve_src(Src b, float* eps, int n, const fr_params& prm, mg_stats* st,
                       Workspace& w, cudaStream_t s, int B = 1);
// u_fine += P(uc - uc2) (27/9/3/1 prolongation; uc2 may be NULL), on B
// boxes back to back.
pm_status prolong_correct_launch(float* u, const float* uc, const float* uc2, int n_fine, int cls,
                                 cudaStream_t s, int B = 1);
// Background constants of the f(R) equation (host, float64).
void fr_background(const fr_params& p, double* fbar, double* kappa, double* c2);

// g = -grad(phi [+ alpha ((1 + eps)^(nh+1) - 1)]); vec4: g interleaved as float4
// (gx, gy, gz, 0) per cell (n >= 64 only), else three planes.
pm_status gradient_launch(const float* phi, const float* eps, float alpha, float* g, int n,
                          int order, bool vec4, cudaStream_t s, int batch = 1, int nh = 1);
// mode 0: acc only; mode 1: kick + drift into Xo/Vo (and acc if non-NULL);
// vec4: g interleaved as float4.  With max_out (2 doubles, device) also the
// largest |a| and |v after the kick| (blockmax: one float2 per block).
pm_status interp_launch(const float* g, const uint32_t* Xs, const float* Vs, const uint32_t* ids_in,
                        int64_t np, int n, float* acc, uint32_t* Xo, float* Vo, uint32_t* ids_out,
                        float dt_kick, float dt_drift, int mode, bool vec4, cudaStream_t s,
                        const Batch& bt = Batch{}, float2* blockmax = nullptr, double* max_out = nullptr);

// The force g = -grad(phi [+ alpha ((1 + eps)^(nh+1) - 1)]) (order 3, 5 or
// 7) computed in shared memory and interpolated at the cell-sorted particles
// (with their cell starts; n >= 32) in one pass, as gradient_launch followed
// by interp_launch (same arithmetic), without the force field in HBM.
pm_status force_interp_launch(const float* phi, const float* eps, float alpha, int nh, int order,
                              const uint32_t* cellstart, const uint32_t* Xs, const float* Vs, const uint32_t* ids_in,
                              int64_t np, int n, float* acc, uint32_t* Xo, float* Vo, uint32_t* ids_out,
                              float dt_kick, float dt_drift, int mode, cudaStream_t s, const Batch& bt = Batch{},
                              float2* blockmax = nullptr, double* max_out = nullptr);

// phi = scale * IFFT[G FFT[rho - mean]], G(0) = 0; kind 1: FFT_7pt, 2: FFT
// with the exact kernel and TSC deconvolution (§3.7); mean (device float64)
// may be NULL.  C: n^2 (n/2 + 1) float2.
pm_status fft_poisson_launch(const float* rho, const double* mean, float* phi, float2* C, int n, int kind,
                             double scale, cudaStream_t s);

// 2LPT (1LPT when e2 = v2 = 0) particles on the n^3 lattice from real white
// noise and the spectrum amplitude amp [n][n][n/2+1]: X = q + d1 Psi1 + e2 Psi2,
// V = v1 Psi1 + v2 Psi2 (§3.3).  A, B: half spectra; R: 5 n^3 floats.
pm_status lpt2_launch(const float* noise, const float* amp, int n, double d1, double e2, double v1, double v2,
                      uint32_t* X, float* V, float2* A, float2* B, float* R, cudaStream_t s);

// max_out[1] = the largest |v| of V [3][np] (max_out[0] = 0); blockmax:
// at most 152 * 16 float2.
pm_status max_speed_launch(const float* V, int64_t np, float2* blockmax, double* max_out, cudaStream_t s);

// Adjoint pieces (adjoint.cu).
pm_status divergence_launch(const float* gbar, float* phibar, int n, int order, cudaStream_t s);
pm_status adj_accel_launch(const float* xbar_out, const float* vbar_out, int64_t np, float dt_kick,
                           float dt_drift, float* abar, cudaStream_t s);
pm_status pos_grad_launch(const uint32_t* X, int64_t np, int n, const float* g, const float* abar,
                          const float* psi, float s_rho, const float* xbar_out, const float* vbar_out,
                          float dt_drift, const uint32_t* perm, float* xbar_in, float* vbar_in,
                          cudaStream_t s);

// Copies `count` doubles of device reduction results to host (synchronises).
pm_status fetch_scalars(const double* dev, double* host, int count, cudaStream_t s);

}  // namespace pmgb

// Launch with instrumentation: `bytes` is the kernel's algorithmic (compulsory)
// DRAM traffic for this launch, accumulated per class while timing is on.
#define PM_LAUNCH(cls, bytes, kern, grid, block, smem, st, ...)       \
  do {                                                                 \
    ::pmgb::launch_begin((cls), (double)(bytes), (st));                \
    kern<<<(grid), (block), (smem), (st)>>>(__VA_ARGS__);              \
    ::pmgb::launch_end((cls), (st));                                   \
  } while (0)

#define PM_TRY(expr)                       \
  do {                                     \
    pm_status _st = (expr);                \
    if (_st != PM_OK) return _st;          \
  } while (0)
