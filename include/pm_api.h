/*
 * pm_api.h - C ABI of the GB300 (sm_103a) particle-mesh force step of
 * PySCo (arXiv 2410.20501).
 *
 * The library computes, on one GPU, the per-step PM force evaluation of §3.4-§3.10
 * and the kick-drift-kick update of §3.4 ("Integrator"):
 *   cell keys + stable cell sort  ->  TSC mass assignment (§3.4)
 *   -> multigrid Poisson solve of the 7-point Laplacian (§3.5, §3.6.1)
 *   -> [f(R)] FAS multigrid for the Hu-Sawicki scalaron (§3.6.2, §3.10)
 *   -> central-difference gradient (Table 1) -> inverse TSC (§3.4)
 *   -> kick-drift-kick with uint32 fixed-point positions.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - n is the number of cells per side, a power of two, 4 <= n <= 1024.
 *  - Scalar grids are float32 [n][n][n] in C order (cell (i,j,k) at index
 *    (i*n + j)*n + k, cell centres at (i + 1/2)/n), as in §3.2.  Vector grids
 *    are three such planes, x then y then z.
 *  - Particle positions are uint32 fixed-point box coordinates, three planes
 *    [3][np]: x = X * 2^-32 in [0, 1), so periodic wrap is exact.  Velocities
 *    and accelerations are float32 planes [3][np] in supercomoving units (§3.1:
 *    box length 1, time unit t_* = a^2/H0).
 *  - Every pointer argument is caller-owned DEVICE memory unless the
 *    description says "host".  The library never allocates device memory: work
 *    buffers come from the caller as one workspace of pm_workspace_size() bytes,
 *    aligned to 256 bytes.  Every other device array must start on a 16-byte
 *    boundary (cudaMalloc and PyTorch allocations start on 256 bytes; a view
 *    at an odd float offset does not): kernels move grids as float2/float4.
 *    A misaligned array is an argument error (PM_EINVAL).  Arrays must not
 *    alias unless stated.
 *  - Work is enqueued asynchronously on `stream` (a cudaStream_t; NULL = the
 *    legacy default stream).  Argument errors are detected synchronously and
 *    nothing is enqueued.  Entry points that test convergence (mg_solve,
 *    fr_solve, pm_step with tolerances) synchronise `stream` once per cycle to
 *    read an 8-byte residual norm; with fixed cycle counts they never sync.
 *    mg_solve_refine synchronises once per refinement step (its float64
 *    residual norm).
 *  - Results are deterministic: no floating-point atomics are used anywhere,
 *    every reduction has a fixed order, so reruns are bitwise identical.
 *  - Not thread-safe: calls must come from one host thread at a time.  The
 *    library's per-device state (kernel shared-memory limits, its second
 *    streams, the scratch address of pm_deposit_noalloc) is kept per device,
 *    so one process may drive several GPUs, one call at a time.
 */
#ifndef PM_API_H
#define PM_API_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int pm_status;
enum {
  PM_OK = 0,
  PM_EINVAL = 1,    /* bad size, null or misaligned pointer, or bad parameter    */
  PM_ENOMEM = 2,    /* workspace smaller than pm_workspace_size()                 */
  PM_ENOCONV = 3,   /* solver hit max_cycles without meeting its tolerance        */
  PM_ENAN = 4,      /* a residual norm was not finite                             */
  PM_ETIMEOUT = 5,  /* a device-side bounded wait gave up                         */
  PM_ECUDA = 6,     /* a CUDA runtime call failed (see pm_last_cuda_error)        */
  PM_EIO = 7        /* a checkpoint file could not be written, read or matched    */
};

/* Human-readable name of a status code (static string). */
const char* pm_status_string(pm_status s);
/* Last CUDA error string seen by the library (static string, "" if none). */
const char* pm_last_cuda_error(void);
/* Library version, e.g. "1.0.0". */
const char* pm_version(void);

/* Flags for pm_workspace_size: which entry points the workspace must serve. */
enum {
  PM_WS_SORT = 1,      /* pm_sort, pm_deposit                                  */
  PM_WS_MG = 2,        /* mg_solve                                             */
  PM_WS_FR = 4,        /* fr_solve                                             */
  PM_WS_STEP = 8,      /* pm_step, pm_step_host (includes all of the above)    */
  PM_WS_IDS = 16,      /* pm_step carries particle ids (pm_state.id != NULL)   */
  PM_WS_ADJ = 32,      /* adjoint entry points (with PM_WS_SORT or PM_WS_STEP) */
  PM_WS_FFT = 64,      /* FFT Poisson solver (pm_poisson_fft, pm_step with
                          poisson != PM_POISSON_MG): the half spectrum          */
  PM_WS_LPT = 128,     /* pm_lpt2: two half spectra and five grids             */
  PM_WS_REFINE = 256   /* mg_solve_refine (with PM_WS_MG): residual and
                          correction grids                                      */
};

/* Bytes of workspace needed for grids of n^3 cells and np particles.
 * Returns PM_EINVAL for a bad n or np < 0.  *bytes is a host pointer. */
pm_status pm_workspace_size(int n, int64_t np, uint32_t flags, size_t* bytes);

/* ---------------------------------------------------------------- sorting --
 * Cell ordering that replaces the periodic Morton reordering of §3.2 and
 * Appendix E: key = (i*n + j)*n + k of the cell containing each particle
 * (i = floor(x n)), then a stable sort (ties keep input order).
 *   X          [3][np] uint32 positions (read)
 *   perm       [np]    out: perm[r] = input index of the particle of rank r
 *   cellstart  [n^3+1] out: particles of cell c are ranks cellstart[c] ..
 *                      cellstart[c+1]-1 (cellstart[n^3] = np)
 * Either output may be NULL (not written).  Integer results are bit-exact. */
pm_status pm_sort(const uint32_t* X, int64_t np, int n, uint32_t* perm,
                  uint32_t* cellstart, void* ws, size_t ws_bytes, void* stream);

/* --------------------------------------------------------------- deposit --
 * TSC mass assignment (§3.4, W_TSC) as a deterministic cell-sorted gather:
 *   rho[c] = (n^3/np) * sum_p prod_d W_TSC(n x_p,d - (c_d + 1/2)),
 * so the grid sums to n^3 (mean density 1; equals the paper's
 * sum rho = N_part when np = n^3).  np = 0 gives rho = 0.
 *   X    [3][np] uint32 positions (read);  rho [n^3] float32 (written). */
pm_status pm_deposit(const uint32_t* X, int64_t np, int n, float* rho,
                     void* ws, size_t ws_bytes, void* stream);

/* pm_deposit for callers that cannot allocate device memory.  Some callers
 * cannot call cudaMalloc: a host application whose memory pool owns the whole
 * device and forbids other allocations, a code path that must not pay
 * cudaMalloc's implicit device synchronisation, or a foreign-language binding
 * that has no device allocator; they cannot provide the workspace pm_deposit
 * needs.  This entry point computes the same density as pm_deposit but takes
 * its scratch from one static device array of 16 MiB inside the library (held
 * on every GPU that loads the library until the process exits), so it
 * allocates nothing.  The paper has no counterpart.
 *   Limits: n <= 64 and np <= 262144 (2^18); larger sizes return PM_EINVAL.
 *   The caller still passes X (device, [3][np] uint32) and rho (device,
 *   [n^3] float32).
 *   Each call made outside stream capture looks up the array's device
 *   address with cudaGetSymbolAddress (with the calling device current); a
 *   call captured into a CUDA graph uses the address found by the last
 *   uncaptured call on that device.  So make the first call on a device, and
 *   the first call after a device reset, before any stream capture (a
 *   captured call with no address on record returns PM_EINVAL).
 *   Every call shares the array: calls that overlap on the GPU (different
 *   streams, or different host threads) race on it and give wrong results. */
pm_status pm_deposit_noalloc(const uint32_t* X, int64_t np, int n, float* rho, void* stream);

/* ------------------------------------------------------------- multigrid -- */
enum { MG_GUESS_INPUT = 0, MG_GUESS_JACOBI = 1, MG_GUESS_SCALED = 2 };

typedef struct {
  int npre, npost;        /* Gauss-Seidel sweeps before / after the coarse
                             correction (§3.6.1 Npre / Npost)                    */
  float omega;            /* SOR factor (§3.6.1, 1.25); omega = 1 is applied on
                             the first pre-sweep and the last post-sweep         */
  int coarsest;           /* size of the coarsest level (§3.6.1: 16)           */
  int coarse_max_sweeps;  /* coarsest level: at most this many sweeps ...      */
  float coarse_drop;      /* ... or until its residual dropped by this factor  */
  int max_cycles;         /* cap on cycles (PM_ENOCONV beyond)                  */
  int fixed_cycles;       /* > 0: run exactly this many cycles, no norms, no
                             host synchronisation (CUDA-graph capturable)       */
  double tol;             /* stop when ||f - L phi||_2 <= tol ||f||_2           */
  double stall;           /* also stop (PM_OK) when a cycle reduced the residual
                             by less than 1/stall while it is below 1e-3 ||f||:
                             the float32 floor of the stored iterate           */
  int first_guess;        /* MG_GUESS_INPUT: phi holds the guess;
                             MG_GUESS_JACOBI: -h^2 f / 6 (Eq. multigrid_initial_guess);
                             MG_GUESS_SCALED: guess_scale * phi (the warm start
                             of Eq. rescaming_newtonian_potential)              */
  float guess_scale;
  int smoother;           /* 2: one fused red-black sweep per pass over memory
                             on levels with n >= 128 (bitwise equal to the
                             colour passes), colour passes below;
                             1: colour passes (one kernel per colour)
                             everywhere; 0: two sweeps per pass on levels with
                             n >= 128 (streaming kernel)                       */
  float coarse_omega;     /* SOR factor of the coarsest-level sweeps; 0: the
                             optimal one for that grid, 2/(1 + sqrt(1 - mu^2)),
                             mu = (2 + cos(2 pi/n))/3 (1.634 at 16^3)          */
} mg_params;

typedef struct {
  int status;             /* pm_status of the solve                            */
  int cycles;             /* cycles run                                        */
  double norm_f;          /* ||f - <f>||_2                                      */
  double res0;            /* residual norm before the first cycle (only with
                             tolerances; computed after the first cycle
                             otherwise: -1)                                      */
  double res;             /* residual norm after the last cycle (-1 if fixed)  */
} mg_stats;

/* Default parameters: npre = npost = 2, omega = 1.25, coarsest = 16,
 * coarse_max_sweeps = 200, coarse_drop = 1e-3, max_cycles = 30,
 * fixed_cycles = 0, tol = 1e-7, stall = 0.5, first_guess = MG_GUESS_INPUT,
 * smoother = 2, coarse_omega = 0. */
void mg_default_params(mg_params* p);

/* Solve the periodic Poisson problem (L(phi) - 6 phi)/h^2 = f - <f>, h = 1/n,
 * with red-black SOR V-cycles (§3.5, §3.6.1): restriction by 8-child average,
 * prolongation 27/9/3/1 over 64, zero initial guess for the coarse error,
 * red-black SOR sweeps on the coarsest level (see coarse_drop / coarse_omega).  Smoothing and transfers run in
 * float32; the finest-level residual is evaluated with compensated float32
 * arithmetic and its norm accumulated in float64.
 *   f    [n^3] float32 right-hand side (read; its float64 mean is removed)
 *   phi  [n^3] float32 in: guess (see first_guess), out: solution
 *   st   host mg_stats (may be NULL) */
pm_status mg_solve(const float* f, float* phi, int n, const mg_params* prm,
                   mg_stats* st, void* ws, size_t ws_bytes, void* stream);

/* The same Poisson problem by mixed-precision iterative refinement: float32
 * multigrid inside, float64 only for the outer residual, the iterate's update
 * and the global reductions.  Each of `outer` steps forms, in float64,
 *   r = (f - <f>) - (L(phi) - 6 phi)/h^2
 * of the float64 iterate (the neighbour sum minus 6 phi, in float64),
 * solves (L(e) - 6e)/h^2 = r - <r> in float32 from e = 0 with prm's cycles
 * (fixed_cycles, or tol relative to ||r||), and adds e to phi in float64.  The
 * float32 solve of mg_solve stops at the float32 resolution of its stored
 * iterate; this one keeps converging to the float64 level (measured against
 * the exact inverse in the tests).
 *   f      [n^3] float32 right-hand side (read; its float64 mean is removed)
 *   phi    [n^3] float64 in: guess (zeros: none), out: solution; 16-byte aligned
 *   outer  refinement steps (>= 1)
 *   prm    multigrid parameters of each correction solve (first_guess is
 *          ignored: the correction starts from 0; MG_GUESS_SCALED is rejected)
 *   st     host mg_stats (may be NULL): res0 / res = float64 residual norms
 *          before the first and after the last step, norm_f = ||f - <f>||,
 *          cycles = V-cycles of all correction solves
 * Workspace: pm_workspace_size(n, 0, PM_WS_MG | PM_WS_REFINE).  Synchronises
 * with the host once per step (the residual norm).  Errors: PM_EINVAL,
 * PM_ENOMEM (ws too small), PM_ENAN (a residual not finite). */
pm_status mg_solve_refine(const float* f, double* phi, int n, int outer, const mg_params* prm, mg_stats* st,
                          void* ws, size_t ws_bytes, void* stream);

/* Poisson solve by 3-D FFT (§3.7): phi = scale * G * (rho - <rho>), with the
 * Green's function of kind PM_POISSON_FFT7 (FFT_7pt: 1 / the Fourier symbol
 * -(4/h^2) sum_d sin^2(pi m_d / n) of the 7-point Laplacian, no mass-
 * assignment compensation: the exact inverse that converged multigrid
 * approaches) or PM_POISSON_FFT (-1 / (k^2 W_TSC(k)^2), k = 2 pi m,
 * W_TSC = prod_d sinc(pi m_d / n)^3: the exact Laplacian with the TSC
 * window deconvolved).  G(0) = 0, so phi has zero mean.  The FFTs are the
 * library's own (shared-memory Stockham, float32).
 *   rho [n^3] (read), phi [n^3] (written); 16 <= n <= 1024.
 * Workspace: pm_workspace_size(n, 0, PM_WS_FFT). */
pm_status pm_poisson_fft(const float* rho, float* phi, int n, int kind, double scale, void* ws, size_t ws_bytes,
                         void* stream);

/* Initial conditions by Lagrangian perturbation theory (§3.3): one particle
 * per cell centre q of the n^3 lattice (lattice order, index (i n + j) n + k),
 * moved to X = q + d1 Psi1 + e2 Psi2 with velocity V = v1 Psi1 + v2 Psi2,
 * where delta_k = amp_k FFT(noise)_k, phi1 = grad^-2 delta, Psi1 = -grad phi1,
 * phi2 = (1/2) grad^-2 [phi1_ii phi1_jj - phi1_ij phi1_ij], Psi2 = grad phi2
 * (spectral derivatives, k = 2 pi m in box units, modes on Nyquist planes set
 * to zero).  e2 = v2 = 0 gives first order (no second-order work).  The
 * factors are the caller's: d1 = D(a)/D(1), e2 the second-order growth
 * factor, v1 = a^2 E(a) d1 f1, v2 = a^2 E(a) e2 f2 (§3.1 velocity units).
 *   noise [n^3] real white noise, amp [n][n][n/2+1] = sqrt(P(k) n^3 / L^3)
 *   (read); X [3][n^3] uint32 fixed point, V [3][n^3] (written); n >= 16.
 * Workspace: pm_workspace_size(n, 0, PM_WS_LPT). */
pm_status pm_lpt2(const float* noise, const float* amp, int n, double d1, double e2, double v1, double v2,
                  uint32_t* X, float* V, void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------ f(R) -- */
typedef struct {
  double a;          /* scale factor                                          */
  double Om, OL;     /* density parameters today (flat)                       */
  double fR0;        /* f_R0 < 0 (Hu-Sawicki)                                  */
  double boxsize;    /* box size in Mpc/h (sets c~ = c / (H0 L))              */
  int cycle;         /* 0 = V-cycle, 1 = F-cycle (default: one F-cycle, §3.10) */
  int npre, npost, coarsest, coarse_max_sweeps;
  float coarse_drop;
  int cycles;        /* cycles to run when tol <= 0                           */
  double tol;        /* > 0: cycle until ||b - N(u)|| <= tol ||b|| (synchronises) */
  int max_cycles;
  int smoother;      /* as mg_params.smoother                                   */
  int nhs;           /* Hu-Sawicki exponent n: 1 (cubic per cell) or 2 (quartic,
                        §3.10); 0 is taken as 1                                 */
} fr_params;

void fr_default_params(fr_params* p);

/* Hu-Sawicki n = 1 scalaron (§3.10, Eq. fr_sim_2) by non-linear FAS multigrid
 * (§3.6.2).  With u = (f~_R / fbar)^(1/2) the discrete equation is
 *   (fbar/h^2)(L(u^2) - 6u^2) - kappa (1/u - 1) = -(Om a / c~^2)(rho - <rho>),
 * kappa = a^4 R~ / (3 c~^2), R~ = 3 Om (a^-3 + 4 OL/Om), fbar = a^2 fR0 (R~0/R~)^2,
 * each Gauss-Seidel update being the positive root of the depressed cubic of
 * Eq. fr_depressed_equation.  The unknown is stored as eps = u - 1 and the
 * cubic solved in that variable in float32 (safeguarded Newton).
 *   rho  [n^3] float32 density (read)
 *   eps  [n^3] float32 in: guess (0 = background), out: solution
 *   st   host mg_stats (may be NULL) */
pm_status fr_solve(const float* rho, float* eps, int n, const fr_params* prm,
                   mg_stats* st, void* ws, size_t ws_bytes, void* stream);

/* -------------------------------------------------------------- gradient --
 * g = -grad(phi) with the central stencils of Table 1 (order 3, 5 or 7),
 * periodic.  phi [n^3] (read), g [3][n^3] (written). */
pm_status pm_gradient(const float* phi, float* g, int n, int order, void* stream);

/* ---------------------------------------------------------- interpolation --
 * Inverse TSC (§3.4): acc_p = sum_c W_TSC(x_p - x_c) g_c over the 27 cells.
 *   g [3][n^3] (read), X [3][np] (read), acc [3][np] (written). */
pm_status pm_interp(const float* g, const uint32_t* X, int64_t np, int n,
                    float* acc, void* stream);

/* ------------------------------------------------------------------ step -- */
typedef struct {
  int n;
  int64_t np;
  uint32_t* X;     /* [3][np] positions, updated in place                     */
  float* V;        /* [3][np] velocities, updated in place                    */
  uint32_t* id;    /* [np] particle ids permuted along, or NULL               */
  float* phi;      /* [n^3] potential: previous step's on input (warm start),
                      this step's on output                                   */
  float* eps;      /* [n^3] f(R) eps = u - 1 (previous / this step), or NULL  */
  float* acc;      /* [3][np] if not NULL: accelerations of this step, in the
                      particles' new (sorted) order                           */
  void* ws;
  size_t ws_bytes;
  int have_prev;   /* 0 before the first step: Jacobi first guess for phi and
                      u = 1 for f(R); set to 1 by pm_step                     */
} pm_state;

enum { PM_GRAVITY_NEWTON = 0, PM_GRAVITY_FR = 1, PM_GRAVITY_PARAM = 2 };
enum { PM_POISSON_MG = 0, PM_POISSON_FFT7 = 1, PM_POISSON_FFT = 2 };

typedef struct {
  double a;            /* scale factor of this force evaluation              */
  double Om, OL;       /* cosmology (flat)                                   */
  double boxsize;      /* Mpc/h                                              */
  int gravity;         /* PM_GRAVITY_NEWTON, PM_GRAVITY_FR or PM_GRAVITY_PARAM
                          (parametrised: the Poisson source times
                          mu(a) = 1 + mu0 Omega_L(a)/Omega_L,0 = 1 + mu0/E(a)^2,
                          §2.4, Eq. mu_parametrized_gravity)                  */
  double fR0;          /* for PM_GRAVITY_FR                                  */
  int grad_order;      /* 3, 5 or 7 (Table 1); 5 by default                  */
  double dt_kick;      /* v += acc * dt_kick (sum of the two half kicks of
                          the leapfrog around this force evaluation)         */
  double dt_drift;     /* then x += v * dt_drift (0: kick only)              */
  double phi_rescale;  /* warm start: phi_guess = phi_rescale * phi_prev     */
  mg_params mg;        /* Poisson multigrid; fixed_cycles applies to warm-
                          started steps only (have_prev = 1): the first step
                          always cycles to tol from the Jacobi guess         */
  fr_params fr;        /* f(R) solver (a, Om, OL, fR0, boxsize taken from above) */
  int poisson;         /* PM_POISSON_MG (multigrid, mg above), PM_POISSON_FFT7
                          or PM_POISSON_FFT (pm_poisson_fft; workspace with
                          PM_WS_FFT); the f(R) scalaron always uses FAS
                          multigrid                                           */
  double mu0;          /* PM_GRAVITY_PARAM: the coupling today minus one      */
  int report_max;      /* 1: fill pm_stats.max_acc / max_vel (one 16-byte
                          device-to-host read: the call synchronises)        */
  int serial;          /* f(R): 0 (default) runs the scalaron solve on a
                          second stream beside the Newtonian Poisson solve
                          (both depend on the density only); 1 runs it on
                          `stream` before the Poisson solve (same results;
                          per-kernel timing without overlap)                 */
} pm_step_params;

typedef struct {
  int status;
  mg_stats mg;         /* Poisson solve                                      */
  mg_stats fr;         /* f(R) solve                                         */
  double max_acc;      /* with report_max: max |acceleration| of the step and */
  double max_vel;      /* max |velocity| after its kick (the inputs of the
                          free-fall and velocity time-step criteria, §3.4)   */
} pm_stats;

/* One PM step on the device-resident state (§3.4-§3.10): sort particles by
 * cell (X, V and id are permuted into cell order), deposit, solve (f(R) first
 * if requested, then Poisson for phi), force g = -grad(phi - (c~^2/2) f~_R),
 * inverse TSC, then v += acc dt_kick and x += v dt_drift with exact periodic
 * wrap.  Kicks of consecutive leapfrog steps are merged by the caller through
 * dt_kick = (dt_{i-1} + dt_i)/2.  `st` is a host pointer (may be NULL). */
pm_status pm_step(pm_state* s, const pm_step_params* prm, pm_stats* st, void* stream);

/* pm_step with HOST particle buffers: copies X_in, V_in (host, ideally pinned)
 * into s->X, s->V, runs pm_step and copies the new X, V back into X_out, V_out
 * (host); same results as the copies around pm_step.  X travels on `stream`
 * before the sort; V travels on a second, library-owned stream while the
 * positions are sorted and the potentials solved (V enters only the force
 * pass), and on the way back V and X travel on the two streams at once.  The
 * call returns after all copies have completed, also on error (the host
 * arrays are then free).  X_in may equal X_out and V_in V_out. */
pm_status pm_step_host(pm_state* s, const pm_step_params* prm, pm_stats* st,
                       const uint32_t* X_in, const float* V_in,
                       uint32_t* X_out, float* V_out, void* stream);

/* --------------------------------------------------------- checkpointing --
 * Checkpoint and resume of a device-resident state (not part of the paper's
 * method: a run of many steps can stop and continue).  The file holds a
 * header (magic "PMGBCKP1", n, np, which optional arrays are present,
 * have_prev) and then X [3][np] uint32, V [3][np] float32, id [np] (if
 * s->id), phi [n^3] and eps [n^3] (if s->eps), in the host's byte order,
 * copied through a host staging buffer of at most 64 MiB (host memory, freed
 * before return).  Both calls synchronise `stream` first and are
 * synchronous.  A step continued from a loaded state is bitwise the step the
 * saved run would have taken (same library, same GPU model). */
/* Writes s to the file at `path` (host string).  PM_EINVAL for bad
 * arguments, PM_EIO if the file cannot be written. */
pm_status pm_state_save(const pm_state* s, const char* path, void* stream);
/* Reads the file at `path` into s, whose n, np and optional arrays (id,
 * eps) must match the file's; sets s->have_prev from the file.  PM_EIO if
 * the file cannot be read or does not match. */
pm_status pm_state_load(pm_state* s, const char* path, void* stream);

/* -------------------------------------------------------------- adjoints --
 * Reverse-mode derivatives of the Newtonian step, for gradients of losses
 * with respect to particle positions and velocities (and, through the
 * initial conditions, the white noise).  Position cotangents are float32
 * [3][np] in box units (derivative with respect to x = X * 2^-32). */

/* Deposit adjoint: with rho = pm_deposit(X), dX_bar[d][p] =
 * sum_c d rho_c / d x_p,d * rho_bar[c] = (n^3/np) n sum_c dW_pc/d(offset_d) rho_bar[c]
 * (W_TSC is C1, §3.4).  rho_bar [n^3], dX_bar [3][np] (written). */
pm_status pm_deposit_adj(const uint32_t* X, int64_t np, int n, const float* rho_bar, float* dX_bar,
                         void* stream);

/* Interpolation adjoint: with acc = pm_interp(g, X), g_bar = sum_p W_pc acc_bar_p
 * (a TSC deposit of acc_bar, deterministic like pm_deposit) and
 * dX_bar[d][p] = n sum_c dW_pc/d(offset_d) (g_c . acc_bar_p).
 *   g [3][n^3], acc_bar [3][np] (read); g_bar [3][n^3], dX_bar [3][np] (written).
 * Workspace: pm_workspace_size(n, np, PM_WS_SORT | PM_WS_ADJ). */
pm_status pm_interp_adj(const float* g, const uint32_t* X, int64_t np, int n, const float* acc_bar,
                        float* g_bar, float* dX_bar, void* ws, size_t ws_bytes, void* stream);

/* Gradient adjoint: with g = pm_gradient(phi, order) (g = -G phi, Table 1),
 * phi_bar = -G^T g_bar = sum_d G_d g_bar_d (the stencil is antisymmetric).
 * g_bar [3][n^3] (read), phi_bar [n^3] (written). */
pm_status pm_gradient_adj(const float* g_bar, float* phi_bar, int n, int order, void* stream);

/* Multigrid adjoint: the 7-point Laplacian is self-adjoint, so the cotangent of
 * the right-hand side of mg_solve is the solution of the same problem with the
 * cotangent of phi as right-hand side: this is mg_solve applied to phi_bar. */
pm_status mg_solve_adj(const float* phi_bar, float* f_bar, int n, const mg_params* prm, mg_stats* st,
                       void* ws, size_t ws_bytes, void* stream);

/* Adjoint of one Newtonian pm_step taken from the state s (s->X, s->V are the
 * step's INPUTS; nothing in s is modified).  X_bar_out, V_bar_out are the
 * cotangents of the step's outputs, in the output order of pm_step (cell
 * order); X_bar_in, V_bar_in receive the cotangents of the inputs, in the
 * input order.  phi_fwd: the potential the forward step used (what pm_step
 * left in s->phi, [n^3]), kept by the caller; NULL recomputes it here
 * (deposit and a Poisson solve to prm->mg.tol from the Jacobi guess), which
 * matches a forward step taken with s->have_prev = 0.  Then a_bar =
 * dt_kick (V_bar' + dt_drift X_bar'), g_bar = deposit of a_bar,
 * phi_bar = -G^T g_bar, rho_bar = 3/2 a Om A^+ phi_bar (a Poisson solve to
 * prm->mg.tol from the Jacobi guess), and X_bar = X_bar' + the interpolation
 * and deposit position terms, V_bar = V_bar' + dt_drift X_bar'.
 * Workspace: PM_WS_STEP | PM_WS_ADJ (| PM_WS_IDS if s->id).  Newtonian
 * gravity only (PM_EINVAL otherwise). */
pm_status pm_step_adj(pm_state* s, const pm_step_params* prm, const float* phi_fwd, const float* X_bar_out,
                      const float* V_bar_out, float* X_bar_in, float* V_bar_in, void* stream);

/* ----------------------------------------------------- batched ensembles -- */
/* B independent boxes of the same size advanced together: the ensembles of
 * runs with different seeds and cosmologies that the paper's speed is meant
 * for (§1, §5).  One launch of each kernel serves every box (the box is the
 * third grid dimension), so small boxes fill the GPU and a step is a few dozen
 * launches instead of B times as many.  The boxes do not interact: box b
 * evolves bitwise as it would alone in a batch of one.  Newtonian gravity;
 * the Poisson solve runs fixed cycle counts and nothing in a step waits on the
 * host, so a step can be captured in a CUDA graph and replayed (the per-box
 * coefficients are read from device memory at run time). */
typedef struct {
  int n;              /* cells per side of every box (power of two, 32..1024) */
  int B;              /* boxes (3 log2 n + ceil(log2 B) <= 32)                 */
  int64_t np_box;     /* particles per box                                      */
  uint32_t* X;        /* [3][B np_box] positions; box b's particles at
                         b np_box .. (b+1) np_box - 1 in every plane; in/out
                         (reordered into cell order within each box)           */
  float* V;           /* [3][B np_box] velocities (same order), in/out         */
  float* phi;         /* [B][n^3] potentials, in/out (warm start)              */
  void* ws;           /* workspace of pm_batch_workspace_size() bytes          */
  size_t ws_bytes;
  int have_prev;      /* 0: phi is not yet a potential (Jacobi first guess)    */
} pm_batch_state;

typedef struct {
  int grad_order;             /* 3, 5 or 7 (Table 1)                             */
  const float* src_scale;     /* [B] device: 3/2 a Om of each box (§3.1)         */
  const float* dt_kick;       /* [B] device: kick interval of each box           */
  const float* dt_drift;      /* [B] device: drift interval of each box          */
  const float* phi_rescale;   /* [B] device: warm-start factor of each box
                                 (a1 D1 / (a0 D0), used when have_prev)          */
  mg_params mg;               /* fixed_cycles > 0: V-cycles of a warm step       */
  int cold_cycles;            /* V-cycles of a step with have_prev = 0           */
} pm_batch_params;

/* Workspace bytes for B boxes of n^3 cells with np_box particles each. */
pm_status pm_batch_workspace_size(int n, int B, int64_t np_box, size_t* bytes);

/* The stages of the step, one launch per kernel for B boxes (the `batch`
 * argument of the boundary): box b's particles at b np_box .. (b+1) np_box - 1
 * of every plane, its grids at b n^3 (scalar) and 3 b n^3 (vector); every box
 * gives bitwise the result of the single-box call on it.  32 <= n.
 *   pm_deposit_batch: rho [B][n^3] of X [3][B np_box]; workspace
 *     pm_batch_workspace_size(n, B, np_box).
 *   mg_solve_batch: exactly prm->fixed_cycles V-cycles per box, each box's
 *     float64 mean of f removed (first_guess MG_GUESS_INPUT or
 *     MG_GUESS_JACOBI); workspace pm_batch_workspace_size(n, B, 0).
 *   pm_gradient_batch: g [B][3][n^3] of phi [B][n^3].
 *   pm_interp_batch: acc [3][B np_box] of g [B][3][n^3] at X [3][B np_box]. */
pm_status pm_deposit_batch(const uint32_t* X, int64_t np_box, int n, int B, float* rho, void* ws, size_t ws_bytes,
                           void* stream);
pm_status mg_solve_batch(const float* f, float* phi, int n, int B, const mg_params* prm, void* ws, size_t ws_bytes,
                         void* stream);
pm_status pm_gradient_batch(const float* phi, float* g, int n, int B, int order, void* stream);

/* The f(R) scalaron of B boxes (§3.6.2, §3.10, the `batch` argument of the
 * boundary): fr_solve's FAS cycles run on every box at once, one launch per
 * kernel and level (box = third grid dimension; the coarsest level is one CTA
 * per box).  The boxes share *prm: one scale factor, cosmology, f_R0 and box
 * size (ensembles over seeds).  Exactly prm->cycles cycles per box (tol and
 * max_cycles are not used: no box waits on a residual, nothing synchronises
 * with the host); smoother 0 is taken as 2.  Box b gives bitwise fr_solve on
 * rho + b n^3 with the same parameters, smoother 2 (or 1) and tol <= 0.
 *   rho  [B][n^3] float32 densities (read); each box's float64 mean is removed
 *   eps  [B][n^3] float32 in: guesses, out: solutions (16-byte aligned)
 *   ws   pm_fr_batch_workspace_size(n, B) bytes, 256-byte aligned
 * Errors: PM_EINVAL (n not a power of two in 32..1024, B < 1, cycles < 1,
 * invalid parameters, misaligned arrays), PM_ENOMEM (ws too small). */
pm_status pm_fr_batch_workspace_size(int n, int B, size_t* bytes);
pm_status fr_solve_batch(const float* rho, float* eps, int n, int B, const fr_params* prm, void* ws,
                         size_t ws_bytes, void* stream);
pm_status pm_interp_batch(const float* g, const uint32_t* X, int64_t np_box, int n, int B, float* acc, void* stream);

/* One fused-kick leapfrog step of every box (pm_step's pipeline, batched):
 * sort by (box, cell), deposit, per-box source 3/2 a Om_b (rho - <rho>_b),
 * multigrid with fixed cycles (Jacobi guess, or phi_rescale[b] phi_b when
 * have_prev), gradient, inverse TSC, kick by dt_kick[b], drift by
 * dt_drift[b]; then have_prev = 1.  Per-box arrays are read on the device
 * when the kernels run.  PM_EINVAL for bad sizes, pointers, parameters
 * (mg.fixed_cycles < 1, cold_cycles < 1, smoother 0 is taken as 2). */
pm_status pm_step_batch(pm_batch_state* s, const pm_batch_params* prm, void* stream);

/* ------------------------------------------------------ host utilities ---- */
/* Supercomoving time between a0 and a1 (§3.1): integral of da/(a^3 E(a)),
 * E(a) = sqrt(Om a^-3 + OL).  Host computation, float64. */
double pm_dt_supercomoving(double Om, double OL, double a0, double a1);
/* Linear growth factor D(a) (Appendix A, growing mode, D ~ a early on). */
double pm_growth_D(double Om, double OL, double a);

/* Adaptive time step of the integrator (§3.4, "Integrator"): the
 * supercomoving step dt = courant * min(dt_a, dt_ff, dt_v), where dt_a lets
 * the scale factor grow by the fraction da_max, dt_ff = sqrt(h / max_acc) is
 * the free-fall time over one cell and dt_v = h / max_vel the time to cross
 * one cell at the largest speed (h = 1/n; a criterion whose maximum is 0 is
 * left out); if the step would pass a_end it ends there instead.  Writes the
 * step (*dt) and the scale factor it reaches (*a_next, by bisection on the
 * monotone t(a)).  Host computation in float64; max_acc and max_vel are the
 * host values pm_step reports with report_max (and pm_max_speed).
 * PM_EINVAL for a <= 0, a_end <= a, negative maxima, courant or da_max <= 0,
 * or NULL outputs. */
pm_status pm_next_timestep(double a, double Om, double OL, int n, double max_acc, double max_vel, double courant,
                           double da_max, double a_end, double* dt, double* a_next);

/* Largest particle speed |v| of V [3][np] (device, float32 planes; computed
 * in float32, returned as float64 in *max_vel, host): the velocity criterion's
 * input before the first step, when no step has reported one yet.
 * Synchronises `stream` (one 16-byte read).  ws: a workspace of
 * pm_workspace_size(n, np, flags) bytes for any flags (its reduction
 * buffers are used; nothing else in it is touched).  PM_EINVAL for bad sizes
 * or pointers, PM_ENOMEM for a short workspace. */
pm_status pm_max_speed(const float* V, int64_t np, int n, uint32_t flags, double* max_vel, void* ws,
                       size_t ws_bytes, void* stream);

/* --------------------------------------------------------- instrumentation */
/* Number of kernels this library has launched since load. */
uint64_t pm_launch_count(void);
/* Enable (1) / disable (0) CUDA-event timing of every launch, recorded on the
 * launch stream.  Enabling clears previous records. */
pm_status pm_timing_enable(int on);
/* Synchronises, then reports per kernel class since pm_timing_enable(1): total
 * milliseconds, launches and algorithmic bytes (the compulsory DRAM traffic
 * of each launch: data read once, results written once).  Arrays are host,
 * length cap (any may be NULL); returns the number of classes written.
 * names[i] are static strings. */
int pm_timing_collect(const char** names, double* ms, int64_t* launches, double* bytes, int cap);

/* ------------------------------------------------------------ autotuning --
 * Batched launches (pm_step_batch) tune how they tile their work, online: for
 * each launch site and shape (n, B) the candidate values of one parameter
 * (the x chunk of the force pass and of the fused multigrid sweep; colour
 * passes or fused sweeps on 64^3 levels) take turns on successive real
 * launches, timed with CUDA events on the launch stream and read back
 * without synchronising; after two timings each the fastest is kept for the
 * rest of the process.  Every candidate computes bitwise the same result, so
 * tuning never changes a result, only when it is ready.  Nothing is timed
 * while a stream is captured into a CUDA graph.  Single-box launches use
 * fixed tilings. */
/* mode 0: fixed default tilings; 1 (the default): tune; 2: forget every
 * choice and timing, then tune.  PM_EINVAL for another mode. */
pm_status pm_autotune(int mode);
/* Reports the tuned sites, five ints each: site (0 force-pass chunk, 1 fused
 * multigrid sweep chunk, 2 multigrid smoother form: 0 colour passes, 1 fused),
 * n, B, the chosen value (-1 while undecided) and the timings read so far.
 * out (host, 5 * cap ints) may be NULL; returns the number of sites. */
int pm_autotune_report(int* out, int cap);

#ifdef __cplusplus
}
#endif
#endif /* PM_API_H */
