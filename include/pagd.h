/*
 * pagd.h -- C ABI of the GB300 (sm_103a) PAGD time-step library.
 *
 * The library advances the phase field crystal (PFC) and functionalized
 * Cahn-Hilliard (FCH) equations of Park, Salgado & Wise (arXiv 2204.07247,
 * Sec. 2) on a periodic Fourier collocation grid (Sec. 3.2) with the fully
 * implicit BDF2 / midpoint (MP) schemes (Sec. 3.1.1, Eqs. eqn:FCH-semidis-implicit,
 * obj:BDF2, obj:MP), each step solved by the preconditioned Nesterov accelerated
 * gradient descent with sweeping friction (Algorithm 2) and the averaged Newton
 * preconditioner (Sec. 3.4.1), or with the linear IMEX schemes LBDF2 / LMP
 * (Eq. eqn:FCH-semidis-simplicit, Sec. 3.3).
 *
 * Conventions (all entry points):
 *  - Grid: n[0] x n[1] (dim 2) or n[0] x n[1] x n[2] (dim 3) points, row-major
 *    with the last index fastest; powers of two from 8 to 512 per axis.  Domain
 *    [0, L[d]) per axis, spacing h_d = L[d] / n[d].
 *  - Fields are FP64, contiguous, caller-owned.  "_dev" pointers are device
 *    memory of the current CUDA device; "_host" pointers are host memory.  The
 *    library never frees caller memory and never calls cudaMalloc: its device
 *    workspace is handed in by the caller (pagd_workspace_size /
 *    pagd_set_workspace).
 *  - Every call returns a pagd_status and never aborts.  On an error during a
 *    step the solver state (u^n, u^{n-1}, step count) is left as it was before
 *    the call and the output field is not written; pagd_last_error() then holds
 *    a one-line description.
 *  - Work is issued on the stream given at init (NULL = legacy default stream).
 *    Calls that return numbers to the host synchronise that stream.
 */
#ifndef PAGD_H
#define PAGD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pagd_solver pagd_solver; /* opaque, library-owned host object */

typedef enum {
    PAGD_OK = 0,
    PAGD_EINVAL = 1,   /* bad argument (size, pointer, parameter) */
    PAGD_ENOMEM = 2,   /* workspace missing or too small; host allocation failed */
    PAGD_ECUDA = 3,    /* a CUDA runtime call failed */
    PAGD_ENOCONV = 4,  /* PAGD hit max_iter before ||d||_inf <= tol (Algorithm 2) */
    PAGD_EPRECOND = 5, /* averaged Newton symbol not positive on some wavenumber */
    PAGD_ENAN = 6,     /* non-finite residual norm */
    PAGD_ESTATE = 7,   /* call out of order (no workspace / no state set) */
    PAGD_ETIMEOUT = 8  /* a device-wide barrier gave up waiting (no hang: error) */
} pagd_status;

enum { PAGD_PFC = 0, PAGD_FCH = 1 };
/* schemes: BDF2 (backward Euler first step), MP, and the linear IMEX LBDF2, LMP */
enum { PAGD_BDF2 = 0, PAGD_MP = 1, PAGD_LBDF2 = 2, PAGD_LMP = 3 };
/* FP64: all arithmetic in FP64.  FP32_MIXED: FFTs and PAGD updates in FP32 on a
 * correction to an FP64 base point; residual norms, energy, mass, the state and
 * the acceptance check of every step stay FP64. */
enum { PAGD_FP64 = 0, PAGD_FP32_MIXED = 1 };

/* Solver settings (Table 1).  Defaults from pagd_default_opts: s = 0.9, the
 * sweeping list eta = sqrt(0.1, 0.575, 1.05, 1.525, 2), max_iter = 1000,
 * theta_mode = 0, accel = 1. */
typedef struct {
    double s;         /* step size of Algorithms 1/2, > 0 */
    int n_eta;        /* 1..16 */
    double eta[16];   /* sweeping friction values, > 0 */
    int max_iter;     /* residual evaluations per step before PAGD_ENOCONV, >= 1 */
    int theta_mode;   /* MP preconditioner: 0 = second variation of 2E((v+u^n)/2)
                         (energy terms x 1/2), 1 = the printed form (x 1) */
    int accel;        /* 1 = PAGD (Algorithm 2), 0 = PGD (Algorithm 1) */
} pagd_opts;

pagd_status pagd_default_opts(pagd_opts* opts);

/* PFC model (Sec. 2.1, Eqs. obj:PFC-egy, eqn:PFCsystem): energy
 * 1/4 u^4 + (1-eps)/2 u^2 - |grad u|^2 + 1/2 (Lap u)^2, mobility M > 0.
 * stream: a cudaStream_t cast to void* (NULL for the default stream).
 * On success *out receives a new solver; release it with pagd_destroy. */
pagd_status pfc_init(pagd_solver** out, int dim, const int* n, const double* L, double eps,
                     double M, int scheme, int precision, const pagd_opts* opts /* nullable */,
                     void* stream);

/* FCH model (Sec. 2.2, Eqs. obj:FCHegy, eqn:FCHPDE): energy
 * 1/2 (eps^2 Lap u - F'(u))^2 - (eps^2 eta1/2 |grad u|^2 + eta2 F(u)),
 * F(z) = 1/2 (z+1)^2 (1/2 (z-1)^2 + 2/3 tau (z-2)). */
pagd_status fch_init(pagd_solver** out, int dim, const int* n, const double* L, double eps,
                     double eta1, double eta2, double tau, double M, int scheme, int precision,
                     const pagd_opts* opts /* nullable */, void* stream);

/* Device workspace: query the size in bytes, allocate it (e.g. a torch uint8
 * tensor on the device, 256-byte aligned) and hand it in.  It must stay valid
 * until pagd_destroy or the next pagd_set_workspace. */
pagd_status pagd_workspace_size(const pagd_solver* s, size_t* bytes);
pagd_status pagd_set_workspace(pagd_solver* s, void* dev_ptr, size_t bytes);

/* Set u^0 (and u^{-1} := u^0, Sec. 3.1.1) from a device field; resets the step
 * counter.  Copies: the caller may reuse u0_dev afterwards. */
pagd_status pagd_set_state(pagd_solver* s, const double* u0_dev);

/* Advance one step of size dt (dt_{n+1}; the previous step size is remembered).
 * Implicit schemes iterate PAGD until ||d_i||_inf <= tol (Algorithm 2; for
 * FP32_MIXED the accepted step also passes that test in FP64).  Writes u^{n+1}
 * to u_dev (device, n_pts doubles).  iters_out: residual evaluations taken
 * (0 for IMEX); resid_out: the accepted ||d||_inf.  Both nullable.
 * Synchronises the stream. */
pagd_status pagd_step(pagd_solver* s, double* u_dev, double dt, double tol, int* iters_out,
                      double* resid_out);

/* One implicit step (as pagd_step) started from a caller's initial iterate,
 * e.g. a learned predictor of u^{n+1}.  The guess (device, n_pts doubles) is
 * first moved to the mass of u^n (the discrete solution keeps it and every
 * PAGD update has zero mean), and the first direction d_0 of Algorithm 2 is
 * evaluated there.  The solver keeps a record R: ||d_0||_inf of the last step
 * it started from the extrapolated guess of Sec. 3.4.2 (reset by
 * pagd_set_state).  With a record, the guess is kept when its ||d_0||_inf <= R
 * and PAGD continues from it at no extra cost; otherwise the step starts over
 * from the extrapolation (the probe counts in iters_out).  Without a record,
 * d_0 is also evaluated at the extrapolation and PAGD continues from the one
 * with the smaller ||d_0||_inf (both evaluations count).  used_guess_out
 * (nullable): 1 if the caller's guess was kept.  Implicit schemes only
 * (PAGD_EINVAL for LBDF2 / LMP).  Synchronises the stream. */
pagd_status pagd_step_with_guess(pagd_solver* s, double* u_dev, const double* guess_dev, double dt, double tol,
                                 int* iters_out, double* resid_out, int* used_guess_out);

/* Advance nsteps steps of size dt in one device launch per chunk of at most
 * 4096 steps.  u_dev (nullable) receives the final field.  iters_out and
 * resid_out (nullable, host arrays of nsteps) receive per-step values.
 * On an error the steps before the failing one are kept. */
pagd_status pagd_run(pagd_solver* s, double* u_dev, double dt, int nsteps, double tol,
                     int* iters_out, double* resid_out);

/* Same as pagd_run with host buffers: copies u0_host in (as pagd_set_state),
 * runs, and copies the final field to u_host_out. */
pagd_status pagd_run_host(pagd_solver* s, const double* u0_host, double* u_host_out, double dt,
                          int nsteps, double tol, int* iters_out, double* resid_out);

/* Discrete energy E_N (Fourier differentiation, trapezoidal rule, Sec. 3.2)
 * and mass (u, 1)_N of a device field. */
pagd_status pagd_energy(pagd_solver* s, const double* u_dev, double* E);
pagd_status pagd_mass(pagd_solver* s, const double* u_dev, double* m);

/* R(v) = M Lap_N mu(v) (the right-hand side of the gradient flow, Sec. 2) of a
 * device field v into r (device; may not alias v). */
pagd_status pagd_rhs(pagd_solver* s, const double* v_dev, double* r_dev);

/* Adaptive time stepping (Sec. 3.1.2, Algorithm 3) from the current state to
 * time T (or max_steps accepted steps): each tentative step of size dt is
 * taken by the solver's scheme, a higher-order value is formed (AM3: the
 * explicit third-order Adams-Moulton variant with R at the tentative, current
 * and previous solutions; for MP from the third step on, midAB2: the quadratic
 * extrapolation through the last three solutions with its truncation factor),
 * ERR = ||u_tentative - u_high|| / ||u_high|| (discrete L2); the step is
 * accepted when ERR <= step_tol or dt <= dt_min, and the next tentative size
 * is clamp(0.9 (step_tol / ERR)^(1/3) dt, dt_min, dt_max).  The first
 * tentative size is dt_min.  A rejected step leaves no trace in the solver
 * state.  scratch_dev: device, 6 n_pts doubles (caller-owned).  Outputs
 * (nullable, host): t_out [max_steps + 1] accepted times (t_out[0] = 0),
 * dt_out / iters_out [max_steps] accepted sizes and PAGD evaluations,
 * nsteps_out, rejected_out; u_dev (device) the final field.  tol is the PAGD
 * tolerance of each step (ignored by IMEX schemes). */
pagd_status pagd_run_adaptive(pagd_solver* s, double T, double dt_min, double dt_max, double step_tol, double tol,
                              int max_steps, double* scratch_dev, double* u_dev, double* t_out, double* dt_out,
                              int* iters_out, int* nsteps_out, int* rejected_out);

/* Unnormalised forward DFT of a real device field (Sec. 3.2): writes the half
 * spectrum n[0] x ... x (n[dim-1]/2 + 1) complex (interleaved re, im doubles),
 * row-major.  pagd_fft_c2r inverts it including the 1/n_pts factor. */
pagd_status pagd_fft_r2c(pagd_solver* s, const double* u_dev, double* spec_dev);
pagd_status pagd_fft_c2r(pagd_solver* s, const double* spec_dev, double* u_dev);

/* Copy the current u^n / u^{n-1} to device buffers (either nullable), and the
 * number of steps taken since pagd_set_state. */
pagd_status pagd_get_state(pagd_solver* s, double* un_dev, double* unm1_dev, int* step);

/* One time step with no device allocation and no caller workspace.  The paper
 * has no counterpart.  It is for callers that cannot allocate device memory
 * when they need a step: runtimes that own the device allocator and forbid
 * the libraries they host to allocate, and programs that fix their device
 * memory budget up front.  It runs on a file-scope static device array of
 * 8 MiB that the library carries; every GPU that loads the library holds that
 * array until the process exits.  The array's head keeps the twiddle tables;
 * the rest, 8,364,032 bytes, holds the step's scratch, so the solver's
 * pagd_workspace_size must not exceed that: every 2D grid up to 128 x 128
 * points and every 3D grid up to 16 x 16 x 16 fits in either precision
 * (FP32_MIXED also up to 128 x 256 and 32 x 32 x 32).  Larger grids are
 * rejected with PAGD_EINVAL and a message giving both sizes.
 * The solver object comes from pfc_init / fch_init and supplies only the
 * model, grid, scheme and solver settings: its own state, workspace and
 * trace setting are neither needed nor touched (no phase trace is recorded).
 * Inputs: un_dev = u^n, unm1_dev = u^{n-1} (device, n_pts doubles; for
 * step_index 0 pass u^0 twice), step_index = n, dt = dt_{n+1}, dt_prev = dt_n
 * (ignored when step_index is 0).  Output: unp1_dev = u^{n+1} (device); it may
 * not alias un_dev or unm1_dev.  iters_out / resid_out as for pagd_step.
 * Each call is one step on its own: the running mass correction that
 * pagd_run / pagd_step carry from step to step (the FP64 mean removal's
 * rounding fed back into the next step) starts from zero in every call, so
 * over a long chain of calls the mass drifts by the rounding of one mean
 * removal per step (about 1e-16 relative each) instead of staying at one.
 * The first call on each device looks up the array's device address and
 * writes the twiddle tables there (make that first call before any stream
 * capture).  All calls share the array and it keeps the previous call's
 * contents (each call clears what must start at zero); calls that overlap on
 * the GPU race on it, so the caller must serialise them.  Synchronises the
 * stream before returning. */
pagd_status pagd_step_static(pagd_solver* s, const double* un_dev, const double* unm1_dev,
                             int step_index, double dt, double dt_prev, double tol, double* unp1_dev,
                             int* iters_out, double* resid_out);

/* Phase tracing (instrumentation, not in the paper).  With tracing enabled,
 * every launch records, for each phase of the persistent kernel, the phase
 * identifier and the device time at which all CTAs finished it (up to 8192
 * records per launch).  pagd_get_trace copies the records of the last launch:
 * phase[i] and t_us[i] (microseconds since the launch started; record 0 is the
 * start marker), at most cap records, and the number recorded to *count.
 * Phase identifiers are those of the kernel's control machine (see
 * paper_2204_07247_gb300/pagd.py PHASES); bit 16 is set on the phases B..E of
 * an incremental base evaluation (transforms of the shift in the iteration
 * precision, FP32-mixed only).  With tracing enabled on the first
 * member of a batch, pagd_batch_run records its global phases in that member
 * instead: phase[i] is then a bit mask (bit p set: some member ran phase p). */
pagd_status pagd_set_trace(pagd_solver* s, int enable);
pagd_status pagd_get_trace(pagd_solver* s, int* phase, double* t_us, int cap, int* count);

/* Device barrier probe (instrumentation, not in the paper): one launch of the
 * solver's persistent kernel, with the solver's launch plan, that runs `count`
 * (1..1000000) empty phases, each ended by the device-wide barrier that also
 * ends every phase of a time step.  *us_per_phase receives the launch's device
 * time divided by count (CUDA events on the solver's stream).  Needs the
 * workspace; leaves the solver state alone.  Synchronises the stream. */
pagd_status pagd_barrier_probe(pagd_solver* s, int count, double* us_per_phase);

/* Iteration pass probe (instrumentation, not in the paper): one launch of the
 * solver's persistent kernel that repeats one pass of a PAGD iteration `count`
 * (1..1000000) times, each ended by the device-wide barrier, so that a
 * profiler capturing that launch sees the pass alone.  pass: 0 the row pass
 * (RI: correction update, nonlinear term, forward transforms along the last
 * axis), 1 the column pass (CI: spectral residual, preconditioner, state
 * update, inverse transforms along the first axis), 2 / 3 the forward /
 * inverse middle pass (MF / MI, 3D only).  The pass runs as iteration 1 of
 * the last completed step, on the iteration buffers that step left (their
 * contents are overwritten; u^n, u^{n-1} and the step count are kept, and
 * the next pagd_run starts from them as usual).  *us_per_pass: the launch's
 * device time / count, barrier included (pagd_barrier_probe gives the
 * barrier alone).  PAGD_EINVAL for a bad argument or a middle pass in 2D,
 * PAGD_ESTATE without a completed step of BDF2 or MP.  Synchronises the
 * stream. */
pagd_status pagd_pass_probe(pagd_solver* s, int pass, int count, double* us_per_pass);

/* Launch plan of the solver's persistent kernel (instrumentation, not in the
 * paper): CTAs of the last launch (0 before the first), threads per CTA, the
 * cluster size of the cluster-resident iterations (0: every phase is
 * device-wide; else the PAGD iterations of square 64^2, 128^2 and 256^2 grids
 * run inside one thread-block cluster of n/16 CTAs with their state in
 * distributed shared memory), whether the passes with FP64 lines run
 * CTA-cooperative units, the dynamic shared memory per CTA, and whether the
 * FP32 iteration passes stage their inputs through shared memory by
 * asynchronous copies (PFC, FP32-mixed, square power-of-two grids; the same
 * arithmetic either way).  Every output nullable. */
pagd_status pagd_launch_info(const pagd_solver* s, int* grid, int* threads, int* cluster, int* coop,
                             size_t* smem, int* staged);

const char* pagd_last_error(const pagd_solver* s);
void pagd_destroy(pagd_solver* s);

/* ---- Batches: many independent instances in one persistent launch.
 * The paper solves one instance at a time; a batch runs the same per-instance
 * computation (Algorithm 2 on every time step of every member) for a set of
 * solvers of possibly different grids, models, parameters, schemes and
 * initial data.  Members keep running independently: each takes its own number
 * of PAGD iterations per step, and a member that fails (PAGD_ENOCONV, ...)
 * stops while the others go on.  Results equal those of pagd_run on each member
 * up to the summation order of the grid reductions.
 *
 * members: solvers from pfc_init / fch_init, all of one precision and one
 * stream, each with its workspace and state set (pagd_set_state); the batch
 * borrows them (does not own or copy them) and they must outlive it.  count:
 * 1..4096, limited further by shared memory (PAGD_EINVAL when the largest
 * member's passes and the per-member control state do not fit one CTA).  A
 * member may appear once. */
typedef struct pagd_batch pagd_batch; /* opaque, library-owned host object */

pagd_status pagd_batch_create(pagd_batch** out, pagd_solver* const* members, int count);

/* Device workspace of the batch (member parameter blocks and the launch's
 * barrier state), handed in like a solver's workspace (256-byte aligned). */
pagd_status pagd_batch_workspace_size(const pagd_batch* b, size_t* bytes);
pagd_status pagd_batch_set_workspace(pagd_batch* b, void* dev_ptr, size_t bytes);

/* Advance every member nsteps steps of size dt to tolerance tol (as pagd_run),
 * in one device launch per chunk of at most 4096 steps.  When every member
 * alone fills every warp of the batched launch in every phase (e.g. 3D grids
 * of 256^3), one launch adds no concurrency and members that drift apart in
 * their phases would slow every global phase to its slowest part; such
 * batches run member after member through the single-instance kernel
 * (pagd_batch_launch_info reports it); pagd_batch_step_with_guess likewise.  Outputs, all
 * nullable host arrays: iters_out / resid_out [count x nsteps], member-major
 * (entries after a member's failing step are not written); status_out [count]
 * per-member status.  Returns PAGD_OK when every member completed, else the
 * status of the first member (by index) that failed, or the launch's error.
 * Each member's u^n, u^{n-1} and step count advance as with pagd_run (read them
 * with pagd_get_state).  Synchronises the stream. */
pagd_status pagd_batch_run(pagd_batch* b, double dt, int nsteps, double tol, int* iters_out, double* resid_out,
                           int* status_out);

/* Launch shape of the batched kernel (not in the paper): warps per CTA
 * (1..8; each warp has its own shared-memory slice for one unit's lines) and
 * CTAs per SM (1..8; the grid is that many per SM, capped at the co-resident
 * count).  Together they fix how the units of every global phase are tiled
 * over the machine.  PAGD_EINVAL when the slices or the CTAs do not fit.
 * pagd_batch_create chooses as many warps per CTA as fit, one CTA per SM;
 * paper_2204_07247_gb300/autotune.py times candidate shapes and keeps the
 * fastest.  pagd_batch_launch_info: CTAs of the last launch (the planned grid
 * before the first), warps per CTA, dynamic shared memory per CTA, and
 * whether the last run went member after member (see pagd_batch_run), and
 * how many members' FP32 iteration passes stage their inputs through shared
 * memory (see pagd_launch_info).  Nullable outputs. */
pagd_status pagd_batch_set_shape(pagd_batch* b, int warps_per_cta, int ctas_per_sm);
pagd_status pagd_batch_launch_info(const pagd_batch* b, int* grid, int* warps_per_cta, size_t* smem,
                                   int* sequential, int* staged);

/* One step of every member in one launch, each from its own initial iterate
 * (the batched form of pagd_step_with_guess, with the same judging of each
 * guess against that member's record): guesses[count] device fields (n_pts
 * doubles each, a null entry starts that member from the extrapolation).
 * Outputs as pagd_batch_run with nsteps = 1, and used_guess_out [count]
 * (nullable): 1 where the member's guess was kept.  Synchronises the stream. */
pagd_status pagd_batch_step_with_guess(pagd_batch* b, const double* const* guesses, double dt, double tol,
                                       int* iters_out, double* resid_out, int* status_out, int* used_guess_out);

const char* pagd_batch_last_error(const pagd_batch* b);
void pagd_batch_destroy(pagd_batch* b);

#ifdef __cplusplus
}
#endif
#endif /* PAGD_H */
