/*
 * mgrit_sl.h -- C ABI of a single-GPU (GB300, sm_103a) implementation of
 * multigrid reduction-in-time (MGRIT) for periodic linear advection with
 * semi-Lagrangian (SL) time steps and the modified SL coarse-grid operator of
 * H. De Sterck, R. D. Falgout, O. A. Krzysik, "Fast multigrid reduction-in-time
 * for advection via modified semi-Lagrangian coarse-grid operators" (2022).
 *
 * Problem statement (Sec. 2.1, eq. (ad); Sec. 4.1, eq. (ad_2D)):
 *   u_t + alpha(x,t) u_x = 0             on the periodic interval [xmin, xmax)
 *   u_t + alpha u_x + beta u_y = 0       on the periodic square [xmin, xmax)^2
 * discretised on nx (x nx) equispaced nodes x_i = xmin + i h, h = (xmax-xmin)/nx,
 * and nt time steps of size dt = cfl * h; the wave speed is one of a fixed set
 * of analytic families ("readily computable for any x and t", Sec. 2.1).
 *
 * Conventions for every call below.
 *   Pointers named d_* are DEVICE pointers to FP64 arrays owned by the caller
 *   (for instance allocated by PyTorch); the library never frees them.  h_*
 *   pointers are HOST pointers.  Arrays are time-major and row-major:
 *   u[n][j][i] with x (index i) fastest, i.e. the row-wise lexicographic
 *   ordering of Sec. 4.2; a 1D slice has nx entries, a 2D slice nx*nx.
 *   The library owns the handle and the device workspace it allocates in
 *   mgrit_setup (released by mgrit_destroy).  All work is issued on the CUDA
 *   stream given to mgrit_setup.  Calls return a status and never throw or
 *   abort; argument errors are detected before any launch.  mgrit_last_error()
 *   returns a human-readable message for the last failing call on this thread.
 *   A handle is not thread-safe: one call at a time per handle.
 */
#ifndef MGRIT_SL_H
#define MGRIT_SL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MGRIT_OK = 0,
  MGRIT_EINVAL = 1,         /* bad argument (checked before any launch) */
  MGRIT_ENOMEM = 2,         /* device allocation failed */
  MGRIT_ECUDA = 3,          /* a CUDA runtime error */
  MGRIT_ENOTCONVERGED = 4,  /* max_iter cycles without reaching rtol */
  MGRIT_EDIVERGED = 5,      /* residual non-finite or grew by more than 1e3 */
  MGRIT_ETIMEOUT = 6,       /* a bounded device wait gave up */
  MGRIT_EUNSUPPORTED = 7,   /* valid but not implemented combination */
  MGRIT_ESINGULAR = 8       /* a correction matrix had a (near) zero pivot */
} mgrit_status;

/* Periodic space-time grid (Sec. 2.1).  dim = 1 or 2 (ny = nx in 2D). */
typedef struct {
  int dim;
  int nx;
  int nt;
  double xmin;
  double xmax;
  double cfl; /* dt = cfl * h; the paper uses 0.85 */
} mgrit_grid;

/* Analytic wave-speed families. */
typedef enum {
  MGRIT_A_CONST = 0,        /* alpha = a                                   eq. (alpha1) with a = 1 */
  MGRIT_A_COS_T = 1,        /* alpha = cos(2 pi t)                          eq. (alpha2) */
  MGRIT_A_COS_T_COS_X = 2,  /* alpha = cos(2 pi t) cos(2 pi x)              eq. (alpha4) */
  MGRIT_A_SIN_KX_COS_T = 3, /* alpha = 1 + a sin(2 pi k x) cos(2 pi t) */
  MGRIT_A2D_CONST = 10,     /* (alpha, beta) = (a, a2)                      eq. (alpha-const_2D) with a = a2 = 1 */
  MGRIT_A2D_PAPER = 11,     /* (sin^2(pi y) cos(2pi t/3.4), -cos^2(pi x) cos(2pi t/3.4))  eq. (alpha-var_2D) */
  MGRIT_A2D_SIN_COS = 12    /* (1 + a sin(2 pi y) cos(2 pi t), 1 + a cos(2 pi x) sin(2 pi t)) */
} mgrit_wave_kind;

typedef struct {
  int kind; /* mgrit_wave_kind */
  double a;
  double k;
  double a2;
} mgrit_wavespeed;

/* Solver options; mgrit_default_options() fills the defaults noted here. */
typedef struct {
  int precision;    /* 0: FP64 throughout (default).  1: FP32 bulk -- relaxation, interpolation
                       and the coarse cycle act on the error in FP32, while departure points, the
                       fine-level residual (one FP64 sweep per cycle), the C-point state and the
                       residual norms stay FP64. */
  int coarse_op;    /* 0: corrected operator [I - diag(sigma) D_{p+1}]^{-1} S (eq. (Phi_multilevel), default);
                       1: plain coarse SL step S with the same departure points (Sec. 2.3). */
  int norm_mode;    /* 1 (default): residual after the FCF relaxation of each cycle, counted as in
                       Tables 1-3; 0: residual after the full cycle, r0 from the initial iterate. */
  int max_iter;     /* default 200 */
  double rtol;      /* relative residual reduction to stop at, default 1e-10 (Sec. 2.2) */
  int max_coarsest; /* levels == 0: stop coarsening once a level has <= this many steps (default 1,
                       the paper's rule: coarsen until fewer than two time points would remain) */
  int m_first;      /* 0 (default): factor m on every level; > 0: this factor on level 1 and m below
                       (the aggressive coarsening of Sec. 5) */
  int coarse_fp64;  /* precision == 1 only: 1 = the coarse cycle (levels >= 1: relaxation, coarse
                       residuals, correction solves, coarsest solve) in FP64 with only level 0's
                       error relaxation in FP32; 0 (default) = FP32 like the rest of the error
                       cycle.  Single-problem solves only. */
  int use_graph;    /* 1 (default): each MGRIT cycle's launches are captured once per mgrit_solve call as
                       a CUDA graph and replayed (one host launch per cycle); 0: launched one by one.
                       Results are identical either way. */
  int profile;      /* 1: time each phase with CUDA events on the handle's stream (mgrit_stats.phase_ms) */
  int gmres_maxit;  /* 2D coarse correction solves: GMRES from a zero guess with at most this many
                       iterations (default 10, at most 10) ... */
  double gmres_rtol;/* ... stopped at this relative residual (default 1e-2): the paper's setting for
                       multilevel and 2D runs (Sec. 3.4, 4.3).  1D correction solves are exact unless
                       solve_mode = 1. */
  int relax;        /* 0 (default): FCF relaxation on every level (Sec. 2.2, the paper's runs);
                       1: F-relaxation only on every level -- with two levels this is Parareal
                       (Sec. 2.2), which after k cycles reproduces the first k coarse intervals of
                       sequential stepping exactly.  Single-problem solves only. */
  int cluster_coarse; /* 1 (default): on 1D FP64 coarse levels with few intervals (and the FP64
                       coarsest solve) each interval's slice is split over a thread-block cluster of
                       up to 16 CTAs, so more SMs share its FP64 steps, sized so that the level's
                       clusters are resident at once; 2, 4, 8, 16: that cluster size on every FP64
                       coarse pass (where the slice allows it); 0: one CTA per interval.  Results
                       are identical either way. */
  double diverge_ratio; /* MGRIT_EDIVERGED once a residual norm exceeds this multiple of the first
                       (default 1e3); 0: only a non-finite norm ends the iteration (rediscretised coarse
                       operators can grow the residual for many cycles before converging) */
  int fine_only;    /* 1D only.  0 (default): the whole MGRIT hierarchy.  1: only what sequential stepping
                       needs -- the fine departure points and the fine level's gather tables (in the
                       handle's precision); sl_step_sequential, sl_step_sequential_batched and
                       mgrit_apply_step at level 0 work, the solves return MGRIT_EUNSUPPORTED. */
  int solve_mode;   /* correction solves [I - diag(sigma) D]^{-1} of 1D coarse levels: 0 (default) exact
                       (partitioned banded solver); 1: the paper's inexact solve (Sec. 3.3, 3.4), GMRES
                       from a zero guess with gmres_maxit / gmres_rtol as in 2D (two-level runs of Table 1:
                       10 iterations, gmres_rtol = 0; multilevel: rtol 1e-2 or 10 iterations) -- FP64 coarse
                       levels only (precision 0, or coarse_fp64 = 1), single problems, no adjoint.
                       2D correction solves take GMRES(gmres_maxit, gmres_rtol) in modes 0 and 1;
                       2: exact solves everywhere -- 1D as mode 0, 2D restarted GMRES(10) to a relative
                       residual of 1e-14 (FP64 coarse levels only), which keeps MGRIT a linear iteration. */
  int coarse_band;  /* 1D FP32 coarse levels.  1 (default): where the separator block of M^{-1} (M = I -
                       diag(sigma) D, 8-row partitions) falls below 1e-8 of its diagonal blocks (under the
                       FP32 unit roundoff of the solve) beyond at most 6 partitions (probed with 8 colours,
                       and again with 16 where the decay is slower), setup stores it as a band and each
                       correction solve applies it in one banded product; 0 (or where the band would be wider
                       or its record does not fit in shared memory): block cyclic reduction of the separator
                       system (p <= 3) or the on-the-fly factorisation (p = 5). */
  int test_wait_cycles; /* testing the timeout path only; 0 (default): off.  > 0: in every 1D FP32 pass
                       whose tables are staged into shared memory by bulk copies, each CTA's first bounded
                       wait is made on a barrier that nothing completes, with this limit in SM cycles, so
                       it gives up; the CTA then lets its copies in flight land (normal limit) and stops,
                       and mgrit_solve returns MGRIT_ETIMEOUT.  The handle stays usable. */
} mgrit_options;

/* Phases timed when mgrit_options.profile = 1 (indices into mgrit_stats.phase_ms / phase_launches). */
enum {
  MGRIT_PHASE_DEPARTURE = 0,  /* fine ERK departure points */
  MGRIT_PHASE_BACKTRACK = 1,  /* coarse departure points, phi, sigma */
  MGRIT_PHASE_TABLES = 2,     /* gather tables */
  MGRIT_PHASE_FACTOR = 3,     /* correction-matrix factorisation */
  MGRIT_PHASE_FINE64_FC = 4,  /* level 0, FP64 F+C relaxation pass */
  MGRIT_PHASE_FINE64_RES = 5, /* level 0, FP64 F-relaxation + C-point residual pass */
  MGRIT_PHASE_FINE64_POST = 6,/* level 0, FP64 final F-relaxation into the output */
  MGRIT_PHASE_FINE32_RES = 7, /* level 0, FP32 error propagation + residual pass */
  MGRIT_PHASE_COARSE = 8,     /* relaxation passes on levels 1 .. L-2 */
  MGRIT_PHASE_COARSEST = 9,   /* sequential solve on the coarsest level */
  MGRIT_PHASE_MISC = 10,      /* norms and elementwise updates */
  MGRIT_PHASE_SEQUENTIAL = 11,/* sl_step_sequential */
  MGRIT_NUM_PHASES = 12
};

typedef struct {
  int iterations;     /* V-cycles performed */
  int converged;      /* 1 if the residual dropped by rtol */
  int levels;         /* levels in the hierarchy (>= 2) */
  int history_len;    /* entries of residual_history written */
  double r0;          /* reference residual norm */
  double r_final;     /* last residual norm */
  double residual_history[256];
  double setup_ms;    /* wall time of mgrit_setup */
  double solve_ms;    /* wall time of the last mgrit_solve */
  int64_t device_bytes; /* workspace held by the handle */
  int64_t kernel_launches;  /* kernels launched by this handle: mgrit_setup plus this call */
  double phase_ms[12];      /* profile = 1: summed event time per phase (setup phases from mgrit_setup) */
  int phase_launches[12];   /* kernels per phase (setup phases from mgrit_setup, others from this call) */
  double final_error;       /* mgrit_solve_to_reference: the last distance of u(T) to the reference */
} mgrit_stats;

typedef struct mgrit_handle mgrit_handle;

/* Fills *opt with the defaults above.  Returns MGRIT_EINVAL on NULL. */
mgrit_status mgrit_default_options(mgrit_options* opt);

/*
 * Builds everything the solver needs for one problem (Sec. 2.1, 3.3.1, 3.4):
 *  - fine departure points: one backward explicit Runge-Kutta step of order r = order
 *    per arrival node and step (eq. (depart_ODE); r = 1 forward Euler, r = 3 Kutta's
 *    third-order method, r = 5 Butcher's six-stage fifth-order method), in FP64;
 *  - the level hierarchy: factor m per level (m_first on level 1 if set) until the
 *    coarsest level has <= max_coarsest steps, or exactly `levels` levels if levels > 0;
 *  - coarse departure points by linear (1D) / bilinear (2D) backtracking
 *    (eq. (coarse_depart_interp), Sec. SM6), phi and sigma (eq. (varphi_p_multilevel_def),
 *    (nu_p_def)) and the factorised correction matrices I - diag(sigma) D_{p+1}.
 * order: odd interpolation degree p in {1, 3, 5} (r = p, Sec. 2.1).
 * m: coarsening factor >= 2; nt must be divisible by the factors used.
 * stream: a cudaStream_t (NULL = the legacy default stream).
 * Errors: MGRIT_EINVAL for bad sizes / kinds / order, MGRIT_ENOMEM, MGRIT_ECUDA,
 *         MGRIT_ESINGULAR if a correction matrix cannot be factorised without pivoting.
 */
mgrit_status mgrit_setup(const mgrit_grid* grid, const mgrit_wavespeed* wave, int order, int m, int levels,
                         const mgrit_options* opt, void* stream, mgrit_handle** out);

/*
 * Solves u_{n+1} = Phi_n u_n, n = 0..nt-1, with u_0 = d_u0 by MGRIT V-cycles with FCF
 * relaxation (Sec. 2.2) until the space-time residual has dropped by rtol.
 * d_u0:     [N] initial condition (N = nx or nx*nx).
 * d_u_init: [(nt+1) x N] initial iterate (row 0 ignored); only rows n = j*m_1 (the C-points)
 *           are read.  NULL means zero.
 * d_u_out:  [(nt+1) x N] the solution at every time point (row 0 = u0).  May alias d_u_init.
 * stats:    optional (NULL allowed), filled on return.
 * The call is synchronous (it returns once convergence is known).
 * Errors: MGRIT_ENOTCONVERGED (d_u_out then holds the last iterate), MGRIT_EDIVERGED,
 *         MGRIT_EINVAL, MGRIT_ECUDA.
 */
mgrit_status mgrit_solve(mgrit_handle* h, const double* d_u0, const double* d_u_init, double* d_u_out,
                         mgrit_stats* stats);

/*
 * mgrit_solve with the alternative stopping rule of the paper's strong-scaling supplement (Sec. SM4):
 * instead of the residual reduction, iterate until the final time slice of the iterate, u(T) after a
 * cycle's correction, is within tol of d_u_final_ref (N values, e.g. the exact PDE solution at T) in
 * the discrete l2 norm e = (h^d sum_i (u_i(T) - ref_i)^2)^(1/2), i.e. to discretisation accuracy.
 * The residual norms are still recorded; stats->final_error holds the last e and stats->converged
 * is 1 when e <= tol.  opt.max_iter bounds the cycles (then MGRIT_ENOTCONVERGED).  Other arguments,
 * results and errors as mgrit_solve; tol < 0 gives MGRIT_EINVAL.
 */
mgrit_status mgrit_solve_to_reference(mgrit_handle* h, const double* d_u0, const double* d_u_init, double* d_u_out,
                                      const double* d_u_final_ref, double tol, mgrit_stats* stats);

/*
 * Sequential SL time stepping (eq. (one-step) with g = 0), the comparator of MGRIT:
 * u_{n+1} = S_{p,r}^{(t_n, dt)} u_n on the fine level, FP64 (precision 0) or FP32 (1).
 * d_u_out: store_all = 1: [(nt+1) x N] every slice; store_all = 0: [N] the final slice only.
 * Asynchronous on the handle's stream.
 */
mgrit_status sl_step_sequential(mgrit_handle* h, const double* d_u0, double* d_u_out, int store_all);

/*
 * Same as mgrit_solve, but d_u0 / d_u_init / h_u_out are HOST arrays: the call copies the
 * inputs to the device, solves, and copies the full solution back (end-to-end timing).
 */
mgrit_status mgrit_solve_host(mgrit_handle* h, const double* h_u0, const double* h_u_init, double* h_u_out,
                              mgrit_stats* stats);

/*
 * Discrete adjoint of the fine-level one-step system for J = 1/2 ||u_nt - u_target||^2.  The paper has no
 * adjoint; this follows from its one-step system (eq. (one-step)): lambda_nt = u_nt - u_target,
 * lambda_n = Phi_n^T lambda_{n+1}, solved backward in time by MGRIT (the reversed problem
 * mu_k = lambda_{nt-k} with the transposed operators; coarse levels use Psi^T = S^T M^{-T} of the
 * forward hierarchy), same cycle and stopping rule as mgrit_solve, from a zero initial iterate.
 * S^T is a deterministic transposed gather (1D: a window of arrival points per node; 2D: the arrival
 * points grouped by the base node of their tensor-product stencil, Sec. 4.1, in sorted buckets).
 * M^{-T}: 1D the partitioned banded solver factorising M^T; 2D the same inexact GMRES as the forward
 * coarse operator (Sec. 4.3), applied to M^T.
 * Outputs dJ/du0 = lambda_0 and dJ/da = sum_n lambda_{n+1}^T (dPhi_n/da) u_n, where a is wave.a of the
 * kinds with an amplitude (MGRIT_A_CONST: alpha = a; MGRIT_A_SIN_KX_COS_T; 2D: the x speed of
 * MGRIT_A2D_CONST and the amplitude of both components of MGRIT_A2D_SIN_COS) and dJ/da is 0 for the
 * others; dPhi/da acts through d s/d a of a tangent-linear ERK step, and u_n is recomputed from the
 * checkpoints.
 * d_C_checkpoints: [(nt/m_1 + 1) x N] the C-point rows u_{j m_1} of a converged forward solve.
 * d_dJ_du0: [N]; d_dJ_dparams: [1] device array receiving dJ/da (both stay on the device, so a caller
 * can chain further device work on the handle's stream).  FP64 handles (precision 0), 1D and 2D.  The first call builds
 * the transposed data (1D: floor ranges and M^T factors; 2D: buckets, 8 bytes per point and step of
 * every level) and d s/d a (8 bytes per fine point, step and dimension).  Synchronous.
 * stats (optional) describes the adjoint MGRIT solve.
 */
mgrit_status mgrit_adjoint_solve(mgrit_handle* h, const double* d_u_target, const double* d_C_checkpoints,
                                 double* d_dJ_du0, double* d_dJ_dparams, mgrit_stats* stats);

/* ---- Introspection (for tests): copies of intermediate setup data --------------------------- */

/* Number of levels and, for a level l, its step count and coarsening factor (0 on level 0). */
mgrit_status mgrit_level_info(const mgrit_handle* h, int level, int* nt_level, int* m_level);

/* Half-width, in 8-row partitions, of the banded separator inverse that level l's FP32 correction solves
 * apply (mgrit_options.coarse_band); 0 where the level solves otherwise.  decay (NULL or 4 floats): the
 * decay of that inverse from the first (8-colour) probe, decay[t - 1] = the largest entry at partition
 * distance t (t = 4: the sum of the two entries at +-4) over the largest diagonal-block entry, maximised
 * over the level's steps; zeros where the level was not probed. */
mgrit_status mgrit_level_band(const mgrit_handle* h, int level, int* half_width, float* decay);

/* Departure offsets s[n][pt] = (x_pt - xi_pt) / h of level l in grid units (2D: x then y
 * component blocks, each [nt_l x N]); d_out has nt_l * N (2D: 2 * nt_l * N) doubles. */
mgrit_status mgrit_copy_offsets(const mgrit_handle* h, int level, double* d_out);

/* sigma of level l >= 1 (eq. (nu_p_def)); same layout as mgrit_copy_offsets. */
mgrit_status mgrit_copy_sigma(const mgrit_handle* h, int level, double* d_out);

/* Applies Phi_{l,n} (level 0: the SL step; level >= 1: the coarse operator) to `count` slices:
 * d_out[c] = Phi_{l, n0 + c} d_in[c], c = 0..count-1, each slice N doubles, in the handle's
 * working precision.  Synchronous. */
mgrit_status mgrit_apply_step(mgrit_handle* h, int level, int n0, int count, const double* d_in, double* d_out);

/*
 * mgrit_apply_step without any device allocation.  The paper has no counterpart: this is a service
 * for callers that cannot allocate device memory -- for instance an application whose framework
 * reserves the GPU's memory up front (a cudaMalloc from this library would fail or fragment that
 * pool), or a latency-sensitive caller that cannot accept the device-wide synchronisation of
 * cudaFree.  Same arguments, layout and result as mgrit_apply_step.  Levels that work in FP32 are
 * staged through an 8 MiB buffer in file-scope device memory that every GPU loading this library
 * holds until the process exits; count * N must not exceed 1048576 (MGRIT_EINVAL otherwise, before
 * any launch).  Every call looks up that buffer's address on the current device (cudaGetSymbolAddress),
 * and the current device must be the handle's device (MGRIT_EINVAL otherwise, before any launch).
 * All calls share the buffer: calls that overlap on the GPU (other streams, other threads, other
 * handles) race; calls issued one after another are safe, as each call overwrites every staged value
 * it reads.  Synchronous.
 */
mgrit_status mgrit_apply_step_noalloc(mgrit_handle* h, int level, int n0, int count, const double* d_in,
                                      double* d_out);

void mgrit_destroy(mgrit_handle* h);

/*
 * Batched independent 1D problems (each as in mgrit_setup, levels chosen by the rule of mgrit_setup):
 * grids[q], waves[q], orders[q], ms[q] for q < nprob; the shared options must select the FP32-bulk mode
 * (precision 1; precision 0 only with fine_only, for FP64 sequential stepping) and the corrected coarse
 * operator.  A fine_only batch sets up the fine levels alone (sl_step_sequential_batched; its solves return
 * MGRIT_EUNSUPPORTED).  mgrit_solve_batched runs the V-cycles of all problems
 * in lockstep with one kernel launch per cycle phase over (problem, interval) tiles; each problem stops
 * when its own residual criterion is met (a per-problem mask).  d_u0[q], d_u_init[q] (or NULL),
 * d_u_out[q] as in mgrit_solve; stats: NULL or an array of nprob.  MGRIT_ENOTCONVERGED if any problem did
 * not converge.  The paper solves one problem at a time; batching follows from its one-step system.
 */
typedef struct mgrit_batch mgrit_batch;
mgrit_status mgrit_setup_batched(int nprob, const mgrit_grid* grids, const mgrit_wavespeed* waves, const int* orders,
                                 const int* ms, const mgrit_options* opt, void* stream, mgrit_batch** out);
mgrit_status mgrit_solve_batched(mgrit_batch* b, const double* const* d_u0, const double* const* d_u_init,
                                 double* const* d_u_out, mgrit_stats* stats);
/*
 * With mgrit_options.profile = 1, stats[q].phase_ms / phase_launches hold problem q's own setup phases
 * (departure .. factor) and, for the cycle phases, the totals of the batch's launches, which serve every
 * problem at once (the same figures in every stats[q]); stats[0].kernel_launches counts every kernel of
 * the batch (the problems' setups, the tuner's timed runs, this call), the other entries 0.
 *
 * mgrit_solve_batched_host: the same solve from HOST arrays (end-to-end timing): h_u0[q] [N];
 * h_u_init_c[q] the initial iterate at the C-points only, [(nt/m_1 + 1) x N] with row j the iterate at
 * time index j m_1 (row 0 ignored), or NULL (zero) -- the solver reads nothing else of the iterate;
 * h_u_out[q] [(nt + 1) x N] the full solution.  The call copies in, solves, and copies every solution
 * back before it returns; device staging comes from the library's pool.
 */
mgrit_status mgrit_solve_batched_host(mgrit_batch* b, const double* const* h_u0, const double* const* h_u_init_c,
                                      double* const* h_u_out, mgrit_stats* stats);
/*
 * Sequential SL time stepping of every problem of the batch (eq. (one-step) with g = 0), the comparator
 * of the batched solve: u_{n+1} = S_{p,r}^{(t_n, dt)} u_n on each problem's fine level, all problems in one
 * launch (one CTA per problem, slice in shared memory): FP32 on FP32-bulk batches, FP64 on fine_only batches
 * set up with precision 0 (mgrit_setup_batched accepts precision 0 only with fine_only).
 * d_u0[q] [N] FP64 start slices; d_u_out[q] [N] FP64 final slices.  Returns once done.
 */
mgrit_status sl_step_sequential_batched(mgrit_batch* b, const double* const* d_u0, double* const* d_u_out);
void mgrit_destroy_batched(mgrit_batch* b);
const char* mgrit_status_string(mgrit_status s);
const char* mgrit_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MGRIT_SL_H */
