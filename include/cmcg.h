/*
 * cmcg.h -- C ABI of the GB300 controllability conjugate-gradient (CMCG) Helmholtz solver.
 *
 * The solver computes the time-harmonic field u of the Helmholtz problem of Sec. 2.1
 * (Eq. HE: -Lap u - k^2 u = f in Omega, du/dn - i k u = g_S on the absorbing faces,
 * du/dn = 0 on Neumann faces, u = 0 on Dirichlet faces and obstacle nodes, k = omega/c)
 * by the CMCG Algorithm of Sec. 2.3: conjugate gradients on the initial data (v0, v1) of
 * the wave equation of Eq. WE so that its solution is T-periodic, T = 2 pi / omega.
 *
 * Discretisation (fixed by this library, identical for every entry point):
 *   - nodes x_j = j h, j in {0..n_x} x {0..n_y} (x {0..n_z}); node index
 *     j = ix + (n_x+1) (iy + (n_y+1) iz), x fastest.  N_p = prod (n_a + 1).
 *   - mass-lumped vertex-centred finite differences: lumped volume W_j = h^d prod_a w(j_a),
 *     w = 1/2 on the two end nodes of an axis, 1 elsewhere; stiffness K = W (-Lap_h) with
 *     mirror (Neumann) ghosts, 2nd order (5/7-point) or 4th order (9/13-point, even
 *     reflection); M = diag(W/c^2); absorbing faces add B = diag(A/c), A = lumped face area.
 *   - leapfrog in time with the absorbing term centred (Sec. 4.3.1: explicit, T/dt an
 *     integer): N = ceil(T/dt_target - 1e-9) steps of dt = T/N per period.
 *   - discrete time-harmonic solution: (K - wt^2 M - i wh B) U = W f + A g with
 *     wt = (2/dt) sin(omega dt/2), wh = sin(omega dt)/dt; returned U = v0 + i v1 / wh
 *     after removing the constant shift lambda of Theorem 1 when there is no Dirichlet
 *     node (compatibility condition of Sec. 2.1, discrete form).
 *
 * Memory: every array argument is a DEVICE pointer to caller-owned memory unless its name
 * ends in _host.  Real fields are double[N_p]; complex fields are interleaved (re, im)
 * double[2 N_p] (C99 double _Complex layout).  The library allocates no device memory
 * itself: all state lives in the caller-allocated workspace passed to cmcg_create (size
 * from cmcg_workspace_size).  Work is enqueued on the handle's stream; the calls return
 * after the stream has finished the call's work.  A handle is not thread-safe; use one
 * handle per stream.
 *
 * Errors: every int-returning call returns CMCG_OK (0), CMCG_NOT_CONVERGED (1, output holds
 * the last iterate) or a negative error code; cmcg_status_string names it.  A call that
 * fails leaves its outputs unspecified and the handle usable unless the code is
 * CMCG_ERR_CUDA.
 */
#ifndef CMCG_H
#define CMCG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------- */
#define CMCG_OK 0
#define CMCG_NOT_CONVERGED 1
#define CMCG_ERR_INVALID_ARG (-1)
#define CMCG_ERR_CFL (-2)
#define CMCG_ERR_WORKSPACE (-3)
#define CMCG_ERR_UNSUPPORTED (-4)
#define CMCG_ERR_CUDA (-5)
#define CMCG_ERR_DIVERGED (-6)
#define CMCG_ERR_DEVICE_TIMEOUT (-7) /* a bounded device-side wait ran out (batched kernel barrier) */

/* ---- boundary codes (face order -x, +x, -y, +y, -z, +z) --------------------------- */
#define CMCG_BC_ABC 0       /* first-order absorbing (impedance) face, Eq. HE_ABC      */
#define CMCG_BC_NEUMANN 1   /* homogeneous Neumann face, Eq. HE_NBC                      */
#define CMCG_BC_DIRICHLET 2 /* homogeneous Dirichlet face, Eq. HE_DBC                    */

/* ---- option flags ------------------------------------------------------------------ */
#define CMCG_FLAG_HOST_IO 1 /* reserve a staging buffer in the workspace for cmcg_solve_host */
#define CMCG_FLAG_TIMING 2  /* time the leapfrog step kernels with CUDA events on the handle's
                               stream; results in cmcg_stats.step_seconds_* / step_launches_*.
                               Flexible-CG iterations are still replayed as CUDA graphs: the
                               events are recorded by nodes of the captured iteration */
#define CMCG_FLAG_INEXACT_RIESZ 4 /* apply the Riesz map of Eq. CMCG_PRECONDITIONIER approximately:
                               one multigrid V-cycle per CG iteration on the dual residual,
                               with flexible (Polak-Ribiere) CG; the fixed point is unchanged
                               (the gradient of J is still evaluated exactly) */
#define CMCG_FLAG_FILTER 8  /* recover U with the fundamental-frequency filter of Sec. 2.2: one
                               extra forced FP64 period from the converged (v0, v1) accumulates
                               (1/N) sum_n (y^n + (i/wh) v^n) e^{i w t_n}, which removes the constant
                               shift of Theorem 1 without the compatibility condition (stats
                               lambda = 0).  In the pure Neumann case (no absorbing face, no
                               Dirichlet node) the minimiser's linear growth eta t leaves a
                               constant, removed with the discrete compatibility condition
                               (Eq. cc_neumann_eta); stats lambda then holds that constant */
#define CMCG_FLAG_NO_CG 16  /* "do-nothing" long-time solver of Sec. 4.2 (Eq. AP_SOLUTION), the
                               comparator the paper uses to show why controllability is needed:
                               integrate the forced wave equation from rest for runup_periods = l
                               periods (or the automatic count for -k; 0 is CMCG_ERR_INVALID_ARG)
                               with the sources ramped by theta_tr over [0, l T] (Sec. 4.2.3) and
                               recover U from the state at t = l T as in step (6), without CG.
                               Near trapped modes (nonconvex obstacles) U converges very slowly
                               in l; stats J_final is the periodicity misfit of that state. */

#define CMCG_FLAG_FIRST_ORDER 32 /* the first-order (mixed) formulation of Sec. 3 on a staggered
                               grid: v = y_t on the nodes, p = grad y on the grid links
                               (Eq. mixWE), staggered leapfrog, J^ of Eq. mix_cost_functional_J
                               with its gradient from the backward first-order period
                               (Eq. mixJ_deriative_2); the energy inner product is diagonal, so
                               no Riesz solve runs.  U by Eq. mix_solution, or with
                               CMCG_FLAG_FILTER by Eq. TH_FILTERED_MIXED_SOLUTION.  The discrete
                               fixed point is the same U as the second-order scheme's.  Supports
                               CMCG_FP64, CMCG_FP32 and CMCG_MIXED (FP64 defect correction around
                               FP32 CG, as for the second-order scheme; with FP32 periods use
                               CMCG_FLAG_FILTER: rounding excites the nearly periodic spurious
                               modes of Sec. 3.2, which Eq. mix_solution keeps and the filter
                               removes), order 2, and the run-up of Sec. 4.2.3 (runup_periods);
                               order 4, CMCG_FLAG_INEXACT_RIESZ and CMCG_FLAG_NO_CG are
                               CMCG_ERR_UNSUPPORTED.  cmcg_wave_period, cmcg_adjoint_period and
                               cmcg_riesz return CMCG_ERR_UNSUPPORTED on such a handle; use
                               cmcg_fo_period and cmcg_fo_adjoint_period. */
#define CMCG_FLAG_L2_KAPPA 64 /* keep the FP32 coefficient kappa (4 bytes per node, read by
                               every FP32 leapfrog step and never written) resident in the L2
                               cache across steps: the handle's stream gets an access-policy
                               window on it and the process's persisting-L2 set-aside is raised
                               to its size (restored when the last such handle is destroyed).
                               Applies to CMCG_FP32 / CMCG_MIXED handles on a created stream
                               whose kappa fits the device's largest set-aside (84.7 MB on a
                               GB300: grids up to 21 M nodes); otherwise ignored.  Side effects
                               beyond the handle: the stream attribute (cleared at destroy) and
                               the set-aside, which other work in the process shares. */

/* ---- precision of the wave stepping ------------------------------------------------ */
#define CMCG_FP64 0  /* every operation in FP64                                            */
#define CMCG_FP32 1  /* leapfrog fields and stencil arithmetic in FP32; CG vectors, inner
                        products, energy functional and Riesz solve in FP64               */
#define CMCG_MIXED 2 /* CMCG_FP32 inner CG inside an FP64 defect-correction loop whose
                        residual (gradient of J) is evaluated with FP64 stepping         */

typedef struct cmcg_handle cmcg_handle;

typedef struct {
    int dim;      /* 2 or 3                                                              */
    int n[3];     /* intervals per axis (n[2] ignored in 2D); nodes per axis = n + 1      */
    double h;     /* grid spacing, equal on all axes                                      */
    int order;    /* spatial order of the Laplacian: 2 or 4                               */
} cmcg_grid;

typedef struct {
    unsigned char face[6];               /* CMCG_BC_* per face (-x,+x,-y,+y,-z,+z)        */
    const unsigned char* dirichlet_mask; /* device uint8[N_p], 1 = sound-soft obstacle
                                            node (u = 0); NULL = none.  Read at create.  */
} cmcg_bc;

typedef struct {
    int precision;          /* CMCG_FP64 / CMCG_FP32 / CMCG_MIXED                        */
    double dt;              /* target time step; 0 = 0.5 h / (sqrt(d) c_max)             */
    int max_iter;           /* CG iteration cap (0 = 10000)                                */
    double riesz_tol;       /* relative residual of the Riesz (Laplace) solve (0 = 1e-12) */
    int riesz_max_iter;     /* PCG iteration cap of the Riesz solve (0 = 60)              */
    double inner_tol;       /* CMCG_MIXED: relative tolerance of each inner FP32 solve
                               (0 = 1e-3)                                                 */
    int flags;              /* CMCG_FLAG_* bits; other bits must be 0                      */
    int runup_periods;      /* initial run-up of Sec. 4.2.3: integrate the wave equation from rest
                               for this many periods with the sources ramped in by
                               theta(t) = (2 - sin(pi t / (2 t_tr))) sin(pi t / (2 t_tr)),
                               t_tr = runup_periods T, and start CG from the final state.
                               0 = none; -k (1 <= k <= 64) = ceil(k diam(Omega) / (T c_min)),
                               the periods waves at the slowest speed need to cross the
                               domain's diagonal k times.  With a run-up, the
                               relative tolerance of cmcg_solve refers to the residual of the
                               zero initial guess (one extra gradient evaluation), so the accuracy
                               at a given tol does not depend on the run-up.                  */
    int tile[4];            /* launch shape of the leapfrog kernels, 0 = default.  [3] selects
                               the step scheme of 3D 7-point steps (the others keep one step per
                               launch): 0 = the default, scheme 3 on 3D 7-point grids and
                               scheme 5 on 2D 5-point grids (the fastest measured); 1 = one
                               step per launch, [0] z-planes per thread
                               (16); 2 = two FP32 steps per launch (temporal blocking), [0]
                               planes staged ahead (1..3, 0 = 2), [1] z-planes per block
                               (0 = 16), [2] interior tile height (0 = the fewest tiles, at
                               most 60); 3 = one step per launch with [2] = 2 (default) or 4
                               z-planes per loop iteration, [0] z-planes per thread; 4 = FP32
                               steps with operands staged by TMA bulk copies, [0] z-planes per
                               CTA and [1] rows per band (0 = automatic); 5 = FP32 steps in
                               vector form, one aligned float4 of the flat node index per
                               thread, also for 2D 5-point steps (FP64 steps: scheme 1);
                               6 = FP32 steps with operands staged in shared memory by
                               asynchronous copies several planes ahead, [0] z-planes per
                               CTA, [1] rows per band, [2] planes in flight (2 or 3; 0 =
                               automatic).  Chosen per grid class by the autotuner
                               (paper_1903_12522_gb300/autotune.py). */
} cmcg_options;

typedef struct {
    int iterations;          /* CG iterations (CMCG_MIXED: summed over inner solves)       */
    int outer_iterations;    /* CMCG_MIXED defect-correction rounds (else 0)              */
    int periods;             /* wave periods integrated (forward + adjoint)               */
    int riesz_iterations;    /* PCG iterations summed over all Riesz solves               */
    int steps_per_period;    /* N                                                         */
    double dt;               /* T / N                                                     */
    double omega_tilde;      /* (2/dt) sin(omega dt / 2)                                  */
    double omega_hat;        /* sin(omega dt) / dt                                        */
    double rel_residual;     /* sqrt(||r||_E^2 / ||r0||_E^2) at exit (Step 5.8)             */
    double J0;               /* J at the initial guess (Eq. cost_functional_J)            */
    double J_final;          /* J at the returned iterate (one extra forward period)      */
    double lambda_re;        /* removed constant shift (0 if Dirichlet nodes exist)       */
    double lambda_im;
    long long point_updates; /* grid-point leapfrog updates performed                      */
    double seconds;          /* wall time of the call                                     */
    long long kernel_launches; /* CUDA kernels this library launched during the call       */
    int runup_periods;       /* periods integrated by the run-up (0 if none)              */
    /* CMCG_FLAG_TIMING: summed device time and launch count of the leapfrog step kernels
       (forward and adjoint), split by stepping precision; 0 otherwise */
    double step_seconds_fp32, step_seconds_fp64;
    long long step_launches_fp32, step_launches_fp64;
    /* flexible-CG iterations (CMCG_FLAG_INEXACT_RIESZ) replayed as one captured CUDA graph
       each; the rest ran as separate launches (the solve's stream was 0, the legacy or the
       per-thread default stream, or capture failed) */
    long long graph_replays;
} cmcg_stats;

typedef struct {
    int steps_per_period;    /* N                                                         */
    double dt, omega_tilde, omega_hat;
    long long num_nodes;     /* N_p                                                       */
    int mg_levels;           /* levels of the multigrid preconditioner of the Riesz solve */
    int has_dirichlet;       /* 1 if any node is Dirichlet                                */
} cmcg_info;

/* Bytes of device workspace cmcg_create needs for this grid and options (0 on invalid
 * arguments).  Exact: serving code admits solves by this number. */
size_t cmcg_workspace_size(const cmcg_grid* grid, const cmcg_options* opts);

/* Build a solver.  c: device double[N_p] wave speed c(x) > 0 (copied).  omega > 0: angular
 * frequency (T = 2 pi / omega).  workspace: device memory of ws_bytes >= cmcg_workspace_size,
 * 256-byte aligned, owned by the caller and kept alive until cmcg_destroy.  stream: a
 * cudaStream_t (NULL = default stream).  Validates sizes and the CFL condition
 * dt^2 c_max^2 rho < 4 (rho = 4d/h^2, 2nd order; 16d/(3h^2), 4th order) and returns
 * CMCG_ERR_CFL if violated.  4th order with Dirichlet nodes is CMCG_ERR_UNSUPPORTED.
 * Sec. 2.1 (problem), Sec. 4.3.1 (leapfrog, mass lumping, T/dt integer). */
int cmcg_create(const cmcg_grid* grid, const double* c, double omega, const cmcg_bc* bc,
                const cmcg_options* opts, void* workspace, size_t ws_bytes, void* stream,
                cmcg_handle** out);

int cmcg_destroy(cmcg_handle* h);

int cmcg_get_info(const cmcg_handle* h, cmcg_info* info);

/* Residual history of the last cmcg_solve / cmcg_solve_host on this handle (the quantity the
 * stopping criterion of the CMCG Algorithm, Step 5.8, tests, studied along the iterations in
 * Sec. 4.2): entry k is sqrt(gamma_k / gamma_0) after CG iteration k (k = 0: the start),
 * relative to the zero initial guess (also with a run-up).  CMCG_MIXED: the inner FP32
 * iterations' estimates scaled by the FP64 residual they started from, and at the end of each
 * inner solve the recomputed FP64 residual.  First-order solves record none.  rel_host: host,
 * capacity doubles; *count receives the number of entries (copies min(count, capacity)). */
int cmcg_get_history(const cmcg_handle* h, double* rel_host, int capacity, int* count);

/* One period of the forced wave equation (Eq. WE) by leapfrog: from y(0) = u0, y_t(0) = v0
 * to (uT, vT) = (y(T), y_t(T)).  f: interior source amplitude, g: boundary datum g_S on
 * absorbing nodes (complex double[N_p] each, NULL = 0); the forcing is
 * Re((W f + A g) exp(-i omega t)).  At edge and corner nodes g is the mean of the faces'
 * values.  Dirichlet entries of the inputs are ignored and zero in the outputs.  Runs in the
 * handle's stepping precision (CMCG_MIXED steps in FP64 here).  Outputs must not alias
 * inputs. */
int cmcg_wave_period(cmcg_handle* h, const double* u0, const double* v0, const double* f,
                     const double* g, double* uT, double* vT);

/* Transpose of the homogeneous period map, P^T (a, b): the discrete backward (adjoint) wave
 * equation of Eq. AWE that yields J' (Eq. J1_derivative_final).  a, b: dual vectors (the
 * cotangents of y(T) and y_t(T)); q0, q1: cotangents of y(0), y_t(0).  Satisfies
 * <P x, (a,b)> = <x, (q0,q1)> to rounding. */
int cmcg_adjoint_period(cmcg_handle* h, const double* a, const double* b, double* q0, double* q1);

/* Riesz map of Eq. CMCG_PRECONDITIONIER for the v0 component: s = K^+ rhs (K = W (-Lap_h),
 * Dirichlet rows removed).  Without Dirichlet nodes K is singular; rhs is projected onto
 * range(K) and s has W-weighted mean zero.  FP64 flexible PCG preconditioned by a geometric
 * multigrid V-cycle.  Returns CMCG_NOT_CONVERGED if riesz_tol is not met. */
int cmcg_riesz(cmcg_handle* h, const double* rhs, double* s);

/* Full CMCG solve (Sec. 2.3, steps (1)-(6)).  f, g as in cmcg_wave_period.  tol: Step 5.8
 * relative E-norm residual.  u: device complex double[N_p] output U.  stats: host, nullable.
 * Returns CMCG_OK, CMCG_NOT_CONVERGED (max_iter reached, u holds the last iterate) or an
 * error (CMCG_ERR_DIVERGED if a CG scalar becomes NaN/Inf or non-positive). */
int cmcg_solve(cmcg_handle* h, const double* f, const double* g, double tol, double* u,
               cmcg_stats* stats);

/* cmcg_solve started from a given field instead of zero or the run-up: on entry u (device,
 * complex interleaved, N_p) holds the start field, for example a checkpointed iterate or the
 * solution at a nearby frequency; CG starts from its periodic initial state (v0, v1) =
 * (Re u, omega_hat Im u), the relation of step (6) read backwards.  On exit u holds the
 * solution, as with cmcg_solve.  The tolerance stays relative to the zero guess's gradient
 * (one extra gradient evaluation), so tol means the same as in a cold solve; the run-up
 * option is not used.  CMCG_ERR_UNSUPPORTED for the first-order formulation and the
 * do-nothing solver. */
int cmcg_solve_warm(cmcg_handle* h, const double* f, const double* g, double tol, double* u,
                    cmcg_stats* stats);

/* cmcg_solve with HOST buffers: f_host, g_host (nullable) and u_host are host complex
 * double[N_p] arrays (pinned memory gives full copy speed).  Copies the inputs into the
 * workspace, solves, copies U back; all copies are on the handle's stream.  Needs a handle
 * created with CMCG_FLAG_HOST_IO (else CMCG_ERR_INVALID_ARG). */
int cmcg_solve_host(cmcg_handle* h, const double* f_host, const double* g_host, double tol,
                    double* u_host, cmcg_stats* stats);

const char* cmcg_status_string(int status);

/* ---- first-order formulation -------------------------------------------------------- */
/* First-order state (handles created with CMCG_FLAG_FIRST_ORDER): (dim + 1) * N_p doubles,
 * laid out p_x | p_y | (p_z) | v; p_a[j] is the link from node j to node j + e_a (entries
 * with j_a = n_a carry no link: ignored on input, 0 on output), v[j] the velocity at node j
 * (ignored and returned 0 on Dirichlet nodes).  All pointers are device, caller-owned.
 *
 * One forward staggered-leapfrog period from s0 (Eq. mixWE) into sT; f, g (nullable) are the
 * sources as in cmcg_wave_period.  CMCG_ERR_UNSUPPORTED for a second-order handle. */
int cmcg_fo_period(cmcg_handle* h, const double* s0, const double* f, const double* g, double* sT);
/* The plain (Euclidean) transpose of the homogeneous first-order period map applied to y:
 * the backward first-order wave equation of Eq. mixJ_deriative_2 in its discrete form. */
int cmcg_fo_adjoint_period(cmcg_handle* h, const double* y, double* out);

/* Self-test of the bounded wait used by the bulk-copy step kernel (cmcg_options.tile[3] == 4):
 * one CTA waits, with at most spin_limit polls, on an mbarrier phase that nothing completes.
 * Returns CMCG_ERR_DEVICE_TIMEOUT (the expected outcome), CMCG_OK if the wait wrongly
 * succeeded, CMCG_ERR_INVALID_ARG for spin_limit < 1, CMCG_ERR_CUDA on a CUDA error.  The
 * context stays usable. */
int cmcg_bulk_wait_selftest(int spin_limit, void* stream);

/* Compiled-in bounds checks.  libcmcg_checked.so is the same library built with -DCMCG_CHECKED:
 * its step, period-end, source, two-step, batched-step and multigrid kernels test, per thread,
 * that every node index they will touch lies inside its array; a thread that fails records the
 * check site and the index and skips its accesses.  This reads the records since the last call
 * and clears them (synchronising the device): *count failed checks, *site the first one's site
 * (1 column kernels, 2 float4 step, 3 batched step, 4 two-step node or plane, 5 two-step shared
 * neighbour, 6 multigrid; -1 when none), *index its offending index.  Any pointer may be null.
 * Returns CMCG_OK in the checked build; in the normal build (no checks compiled) it writes
 * zeros and returns CMCG_ERR_UNSUPPORTED. */
int cmcg_check_status(long long* count, long long* site, long long* index);

/* ---- multi-solve engine (batched solves and serving) -------------------------------- */
/* Many solves advance together, one CG iteration per cmcg_engine_tick.  Each admitted solve
 * keeps its own handle (its workspace holds the resident CG state).  Per tick, the FP32
 * leapfrog step loops of all solves in their inner iterations run in one batched persistent
 * kernel per period (forward, then adjoint; uneven grids and step counts step together and
 * idle when done); the rest of each iteration is per-solve kernels.  The tick is captured as
 * a CUDA graph and replayed while the set of active solves and their phases stay the same.
 * Solves finish independently; a finished solve's result is read with cmcg_engine_result,
 * which frees its slot.  Requirements: every handle uses the engine's stream, precision
 * CMCG_FP32 or CMCG_MIXED and CMCG_FLAG_INEXACT_RIESZ, none of CMCG_FLAG_FILTER,
 * CMCG_FLAG_NO_CG and CMCG_FLAG_FIRST_ORDER, and a run-up only with CMCG_MIXED (else
 * CMCG_ERR_UNSUPPORTED).  A mixed-precision slot with runup_periods != 0 runs its run-up as one
 * unit after the zero guess's outer gradient (the tolerance reference).  The
 * batched kernel is a cooperative launch whose grid barrier waits are bounded; a wait that
 * runs out returns CMCG_ERR_DEVICE_TIMEOUT from cmcg_engine_tick. */
typedef struct cmcg_engine cmcg_engine;
#define CMCG_ENGINE_NO_GRAPH 1 /* run ticks as plain launches instead of CUDA graphs */

/* Device workspace bytes for an engine of max_slots slots (0 if max_slots is not 1..4096). */
size_t cmcg_engine_workspace_size(int max_slots);
/* workspace: device, 256-byte aligned, caller-owned; stream: cudaStream_t shared with the
 * handles (CUDA graphs need a created stream: on the legacy default stream, NULL, ticks run as
 * plain launches); flags: CMCG_ENGINE_* bits. */
int cmcg_engine_create(int max_slots, void* workspace, size_t ws_bytes, void* stream, int flags,
                       cmcg_engine** out);
int cmcg_engine_destroy(cmcg_engine* e);
/* Launch shape of the batched step kernel (tuned per workload class by the autotuner):
 * blocks_per_sm resident blocks per SM (0 = as many as fit, the default; larger values are
 * capped there), z_planes = z-planes per work item on 3D grids (0 = 16, at most 256).  Only
 * while no solve is active (else CMCG_ERR_INVALID_ARG). */
int cmcg_engine_set_shape(cmcg_engine* e, int blocks_per_sm, int z_planes);
/* Admit a solve: f, g sources as in cmcg_solve (device, nullable, read now); tol as in
 * cmcg_solve; u: device complex double[N_p] written when the solve finishes.  Returns the slot
 * (>= 0), or CMCG_ERR_WORKSPACE when no slot is free, CMCG_ERR_INVALID_ARG when h is already
 * in a slot. */
int cmcg_engine_submit(cmcg_engine* e, cmcg_handle* h, const double* f, const double* g, double tol, double* u);
/* One iteration of every active solve.  finished[0..max_finished) receives the slots that
 * finished in this tick, *n_finished their number. */
int cmcg_engine_tick(cmcg_engine* e, int* finished, int max_finished, int* n_finished);
/* Status and statistics of a finished slot (CMCG_OK, CMCG_NOT_CONVERGED or an error); frees
 * the slot.  CMCG_ERR_INVALID_ARG if the slot has not finished.  After it returns, the engine
 * holds nothing of the solve (a cached tick graph that included the slot is dropped): the
 * caller may destroy the handle and free its workspace, and a new solve admitted into the
 * same slot, even with a handle at the same address, never replays the old solve's graph.
 * A handle must not be destroyed while its slot is still active or unread. */
int cmcg_engine_result(cmcg_engine* e, int slot, cmcg_stats* stats);
/* Number of solves in progress. */
int cmcg_engine_active(const cmcg_engine* e);
/* Ticks run and CUDA graphs built so far. */
int cmcg_engine_info(const cmcg_engine* e, long long* ticks, long long* graph_builds);
/* Name of the CUDA error behind the engine's last CMCG_ERR_CUDA ("cudaSuccess" if none). */
const char* cmcg_engine_cuda_error(const cmcg_engine* e);
/* Failure-path self-test: launches a one-block grid barrier that expects one block more than
 * exists, so its bounded wait must run out after spin_limit polls (1..2^24).  Returns
 * CMCG_ERR_DEVICE_TIMEOUT when the time-out path works, CMCG_OK if it (wrongly) did not fire. */
int cmcg_engine_barrier_selftest(cmcg_engine* e, long long spin_limit);

/* Allocation-free FP64 wave period (the paper has no counterpart; this entry point exists for
 * callers that cannot allocate device memory, such as a plug-in inside a host application
 * that owns the whole device-memory budget, or a real-time loop that must not take
 * cudaMalloc's implicit device-wide synchronisation).  Computes what cmcg_wave_period computes
 * for a handle of the same grid, c, omega, bc and dt with precision CMCG_FP64, without a handle
 * or workspace: arguments as in cmcg_create and cmcg_wave_period (device pointers; stream is a
 * cudaStream_t, NULL = default stream).  It calls no cudaMalloc, cudaFree or other allocating
 * routine.  Its scratch is one static 18 MiB device array inside this library, which every GPU
 * that loads the library holds until the process exits; grids above 262,144 nodes (for example
 * larger than 511^2 in 2D or 63^3 in 3D) are rejected with CMCG_ERR_WORKSPACE.  Every call
 * reads scalars back to the host and synchronises its stream, so no call may be made while its
 * stream is being captured into a CUDA graph.  The first call on a device looks up the
 * array's device address with cudaGetSymbolAddress; the address is kept for the life of the
 * process, so a device reset (cudaDeviceReset) on a device this entry point has used leaves
 * it unusable on that device.  Every call on a device shares the array and
 * clears the parts that must start at zero; calls that overlap on the GPU (other streams or
 * threads) race.  Returns after the stream has finished the call's work. */
int cmcg_wave_period_static(const cmcg_grid* grid, const double* c, double omega, const cmcg_bc* bc,
                            double dt, const double* u0, const double* v0, const double* f,
                            const double* g, double* uT, double* vT, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* CMCG_H */
