/*
 * mqs.h - C ABI of the GB300 (sm_103a) library for the semi-explicit
 * eddy-current time stepper with multiple right-hand side start vectors.
 *
 * Method (Dutine, Clemens, Schoeps, "Multiple Right-Hand Side Techniques in
 * Semi-Explicit Time Integration Methods for Transient Eddy Current
 * Problems"):
 *   Sec. II, eq. (DAE)   edge unknowns split into conducting a_c and
 *                        nonconducting a_n;
 *   Sec. II, eq. (SC)    generalised Schur complement
 *                        K_S(a_c) = K_c(a_c) - K_cn K_n^+ K_cn^T;
 *   Sec. II, eq. (ODE)   M_c da_c/dt + K_S a_c = -K_cn K_n^+ j;
 *   Sec. II, eq. (acm)   explicit Euler update of a_c (source sign as in (ODE));
 *   Sec. II, eq. (CFL)   dt <= 2 / lambda_max(M_c^-1 K_S), power method;
 *   Sec. III, eq. (mrhs) K_n a_p = j_p solved by PCG every step;
 *   Sec. III, eq. (SPE_x0) subspace projection extrapolation start vector;
 *   Sec. III, eqs. (SVD),(relSV2),(keepInfo),(POD_x0) POD start vector.
 *
 * Discretisation: Cartesian finite-integration grid of n^3 cells of spacing
 * h, lowest-order edge unknowns, homogeneous Dirichlet on the outer surface.
 *
 * DEVICE / EDGE LAYOUT.  Every full edge vector ("layout vector") holds
 * 3 n^3 doubles: component c in {x, y, z} occupies [c n^3, (c+1) n^3), and
 * the edge of component c whose lower node is (i, j, k) sits at
 *     c n^3 + i + n (j + n k),   0 <= i, j, k < n.
 * Edges with a node index n (all of them Dirichlet) are not stored; stored
 * Dirichlet edges (index 0 in a direction normal to the edge) hold zero.
 * "n-edges" are interior edges none of whose four cells conducts; "c-edges"
 * are the other interior edges.  Compact conducting vectors (a_c) list the
 * c-edges in increasing layout index, i.e. ordered by (component, k, j, i).
 *
 * Cell arrays are n^3 entries, flat index i + n (j + n k).
 *
 * CONVENTIONS.  Every call returns an int status: MQS_OK (0) or a negative
 * MQS_ERR_* code; mqs_last_error() gives a text for the last failure on a
 * handle.  A handle owns all its device memory (allocated in mqs_setup,
 * released by mqs_destroy).  Pointers without a _dev suffix are host
 * pointers; _dev calls take device pointers and a cudaStream_t passed as
 * void* (NULL = the handle's stream) and do not synchronise the host.  No
 * caller pointer is retained after a call returns.  All arithmetic is
 * IEEE FP64.  A handle is not thread-safe; distinct handles are independent.
 */
#ifndef MQS_H
#define MQS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MQS_OK                  0
#define MQS_ERR_ARG            -1   /* invalid argument or size            */
#define MQS_ERR_CUDA           -2   /* CUDA runtime error                  */
#define MQS_ERR_OOM            -3   /* device allocation failed            */
#define MQS_ERR_NOT_CONVERGED  -4   /* PCG reached maxit                   */
#define MQS_ERR_BREAKDOWN      -5   /* PCG p.Kp <= 0                       */
#define MQS_ERR_NAN            -6   /* non-finite value met                */
#define MQS_ERR_UNSTABLE       -7   /* explicit Euler state blew up        */
#define MQS_ERR_TIMEOUT        -8   /* a bounded device wait gave up       */
#define MQS_ERR_UNIMPLEMENTED  -9
#define MQS_ERR_HALTED        -10   /* step not run: an earlier step of the
                                       same call failed                    */

#define MQS_START_ZERO 0            /* x0 = 0                              */
#define MQS_START_PREV 1            /* x0 = solution of the previous step  */
#define MQS_START_SPE  2            /* eq. (SPE_x0), last spe_depth sols   */
#define MQS_START_POD  3            /* eq. (POD_x0), last pod_snapshots    */
#define MQS_START_CSPE 4            /* eq. (SPE_x0) on the cascaded basis:
                                       frozen past solutions + the newest  */

typedef struct mqs_handle mqs_handle;

/* Grid: nx x ny x nz cells of spacing h metres.  This build runs cubic grids,
 * nx = ny = nz = n with 2 <= n <= 800 (every kernel indexes one n for all three
 * axes); other shapes return MQS_ERR_UNIMPLEMENTED from mqs_setup. */
typedef struct { int nx, ny, nz; double h; } mqs_grid;

/* Materials.  sigma_cell: n^3 conductivities (S/m, >= 0).  brauer_cell:
 * n^3 flags (1 = reluctivity nu(B) = k1 exp(k2 B^2) + k3, else nu0), or
 * NULL; a flagged cell must conduct.  nu0 = reluctivity of every other cell. */
typedef struct {
    const double*  sigma_cell;
    const uint8_t* brauer_cell;
    double nu0, k1, k2, k3;
} mqs_materials;

/* Coil: one loop of edges in node plane plane_k around the node square
 * [i0, i1] x [j0, j1], counter-clockwise seen from +z (the distribution X_S
 * of Sec. II, J_S = X_S i_S(t)); current i(t) = amplitude sin(2 pi freq t)
 * (waveform 0) or amplitude (1 - exp(-t / tau)) (waveform 1, Sec. IV).
 * The loop must lie on interior n-edges. */
typedef struct {
    int plane_k, i0, j0, i1, j1;
    double amplitude, freq_hz;
    int waveform;
    double tau;
} mqs_coil;

/* Options.  tol: PCG stopping rule ||b - K_n x||_2 <= tol ||b||_2 (true
 * residual).  maxit: PCG iteration cap.  start_mode: MQS_START_*.
 * spe_depth (1..16; CSPE 1..19), pod_snapshots (1..40), eps_pod (POD truncation
 * sigma_i/sigma_1 >= eps_pod, eq. (relSV2)), eps_lin (SPE drop tolerance).
 * dt: explicit Euler step (s); may be set later with mqs_set_dt.  With dt <= 0
 * and cfl_factor > 0, mqs_setup sets it from eq. (CFL) (see cfl_factor).
 * rhs_time: 0 = source at t_m (as printed in eq. (acm)), 1 = at t_{m-1}.
 * pcg_variant: see the field. */
typedef struct {
    double tol;
    int    maxit;
    int    start_mode;
    int    spe_depth;
    int    pod_snapshots;
    double eps_pod;
    double eps_lin;
    double dt;
    int    rhs_time;
    int    pcg_variant;   /* 0: two grid reductions per iteration (Hestenes-Stiefel
                             recurrences, default); 1: one reduction (Chronopoulos-
                             Gear recurrences, one fused stencil pass per
                             iteration). Same iterates in exact arithmetic.
                             With precision 1 it selects the form of the FP32
                             inner CG the same way.  2: with precision 1, the
                             one-reduction inner CG whose pass carries x, r and p
                             only (s = L p and w = L r formed in the pass: 24 bytes
                             per unknown and iteration instead of 40); with
                             precision 0 the same as 1. */
    int    precision;     /* 0: FP64 PCG (default); 1: FP64 iterative refinement
                             around FP32 CG inner solves (stencil, vectors and
                             products in FP32; residual, norms, convergence test
                             and solution update in FP64; same tol); 2: the same
                             refinement around float-float inner solves (value
                             = FP32 hi + FP32 lo, about 48 bits, FP32 pipes;
                             one-reduction form), which converge like FP64 CG. */
    double inner_tol;     /* precision 1/2: smallest residual reduction an inner
                             solve aims at (<= 0: 1e-5 / 1e-12) */
    int    cspe_period;   /* MQS_START_CSPE (Sec. III "cascaded SPE", Sec. IV):
                             the basis holds frozen past solutions and one live
                             column, the newest solution, replaced every step;
                             every cspe_period steps (<= 0: 25) the live column
                             is frozen and the basis grows, up to spe_depth
                             columns (1..19, "below 20").  Frozen columns are
                             kept K-orthonormal (two-pass Gram-Schmidt in the K
                             inner product with the stored K-images, no stencil),
                             the newest solution is projected against them every
                             step.  mqs_push_history makes the pushed solution the
                             newest column; columns are frozen only by steps. */
    int    rhs_split;     /* 1: solve the separate right-hand sides listed after
                             eq. (mrhs) - the conductor type -K_cn^T a_c^{m-1} and
                             the coil type j^m_{s,n} - one PCG solve each, each
                             started from the SPE projection on past solutions of
                             its own type (two difference tables), w = sum; needs
                             start_mode ZERO or SPE; the adjoint refuses it.
                             mqs_push_history / spe_start act on the conductor
                             type's table.  0 (default): one fused solve (exact
                             by linearity). */
    int    graph;         /* 1: once the SPE table is full, steps are replayed
                             from CUDA graphs (one per parity of the conductor
                             buffers, captured on first use and again whenever
                             the stream, block count, options, dt or a buffer
                             the step uses changes): the same launches with the
                             same arguments, so the results are bitwise those
                             of 0.  Only SPE starts without rhs_split, timing or
                             adjoint recording, and a stream that can be
                             captured (not the legacy default stream); other
                             steps are issued launch by launch.  0 (the C
                             default of a zeroed struct; the Python binding's
                             SolverOptions defaults to 1): every step launch
                             by launch. */
    double cfl_factor;    /* eq. (CFL): with dt <= 0 and cfl_factor > 0, mqs_setup
                             runs the power method of mqs_lambda_max (PCG tol 1e-12,
                             stop at |dlambda| < 1e-8 lambda or 2000 iterations; its
                             start vector is the library's own: uniform numbers in
                             [-1, 1) from the SplitMix64 generator, seed 1611) and
                             sets dt = cfl_factor * 2 / lambda_max (0.9 in the
                             paper's setting); mqs_get_dt returns lambda_max.  0
                             (a zeroed struct): dt stays unset until mqs_set_dt. */
    int    monitor_steps; /* instability monitor of the explicit Euler update
                             (eq. (CFL) violated): a step fails with
                             MQS_ERR_UNSTABLE once the M_c-energy of the state
                             increment a^m - a^{m-1} has grown, with the sign of
                             the increment alternating (M_c-inner product of
                             successive increments < 0), over monitor_steps
                             consecutive steps (above 1e-20 of the largest
                             increment energy seen), or when the state is not
                             finite.  That is the signature of the explicit Euler
                             factor 1 - dt lambda < -1 of the top mode; stable
                             steps (|1 - dt lambda| <= 1 for every mode) shrink the
                             alternating part instead.  0: 8 steps; < 0: off (the
                             non-finite test stays). */
    int    tile_groups;   /* stencil groups per block of the one-reduction FP64
                             pass (precision 0, pcg_variant 1): each group marches
                             one 32 x 4 tile of positions at a time.  0 or 2
                             (default): 320-thread blocks; 3: 480-thread blocks
                             (more warps to hide latency, fewer registers per
                             thread).  mqs_tune_pcg chooses it with the form.
                             Other precisions and forms use 2. */
    int    halo_warps;    /* warps per tile group of that pass, and of the FP32
                             inner pass of precision 1 with pcg_variant 1 below
                             96^3, that form the tile's halo (the sources and
                             fluxes of the positions next to the tile, which the
                             neighbouring tiles own).  0 or 1 (default): one; 2
                             (with two tile groups only): two, each over half of
                             the halo, in 384-thread blocks (three warps on each
                             of the SM's four schedulers).  The iterates are
                             bitwise the same.  Other forms ignore it.
                             mqs_tune_pcg chooses it with the form. */
} mqs_options;

typedef struct {
    int    n;             /* cells per axis                                 */
    long   n_layout;      /* 3 n^3: length of a layout vector               */
    long   n_c;           /* number of c-edges (length of a_c)              */
    long   n_n;           /* number of n-edges (unknowns of K_n)            */
    int    box_lo[3];     /* node range of the conducting region [lo, hi)   */
    int    box_hi[3];
} mqs_layout_info;

typedef struct {
    int    iterations;    /* products K_n p inside the PCG loop             */
    int    status;        /* MQS_OK or MQS_ERR_*                            */
    int    rank;          /* SPE columns kept / POD k (0 otherwise)         */
    int    refinements;   /* FP64 refinement steps (precision 1; else 0)    */
    double relres;        /* final true ||b - K_n w|| / ||b||               */
    double start_relres;  /* ||b - K_n x0|| / ||b||                          */
    double pod_info;      /* eq. (keepInfo) ratio, POD mode (else 0)        */
} mqs_step_stats;

typedef struct {
    int    iterations;
    int    status;
    double relres;
    double start_relres;
} mqs_pcg_info;

/* mqs_setup: Sec. II eq. (DAE).  conductor_mask: n^3 flags selecting the
 * conducting region Omega_c (flagged cells must have sigma > 0, the others
 * are treated as nonconducting whatever their sigma), or NULL to take
 * sigma > 0.  Classifies edges, builds the per-edge
 * conductivity M_c (h * mean sigma of the four cells of an edge), the coil
 * distribution and all device buffers.  K_n = C_n^T M_nu C_n is applied
 * matrix-free: every face touching an n-edge has reluctivity nu0, so K_n is
 * (nu0/h) times an integer stencil and its Jacobi diagonal is the uniform
 * 4 nu0/h.  State after setup: a_c = 0, t = 0, m = 0, empty history.
 * Errors: MQS_ERR_ARG (sizes, coil not on n-edges, nonconducting Brauer
 * cell, no conducting cell), MQS_ERR_OOM, MQS_ERR_CUDA.  On failure *out is
 * NULL and nothing is leaked. */
int mqs_setup(const mqs_grid* grid, const mqs_materials* mat,
              const uint8_t* conductor_mask, const mqs_coil* coil,
              const mqs_options* opts, mqs_handle** out);

int mqs_destroy(mqs_handle* h);

/* Copies a NUL-terminated text of the last error (possibly empty). */
int mqs_last_error(const mqs_handle* h, char* buf, size_t len);

int mqs_layout(const mqs_handle* h, mqs_layout_info* info);

/* mqs_set_dt / mqs_get_dt: the explicit Euler step (eq. (acm)).  mqs_get_dt
 * also returns (lambda_max, nullable) the largest eigenvalue of M_c^-1 K_S(0)
 * of eq. (CFL) found on this handle (by mqs_setup with cfl_factor, or the last
 * mqs_lambda_max), 0 if none was computed.  dt (nullable) is 0 while unset. */
int mqs_set_dt(mqs_handle* h, double dt);
int mqs_get_dt(const mqs_handle* h, double* dt, double* lambda_max);

/* mqs_set_options: replaces every option (dt is kept unless > 0).
 * Changing start_mode, spe_depth, pod_snapshots, cspe_period or rhs_split
 * clears the history.
 * mqs_get_options: the handle's current options (after a tuner's choice);
 * opts->dt receives the current step.  Errors: MQS_ERR_ARG (NULL). */
int mqs_set_options(mqs_handle* h, const mqs_options* opts);
int mqs_get_options(const mqs_handle* h, mqs_options* opts);

/* mqs_lambda_max: eq. (CFL) - power method on M_c^-1/2 K_S(0) M_c^-1/2,
 * Rayleigh quotient, every application of K_S using one PCG solve of K_n
 * (tolerance pcg_tol).  v0: host vector of n_c entries (the start vector;
 * random numbers are the caller's).  Stops when |dlambda| < rtol lambda or
 * after maxit iterations.  Returns lambda_max (1/s) and the iterations. */
int mqs_lambda_max(mqs_handle* h, const double* v0, double pcg_tol,
                   double rtol, int maxit, double* lambda_max, int* iters);

/* mqs_step: nsteps explicit Euler steps (eq. (acm) with the source sign of
 * eq. (ODE)); each step m:
 *   b   = i(t) X_s - K_cn^T a_c^{m-1}        on n-edges   (eq. (mrhs))
 *   x0  = start vector (zero / previous / SPE / POD)
 *   w   = PCG(K_n, b, x0)                    (= a_n, eq. (a_n))
 *   a_c = a_c - dt M_c^-1 (K(a)[a_c; w])_c   (Brauer nu re-evaluated per cell)
 * then w and K_n w join the start-vector history.  per_step: host array of
 * nsteps records or NULL.  The loop stops at the first failing step (a PCG
 * status other than MQS_OK, a timed-out device wait, or MQS_ERR_UNSTABLE from
 * the instability monitor, see mqs_options.monitor_steps): on the device, every
 * later step of the call skips its solve and its conductor update, and its
 * record carries MQS_ERR_HALTED.  The handle is then left at the last step that
 * succeeded: a_c, t and m as after that step (the failing step's update is
 * discarded), with an empty start-vector history.  Returns the failing step's
 * status (MQS_OK if none), MQS_ERR_ARG if dt is unset. */
int mqs_step(mqs_handle* h, int nsteps, mqs_step_stats* per_step);

/* mqs_step in two halves.  mqs_step_enqueue issues the launches of nsteps
 * steps on the handle's stream (the side stream of the SPE table push joined
 * back at the end) and returns without waiting for the device, so the host can
 * work (or record events in stream order) while the steps run; it may be called
 * again before the finish (the steps queue up behind each other).
 * mqs_step_finish(h, nsteps, per_step) then copies the statistics of all
 * enqueued steps, waits for the stream and returns what mqs_step would have;
 * nsteps must equal the total enqueued count.  A finish without an enqueue, or
 * mqs_step while steps are enqueued, returns MQS_ERR_ARG; no other call may use
 * the handle in between. */
int mqs_step_enqueue(mqs_handle* h, int nsteps);
int mqs_step_finish(mqs_handle* h, int nsteps, mqs_step_stats* per_step);

/* State access.  a_c: n_c doubles in compact c-edge order. */
int mqs_get_state(mqs_handle* h, double* a_c, size_t n_c, double* t, long* m);
int mqs_set_state(mqs_handle* h, const double* a_c, size_t n_c, double t, long m);
int mqs_get_state_dev(mqs_handle* h, double* a_c_dev, size_t n_c, void* stream);
int mqs_set_state_dev(mqs_handle* h, const double* a_c_dev, size_t n_c, void* stream);
/* Copies the latest PCG solution w (layout vector, zero off n-edges). */
int mqs_get_solution(mqs_handle* h, double* w_layout);
/* mqs_solve_an: a_n^m of eq. (anm) for the current state: one PCG solve of
 * K_n a_n = j^m_{s,n} - K_cn^T a_c^m (source at the time level the last step
 * used, new conductor state), started from the step's solution w and run to
 * the handle's tol.  (The step itself needs only w = K_n^+ (j^m - K_cn^T
 * a_c^{m-1}); a_n^m is an output on request.)  a_n (host, layout vector,
 * nullable) receives the solution; info (nullable) the PCG result.  The time
 * loop's state, history and w are left as they were.  Errors: MQS_ERR_ARG,
 * MQS_ERR_CUDA and the PCG statuses. */
int mqs_solve_an(mqs_handle* h, double* a_n_layout, mqs_pcg_info* info);
int mqs_reset_history(mqs_handle* h);

/* pcg_solve: Sec. III eq. (mrhs) - Jacobi-preconditioned CG for K_n x = b
 * with the handle's K_n.  b, x: layout vectors (host); entries of b off
 * n-edges are ignored, x is read as the start vector and overwritten with
 * the solution (zero off n-edges).  Stops on the true relative residual.
 * info may be NULL.  Returns MQS_OK, MQS_ERR_NOT_CONVERGED,
 * MQS_ERR_BREAKDOWN, MQS_ERR_NAN or MQS_ERR_TIMEOUT. */
int pcg_solve(mqs_handle* h, const double* b, double* x, double tol,
              int maxit, mqs_pcg_info* info);
int pcg_solve_dev(mqs_handle* h, const double* b_dev, double* x_dev,
                  double tol, int maxit, mqs_pcg_info* info, void* stream);

/* mqs_apply_kn: y = K_n x for layout vectors (host); entries off n-edges of
 * x are ignored and those of y are set to zero. */
int mqs_apply_kn(mqs_handle* h, const double* x, double* y);
int mqs_apply_kn_dev(mqs_handle* h, const double* x_dev, double* y_dev, void* stream);

/* mqs_conductor_rate: F = (K(a)[a_c; w])_c with the Brauer reluctivity
 * evaluated at a (the bracket of eq. (acm) after the single solve).  a_c:
 * n_c doubles, w: layout vector, F: n_c doubles (host). */
int mqs_conductor_rate(mqs_handle* h, const double* a_c, const double* w, double* F);

/* mqs_set_stream: later work of the handle goes to `stream` (a
 * cudaStream_t passed as void*; NULL = the handle's own stream).  Work already
 * queued on the previous stream is waited for first. */
int mqs_set_stream(mqs_handle* h, void* stream);

/* Per-phase device time of mqs_step, measured with CUDA events recorded on
 * the handle's stream around each phase of every step while timing is on:
 * right-hand side (a2), start vector (a3), PCG (a4), history (a6; issued
 * before the conductor update: with SPE only the fork of the table push to the
 * side stream, whose time then shows where the main stream waits for it),
 * conductor update (a5, with the step's statistics record).  `launches` counts
 * every kernel the library launched inside those steps and `pcg_launches` the
 * PCG kernels among them. */
typedef struct {
    double ms_rhs, ms_start, ms_pcg, ms_conductor, ms_history;
    long   launches;
    long   pcg_launches;
    long   steps;
} mqs_timing;

/* on != 0 starts (and resets) the accumulation, 0 stops it. */
int mqs_timing_enable(mqs_handle* h, int on);
/* Waits for the stream and returns the accumulated times and counts. */
int mqs_timing_get(mqs_handle* h, mqs_timing* out);

/* mqs_graph_steps: steps of the handle replayed from (or captured into) a CUDA
 * graph since setup (options.graph); mqs_batch_graph_steps: the same count of
 * batch steps (each advances every handle of the batch).  *steps (host). */
int mqs_graph_steps(const mqs_handle* h, long* steps);

/* mqs_part_ranges: the plane-tile ranges that the one-reduction PCG pass (the
 * solve of Sec. III, eq. (mrhs), pcg_variant 1) gives to its tile groups on an n^3 grid with nblk blocks of `groups` tile groups
 * each (groups 0 counts as 2).  Host only: no CUDA call, no handle.  A plane-tile is 32 x 4
 * positions of one z-plane; tiles are numbered column by column (tile column
 * t = x-tile + (n+31)/32 y-tile, plane k: index t n + k), so a group marches z.
 * Part p = block b x groups + group g gets [ranges[2p], ranges[2p+1]).  The
 * parts cover every tile once, in order; parts past the last tile are empty.
 * A part costs its tiles plus one warm-up plane per segment (a segment starts
 * at the part's first tile, at every column's first plane and after 32 planes
 * of a column); the ranges minimise the largest part cost (binary search on the
 * cost with a greedy fill).  ranges: 2 nblk groups ints (host).  Errors:
 * MQS_ERR_ARG (n, nblk or groups < 1, ranges NULL, or more than 2^31 tiles or
 * parts). */
int mqs_part_ranges(int n, int nblk, int groups, int* ranges);

/* mqs_selftest_barrier_timeout: launches the persistent kernels' grid
 * barrier with an arrival count that can never be reached and a wait limit
 * of `polls` polls (about 100 ns each), so every block gives up, records
 * MQS_ERR_TIMEOUT and returns (a poll is one L2 round trip, under a
 * microsecond).  Used to test that a stuck device wait ends with an error
 * status while the context stays usable.  Returns the status
 * the kernel recorded (MQS_ERR_TIMEOUT expected), MQS_ERR_CUDA on a launch
 * failure.  Allocates a few bytes of device memory for the flag. */
int mqs_selftest_barrier_timeout(long long polls);

/* History for the start vectors (Sec. III).  mqs_push_history appends a
 * solution w (layout vector, host) as the newest entry; K_n w is computed
 * by the library (during mqs_step it is a by-product of the PCG residual). */
int mqs_push_history(mqs_handle* h, const double* w);

/* spe_start: eq. (SPE_x0) for right-hand side b (layout, host) over the
 * span of the newest spe_depth history entries.  x0: layout output.
 * rank_used: columns kept after the linear-dependence drop (may be NULL). */
int spe_start(mqs_handle* h, const double* b, double* x0, int* rank_used);

/* pod_basis: eqs. (SVD), (relSV2), (keepInfo) for the newest pod_snapshots
 * history entries: *k kept singular values, sigma (pod_snapshots doubles,
 * descending, zero-filled), *info_ratio.  Any output may be NULL. */
int pod_basis(mqs_handle* h, int* k, double* sigma, double* info_ratio);

/* pod_start: eq. (POD_x0) for right-hand side b (layout, host). */
int pod_start(mqs_handle* h, const double* b, double* x0, int* k);

/* mqs_pcg_solve_noalloc: the same Jacobi-PCG solve as pcg_solve_dev, as a
 * stateless call that allocates no device memory.  (The paper has no
 * counterpart; this exists for callers that cannot call cudaMalloc, e.g. a
 * host application whose device memory belongs to its own pool allocator, or
 * a real-time loop where an allocation, which may synchronise the device, is
 * not allowed.)
 * Inputs and outputs are the caller's device pointers: cell_mask_dev (n^3
 * bytes, nonzero = conducting cell), b_dev (layout vector, K_n units),
 * x_dev (layout vector: start vector in, solution out; entries off n-edges
 * are set to zero; 16-byte aligned, as cudaMalloc returns).  n, h, nu0: grid cells per axis, spacing, reluctivity.
 * Scratch: one file-scope device array sized for n <= MQS_NOALLOC_MAX_N
 * (about 13.4 MB), held by every GPU that loads the library until the
 * process exits.  Larger n returns MQS_ERR_ARG (message on stderr).  Set-up:
 * the first call in a CUDA context (per device, and again after a device
 * reset, which makes a new context) looks the array's address up
 * (cudaGetSymbolAddress) with that device current, under a lock, and keeps it
 * for later calls in that context.  All calls share the array: calls that overlap on the GPU (other
 * streams, other host threads) race; serialise them.  Every call starts its
 * own scratch state afresh (the barrier counter and error word are cleared).
 * Blocks the host until the solve finishes; info (host) may be NULL.
 * Returns MQS_OK or the PCG status (MQS_ERR_NOT_CONVERGED, _BREAKDOWN,
 * _NAN, _TIMEOUT), MQS_ERR_ARG or MQS_ERR_CUDA. */
#define MQS_NOALLOC_MAX_N 48
int mqs_pcg_solve_noalloc(int n, double h, double nu0, const uint8_t* cell_mask_dev,
                          const double* b_dev, double* x_dev, double tol, int maxit,
                          mqs_pcg_info* info, void* stream);

/* ---- Discrete adjoint of the time loop ----------------------------------
 * The paper's motivation for fast time stepping includes optimisation
 * (Sec. I); this computes the gradient of the time-integrated eddy-current
 * loss over the explicit-Euler steps of eqs. (ODE)/(acm)
 *
 *   J = sum_m dt e_m^T M_c e_m,  e_m = (a_c^m - a_c^{m-1}) / dt,
 *
 * (the FIT edge form of sum over cells of sigma |E|^2 dV with E = -da/dt on
 * the conducting edges; J = sum_m dt F_m^T M_c^-1 F_m with F_m the bracket of
 * eq. (acm)) with respect to every cell conductivity and the coil amplitude,
 * by the reverse sweep of the discrete adjoint: per step one PCG solve with
 * K_n (same kernels and start vectors as the time loop) and the transposed
 * Jacobian of the Brauer face law on the conductor box.  dt, the edge classes
 * and the coil waveform are held fixed.
 *
 * mqs_adjoint: runs nsteps steps from the handle's current state (recording
 * a_c^{m-1} and F_m of every step on the device: 16 n_c bytes per step; no
 * recomputation), evaluates J, then the reverse sweep.  grad_sigma_cell
 * (host, n^3 in cell order i + n (j + n k), nullable) receives dJ/dsigma per
 * cell (J per S/m, 0 for nonconducting cells).  info (nullable) receives J
 * (in joules: W s of dissipated power, SI units of the grid), dJ/d
 * amplitude and the PCG iteration totals.  Afterwards the handle is at the
 * forward end state (time and step count advanced by nsteps) with an empty
 * start-vector history (the reverse sweep used it for the adjoint solves) and
 * mqs_get_solution holding the last adjoint solve.  Errors: MQS_ERR_ARG,
 * MQS_ERR_OOM, MQS_ERR_CUDA and the PCG statuses of either sweep. */
typedef struct {
    double objective;        /* J                                               */
    double grad_amplitude;   /* dJ / d(coil amplitude)                          */
    long   forward_iterations;   /* PCG iterations of the forward steps         */
    long   adjoint_iterations;   /* PCG iterations of the adjoint solves        */
    long   recompute_iterations; /* PCG iterations of recomputed forward steps  */
} mqs_adjoint_info;
int mqs_adjoint(mqs_handle* h, int nsteps, double* grad_sigma_cell, mqs_adjoint_info* info);

/* mqs_adjoint with checkpoints: the forward sweep keeps a_c at every
 * checkpoint_every-th step (8 n_c bytes each) and the record of one segment
 * (16 n_c bytes per step of it) instead of the whole trajectory; the reverse
 * sweep recomputes each segment's forward steps from its checkpoint, with a
 * start-vector history that starts empty at each segment, before the segment's
 * adjoint steps, whose history (with SPE a second table) runs on across
 * segments.  J is the forward sweep's.  checkpoint_every = 0 (or >= nsteps) is
 * mqs_adjoint.  The recomputed steps' PCG total goes to
 * info->recompute_iterations.  Same end state and errors as mqs_adjoint. */
int mqs_adjoint_ckpt(mqs_handle* h, int nsteps, int checkpoint_every, double* grad_sigma_cell,
                     mqs_adjoint_info* info);

/* mqs_loss: the forward part of mqs_adjoint alone: nsteps steps from the
 * current state and J over them (*objective, host, nullable); the handle
 * advances as with mqs_step.  Errors as mqs_step. */
int mqs_loss(mqs_handle* h, int nsteps, double* objective);

/* ---- Batched multi-query ------------------------------------------------
 * Sec. I motivates fast time stepping by many-query work (uncertainty
 * quantification, optimisation: many runs of one model with different
 * parameters).  A batch advances several handles -- each its own problem
 * (grid, materials, coil, options, dt) -- together on one GPU.  Each handle's
 * launches go to a stream of its own, and its persistent PCG kernels use a
 * block count proportional to its unknowns, so that the solves of small
 * problems run side by side on disjoint SMs instead of each taking the whole
 * GPU in turn.  Per handle, the result equals an mqs_step run up to the
 * summation order of the grid-wide reductions (which depends on the block
 * count).
 *
 * mqs_set_blocks: persistent blocks of the handle's PCG kernels, 1 .. the SM
 * count (0 = one block per SM, the default).  MQS_ERR_ARG above the SM count.
 *
 * mqs_batch_create: handles[0..count) stay owned by the caller, must be
 * distinct, must outlive the batch and must not be stepped outside it while
 * it exists.  blocks_scale (> 0; <= 0 selects 2.0) makes the block counts add
 * up to about blocks_scale blocks per SM (each at least 1, at most one per
 * SM): values above 1 oversubscribe, so that SMs released by solves that
 * converge early are taken by others.  The batch creates min(count, 32)
 * streams, shared by the handles round-robin (CUDA maps streams onto
 * CUDA_DEVICE_MAX_CONNECTIONS hardware queues, 8 unless the environment sets
 * up to 32 before the CUDA context is created; set it to 32 for batches), and
 * restores each handle's stream and block count on destroy.
 * Errors: MQS_ERR_ARG, MQS_ERR_OOM, MQS_ERR_CUDA; on failure *out is NULL.
 *
 * mqs_batch_step: nsteps explicit-Euler steps (as mqs_step) of every handle.
 * per_step (host, nullable) receives nsteps*count stats, step-major:
 * per_step[s*count + i] is step s of handles[i].  Blocks until all finish.
 * Returns MQS_OK or the first failing handle's status (its mqs_last_error
 * holds the text).
 *
 * mqs_batch_last_ms: device time of the last mqs_batch_step (CUDA events from
 * the fork of the streams to their join).
 *
 * mqs_batch_tune: tries blocks_scale 1, 2, 4 and 8 with the current block
 * shares, for trial_steps steps each -- real steps that advance every problem
 * -- once in that order and once in reverse.  A candidate's score is its
 * device time per unit of PCG work (unknowns x iterations) summed over its two
 * trials, so the falling iteration counts of a starting transient favour no
 * candidate.  It keeps the best (its scale in *best_scale, nullable).
 * mqs_batch_set_scale: sets blocks_scale (> 0) and reassigns the counts.
 * mqs_batch_tune_pcg: mqs_tune_pcg on the first handle of every group of
 * handles with the same grid size and precision (on its batch stream and its
 * block share), the winner set on the whole group; chosen (host, nullable)
 * receives every handle's pcg_variant in the batch's order.
 * mqs_batch_set_weighting: by_work 0 (shares by unknowns, the default) or 1
 * (by unknowns x the last call's iterations per step) and reassigns the
 * counts; mqs_batch_get_weighting reads it back.  MQS_ERR_ARG otherwise.
 *
 * mqs_batch_tune_depth: the SPE depth per grid size.  The handles with the SPE
 * start are grouped by n.  Group by group, in increasing n, the depths in
 * depths[0..ndepths) (each 1..16) are tried in the order d_0 .. d_last, then
 * d_last .. d_0.  Each trial sets the depth on the group's handles (through
 * mqs_set_options: a new history), refills the tables with dmax + 1 steps and
 * times trial_steps steps (mqs_batch_last_ms).  A depth's two trial times are
 * added, so a linear drift of a transient's iteration counts cancels.  The group
 * keeps its fastest depth while the next group is searched.  These are real
 * steps: every problem advances.  chosen (host, nullable) receives the final spe_depth of every
 * handle, in the batch's order.  Other handles keep their options.  Errors:
 * MQS_ERR_ARG, or the status of a failing step. */
int mqs_set_blocks(mqs_handle* h, int nblk);
/* mqs_tune_pcg: the PCG kernel form for this handle's grid, precision and block
 * count.  The candidates compute the same iterates and differ in their tiles'
 * halo depth, staging and traffic: precision 0, pcg_variant 0 (two reductions
 * per iteration) and 1 (one fused pass carrying x, p, r, w, s) on 2 tile groups
 * per block with one or two halo warps each and on 3 (tile_groups,
 * halo_warps); precision 1,
 * pcg_variant 0, 1 (one reduction, five carried vectors; one or two halo warps)
 * and 2 (three carried vectors, a two-deep halo staged by cp.async); precision 2
 * has one form.
 * Each candidate solves K_n x = b from x = 0, b the coil's pattern at unit
 * current with the conductors at rest, trials + 1 times on the handle's stream
 * and block count; the first solve is untimed and the fastest median (CUDA
 * events) sets opts.pcg_variant (and tile_groups, halo_warps).  The state, the start-vector history and the
 * step's right-hand side are untouched.  chosen (host, nullable) receives the
 * variant.  Blocks the host.  Errors: MQS_ERR_ARG (trials < 1), a failing trial
 * solve's status (the previous variant is kept), MQS_ERR_CUDA. */
int mqs_tune_pcg(mqs_handle* h, int trials, int* chosen);
typedef struct mqs_batch mqs_batch;
int mqs_batch_create(mqs_handle* const* handles, int count, double blocks_scale,
                     mqs_batch** out);
int mqs_batch_set_scale(mqs_batch* b, double blocks_scale);
int mqs_batch_step(mqs_batch* b, int nsteps, mqs_step_stats* per_step);
int mqs_batch_last_ms(mqs_batch* b, double* ms);
int mqs_batch_tune(mqs_batch* b, int trial_steps, double* best_scale);
int mqs_batch_set_weighting(mqs_batch* b, int by_work);
int mqs_batch_tune_pcg(mqs_batch* b, int trials, int* chosen);
int mqs_batch_get_weighting(const mqs_batch* b, int* by_work);
int mqs_batch_tune_depth(mqs_batch* b, int trial_steps, const int* depths, int ndepths,
                         int* chosen);
int mqs_batch_destroy(mqs_batch* b);
int mqs_batch_graph_steps(const mqs_batch* b, long* steps);

/* ---- debug build checks --------------------------------------------------
 * The library is also built as a debug variant (compiled with
 * MQS_DEBUG_CHECKS) in which every index a hot kernel computes -- the
 * stencil sweeps and fused passes, the FP32 inner pass, the conductor,
 * right-hand-side, SPE and adjoint kernels, the step records -- is tested
 * against the length of the array it addresses.  An access out of range is
 * skipped (a load reads 0) and the first one per translation unit is kept
 * with its site number and index: nothing traps.  Every device buffer a
 * handle allocates is followed by 256 guard bytes of a fixed pattern.
 *
 * mqs_debug_check(h, report): synchronizes the device, reads and clears the
 * recorded index faults of all translation units, and (h non-NULL) compares
 * the guard bytes of every buffer of h with the pattern.
 *   report (host, non-NULL): receives enabled = 1 in the debug variant and 0
 *     in the release library (where everything else reads 0);
 *   site / index: the first fault found (site 0: none); faults: how many
 *     translation units recorded one; canaries_bad: buffers of h whose guard
 *     bytes changed (buffers: how many were checked).
 * Returns MQS_OK, MQS_ERR_ARG (report NULL) or MQS_ERR_CUDA. */
typedef struct {
  int enabled;
  int site;
  long long index;
  int faults;
  int canaries_bad;
  int buffers;
} mqs_debug_report;
int mqs_debug_check(mqs_handle* h, mqs_debug_report* report);

#ifdef __cplusplus
}
#endif
#endif /* MQS_H */
