/*
 * lbm_stefan.h -- C ABI of the GB300 IREBM library.
 *
 * The library advances the implicit regularized enthalpy based lattice
 * Boltzmann method (IREBM) of Luddens, Lothode and Danaila, "An implicit
 * regularized enthalpy Lattice Boltzmann Method for the Stefan problem"
 * (arXiv 2505.13097), on one GPU.  One call of lbm_stefan_step() runs
 * Algorithm 3 of the paper once per step: collision (Eq. 12), pull
 * streaming, the boundary closures of Sec. 4.2 on q, the zeroth moment, the
 * local Newton solve of Eq. (14), the source of Eq. (13), and the next
 * collision.  Kernel launches per step: D2Q9 with FP32 populations, four on
 * the legacy default stream (the nodes on or next to a wall in two, rows 1 .. ny-2
 * of every 128-column strip, then the kernel that solves the list of nodes
 * that need the Newton iteration and publishes the step), six on a stream of
 * the handle's own (rows 1 .. ny-2 of the left and of the right half of the
 * strips; on a second, higher-priority stream the S / N wall rows and the
 * W / E wall groups, then Newton solves of those and of the left half beside
 * the right half; then a launch that solves the rest and publishes the step);
 * D2Q9 in FP64 and D2Q5, two (the stream/collide kernel, which hands the
 * nodes that need the Newton iteration to a list, then the kernel that
 * solves that list); D1Q3, one launch for all the steps of a call.
 *
 * Problem statement (Sec. 2, Eq. 1): dimensionless temperature theta with
 * melting temperature 0, Stefan number Ste, equal phase properties; the
 * liquid fraction is regularized as phi(theta) = (1 + tanh(theta/delta))/2
 * (Sec. 4.1).  The lattice spacing is one node; tau - 1/2 = 3 dt/dx^2
 * (end of Sec. 5) maps steps to physical time.
 *
 * Conventions for every entry point:
 *  - Fields are row-major (ny rows of nx values, x fastest); D1Q3 uses ny = 1.
 *  - Host pointers are read or written synchronously.  With on_device = 1 the
 *    pointer is a device address (for instance a torch CUDA tensor), accessed
 *    in order on the handle's stream.
 *  - The library owns all its device buffers; the caller owns what it passes.
 *  - Functions return lbm_status; nothing aborts.  lbm_stefan_last_error()
 *    returns a message for the last failure on the calling thread.
 *  - Kernels run asynchronously on the stream given at creation.  Errors the
 *    device detects (Newton not converged, non-finite values) are sticky and
 *    returned by the next call that synchronizes (lbm_stefan_sync,
 *    lbm_stefan_get_fields, lbm_stefan_get_stats, ...).
 */
#ifndef LBM_STEFAN_H
#define LBM_STEFAN_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_stefan lbm_stefan;             /* one problem, opaque */
typedef struct lbm_stefan_batch lbm_stefan_batch; /* many problems, opaque */

typedef enum {
    LBM_OK = 0,
    LBM_ERR_ARG = 1,     /* invalid argument (sizes, tau <= 1/2, Ste <= 0, delta <= 0, NULL, ...) */
    LBM_ERR_CUDA = 2,    /* a CUDA runtime call failed */
    LBM_ERR_NEWTON = 3,  /* a node's Newton solve hit its iteration limit, or a value was not finite */
    LBM_ERR_TIMEOUT = 4, /* a bounded device wait ran out (the TMA row-pipeline kernel's waits for its row
                            loads: FP32 D2Q9 batches, and single problems under lbm_stefan_set_wait_test) */
    LBM_ERR_STATE = 5    /* call out of order (e.g. step before set_ic) */
} lbm_status;

enum { LBM_D1Q3 = 1, LBM_D2Q9 = 2, LBM_D2Q5 = 3 };             /* lattice (Sec. 3.2) */
enum { LBM_FP64 = 0, LBM_FP32 = 1 };                           /* population storage */
enum { LBM_WALL_W = 0, LBM_WALL_E = 1, LBM_WALL_S = 2, LBM_WALL_N = 3 };
enum { LBM_ADIABATIC = 0, LBM_DIRICHLET = 1 };                 /* wall kinds (Sec. 4.2) */
enum { LBM_BB_MIRROR = 0, LBM_BB_LINK = 1, LBM_NEU_EQ17 = 2 }; /* adiabatic-wall closures */
enum { LBM_IREBM = 0, LBM_EEBM = 1, LBM_ILFBM = 2 };           /* step method (Algorithms 3, 2, 1) */

typedef struct {
    int lattice;          /* LBM_D1Q3, LBM_D2Q9 or LBM_D2Q5 */
    int nx, ny;           /* nodes per side, >= 2 (ny = 1 for D1Q3; nx, ny >= 3 for D2Q5) */
    double tau;           /* BGK relaxation time, > 1/2 (Eq. 8) */
    double delta;         /* regularization width of phi, > 0 (Sec. 4.1) */
    double ste;           /* Stefan number, > 0 (Eq. 1) */
    int precision;        /* LBM_FP64: everything FP64; LBM_FP32: populations stored and
                             relaxed in FP32, moments as float-float sums, Newton in FP64 */
    double newton_tol;    /* step tolerance of the Newton solve (Algorithm 3), e.g. 1e-14 */
    int newton_max_iter;  /* iteration limit, e.g. 60; reaching it sets LBM_ERR_NEWTON */
    int bb_mode;          /* closure of the adiabatic walls: LBM_BB_MIRROR: q_i = q_{bar i}
                             (Sec. 4.2.2); LBM_BB_LINK: q_i = Omega_{bar i} at the node;
                             LBM_NEU_EQ17 (D2Q5 only): Eq. (17), M0(q) of a wall node equals
                             M0(q) of the node one step inwards (at a corner of two adiabatic
                             walls the diagonal interior node, the two unknowns sharing the
                             rest equally) */
} lbm_stefan_params;

typedef struct {
    double energy;         /* E = sum_x theta + phi(theta)/Ste after the last step (FP64) */
    double energy_prev;    /* E before the last step */
    double flux;           /* boundary flux of the last step: filled q minus Omega leaving */
    double imbalance;      /* E - energy_prev - flux of the last step (energy balance) */
    double imbalance_max;  /* largest |imbalance| since set_ic */
    long long steps;       /* steps since set_ic */
    long long newton_nodes;/* nodes that ran the Newton iteration in the last step */
    int newton_max_iter;   /* largest iteration count in the last step */
    int error;             /* sticky device error (lbm_status value, 0 if none) */
    long long newton_iters;/* sum of the Newton iteration counts of the last step (its mean is
                              newton_iters / newton_nodes) */
} lbm_stefan_stats;

/* ---------------------------------------------------------------- one problem
 * State buffers (lbm_stefan_layout): q planes of populations (ny + 2 rows of
 * row_stride elements each, the first and last rows zero halo rows); D1Q3
 * adds a fourth plane, the liquid fraction of LBM_ILFBM (D2Q9 / D2Q5 with
 * ILFBM: a plane after the q); then a 256-byte tail.  The populations are the
 * post-collision Omega_i of the stored-Omega form.  FP32 D2Q9 / D2Q5 states
 * store Omega_i - w_i s, s being a float in the first 4 bytes of the tail
 * (M0 = s + the sum of the stored values): set_ic sets s to the mean of the
 * initial M0 (theta0; EEBM: its enthalpy), so that stored values near s are
 * small and round finely.  The tail is zero in the other forms. */

/* Create a problem.  cuda_stream is a cudaStream_t (NULL = legacy default
 * stream).  All walls start adiabatic; the state is undefined until set_ic. */
lbm_status lbm_stefan_create(const lbm_stefan_params* p, void* cuda_stream, lbm_stefan** out);

/* Boundary condition of one wall (Sec. 4.2): kind LBM_DIRICHLET holds theta at
 * theta_wall through the closure of Eq. (15) on q; LBM_ADIABATIC applies
 * bounce-back.  A node on a Dirichlet wall is a Dirichlet node (corners
 * included); its value is that of the first Dirichlet wall in W, E, S, N.
 * Call before set_ic so that Dirichlet nodes start at theta_wall. */
lbm_status lbm_stefan_set_bc(lbm_stefan* h, int wall, int kind, double theta_wall);

/* Change the Stefan number (Eq. 1) of an existing problem, e.g. between the
 * runs of a finite-difference check or of an optimisation over Ste; the
 * state is kept.  LBM_ERR_ARG unless ste > 0 and finite. */
lbm_status lbm_stefan_set_ste(lbm_stefan* h, double ste);

/* Step method.  LBM_IREBM (default): Algorithm 3.  LBM_EEBM: the explicit
 * enthalpy based method of Algorithm 2 (Sec. 3.4), the paper's comparison
 * scheme, on D1Q3, D2Q9 and D2Q5: the populations carry the enthalpy H = M0(f),
 * theta = Theta(H) (H below 0, 0 on [0, 1/Ste], H - 1/Ste above), the
 * equilibrium is w_i theta (i != 0) and H - (1 - w_0) theta (i = 0), no Newton;
 * the closures act on the streamed populations as for IREBM (Eq. 17 included),
 * a Dirichlet node holding M0 at the enthalpy of its wall value
 * (theta_D + [theta_D > 0]/Ste);
 * delta is not used.  For EEBM, get_fields returns theta = Theta(H), phi = the
 * liquid fraction min(max(Ste H, 0), 1) and H; the energy statistics are the
 * sum of H; the adjoint calls return LBM_ERR_STATE.  Discards the state: call
 * lbm_stefan_set_ic afterwards.  LBM_ERR_ARG for an unknown method.
 * LBM_ILFBM: the implicit liquid fraction based method of Algorithm 1
 * (Sec. 3.3), the paper's other comparison scheme, in FP64 on D1Q3 (up to
 * 2,844 nodes, one block) and on D2Q9 / D2Q5 (one launch per inner
 * iteration; the state buffers grow by one plane, so lbm_stefan_layout's
 * state_bytes changes): theta = M0(f), f_i^eq = w_i theta, and a
 * liquid-fraction field l (the plane after the q populations: the fourth
 * plane of the D1Q3 state, zero for the other methods) updated
 * by an inner loop of collision with the source (w_i/Ste)(l - l^(k-1)),
 * streaming, H^(k) = M0(f^(k)) + l^(k-1)/Ste and the lever rule l(H) = 0,
 * Ste H, 1 (H < 0, in [0, 1/Ste], above), until max |l^(k) - l^(k-1)| <=
 * newton_tol; newton_max_iter bounds the loop (reaching it sets
 * LBM_ERR_NEWTON).  Dirichlet nodes hold theta_D with l = [theta_D > 0];
 * set_ic puts l = [theta0 > 0].  get_fields returns theta, phi = l and
 * H = theta + l/Ste; the energy statistics are the sum of H and
 * newton_max_iter the last step's inner iteration count; step_record,
 * step_timed and the adjoint calls return LBM_ERR_STATE / LBM_ERR_ARG;
 * LBM_ERR_ARG for ILFBM in FP32, with the Eq. (17) closure, or on D1Q3
 * beyond 2,844 nodes. */
lbm_status lbm_stefan_set_method(lbm_stefan* h, int method);

/* Initial state: f_i = w_i theta0 (equilibrium), Dirichlet nodes at their wall
 * value.  theta0 holds nx*ny doubles.  Resets the step counter and stats. */
lbm_status lbm_stefan_set_ic(lbm_stefan* h, const double* theta0, int on_device);

/* Advance nsteps >= 0 steps (Algorithm 3), asynchronously on the stream.
 * Every step also forms the energy E and the boundary flux on the device. */
lbm_status lbm_stefan_step(lbm_stefan* h, int nsteps);

/* D2Q9 and D2Q5: advance nsteps >= 1 steps launched one by one (no graph) with a
 * CUDA event before, between and after the kernels of each step, wait for
 * them, and return the mean device time per step of each kernel in ms:
 * ms_kernels (3 doubles): [0] the stream/collide kernel (FP32 D2Q9: every
 * launch of the step but the last Newton launch), [1] the (last) Newton job
 * kernel, [2] FP32 D2Q9: the flat kernel's launches alone (events on the
 * handle's stream around each; 0 for the other forms).  Same result as
 * lbm_stefan_step; for measuring each kernel against its roofline.
 * Synchronizes. */
lbm_status lbm_stefan_step_timed(lbm_stefan* h, int nsteps, double* ms_kernels);

/* Test hook of the TMA row-pipeline kernel (the FP32 D2Q9 kernel whose
 * blocks wait for row loads that they issued themselves; FP32 D2Q9 batches
 * run it).  Only FP32 D2Q9 handles use it; other handles ignore it.
 * wait_limit_s > 0 bounds every such wait (default 2 s).  While
 * withhold_load is in {0, 1, 2}, the handle's steps run that kernel in place
 * of the flat interior / wall-row pair, and its first block skips that row
 * load (its rows are a range of the 128-column strip at x = 0; load 0 is the
 * row above the range, load 1 its first row): the waits for it run out, the
 * block stops after the loads it has in flight have landed (each of those
 * waits bounded too), and the next synchronizing call returns
 * LBM_ERR_TIMEOUT (the handle's state is then undefined; create a new one).
 * withhold_load = -1 restores normal steps (the flat pair).  LBM_ERR_ARG for
 * a value outside [-1, 2] or a wait limit outside (0, 60] s. */
lbm_status lbm_stefan_set_wait_test(lbm_stefan* h, double wait_limit_s, int withhold_load);

/* Advance nsteps steps and write theta(t+1), ..., theta(t+nsteps) to
 * theta_traj (device, nsteps planes of ny*row_stride doubles, row_stride from
 * lbm_stefan_layout).  Used to recompute a checkpoint segment for the adjoint. */
lbm_status lbm_stefan_step_record(lbm_stefan* h, int nsteps, double* theta_traj);

/* Wait for the stream; return the sticky device error, if any. */
lbm_status lbm_stefan_sync(lbm_stefan* h);

/* theta = M0(f), phi(theta) and H = theta + phi/Ste (Sec. 2), nx*ny doubles
 * each; any of the three may be NULL.  Synchronizes. */
lbm_status lbm_stefan_get_fields(lbm_stefan* h, double* theta, double* phi, double* H, int on_device);

/* Interface position of the current state (the paper plots it, Sec. 6.1, but
 * does not define how it is read off the lattice).  Along every lattice line
 * that starts at `wall` (0 W, 1 E, 2 S, 3 N: rows for W/E, columns for S/N;
 * D1Q3 has W and E), node 0 on the wall, in node units (multiply by dx):
 *  - first zero: the first sign change of theta from the wall node's sign,
 *    linearly interpolated between its two nodes; 0 if theta is 0 on the
 *    wall node, n - 1 if the sign never changes;
 *  - integrated: the wall side's phase fraction phi (hot wall) or 1 - phi
 *    (cold wall) summed along the line, minus the wall node's half cell.
 * first_zero / integrated receive the means over the lines; line_* (host,
 * ny or nx doubles, may be NULL) the values per line.  Synchronizes. */
lbm_status lbm_stefan_front_position(lbm_stefan* h, int wall, double* first_zero, double* integrated,
                                     double* line_first_zero, double* line_integrated);

/* Energy, flux, Newton statistics and the sticky error.  Synchronizes. */
lbm_status lbm_stefan_get_stats(lbm_stefan* h, lbm_stefan_stats* out);

/* Device layout: bytes of one state (all populations, with padding) and the
 * row stride, in elements, of state rows and of recorded theta planes. */
lbm_status lbm_stefan_layout(lbm_stefan* h, size_t* state_bytes, int* row_stride);

/* Copy the whole state (populations, step counter kept on the host) to or from
 * buf, state_bytes long.  For checkpoint / resume. */
lbm_status lbm_stefan_get_state(lbm_stefan* h, void* buf, int on_device);
lbm_status lbm_stefan_set_state(lbm_stefan* h, const void* buf, int on_device);

/* theta of the current state written to one recorded-theta plane (device,
 * ny*row_stride doubles): the start of a recorded trajectory. */
lbm_status lbm_stefan_theta_plane(lbm_stefan* h, double* theta_plane);

/* ---------------------------------------------------------------- adjoint
 * Discrete adjoint of the step above, for the misfit
 *     L = 1/2 sum_x (phi(theta_T(x)) - phi_target(x))^2.
 * Adjoint states have the layout and precision of the forward state.  The
 * Newton root enters through the implicit function theorem on
 * F(x) = x + phi(x)/Ste - m0 - phi(theta)/Ste (Eq. 14).  Gradients with
 * respect to the wall temperatures and Ste accumulate on the device.  D1Q3
 * and D2Q9 with the bounce-back closures; LBM_ERR_ARG for D2Q5. */

/* lambda_T = dL/dOmega(T) from theta_T (a recorded plane) and phi_target
 * (device, nx*ny doubles); clears the wall / Ste accumulators.  If loss is
 * not NULL it receives L (synchronizes). */
lbm_status lbm_stefan_adjoint_seed(lbm_stefan* h, const double* theta_T, const double* phi_target,
                                   void* adj, double* loss);

/* One reverse step: adj_out = (dOmega(t+1)/dOmega(t))^T adj_in, with the
 * recorded planes theta_t = theta(t) and theta_t1 = theta(t+1). */
lbm_status lbm_stefan_adjoint_step(lbm_stefan* h, const double* theta_t, const double* theta_t1,
                                   const void* adj_in, void* adj_out);

/* nsteps reverse steps over one recorded segment: theta_traj holds nsteps+1
 * planes theta(t0), ..., theta(t0+nsteps) (device, ny*row_stride doubles each,
 * as written by lbm_stefan_theta_plane and lbm_stefan_step_record); adj holds
 * lambda(t0+nsteps) on entry.  The two state-sized device buffers adj and
 * adj_other alternate; *result_index is 0 if lambda(t0) ends in adj, 1 if in
 * adj_other.  Asynchronous on the handle's stream; LBM_ERR_ARG for NULL
 * pointers, nsteps < 0 or adj == adj_other. */
lbm_status lbm_stefan_adjoint_run(lbm_stefan* h, int nsteps, const double* theta_traj, void* adj,
                                  void* adj_other, int* result_index);

/* One backward segment of a checkpointed run (D2Q9): loads `checkpoint` (a
 * device copy of a state, state_bytes long, from lbm_stefan_get_state) as
 * the current state, recomputes nsteps steps from it recording theta into
 * theta_traj (nsteps + 1 planes), then runs nsteps reverse steps as
 * lbm_stefan_adjoint_run does (adj holds lambda at the segment's end on
 * entry; *result_index tells which buffer holds lambda at its start).  On a
 * non-default stream the launches after the checkpoint copy are captured
 * once per (nsteps, theta_traj, adj, adj_other) and replayed as a CUDA graph
 * (at most 8 kept; set_bc, set_ste and set_method drop them).  Afterwards
 * the current state is the segment's end.  Asynchronous on the handle's
 * stream.  LBM_ERR_ARG for NULL pointers, nsteps < 1, adj == adj_other or
 * another lattice; LBM_ERR_STATE for another method. */
lbm_status lbm_stefan_adjoint_segment(lbm_stefan* h, const void* checkpoint, int nsteps, double* theta_traj,
                                      void* adj, void* adj_other, int* result_index);

/* From lambda_0: dL/dtheta0 (nx*ny doubles, zero on Dirichlet nodes),
 * dL/dtheta_wall[4] (walls that are not Dirichlet get 0) and dL/dSte.
 * Synchronizes. */
lbm_status lbm_stefan_adjoint_finish(lbm_stefan* h, const void* adj0, double* g_theta0, int on_device,
                                     double* g_wall, double* g_ste);

void lbm_stefan_destroy(lbm_stefan* h);

/* ---------------------------------------------------------------- batches
 * Many independent D2Q9 problems of uneven sizes advanced by kernel launches
 * over all problems at once, then the Newton job kernel; the launches of a
 * call are captured in a CUDA graph.  FP32: the kernels of the single-problem
 * FP32 step over tables (the S and N wall rows and the W and E wall groups of
 * every problem, one block per 128-column x 8-row tile of every problem); on
 * a stream of the batch's own, the single problem's split step (the left
 * halves' Newton solves beside the right halves' streaming on a second
 * stream); FP64: the persistent warp-tile kernel over a schedule of warp
 * tiles.  The order of the problems (and, in FP64, the tile height) come from
 * lbm_stefan_batch_autotune (or defaults). */

typedef struct {
    int nx, ny;                 /* >= 2 each */
    double tau, delta, ste;
    int wall_kind[4];           /* W, E, S, N */
    double wall_theta[4];
} lbm_stefan_problem;

lbm_status lbm_stefan_batch_create(int count, const lbm_stefan_problem* problems, int precision,
                                   double newton_tol, int newton_max_iter, void* cuda_stream,
                                   lbm_stefan_batch** out);
lbm_status lbm_stefan_batch_set_ic(lbm_stefan_batch* b, int k, const double* theta0, int on_device);
lbm_status lbm_stefan_batch_step(lbm_stefan_batch* b, int nsteps);
lbm_status lbm_stefan_batch_get_fields(lbm_stefan_batch* b, int k, double* theta, int on_device);
lbm_status lbm_stefan_batch_get_stats(lbm_stefan_batch* b, int k, lbm_stefan_stats* out);
/* Time candidate schedules (FP64: and tile heights) for trial_steps steps
 * each and keep the fastest; the state is saved and restored around the
 * trials.  chosen_tile_h receives the chosen height (FP32: 8; may be NULL). */
lbm_status lbm_stefan_batch_autotune(lbm_stefan_batch* b, int trial_steps, int* chosen_tile_h);
/* Set the tile height (rows per warp tile, FP64; FP32 tiles have 8 rows and
 * ignore it) and schedule (0 = problem order, 1 = largest problems first in
 * FP32, longest tiles first in FP64) explicitly. */
lbm_status lbm_stefan_batch_set_schedule(lbm_stefan_batch* b, int tile_h, int schedule);
void lbm_stefan_batch_destroy(lbm_stefan_batch* b);

/* ---------------------------------------------------------------- one step without allocation
 * The paper has no counterpart to this entry point: it exists for callers that
 * cannot allocate device memory when they step (code running under an
 * allocator or memory budget it does not own, pre-sized real-time loops that
 * must not call cudaMalloc, hosts whose GPU memory is handed out up front).
 *
 * One D2Q9 step, state_in -> state_out, computing what lbm_stefan_step does for
 * one step of a problem created with the same parameters and walls.  It
 * allocates nothing: the scratch of the step (problem descriptor, statistics,
 * counters, the list of nodes whose Newton solve is deferred) lives in one
 * fixed device array of about 6.3 MB inside the library, which every GPU that
 * loads the library holds until the process exits.
 *  - Sizes: nx * ny <= 262,144 nodes; larger problems return LBM_ERR_ARG.
 *  - Buffers (device, caller-owned, distinct): the state layout of
 *    lbm_stefan_layout / lbm_stefan_get_state: 9 planes; each plane has ny + 2
 *    rows of `pitch` elements (pitch = nx rounded up to 128 elements in FP32, 64
 *    in FP64); rows -1 and ny and the padding columns are zero; then the
 *    256-byte tail (FP32: the shift s, see the state buffers above), which the
 *    call copies from state_in to state_out.  Elements are float (LBM_FP32) or
 *    double (LBM_FP64).
 *  - wall_kind[4], wall_theta[4]: W, E, S, N as in lbm_stefan_set_bc.
 *  - The first call in each CUDA context resolves the array's device address
 *    (cudaGetSymbolAddress) and keeps it for that context.
 *  - Every call shares the array: calls that overlap on the GPU (other
 *    streams, other threads) race.  Each call clears what must start at zero.
 *  - Runs on cuda_stream (a cudaStream_t), copies the problem descriptor
 *    from host memory and synchronizes the stream to read the device error
 *    flag (LBM_ERR_NEWTON on a Newton failure or a non-finite value): every
 *    call returns after its step has finished. */
lbm_status lbm_stefan_step_d2q9_noalloc(const lbm_stefan_params* p, const int* wall_kind, const double* wall_theta,
                                        const void* state_in, void* state_out, void* cuda_stream);

const char* lbm_stefan_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LBM_STEFAN_H */
