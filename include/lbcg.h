/*
 * lbcg.h -- C ABI of liblbcg.so: the time step of the two-colour D2Q9 MRT colour-gradient
 * lattice Boltzmann method with the improved geometric wetting condition of
 * Yu, Liu, Zhang & Liang, "Lattice Boltzmann simulation of viscous fingering of immiscible
 * displacement in a channel using an improved wetting scheme" (arXiv 1707.00198).
 *
 * One call of lbcg_step() advances every lattice of a handle by whole time steps, each made
 * of (Sec. II.A-C):
 *   rho_R, rho_B, rho^N from the populations          (Eq. 12, 16)
 *   grad rho^N, virtual values on outermost solid     (Eq. 28, 29)
 *   wetting correction on the outermost fluid nodes   (Eq. 30-36, E8 normal Eq. 32-33)
 *   n, virtual n, grad n, curvature, CSF force        (Eq. 10, 11, 13, 29, 44)
 *   velocity and local viscosity                       (Eq. 5, 17, 18)
 *   MRT collision with Guo forcing                     (Eq. 1-9)
 *   recolouring                                        (Eq. 14)
 *   streaming with half-way bounce-back                (Eq. 15; Sec. II.A after Eq. 6)
 *   optional Zou-He velocity inlet / pressure outlet   (Sec. III.D)
 * on one GPU, entirely in CUDA kernels; nothing of the step runs on the host.
 *
 * Conventions
 *   - Arrays are row-major [ny][nx], x fastest.  Direction order of the populations follows
 *     the paper: e0=(0,0), e1=(1,0), e2=(0,1), e3=(-1,0), e4=(0,-1), e5=(1,1), e6=(-1,1),
 *     e7=(-1,-1), e8=(1,-1).
 *   - Contact angles are in radians, measured through the red fluid.
 *   - All pointers in the structs below are HOST pointers, read during the call and not
 *     kept; the handle owns every device allocation it makes (from cudaMalloc, or from the
 *     caller's allocator, lbcg_set_allocator).
 *   - Every function returns an lbcg_status; no exception or abort crosses the ABI.  After
 *     an error lbcg_last_error() returns a message for the calling thread.  A failed CUDA
 *     call marks the handle dead (later calls return LBCG_E_CUDA).
 *   - Calls on one handle must not be made concurrently from several threads.
 */
#ifndef LBCG_H
#define LBCG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LBCG_OK = 0,
  LBCG_E_ARG = 1,             /* NULL pointer, bad size, bad enum value              */
  LBCG_E_GEOMETRY = 2,        /* no fluid node, fluid on a closed edge, bad normal    */
  LBCG_E_UNSTABLE_PARAM = 3,  /* nu <= 0, theta outside (0, pi), |u_in| >= 1, ...     */
  LBCG_E_CUDA = 4,            /* a CUDA call failed; the handle is dead               */
  LBCG_E_DIVERGED = 5,        /* non-finite density found by lbcg_observables         */
  LBCG_E_TIMEOUT = 6,         /* a bounded device wait ran out (lbcg_set_poll_limit)  */
  LBCG_E_UNSUPPORTED = 7,     /* request outside what this library supports           */
  LBCG_E_NOMEM = 8,           /* device or host allocation failed                     */
  LBCG_E_BOUNDS = 9           /* checked build only: a kernel's range check failed    */
} lbcg_status;

/* Storage and arithmetic of the populations.
 *   LBCG_FP64: populations f_R, f_B stored and computed in double.
 *   LBCG_FP32: populations f_R, f_B stored and computed in float.
 *   LBCG_FP16_STORE / LBCG_BF16_STORE: 16-bit storage of d = f_R + f_B - w_a rho0 (deviation
 *     from the rest state) and g = f_R - f_B, all arithmetic in float.  FP16 stores 1024 d and
 *     1024 g (an exact power of two that keeps small deviations out of FP16's subnormal range).
 *     A step stores them with stochastic rounding (up or down with the probability of the
 *     distance, keyed by a hash of the node and the step), so that changes smaller than
 *     half a unit in the last place accumulate instead of being rounded away; the initial
 *     state and lbcg_set_populations round to nearest.  The keys count graph replays and the
 *     steps within them, so a 16-bit trajectory repeats exactly for the same sequence of
 *     lbcg_step calls on a fresh handle (lbcg_step(h, 64) and 64 calls of lbcg_step(h, 1)
 *     round differently; both are unbiased). */
typedef enum { LBCG_FP64 = 0, LBCG_FP32 = 1, LBCG_FP16_STORE = 2, LBCG_BF16_STORE = 3 } lbcg_precision;

/* x boundaries: periodic; closed (columns 0 and nx-1 must be solid); or a Zou-He velocity
 * inlet carrying pure red fluid at x = 0 and a Zou-He pressure outlet at x = nx-1. */
typedef enum { LBCG_BCX_PERIODIC = 0, LBCG_BCX_CLOSED = 1, LBCG_BCX_INOUT = 2 } lbcg_bc_x;
/* y boundaries: periodic, or closed (rows 0 and ny-1 must be solid). */
typedef enum { LBCG_BCY_PERIODIC = 0, LBCG_BCY_CLOSED = 1 } lbcg_bc_y;

/* Geometry of one lattice (host arrays, copied at create). */
typedef struct {
  int32_t nx, ny;              /* lattice size, 1 <= nx, ny and nx*ny <= 2^31-1           */
  int32_t bc_x, bc_y;          /* lbcg_bc_x, lbcg_bc_y                                    */
  const uint8_t* solid;        /* [ny*nx], nonzero = solid node (Eq. 32 indicator s)      */
  const double* rhoN0;         /* [ny*nx], initial colour field in [-1, 1]; the initial
                                  populations are f_{a,R} = w_a rho0 (1 + rhoN0)/2,
                                  f_{a,B} = w_a rho0 (1 - rhoN0)/2 at rest                 */
  const double* normal;        /* [2][ny*nx] analytic solid normal n_s pointing into the
                                  solid (Sec. II.C.1.a, curved walls), or NULL to use the
                                  E8 estimate of Eq. 32-33                                 */
  const double* theta_node;    /* [ny*nx] contact angle per node in radians, or NULL to use
                                  lbcg_params.theta everywhere                             */
} lbcg_geometry;

/* Parameters of one lattice (Sec. II.A; Eq. 4-6, 10, 14, 18; Sec. III.D). */
typedef struct {
  double nu_R, nu_B;           /* kinematic viscosities of red and blue (Eq. 18)          */
  double sigma;                /* interfacial tension coefficient (Eq. 10)                */
  double theta;                /* prescribed contact angle [rad] (Eq. 34)                 */
  double beta;                 /* segregation parameter, 0.7 in the paper (Eq. 14)        */
  double s_e, s_eps, s_q;      /* fixed MRT rates, 1.64, 1.54, 1.9 in the paper (Eq. 6)   */
  double rho0;                 /* reference density of both fluids                        */
  double u_in;                 /* inlet velocity (LBCG_BCX_INOUT)                         */
  double rho_out;              /* outlet density (LBCG_BCX_INOUT)                         */
  double grad_eps;             /* n = 0 where |grad rho^N| <= grad_eps                    */
  int32_t inlet_profile;       /* LBCG_BCX_INOUT inlet: 0 uniform u_in; 1 Poiseuille profile of
                                  maximum u_in across the inlet column's fluid rows, the walls
                                  half a node beyond its first and last fluid rows (Sec. III.D) */
  int32_t wetting;             /* 0: the paper's improved scheme (a) (Eq. 28-36, grad n with
                                  Eq. 29 virtual n); 1: scheme (b) of Sec. III.A.2, grad n on
                                  the outermost fluid nodes by Eq. 48; 2: the surface-energy
                                  formulation, rho^N = cos(theta) on the outermost solid nodes
                                  and no Eq. 30-36 correction (one global theta)              */
} lbcg_params;

/* What lbcg_observables measures (all rows are 0-based y indices). */
typedef struct {
  double wall_y;               /* flat-wall height for the contact angle (e.g. 0.5)       */
  double cyl_x, cyl_y, cyl_r;  /* if cyl_r > 0: angle against this solid cylinder instead */
  int32_t tip_row0, tip_row1;  /* finger tip: first rho^N >= 0 -> < 0 change along the
                                  mean of these two rows, scanning from x = 0             */
  int32_t cl_row0, cl_row1;    /* contact line: the same change along each of these rows,
                                  averaged over the rows where one is found                */
} lbcg_obs_spec;

/* Observables of one lattice, in FP64 whatever the precision of the populations. */
typedef struct {
  int64_t step;                /* time steps taken since create                           */
  double mass_R, mass_B;       /* sum of rho_R, rho_B over fluid nodes (Eq. 16)           */
  double umax;                 /* max |u| over fluid nodes (Eq. 46, u of Eq. 17)          */
  double n_pts;                /* interface points used by the circle fit                  */
  double xc, yc, R;            /* algebraic circle fit through the rho^N = 0 crossings     */
  double theta_deg;            /* contact angle from the fit (flat wall or cylinder)      */
  double dp_laplace;           /* mean rho/3 over rho^N > 0.9 minus over rho^N < -0.9     */
  double x_tip, x_cl;          /* finger tip and contact line, -1 if not found            */
  double moments[9];           /* n, Sx, Sy, Sxx, Syy, Sxy, Szx, Szy, Sz of the points,
                                  relative to (nx/2, ny/2), z = x^2 + y^2                  */
  int32_t nonfinite;           /* 1 if any fluid density is NaN or Inf                    */
} lbcg_obs;

typedef struct lbcg_handle lbcg_handle;

/* Device memory.  By default a handle allocates its device buffers (the two population pools,
 * node arrays, work lists, reduction scratch, and the temporaries of lbcg_set_populations,
 * lbcg_get_populations, lbcg_diagnostics and lbcg_adjoint) with cudaMalloc and frees them with
 * cudaFree.  A caller that manages device memory itself -- e.g. through PyTorch's caching
 * allocator, so that its accounting sees the pools -- installs callbacks with
 * lbcg_set_allocator; every handle created afterwards takes all its device memory from them
 * and returns it to them (a handle keeps the allocator it was created with, also across later
 * lbcg_set_allocator calls).  alloc(bytes, stream, ctx) returns device memory of the current
 * device aligned to 256 bytes, or NULL (the call then fails with LBCG_E_NOMEM); stream is the
 * handle's cudaStream_t, on which the memory is used; release(ptr, stream, ctx) takes back a
 * block after the work of the handle on it has completed.  The callbacks are not called during
 * lbcg_step (nor during a CUDA graph capture).  lbcg_set_allocator(NULL) restores
 * cudaMalloc / cudaFree.  The setting is process-wide and thread-safe. */
typedef struct {
  void* (*alloc)(size_t bytes, void* stream, void* ctx);
  void (*release)(void* ptr, void* stream, void* ctx);
  void* ctx;
} lbcg_allocator;
lbcg_status lbcg_set_allocator(const lbcg_allocator* allocator);

/* Create a handle with ONE lattice.  `stream` is the cudaStream_t on which all later work
 * of the handle is enqueued; with NULL the handle creates (and later destroys) its own
 * non-blocking stream.  The calls that return data synchronise that stream.  Copies the geometry,
 * classifies nodes (outermost fluid / outermost solid, Sec. II.C), computes solid normals
 * (Eq. 32-33 unless given), initialises the populations and uploads everything. */
lbcg_status lbcg_create(const lbcg_geometry* geom, const lbcg_params* prm, int32_t precision,
                        void* stream, lbcg_handle** out);

/* Create a handle holding `n` independent lattices of any sizes and parameters; every
 * later lbcg_step advances all of them with one kernel launch per kernel of the step. */
lbcg_status lbcg_create_batch(int32_t n, const lbcg_geometry* geoms, const lbcg_params* prms,
                              int32_t precision, void* stream, lbcg_handle** out);

/* Enqueue `nsteps` >= 0 time steps on the handle's stream (asynchronous; replayed from a
 * captured CUDA graph when nsteps is large). */
lbcg_status lbcg_step(lbcg_handle* h, int64_t nsteps);

/* Measure the observables of lattice `lattice` of the current state (synchronises the
 * stream).  Returns LBCG_E_DIVERGED (with *out filled) if a density is not finite. */
lbcg_status lbcg_observables(lbcg_handle* h, int32_t lattice, const lbcg_obs_spec* spec,
                             lbcg_obs* out);

/* Copy the populations of lattice `lattice` to/from host memory as double
 * [2][9][ny][nx] (red block then blue block).  Synchronises the stream.  Values at solid
 * nodes are ignored on input and returned as 0. */
lbcg_status lbcg_get_populations(lbcg_handle* h, int32_t lattice, double* host_out);
lbcg_status lbcg_set_populations(lbcg_handle* h, int32_t lattice, const double* host_in);

/* Per-node fields of the current state of lattice `lattice`, as double [4][ny][nx]:
 * rho, rho^N, u_x, u_y (Eq. 12, 16, 17; zeros on solid nodes).  Synchronises. */
lbcg_status lbcg_get_fields(lbcg_handle* h, int32_t lattice, double* host_out);

/* The raw device state in its storage format: `bytes` must equal lbcg_state_bytes(h);
 * the host buffer should be pinned for full copy speed.  Enqueued on the stream;
 * lbcg_download_state synchronises before returning. */
size_t lbcg_state_bytes(const lbcg_handle* h);
lbcg_status lbcg_upload_state(lbcg_handle* h, const void* host_in, size_t bytes);
lbcg_status lbcg_download_state(lbcg_handle* h, void* host_out, size_t bytes);

/* Host state in, `nsteps` >= 0 steps, host state out: the same result as lbcg_upload_state,
 * lbcg_step(nsteps) with direct launches and lbcg_download_state, but the lattices of a batch
 * move in up to 8 groups of consecutive lattices (about equal node counts) whose copies and
 * steps overlap: group g's steps start when its upload lands, its download when its steps end,
 * while later groups are still uploading (the lattices are independent).  host_in and host_out
 * hold lbcg_state_bytes(h) bytes in the layout of lbcg_upload_state (pinned for full copy
 * speed) and may be the same buffer.  Ordered after the work already on the handle's stream;
 * synchronises before returning (the device error word is checked as in lbcg_download_state).
 * The copies run on two streams of the handle's own. */
lbcg_status lbcg_step_host(lbcg_handle* h, const void* host_in, void* host_out, size_t bytes, int64_t nsteps);

/* Schedule of the fused step kernel.  The default is the y-sweep (k_sweep): blocks of 128
 * threads own strips of 124 columns and walk up `rows`-row segments of them (rows = 0 picks
 * the segment height so that every SM gets several strips).  lbcg_set_tile switches to 2-D
 * tiles of 32 x ty nodes (k_step; ty = 4, 8 or 16, 0 = 8).  Both give the same results to
 * rounding; the choice only changes speed.  Both calls synchronise and drop captured graphs. */
lbcg_status lbcg_set_sweep(lbcg_handle* h, int32_t rows);
lbcg_status lbcg_set_tile(lbcg_handle* h, int32_t ty);

/* Checked build.  Compiled with -DLBCG_BOUNDS_CHECK (paper_1707_00198_gb300.build.build(
 * checked=True), which writes liblbcg_checked.so), the step kernels range-check every
 * population, node-array and staged-row access against the extent of its buffer and skip an
 * access that fails; the next synchronising call then returns LBCG_E_BOUNDS (and clears the
 * record).  The checks change no arithmetic: a checked run that reports nothing produces the
 * same bits as the normal build.  The normal build compiles them out. */

/* Failure detection of the y-sweep's only device-side wait.  In the FP32 and 16-bit y-sweep a
 * block stages each row in shared memory with bulk asynchronous copies that complete on an
 * mbarrier, and every thread waits for the row with a bounded number of polls (default 2^22,
 * about a second; a wait that healthy hardware always finishes in microseconds).  When a wait
 * gives up, the block stops at that row without writing it or any later row, waits (with the
 * default bound) for the copies it already issued, and sets the handle's device error word;
 * the next synchronising call (lbcg_observables, lbcg_get_populations, lbcg_get_fields,
 * lbcg_download_state, lbcg_diagnostics) returns LBCG_E_TIMEOUT, clears the word and leaves
 * the handle usable: the state of the steps since the previous check is unreliable and should
 * be replaced (lbcg_set_populations, lbcg_upload_state).  lbcg_set_poll_limit sets the number
 * of polls (polls < 0 restores the default; 0 makes every wait give up at once, which tests
 * the path without any fault).  Synchronises and drops captured graphs. */
lbcg_status lbcg_set_poll_limit(lbcg_handle* h, int32_t polls);

/* Gradients by the discrete adjoint (reverse mode) of the step.  From the handle's current
 * state, lbcg_adjoint runs `nsteps` steps forward (storing the state every `checkpoint`
 * steps; the handle ends at step T = nsteps), evaluates the objective J of the state at
 * T, then runs hand-written reverse kernels back to the start, recomputing each segment of
 * states from its checkpoint.  It returns J and dJ/d sigma, dJ/d nu_R, dJ/d nu_B and
 * dJ/d theta: the sum over outermost fluid nodes (a change of the global contact angle) and,
 * if dJ_dtheta_node is not NULL, per node [ny*nx] (zero off the outermost fluid nodes).
 * Objectives: LBCG_OBJ_WEIGHTED, J = sum_x weight(x) rho^N(x) (weight: host [ny*nx]);
 * LBCG_OBJ_FINGER_LENGTH, J = x_tip - x_cl (Sec. III.D; rows as in lbcg_obs_spec), whose
 * derivative is taken at the crossing cells found at T; LBCG_OBJ_RED_MASS, J = the red
 * (invading) fluid's mass sum_x rho_R(x), i.e. the displaced mass plus its initial value.
 * Single-lattice FP64 or FP32 handles (else LBCG_E_UNSUPPORTED).  On an FP32 handle the
 * forward steps, checkpoints and segment recomputation are the FP32 step.  The reverse kernels
 * read those states and run in FP64 (reverse_fp32 = 0: the gradient of the trajectory's map
 * evaluated in double) or in FP32 (reverse_fp32 = 1: several times faster on this GPU, whose
 * FP64 latency dominates the reverse sweep); the per-node parameter adjoints are summed in
 * double either way.  A second, internal stream recomputes the states of one segment while the
 * handle's stream reverses the next (the call synchronises both before it returns).  Device
 * memory for nsteps/checkpoint + 2*checkpoint states, one more wall-kernel output and the
 * adjoint arrays is allocated for the call and freed before it returns. */
enum { LBCG_OBJ_WEIGHTED = 0, LBCG_OBJ_FINGER_LENGTH = 1, LBCG_OBJ_RED_MASS = 2 };
typedef struct {
  int64_t nsteps, checkpoint;
  int32_t objective;
  const double* weight;
  int32_t tip_row0, tip_row1, cl_row0, cl_row1;
  int32_t reverse_fp32;   /* 1: reverse kernels in FP32 arithmetic; 0: FP64 */
} lbcg_adjoint_spec;
typedef struct {
  double J, dJ_dsigma, dJ_dnu_R, dJ_dnu_B, dJ_dtheta;
  double* dJ_dtheta_node;
} lbcg_grads;
lbcg_status lbcg_adjoint(lbcg_handle* h, const lbcg_adjoint_spec* spec, lbcg_grads* out);

/* Schedule of the step kernel.  lbcg_create picks the y-sweep over 124-column strips when
 * the strips give each of the 152 SMs a block, else 32-wide tiles (height 4 for FP64,
 * 8 otherwise); lbcg_set_sweep / lbcg_set_tile choose one explicitly.  lbcg_autotune times
 * each candidate (the sweep with automatic segments and with segments of 24, 32, 40, 48, 56,
 * 64 and 80 rows; tiles 4, 8, 16) as lbcg_step runs it, a captured graph of `probe_steps`
 * steps (with a batch's parallel branches) that rewrite the same next state from the current
 * one without advancing it, keeps the fastest and writes it to *schedule (0 = sweep, else the tile height;
 * schedule may be NULL).  It synchronises the handle's stream.  The candidates
 * give the same result up to rounding order (FP32: a few ulp per step; FP64 within 1e-13).
 * lbcg_schedule reports the current choice with the same encoding, lbcg_sweep_rows the
 * sweep's rows per strip segment (0: the automatic height; -1 for a NULL handle). */
lbcg_status lbcg_autotune(lbcg_handle* h, int32_t probe_steps, int32_t* schedule);
lbcg_status lbcg_schedule(const lbcg_handle* h, int32_t* schedule);
int32_t lbcg_sweep_rows(const lbcg_handle* h);

/* Steady-state diagnostics of Sec. III, in FP64 over one lattice's fluid nodes.
 *   e1: Eq. 45, max(|u_x - u_x'|, |u_y - u_y'|) between the current velocity and the one stored
 *     by this lattice's previous lbcg_diagnostics call (taken at step prev_step; NaN and
 *     prev_step = -1 on the first call).  Every call stores the current velocity.  The paper
 *     calls it every 500 steps and stops when e1 < 1e-7.
 *   e_npmt: Eq. 47, read as each colour's mass on the wrong side of the theoretical steady
 *     interface C, the circle (cx, cy, r) in node coordinates (node (x, y) is inside when
 *     (x-cx)^2 + (y-cy)^2 < r^2): sqrt((m_O^in / m_O^all)^2 + (m_D^out / m_D^all)^2), D the colour
 *     inside C (inside_red != 0: red) and O the other; the four masses are returned too.
 * The first call allocates the velocity store (2 doubles per node of the handle); the call
 * synchronises the handle's stream. */
typedef struct {
  double cx, cy, r;
  int32_t inside_red;
} lbcg_diag_spec;
typedef struct {
  int64_t step, prev_step;
  double e1, e_npmt, m_R_in, m_R_out, m_B_in, m_B_out;
} lbcg_diag;
lbcg_status lbcg_diagnostics(lbcg_handle* h, int32_t lattice, const lbcg_diag_spec* spec, lbcg_diag* out);

/* Kernel timing with CUDA events.  While enabled, lbcg_step launches the kernels of each step
 * directly (no graph) in the arrangement its graph replays: a batch's lattice groups as
 * parallel branches, each on its own stream (forked from the handle's stream once per call and
 * joined back when the call returns), with an event recorded before and after each kernel: the
 * wall kernel (rho^N on the wall band, Eq. 28-36 on the outermost fluid nodes) and the step
 * kernel (y-sweep or tiles).  lbcg_kernel_times synchronises and returns in ms2[0..1], for the
 * wall kernels and for the step kernels of the steps taken since the last call (or since
 * enabling), the milliseconds during which at least one of them ran (the length of the union
 * of their event intervals; with one branch, the sum of the kernel times), the number of steps
 * in *steps, and restarts. */
lbcg_status lbcg_profile(lbcg_handle* h, int32_t enable);
lbcg_status lbcg_kernel_times(lbcg_handle* h, double* ms2, int64_t* steps);

/* Number of kernel launches one directly launched time step enqueues (the wall kernel and the
 * bulk kernel), the number of kernel launches lbcg_step has enqueued on the handle since it was
 * created (each kernel node of a replayed graph counts: a batch's graph runs its lattices as
 * up to 3 parallel branches of their own launches), and the number of lattice nodes (fluid and
 * solid) all lattices hold. */
int32_t lbcg_launches_per_step(const lbcg_handle* h);
int64_t lbcg_step_launches(const lbcg_handle* h);
int64_t lbcg_total_nodes(const lbcg_handle* h);

lbcg_status lbcg_destroy(lbcg_handle* h);

/* Observable sums without any device allocation.  The paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc -- code that runs under a fixed
 * device-memory budget or a custom allocator that forbids new allocations, or a thread that
 * must not take the driver's allocation locks -- and that hold the macroscopic fields of a
 * lattice in their own device buffers.  It runs the same reduction lbcg_observables runs
 * internally, with the per-block partial sums kept in a file-scope device array of
 * 304 x 17 doubles (41,344 bytes) that every GPU loading the library holds until exit.
 *
 *   fields : DEVICE pointer, double [4][ny][nx]: rho_R, rho_B, u_x, u_y (caller-owned);
 *   mask   : DEVICE pointer, uint8 [ny][nx]: LBCG_MASK_SOLID marks solid nodes (skipped),
 *            LBCG_MASK_NO_FIT marks nodes whose links give no interface point (caller-owned);
 *   nx, ny : 1 <= nx*ny <= LBCG_NOALLOC_MAX_NODES, else LBCG_E_ARG with a message;
 *   stream : cudaStream_t the two kernels are enqueued on (asynchronous, no synchronisation);
 *   out    : DEVICE pointer to 17 doubles (caller-owned): mass_R, mass_B, |u|max, the nine
 *            interface moments (as lbcg_obs.moments: n, Sx, Sy, Sxx, Syy, Sxy, Szx, Szy, Sz
 *            about (nx/2, ny/2)), sum and count of rho/3 over rho^N > 0.9, sum and count over
 *            rho^N < -0.9, non-finite flag.
 * The values are raw sums; lbcg_observables derives its outputs from the same 17 values:
 * dp_laplace = out[12]/out[13] - out[14]/out[15], and the contact angle from the algebraic
 * circle fit through the moments out[3..11] (the 3x3 normal equations of x^2 + y^2 + D x +
 * E y + F = 0, centre (-D/2 + nx/2, -E/2 + ny/2)).  Interface links that cross a periodic
 * seam are not counted, as in lbcg_observables.
 *
 * Every call looks up the array's device address in the current context
 * (cudaGetSymbolAddress); the first call on a device may load the library's device code, so
 * make it before any stream capture.  All calls on a device share the array; calls whose
 * kernels overlap on the GPU race and must be serialised by the caller.  Each call overwrites
 * every partial before reading it, so no state carries over between calls.  Errors found at
 * the call (arguments, a CUDA error pending from earlier work, a failed launch) are returned
 * with a message in lbcg_last_error(); a fault while the kernels run (e.g. a bad caller
 * pointer) surfaces at the caller's next synchronisation. */
#define LBCG_MASK_SOLID 1
#define LBCG_MASK_NO_FIT 8
#define LBCG_NOALLOC_MAX_NODES 2147483647LL
lbcg_status lbcg_field_moments_noalloc(const double* fields, const uint8_t* mask, int32_t nx, int32_t ny,
                                       void* stream, double* out);

/* Message of the last error on the calling thread ("" if none). */
const char* lbcg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LBCG_H */
