/*
 * ibm.h -- C ABI of the GB300 fractional-step immersed-boundary solver.
 *
 * One call of ibm_step advances incompressible Navier--Stokes on a uniform
 * staggered (MAC) grid by the fractional-step method of Sec. II.B of
 * "Direct numerical simulation of flapping flags in grid-induced turbulence"
 * (Olivieri, Viola, Mazzino, Rosti): AB2 advection and Crank--Nicolson
 * diffusion by approximate factorisation for the provisional velocity, then
 * immersed-boundary direct forcing (regularised delta-kernel interpolation
 * and spreading, the uniform-grid form of the moving-least-squares forcing)
 * for the passive bar grid and the flexible flag, then the pressure Poisson
 * equation (transforms in the periodic y, z directions and a tridiagonal
 * solve along x) and the projection. The flag is a spring network (Sec. II.B,
 * last paragraphs) hinged at its leading edge, advanced in FP64 with
 * velocity-Verlet sub-steps. Boundary conditions follow Sec. II.A: uniform
 * inflow (U, 0, 0) at x = 0, convective outflow at x = Lx, periodic y, z.
 *
 * Units: lengths in flag lengths (L = 1), velocities in inflow speeds
 * (U = 1), fluid density 1, viscosity 1/Re.
 *
 * Layout of every field on the device and in host buffers: x slowest,
 * z fastest, index (i * ny + j) * nz + k.
 *   u, v, w : (nx + 1) * ny * nz values.
 *     u[i] sits on the x-face i (i = 0 inflow, i = nx outflow);
 *     v[i], w[i] sit at x = (i + 1/2) h for i < nx; plane i = nx holds the
 *     ghost values just outside the outflow.
 *   p       : nx * ny * nz values at cell centres.
 *
 * Status codes: every int-returning function returns IBM_OK (0) or a
 * negative IBM_E* code; ibm_strerror names it. Errors leave the state as it
 * was before the call unless stated otherwise. The library never aborts the
 * process and never traps on the GPU.
 *
 * Threading: one ibm_state must not be used from two host threads at once.
 * Streams: all device work of a state is ordered on the stream given at
 * creation (or a stream the library creates). ibm_step is asynchronous with
 * respect to the host; the query calls synchronise that stream.
 */
#ifndef IBM_H
#define IBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define IBM_OK         0
#define IBM_EINVAL    -1   /* an argument is out of range or inconsistent    */
#define IBM_ENOMEM    -2   /* device workspace missing, too small or unallocatable */
#define IBM_ECUDA     -3   /* a CUDA runtime call failed                      */
#define IBM_EDIVERGED -4   /* non-finite velocity or CFL above the limit      */
#define IBM_ETIMEOUT  -5   /* a bounded device-side wait ran out              */
#define IBM_EIO       -6   /* checkpoint file could not be written or read    */

/* arithmetic of the fluid fields */
#define IBM_FP64  0        /* everything in FP64                               */
#define IBM_FP32  1        /* fluid fields and kernels in FP32; flag, sums FP64 */
#define IBM_MIXED 2        /* FP32 fields; Poisson transforms as split-TF32 tensor-core
                              GEMMs (FP32 accumulation) + one refinement sweep on a
                              residual evaluated in double-single (FP64-class)
                              arithmetic */

/* stages for ibm_time_stage (Sec. II.B step order) */
#define IBM_STAGE_STEP      -1  /* the whole captured step                   */
#define IBM_STAGE_RHS        0  /* explicit right-hand side (AB2 + CN half)   */
#define IBM_STAGE_OUTFLOW    1  /* convective outflow plane                   */
#define IBM_STAGE_AF_X       2  /* implicit factor along x                    */
#define IBM_STAGE_AF_Y       3  /* implicit factor along y (periodic), separate */
#define IBM_STAGE_AF_Z       4  /* implicit factor along z (periodic) + u*, separate */
#define IBM_STAGE_IB         5  /* marker interpolation + spreading           */
#define IBM_STAGE_FLAG       6  /* structural sub-steps                       */
#define IBM_STAGE_MASS_DIV   7  /* mass fix + divergence                      */
#define IBM_STAGE_DHT_Y      8  /* transform along y                          */
#define IBM_STAGE_DHT_Z      9  /* transform along z                          */
#define IBM_STAGE_POISSON_X 10  /* tridiagonal solves along x                 */
#define IBM_STAGE_PROJECT   11  /* projection + pressure update               */
#define IBM_STAGE_POISSON   12  /* the whole pressure solve of the precision   */
#define IBM_STAGE_AF_YZ     13  /* y and z factors + u* in one kernel (used by the
                                   step when nz = 32, 64, 128 or 256 and ny is a
                                   multiple of 32 (FP32) or 16 (FP64); otherwise
                                   the step runs AF_Y and AF_Z and this stage
                                   launches nothing)                          */
#define IBM_STAGE_DHT_2D    14  /* both transforms of every x plane in one pass
                                   (used by the pressure solve when ny = nz =
                                   256; otherwise the solve runs DHT_Y and
                                   DHT_Z and this stage launches nothing)     */
#define IBM_STAGE_TC_PASS   15  /* one tensor-core transform pass (X H)^T over every
                                   x plane (IBM_MIXED with square planes of 32,
                                   64, 128 or 256; otherwise nothing), split
                                   products: the correction of the tensor-core
                                   mixed solve runs four                      */
#define IBM_STAGE_RESIDUAL  16  /* the double-single residual D - L_h phi of the
                                   mixed solve's refinement (IBM_MIXED only)  */
#define IBM_STAGE_TC_PASS1  17  /* one single-product (TF32) transform pass, as the
                                   mixed solve's tensor-core predictor runs at
                                   256 x 256 planes (IBM_MIXED with
                                   mixed_tc_predictor; otherwise nothing)     */
#define IBM_STAGE_TC_BF16   18  /* one bfloat16 transform pass, as the mixed
                                   solve's correction runs at 256 x 256 planes
                                   (IBM_MIXED without mixed_tc_predictor;
                                   otherwise nothing): the solve runs four    */
#define IBM_STAGE_POISSON_X16 19 /* the tridiagonal solves along x on bfloat16
                                   storage, as the correction runs them (same
                                   condition as TC_BF16)                      */

/* field selectors for ibm_get_field / ibm_set_field */
#define IBM_FIELD_U 0
#define IBM_FIELD_V 1
#define IBM_FIELD_W 2
#define IBM_FIELD_P 3

/* Cells per direction. The spacing h = lx/nx must equal ly/ny and lz/nz;
 * ny and nz must be powers of two in [4, 1024]; nx >= 4. */
typedef struct { int nx, ny, nz; } ibm_grid;

/* Domain lengths (Sec. II.A: Lx x Ly x Lz box). */
typedef struct { double lx, ly, lz; } ibm_domain;

/* Immersed bodies (Sec. II.A geometry).
 * Bar grid: square rods of side bar_width on a mesh bar_mesh in the plane
 *   x = bar_x, rods along y centred at z = (r + 1/2) bar_mesh and rods along
 *   z centred at y = (r + 1/2) bar_mesh; ly and lz must be whole multiples
 *   of bar_mesh. The rods are filled with markers (ceil(width/h) + 1 across
 *   each short side, ceil(length/h) along), crossings counted once.
 * Flag: flag_len x flag_span sheet hinged along its leading edge at
 *   x = flag_x_le, centred in y and z, pitched by pitch0 about the spanwise
 *   axis, flag_ns x flag_nt vertices (streamwise x spanwise), mass ratio
 *   rho = (rho_s / rho_f)(thickness / L), bending coefficient
 *   beta = B / (rho_f U^2 L^3), stretching spring constant `stretch`. */
typedef struct {
  int    bars_on;
  double bar_x, bar_mesh, bar_width;
  int    flag_on;
  double flag_x_le, flag_len, flag_span;
  int    flag_ns, flag_nt;
  double mass_ratio, bending, pitch0, stretch;
} ibm_bodies;

/* Options (pass NULL for the defaults given in brackets). */
typedef struct {
  int    precision;   /* IBM_FP64, IBM_FP32 or IBM_MIXED [IBM_FP64]              */
  double cfl;         /* Courant number used when ibm_step gets dt <= 0 [0.3]    */
  double cfl_limit;   /* ibm_step reports IBM_EDIVERGED above this CFL [2.0]     */
  void*  stream;      /* cudaStream_t to run on; NULL: the library creates one   */
  /* Initial perturbations added to u = U, v = w = 0 before the initial
   * projection: host arrays of (nx+1)*ny*nz doubles in the field layout, or
   * NULL. The inflow and outflow faces of u and the ghost planes of v, w must
   * hold zeros. Copied during ibm_create; the caller keeps ownership. */
  const double* init_u;
  const double* init_v;
  const double* init_w;
  /* Tile parameters (0: defaults). rhs_planes: x planes per block of the
   * streamed explicit stage [16], in [2, 256]; afx_planes: x planes per
   * segment of the implicit x factor [64]: 16 or 24 hold a segment in each
   * thread's registers; otherwise values up to 40 select 32-plane and larger
   * values 64-plane segments staged in shared memory (range [8, 256]);
   * rhs_stages: depth of the
   * explicit stage's shared-memory ring in x planes [as many as 210 KB
   * holds, at most 8], in [4, 8] (fewer than asked if they do not fit).
   * Results do not depend on them; the package's autotuner picks them per
   * problem shape. */
  int rhs_planes;
  int afx_planes;
  int rhs_stages;
  /* Nonzero: order-independent (bitwise reproducible) forcing. The scatter
   * of the IB forcing accumulates in 64-bit fixed point (resolution 2^-40,
   * partial sums below 2^23 in magnitude) and every touched node receives its
   * sum in a single addition, so results do not depend on the order of the
   * atomic operations. Costs 24 bytes per cell of workspace and one more pass
   * over the markers. [0: floating-point atomic scatter] */
  int deterministic;
  /* Nonzero: the inflow plane x = 0 is prescribed by the caller
   * (ibm_set_inflow / ibm_inflow_planes) instead of the uniform (U, 0, 0).
   * Costs 8 planes of workspace and two small kernels per step. [0] */
  int inflow;
  /* Forcing of the bar grid. 0: delta-kernel markers filling the bars,
   * forced like the flag's. 1: Eulerian direct forcing (Sec. II.B forces the
   * fixed grid on Eulerian nodes): every velocity node whose cell
   * [x - h/2, x + h/2]^3 the bars cut is set to (1 - alpha) u*, alpha the
   * cell's solid fraction (zero inside the solid); the bars then carry no
   * markers. [0] */
  int bar_forcing;
  /* IBM_MIXED with 256 x 256 transverse planes. 0: the refinement's
   * predictor is the FP32 FFT solve and the correction's transforms run on
   * the tensor cores with the single TF32 product. 1: both solves on the
   * tensor cores, the predictor with the single and the correction with the
   * split TF32 products. Both leave the FP32 rounding of the stored result
   * as the error (the final error is the product of the two solves' relative
   * errors); 0 is faster. Other plane sizes always take 1's scheme. [0] */
  int mixed_tc_predictor;
} ibm_options;

/* Diagnostics read by ibm_stats (all FP64). */
typedef struct {
  long long step;        /* steps taken                                         */
  double t;              /* simulated time                                      */
  double dt;             /* last time step                                      */
  double cfl;            /* dt * max_cells(|u|+|v|+|w|) / h at the last step    */
  double max_div;        /* max |div u| over cells (after the last projection)  */
  double q_in, q_out;    /* volume fluxes through the inflow / outflow faces    */
  double ke;             /* kinetic energy 1/2 sum |u|^2 h^3 (face values)      */
  double ib_slip;        /* max |U*_l - U_l| over markers before the last forcing */
  double te_mid[3];      /* position of the flag's trailing-edge mid vertex     */
  double force[3];       /* total fluid force on the flag, sum -F_l dV_l        */
  double max_strain;     /* max |len/len0 - 1| over flag springs                */
  int    n_sub;          /* structural sub-steps used by the last step          */
  int    n_markers;      /* flag vertices + bar markers                         */
  int    kernels_per_step; /* kernel launches in one captured step              */
} ibm_stats_t;

typedef struct ibm_state ibm_state;   /* opaque; owns its device data */

/* Bytes of device workspace ibm_create needs for this problem (all fields,
 * marker data, flag data and scratch). Fails with IBM_EINVAL on the argument
 * checks ibm_create makes. */
int ibm_workspace_bytes(const ibm_grid* grid, const ibm_domain* domain,
                        const ibm_bodies* bodies, const ibm_options* opts,
                        size_t* bytes);

/* Build a solver state: validate, generate the flag lattice and bar markers
 * on the host, upload them, set u = U + init_u, v = init_v, w = init_w,
 * p = 0, apply one projection, and capture one time step as a CUDA graph.
 * workspace: a device pointer of at least ibm_workspace_bytes() bytes,
 * 256-byte aligned, owned by the caller and kept alive until ibm_destroy;
 * or NULL, in which case the library allocates (and later frees) its own.
 * Re > 0 sets the viscosity nu = 1/Re. */
int ibm_create(const ibm_grid* grid, const ibm_domain* domain, double re,
               const ibm_bodies* bodies, const ibm_options* opts,
               void* workspace, size_t workspace_bytes, ibm_state** out);

/* Advance nsteps >= 0 time steps (Sec. II.B step order). dt > 0: fixed step;
 * dt <= 0: each step uses dt = cfl * h / max_cells(|u|+|v|+|w|) computed on
 * the device from the current velocity. Asynchronous: returns after the
 * launches are queued. Divergence is checked once per call, after the last
 * step, and reported as IBM_EDIVERGED (the fields then hold the diverged
 * state). */
int ibm_step(ibm_state* s, double dt, int nsteps);

/* Wait for the state's stream. */
int ibm_sync(ibm_state* s);

/* Copy the flag's vertex positions X, velocities V and the fluid force on
 * each vertex F (each 3 * n_vertices doubles, vertex (a, b) at index
 * a * flag_nt + b, xyz interleaved) to host memory. V and F may be NULL.
 * n_vertices must equal flag_ns * flag_nt. Synchronises. */
int ibm_flag_state(ibm_state* s, double* X, double* V, double* F, size_t n_vertices);

/* Compute and copy the diagnostics (launches small reduction kernels and
 * synchronises). */
int ibm_stats(ibm_state* s, ibm_stats_t* out);

/* Copy one field to / from host memory as doubles (n must equal the field
 * size in the layout above). ibm_set_field converts to the state's precision
 * and does not project. Both synchronise. */
int ibm_get_field(ibm_state* s, int which, double* host, size_t n);
int ibm_set_field(ibm_state* s, int which, const double* host, size_t n);

/* Prescribed, time-dependent inflow (states created with opts->inflow != 0;
 * IBM_EINVAL otherwise). The step that follows uses the pending planes as the
 * inflow of its new time level (the Dirichlet condition of Sec. II.A made
 * time-dependent): u on the inflow face becomes the pending u shifted by a
 * constant so that its mean is U (inflow flux U * ly * lz exactly, as the
 * pressure solve requires); v and w take the pending values on the inflow
 * plane through the ghost q_-1 = 2 q_in - q_0; the changes against the
 * previous level enter the implicit x factor. The explicit terms of a step
 * use the previous level. Planes are ny * nz values, index j * nz + k; the
 * pending planes keep their values until changed (a constant inflow after
 * the first step), and start as u = U, v = w = 0.
 * ibm_set_inflow copies three host planes of doubles (converted to the
 * state's precision) and synchronises. ibm_inflow_planes returns the device
 * addresses of the three pending planes in the state's precision, for
 * callers that generate the inflow on the GPU: write them on the state's
 * stream (or synchronise with it) before ibm_step. */
int ibm_set_inflow(ibm_state* s, const double* u, const double* v, const double* w);
int ibm_inflow_planes(ibm_state* s, void** u, void** v, void** w);

/* One x-plane of the velocity (precursor dumps, probes): u on face i and
 * v, w at x = (i + 1/2) h (i = nx: the outflow ghosts), 0 <= i <= nx, ny * nz
 * values each, index j * nz + k. ibm_get_plane copies them to host doubles
 * and synchronises; ibm_plane_device returns their device addresses in the
 * state's precision, valid until the next ibm_step (the velocity buffers
 * alternate between steps). */
int ibm_get_plane(ibm_state* s, int i, double* u, double* v, double* w);
int ibm_plane_device(ibm_state* s, int i, void** u, void** v, void** w);

/* Number of markers (flag vertices first, then bar markers) and their
 * positions at the start of the next step (3 doubles each). */
int ibm_marker_count(const ibm_state* s, size_t* n);
int ibm_get_markers(ibm_state* s, double* X, size_t n);

/* Virtual probes (time histories for the statistics of Sec. III): set n
 * probes at cells (i, j, k) (host ints, 3 per probe, 0 <= i < nx); each
 * ibm_probe_sample then writes the cell-centred velocity (u averaged over
 * the faces i, i + 1, v over j, j + 1, w over k, k + 1, periodic in y, z) of
 * every probe, (u, v, w) per probe, into the DEVICE buffer dst (3 n values in
 * the state's precision), asynchronously on the state's stream. The state
 * owns the probe list; n = 0 clears it. IBM_EINVAL for cells out of range or
 * a sample without probes. */
int ibm_probes_set(ibm_state* s, const int* ijk, int n);
int ibm_probe_sample(ibm_state* s, void* dst);

/* Checkpoint / restart. ibm_save writes everything the next step reads --
 * the device parameter block (time, step count, previous dt, AB2 and
 * time-step mode), u, v, w, p and the previous advection term N^{n-1} in the
 * state's precision, the per-block CFL speed maxima that set the next dt,
 * and the flag's X, V, F in FP64 -- to the file `path`
 * (created or truncated), after synchronising the state's stream. ibm_load
 * reads such a file into a state created with the same grid, domain,
 * Reynolds number, bodies and precision, so that stepping on gives the same
 * result as never having stopped (up to the order of the atomic additions of
 * the forcing). Errors: IBM_EIO if the file cannot be opened, written or
 * read completely, is not a checkpoint, or has trailing bytes; IBM_EINVAL if
 * it belongs to a different problem or precision. On any error ibm_load
 * leaves the state unchanged. The format is this library's own (native
 * byte order, not meant for exchange between machines). */
int ibm_save(ibm_state* s, const char* path);
int ibm_load(ibm_state* s, const char* path);

/* Benchmarking aid: launch one stage of the step `nrep` >= 1 times back to
 * back on the state's stream, bracketed by CUDA events, and return the mean
 * device time per launch in *ms. IBM_STAGE_STEP replays the captured step
 * (a normal time step). Any other stage runs outside the step order and
 * leaves the fields meaningless: use a state created for timing only.
 * Synchronises. */
int ibm_time_stage(ibm_state* s, int stage, int nrep, double* ms);

/* Diagnostics without any device allocation or workspace scratch (the paper
 * has no counterpart; this is a library facility). Same values as ibm_stats,
 * but the reduction scratch is a fixed device array compiled into the
 * library: 2 x 65,536 partial results plus 16 output values (about 1 MiB),
 * which every GPU that loads the library keeps until the process exits.
 * For callers that cannot allocate device memory at the point where they
 * read diagnostics: code that runs while another part of the program is
 * capturing a CUDA graph (cudaMalloc is not allowed then), loops that must
 * not stall on the implicit device synchronisation of cudaMalloc/cudaFree,
 * and programs whose device memory is wholly owned by another allocator.
 * Sizes: grids needing more than 65,536 reduction blocks
 * (ceil(nz/32) * ceil(ny/8) * ceil((nx+1)/8)) are rejected with IBM_EINVAL.
 * The first call on a device looks the array's device address up once
 * (with that device current); make that first call before any stream
 * capture. The looked-up address is kept for the life of the process: after
 * cudaDeviceReset it is stale, and the library must not be used on that
 * device again. Every call shares the array and overwrites all of it that it
 * reads, so no clearing is needed; calls that overlap on the GPU (from two
 * streams or threads) race on it. Synchronises the state's stream. */
int ibm_stats_static(ibm_state* s, ibm_stats_t* out);

/* Ensembles: several independent states stepped together. One CUDA graph
 * launch per step runs the captured step of every member as concurrent
 * branches, so that small cases of uneven size share the GPU. Members keep
 * their own fields and parameters (grid, Re, bodies, precision); they must
 * not be stepped on their own while they belong to an ensemble, and must
 * outlive it. The ensemble runs on `stream` (cudaStream_t, NULL: a stream
 * the library creates). */
typedef struct ibm_ensemble ibm_ensemble;
int ibm_ensemble_create(ibm_state* const* members, int n, void* stream, ibm_ensemble** out);
/* The same ensemble with the explicit stage (Sec. II.B: AB2 advection, the
 * explicit Crank-Nicolson half, -G p) of every member batched into one
 * persistent launch: a case table lists each member's constants, fields
 * and block grid, and the launch's blocks walk the concatenated block lists
 * of all members. Each member's step is recorded in pieces (start of step,
 * rest of the head, tail with the structural update joined) around that
 * launch, so the members meet at the explicit stage once per step. Same
 * results as ibm_ensemble_create up to rounding order; the table (device
 * memory) belongs to the ensemble. Errors as ibm_ensemble_create, plus
 * IBM_ENOMEM if the table cannot be allocated. */
int ibm_ensemble_create_batched(ibm_state* const* members, int n, void* stream, ibm_ensemble** out);
/* Advance every member nsteps steps (dt as in ibm_step, for every member).
 * Checks every member for divergence at the end; returns the first error. */
int ibm_ensemble_step(ibm_ensemble* e, double dt, int nsteps);
void ibm_ensemble_destroy(ibm_ensemble* e);

/* ---- x-slab decomposition of one case ------------------------------------
 * Sec. II.B runs one case on several GPUs by a one-dimensional domain
 * decomposition: slabs of whole y-z planes along x. Here each rank (one
 * process, one GPU) holds one slab state: its owned cell planes
 * [x_begin, x_end) of the global grid plus `ghosts` overlap planes on each
 * side that has a neighbour. A step is a fixed sequence of phases; between
 * two phases the caller moves one buffer between the ranks with a plain
 * collective (all-reduce, all-gather or a neighbour exchange, e.g. NCCL or
 * gloo through torch.distributed), so the library itself never
 * communicates and no kernel waits on another rank.
 *   step:               FORCE, SOLVE, REDUCE, PROJECT, GHOSTS
 *   initial projection: INIT, REDUCE, PROJECT, GHOSTS (once, before the
 *                       first step; ibm_create_slab does not project)
 * What couples the slabs (the rest is local to the window):
 *   - the pressure equation's x solve per transverse mode, by the partition
 *     method: local solves with the neighbours' values removed, a small
 *     system for the values next to every cut assembled from all ranks' line
 *     data (all-gather), and a corrected local solve (exact, not iterative);
 *     the mode (0, 0) keeps the pinned first row and the gauge mean(phi) = 0
 *     of the single-domain solve;
 *   - the flag's fluid force (each vertex counted by the rank owning its x
 *     position, all-reduce) and the inflow / outflow fluxes of the mass fix;
 *   - the overlap planes of u, v, w and p, refreshed from the owning
 *     neighbours after every step (each rank recomputes the advection
 *     history from the refreshed velocity). The implicit x factor's
 *     dependence on the window's ends decays like rho^d over d planes
 *     (rho < 1), so overlap planes wider than that decay plus the forcing
 *     kernel's support leave the owned planes exact to round-off
 *     (ibm_slab_ghosts).
 * Every rank builds the same flag and advances it identically. Results equal
 * the single-domain solver's up to rounding order. Limits: FP64 fields,
 * fixed dt, uniform inflow, marker forcing of the bars, at most
 * IBM_SLAB_MAX_RANKS ranks. */
#define IBM_SLAB_MAX_RANKS 8

typedef struct {
  int nranks;    /* slabs along x, 1 .. IBM_SLAB_MAX_RANKS                     */
  int rank;      /* this slab, 0 .. nranks - 1, in x order                      */
  int x_begin;   /* first owned cell plane (0 on rank 0)                         */
  int x_end;     /* one past the last owned cell plane (nx on the last rank)     */
  int ghosts;    /* overlap planes on each side with a neighbour: at least
                    ibm_slab_ghosts(), x_end - x_begin >= ghosts + 1, and the
                    window [x_begin - ghosts, x_end + ghosts) inside [0, nx);
                    the same on every rank (the exchange layouts depend on it) */
} ibm_slab;

/* phases (in step order) */
#define IBM_SLAB_INIT    0  /* divergence of the initial velocity, transforms,
                               local x solves                                   */
#define IBM_SLAB_FORCE   1  /* dt, explicit terms, implicit factors, IB forcing */
#define IBM_SLAB_SOLVE   2  /* structure, mass fix, divergence, transforms,
                               local x solves                                   */
#define IBM_SLAB_REDUCE  3  /* cut values, corrected x solves, inverse transforms */
#define IBM_SLAB_PROJECT 4  /* projection (and pressure update after a step)    */
#define IBM_SLAB_GHOSTS  5  /* overlap planes from the neighbours               */

/* exchanges the caller performs on a phase's send buffer (doubles) */
#define IBM_XCHG_NONE   0
#define IBM_XCHG_SUM    1   /* element-wise sum over all ranks (all-reduce)     */
#define IBM_XCHG_GATHER 2   /* every rank's buffer, concatenated in rank order
                               (all-gather): nranks * send_count values         */
#define IBM_XCHG_HALO   3   /* send = [to rank - 1 | to rank + 1], two halves of
                               send_count / 2; recv = [from rank - 1 | from
                               rank + 1] (a half without a neighbour is ignored
                               on send and left as it is on receive)            */

/* Smallest overlap (planes) for which the owned planes are exact to FP64
 * round-off at viscosity 1/re, spacing h and fixed step dt: the decay length
 * of the implicit x factor, ceil(log 1e-17 / log rho) with rho its decay
 * factor at r = dt / (2 re h^2), plus 4 planes of forcing support and
 * explicit stencil. Host only. */
int ibm_slab_ghosts(double re, double h, double dt, int* ghosts);

/* Even split of nx cell planes over nranks slabs with `ghosts` overlap
 * planes (the first nx % nranks slabs one plane longer); IBM_EINVAL if a
 * slab would be too short for its overlap. Host only. */
int ibm_slab_split(int nx, int nranks, int rank, int ghosts, ibm_slab* out);

/* Sizes of a phase's exchange: kind (IBM_XCHG_*), doubles the phase writes
 * into `send`, and doubles the caller passes as `recv` to the next phase
 * (the exchange's result). Depends only on the arguments (host only, no
 * state needed): ny, nz of the global grid, the flag's vertex count
 * (0 without flag) and the slab. */
int ibm_slab_plan(const ibm_grid* grid, int n_flag_vertices, const ibm_slab* slab, int phase, int* xchg,
                  size_t* send_count, size_t* recv_count);

/* Build the slab state of `slab` for the global problem (grid, domain,
 * bodies as for ibm_create; opts: FP64, no prescribed inflow, bar_forcing 0;
 * init_u/v/w, if given, are the WINDOW's perturbations, (nx_w + 1) ny nz
 * values with nx_w = x_end - x_begin + the overlap planes, window plane 0 =
 * global plane x_begin - ghosts, or x_begin on rank 0). The state covers the
 * window: ibm_get_field / ibm_set_field / ibm_get_plane work on window
 * planes; ibm_flag_state reports the shared flag in global coordinates; bar
 * markers are the global grid's within three cells of the window, shifted
 * to window coordinates. No projection is applied: run the initial phase
 * sequence before the first step. workspace: as ibm_create (window size);
 * the slab's solve tables (pivots per mode and row, 6 values per mode, and a
 * scratch of the owned planes) are allocated by the library. ibm_step,
 * ibm_time_stage(IBM_STAGE_STEP) and the ensembles refuse slab states
 * (IBM_EINVAL). */
int ibm_create_slab(const ibm_grid* grid, const ibm_domain* domain, double re,
                    const ibm_bodies* bodies, const ibm_options* opts, const ibm_slab* slab,
                    void* workspace, size_t workspace_bytes, ibm_state** out);
/* Bytes of workspace ibm_create_slab needs. */
int ibm_slab_workspace_bytes(const ibm_grid* grid, const ibm_domain* domain, const ibm_bodies* bodies,
                             const ibm_options* opts, const ibm_slab* slab, size_t* bytes);

/* Run one phase on the state's stream. recv: DEVICE buffer holding the
 * previous phase's exchange result (ibm_slab_plan's recv_count doubles;
 * NULL for IBM_SLAB_INIT and IBM_SLAB_FORCE); send: DEVICE buffer of
 * send_count doubles that this phase fills for the next exchange (NULL when
 * send_count is 0). dt > 0 (FORCE only; ignored otherwise). Phases must come
 * in one of the two sequences above (IBM_EINVAL otherwise, state unchanged).
 * Asynchronous, except GHOSTS, which synchronises and reports device-side
 * errors of the step (IBM_EDIVERGED for a non-finite velocity, IBM_ETIMEOUT,
 * IBM_EINVAL for a step size outside the implicit factor's range). Buffers
 * belong to the caller; `send` may be reused once the exchange has read it.
 * The flag's structural update of SOLVE runs on a second stream of the
 * state and is joined by GHOSTS: queries between FORCE and GHOSTS see a step
 * in progress. */
int ibm_slab_phase(ibm_state* s, int phase, double dt, const double* recv, double* send);

/* ---- Learned inflow generator ------------------------------------------
 * The synthetic-inflow alternative that Sec. V of the paper leaves open: an
 * autoregressive convolutional network that maps the two latest keyframes
 * of inflow velocity fluctuations (q_t, q_{t-s}, each 3 components on the
 * periodic ny x nz plane, s the keyframe stride in recorded planes) to the
 * next one, trained on planes recorded from a grid-resolved (precursor) run,
 * then rolled out as the prescribed inflow of a state created with
 * opts->inflow (keyframes, and planes interpolated between them).
 *
 * Network (periodic 3 x 3 cross-correlations, phi(s) = s for s > 0, s / 8
 * otherwise, width 128, `blocks` residual blocks):
 *   h_1 = conv(W_in, x) + b_in,  x = (q_t, q_{t-s})[:in_channels]
 *   h_{l+1} = h_l + conv(W_l, phi(h_l)) + b_l
 *   delta = conv(W_out, phi(h_{L+1})) + b_out,   q_{t+s} = q_t + delta
 * Convolution operands are bfloat16 (tensor cores), accumulation, residual
 * streams and the Adam master weights FP32. Loss: mean of (delta - target)^2
 * over samples, pixels and the 3 components.
 * Parameters, flat (doubles at the interface): W_in, b_in, then W_l, b_l per
 * block, then W_out, b_out; every W in [dy + 1][dz + 1][out][in] order, where
 * out[y][z] += W[dy + 1][dz + 1][o][c] in[(y + dy) mod ny][(z + dz) mod nz][c].
 * Planes q are normalised: q = (plane - mean) / std per component.
 * All pointers below are DEVICE pointers unless stated otherwise; the
 * generator owns its workspace; calls are ordered on `stream` and the ones
 * that return values synchronise it. Errors: IBM_EINVAL (arguments),
 * IBM_ENOMEM, IBM_ECUDA, IBM_ETIMEOUT (a bounded device wait ran out). */
typedef struct ibm_gen ibm_gen;
typedef struct {
  int ny, nz;         /* plane: ny >= 1, nz a multiple of 128, ny * nz <= 2^24 */
  int width;          /* 128 */
  int blocks;         /* residual blocks, 0 .. 64 */
  int in_channels;    /* input components used, 1 .. 6 (6: q_t and q_{t-s}) */
  int batch;          /* most samples per training step, 1 .. 64 */
  double lr, beta1, beta2, eps;   /* Adam (<= 0: 1e-3, 0.9, 0.999, 1e-8) */
  void* stream;       /* cudaStream_t (NULL: the default stream) */
  int stride;         /* planes between the generator's keyframes (<= 0: 1): it
                         predicts plane t + stride from t and t - stride */
} ibm_gen_config;
int ibm_gen_create(const ibm_gen_config* cfg, ibm_gen** out);
size_t ibm_gen_param_count(const ibm_gen* g);
/* host arrays of ibm_gen_param_count doubles; set_params also resets Adam */
int ibm_gen_set_params(ibm_gen* g, const double* w, size_t n);
int ibm_gen_get_params(ibm_gen* g, double* w, size_t n);
/* gradients of the last ibm_gen_grad / ibm_gen_train_step */
int ibm_gen_get_grads(ibm_gen* g, double* d, size_t n);
/* host arrays of 3: data mean and std of each component (normalisation) and
 * the rms of normalised q that rollouts keep */
int ibm_gen_set_norm(ibm_gen* g, const double* mean, const double* std, const double* rms);
/* q_t, q_prev: [batch][ny][nz][3] normalised; delta out: same layout */
int ibm_gen_forward(ibm_gen* g, const float* q_t, const float* q_prev, float* delta, int batch);
/* loss (host double, nullable) and its gradients for targets [batch][ny][nz][3] */
int ibm_gen_grad(ibm_gen* g, const float* q_t, const float* q_prev, const float* target, int batch,
                 double* loss);
/* one Adam step with the stored gradients */
int ibm_gen_adam_step(ibm_gen* g);
/* one training step on raw planes [n_planes][3][ny][nz] (FP32, e.g. a
 * precursor record): sample b predicts plane t_idx[b] + stride from
 * t_idx[b] and t_idx[b] - stride (host ints, stride <= t < n_planes - stride);
 * gradients, then Adam.
 * loss (host, nullable): the batch loss before the step. */
int ibm_gen_train_step(ibm_gen* g, const float* planes, int n_planes, const int* t_idx, int batch,
                       double* loss);
/* pushforward training step (rollout-aware): a first forward pass predicts
 * q^_t = q_{t-s} + delta(q_{t-s}, q_{t-2s}) (with the training-input noise,
 * no gradients), then the step of ibm_gen_train_step runs on the inputs
 * (q^_t, q_{t-s}) with the target q_{t+s} - q^_t, so that the network learns
 * to correct its own one-step errors, as in a rollout. 2 stride <= t_idx[b]
 * < n_planes - stride; otherwise as ibm_gen_train_step (loss: the second
 * pass's batch loss before the update). */
int ibm_gen_train_step_pushforward(ibm_gen* g, const float* planes, int n_planes, const int* t_idx, int batch,
                                   double* loss);
/* loss (host double) of a batch of raw planes as in ibm_gen_train_step,
 * without gradients or update (validation) */
int ibm_gen_eval(ibm_gen* g, const float* planes, int n_planes, const int* t_idx, int batch,
                 double* loss);
/* training-input noise: ibm_gen_train_step adds std * N(0, 1) to every
 * normalised input value (q_t and q_{t-s}) and takes the target from the
 * noisy q_t, so that the network learns to pull perturbed planes back to
 * the data (a stable rollout). N(0, 1) is Box-Muller of SplitMix64 (Steele,
 * Lea and Flood 2014) with key seed + (Adam steps done) and counter
 * (b * ny * nz + pixel) * 6 + input channel. std = 0 (the default) disables it. */
int ibm_gen_set_noise(ibm_gen* g, double std, unsigned long long seed);
/* learning rate of the following Adam steps (> 0) */
int ibm_gen_set_lr(ibm_gen* g, double lr);
/* mean device time (ms, CUDA events on the generator's stream) over nrep
 * repetitions after one warm-up, on the data in place: what = 0 training
 * step (gradients and Adam) of a full batch, 1 forward pass of a full
 * batch, 2 / 3 / 4 the forward convolution, input-gradient convolution and
 * weight gradient of the first residual block (blocks >= 1). Changes the
 * parameters when what = 0. */
int ibm_gen_time(ibm_gen* g, int what, int nrep, double* ms);
/* rollout relaxation (after ibm_gen_set_norm): each keyframe step becomes
 * q_t + delta - lambda (q_t - q_ref), q_ref the normalised host plane
 * [3][ny][nz] of doubles (e.g. the data's time mean), before the
 * renormalisation; it damps slow drifts of the rollout away from the data.
 * 0 <= lambda <= 1 (0, the default, disables it; plane may then be NULL). */
int ibm_gen_set_relax(ibm_gen* g, const double* plane, double lambda);
/* spectral relaxation of the rollout (256 x 256 planes, after
 * ibm_gen_set_relax with lambda > 0, whose plane is the reference q_ref):
 * after each keyframe step the fluctuation f = q - q_ref of every component
 * is taken to Fourier space (2-D, y and z periodic) and the amplitude of each
 * wavenumber k scaled by (S(k) / P(k))^(lambda / 2), clamped to [1/2, 2],
 * P(k) its current power and S(k) = power[c][ky][kz] the target, e.g. the
 * recorded planes' mean |FFT2(f)|^2 (unnormalised transform, normalised
 * units of ibm_gen_set_norm); the phases are kept. It keeps the rollout's
 * spectrum on the data's where errors would otherwise accumulate in some
 * wavenumbers. 0 <= lambda <= 1 (0, the default, disables it; power may
 * then be NULL). IBM_EINVAL for other plane sizes or without the relaxation
 * plane; IBM_ENOMEM if its buffers (four planes of 3 ny nz floats) cannot be
 * allocated. */
int ibm_gen_set_spectrum(ibm_gen* g, const double* power, double lambda);
/* rollout: start from two raw planes [3][ny][nz] (FP32) */
int ibm_gen_rollout_init(ibm_gen* g, const float* plane_prev, const float* plane_cur);
/* generate the next plane: q = q_t + delta (relaxed, see above), each component's plane mean
 * removed and its rms set to the `rms` of ibm_gen_set_norm; writes
 * mean + std * q into u, v, w ([ny][nz], doubles for IBM_FP64, floats
 * otherwise; any may be NULL), e.g. the pending planes of
 * ibm_inflow_planes. Asynchronous. */
int ibm_gen_rollout(ibm_gen* g, void* u, void* v, void* w, int precision);
/* planes between the last two keyframes of the rollout: writes
 * mean + std ((1 - w) q_prev + w q_t) (0 <= w <= 1) like ibm_gen_rollout,
 * so that a run can take one plane per step with keyframes every `stride`
 * steps. Asynchronous. */
int ibm_gen_emit(ibm_gen* g, double w, void* u, void* v, void* wv, int precision);
/* copy the rollout history (normalised newest and previous keyframes, [ny][nz][3]) */
int ibm_gen_history(ibm_gen* g, float* q_t, float* q_prev);
/* checkpoint of the trainable state: FP32 master weights, Adam moments and
 * step count, normalisation (mean, std, rms). A file of another
 * configuration (plane, blocks, input channels, stride) is refused with
 * IBM_EINVAL; a missing, truncated, foreign or over-long file with IBM_EIO;
 * a refused load leaves the generator as it was. The relaxation plane and
 * the rollout history are not saved. Synchronise. */
int ibm_gen_save(ibm_gen* g, const char* path);
int ibm_gen_load(ibm_gen* g, const char* path);
int ibm_gen_sync(ibm_gen* g);
void ibm_gen_destroy(ibm_gen* g);

/* Self-test of the bounded device-side waits that every kernel waiting on
 * bulk copies or tensor-core work uses (see IBM_ETIMEOUT): one thread waits
 * on an mbarrier that nothing completes, for at most `spins` try-wait rounds
 * (1 .. 2^24), records the time-out in a device flag the way the solver's
 * kernels do, and returns. Result: IBM_ETIMEOUT when the wait ran out (the
 * expected outcome; the CUDA context stays usable), IBM_EINVAL for `spins`
 * outside the range (checked before any CUDA call), IBM_ECUDA if a runtime
 * call fails. Uses the current device and its default stream; synchronises;
 * allocates and frees 4 bytes of device memory. */
int ibm_check_bounded_wait(unsigned int spins);

/* Release the state (and the workspace if the library allocated it). */
void ibm_destroy(ibm_state* s);

const char* ibm_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* IBM_H */
