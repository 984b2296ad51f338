/*
 * hydro.h -- C ABI of the B300 relativistic-hydrodynamics step library.
 *
 * The library advances the (3+1)D ideal relativistic hydrodynamic equations
 * with a jet source, d_mu T^{mu nu} = S^nu (arXiv:1511.02137, Sec. 1, Eq. 1),
 * T^{mu nu} = (e+p) u^mu u^nu - p g^{mu nu}, EOS p = e/3 (Fig. 3 caption), on a
 * uniform Cartesian grid, by third-order Runge-Kutta steps (Sec. 1) of a
 * finite-difference 7th-order WENO scheme (Sec. 1) applied component-wise to
 * local Lax-Friedrichs split fluxes.  Jets are light-speed point sources
 * (Eq. 2) losing energy at the rate of Eq. 3.
 *
 * Conventions shared by every entry point:
 *  - Fields are 5 arrays of nx*ny*nz values each, x fastest, then y, then z
 *    ("SoA"): conserved (E = T^00, M^x, M^y, M^z, R = n gamma) or primitive
 *    (e, u^x, u^y, u^z, n) with u^i the spatial four-velocity.
 *    Units: fm, fm/c, GeV/fm^3 (E, M, e), fm^-3 (R, n), GeV (T).
 *  - Cell (i, j, k) has centre ((i + 1/2 - nx/2) dx, (j + 1/2 - ny/2) dx,
 *    (k + 1/2 - nz/2) dx): the grid is centred on the origin.
 *  - Every function returns a hydro_status and never aborts, prints or throws.
 *  - Field buffers (host, or device where a call says so) are owned by the
 *    caller and only used during the call.
 *  - All device work is issued on the stream given in hydro_config; every
 *    call that returns data synchronises that stream before returning.  The
 *    library does not link PyTorch: in C a NULL stream is the legacy default
 *    stream, and the Python binding passes PyTorch's current stream.
 *  - Device memory: the caller may pass every buffer the library needs
 *    (hydro_config.workspace; the Python binding passes PyTorch tensors, so
 *    PyTorch's caching allocator provides all device memory); with a NULL
 *    workspace the library calls cudaMalloc itself.
 *  - A context is not thread safe; use one context per thread.
 */
#ifndef HYDRO_H
#define HYDRO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HYDRO_OK = 0,
  HYDRO_EINVAL = 1,      /* bad argument or configuration */
  HYDRO_ENOMEM = 2,      /* device allocation failed, or the given workspace is too small */
  HYDRO_ECUDA = 3,       /* a CUDA runtime call or kernel launch failed */
  HYDRO_EUNPHYSICAL = 4, /* NaN or Inf appeared in the state during a step */
  HYDRO_ECFL = 5,        /* max signal speed * dt / dx exceeded cfl_limit */
  HYDRO_ETIMEOUT = 6,    /* a bounded device-side wait expired (hydro_config.wait_limit_s); the
                            fields written by that step are invalid: set a new initial state */
  HYDRO_ESTATE = 7,      /* call out of order (e.g. hydro_step before hydro_set_initial) */
  HYDRO_ECHECK = 8       /* bounds-checked build only (libhydro_check.so, compiled with
                            -DHYDRO_CHECK): a sweep kernel computed a global-memory index outside
                            its buffer or a TMA coordinate the copy rules forbid; the access was
                            redirected inside the buffer or the copy skipped, hydro_diag names the
                            first one (check_site, check_index), and the step's results are invalid */
} hydro_status;

enum { HYDRO_FP64 = 0, HYDRO_FP32 = 1, HYDRO_MIXED = 2 };     /* hydro_config.precision */
enum { HYDRO_OUTFLOW = 0, HYDRO_PERIODIC = 1 };              /* hydro_config.boundary */
enum { HYDRO_PRIMITIVE = 0, HYDRO_CONSERVED = 1 };           /* field kinds */

#define HYDRO_MAX_JETS 16

/* Run configuration.  hydro_config_default() fills the paper's values. */
typedef struct {
  int32_t nx, ny, nz;   /* cells per axis, each >= 1; ny, nz <= 65535 and nx ny nz <= 4e8
                           (32-bit element indices in the kernels) */
  int32_t precision;    /* HYDRO_FP64: everything in FP64.
                           HYDRO_FP32: storage and arithmetic in FP32.
                           HYDRO_MIXED: FP64 storage, FP64 conserved-to-primitive recovery
                           and RK3 accumulation; FP32 WENO weights, fluxes and divergence. */
  int32_t boundary;     /* HYDRO_OUTFLOW (zero-gradient ghosts) or HYDRO_PERIODIC */
  int32_t weno_order;   /* 7 (WENO7, Sec. 1) or 5 (WENO5, Sec. 1) */
  double dx;            /* cell edge [fm] (0.1 in Fig. 3 caption) */
  double dt;            /* time step [fm/c] (0.02 in Fig. 3 caption) */
  double t0;            /* time of the initial state [fm/c] (1 in Sec. 2) */
  double k_rad;         /* kappa_rad of Eq. 3 (4) */
  double k_coll;        /* kappa_coll of Eq. 3 (2.5) */
  double cr_over_cf;    /* C_R/C_F of Eq. 3 (1) */
  double hbarc;         /* hbar c [GeV fm] (0.1973) */
  double dof;           /* degrees of freedom in e = (pi^2/30) dof T^4/(hbar c)^3 (47.5) */
  double e_floor;       /* floor on E in the primitive recovery [GeV/fm^3] */
  double weno_eps;      /* epsilon of the WENO weights (1e-6); must lie in [1e-20, 1e20] for
                           HYDRO_FP64 and in [1e-18, 1e18] for HYDRO_FP32 and HYDRO_MIXED, whose
                           FP32 weights 1/(eps + beta)^2 must stay finite and normal */
  double cfl_limit;     /* hydro_step returns HYDRO_ECFL when max speed * dt/dx exceeds it; <= 0: off */
  void* cuda_stream;    /* cudaStream_t for all device work; NULL = legacy default stream */
  void* workspace;      /* device buffer of >= hydro_workspace_size() bytes, 256-byte aligned,
                           owned by the caller and kept alive until hydro_destroy; NULL: the
                           library allocates (cudaMalloc) and frees it itself */
  size_t workspace_bytes;
  double wait_limit_s;  /* time limit of each bounded device-side wait, in seconds of the GPU's
                           global timer: a tile's wait for its TMA copies into shared memory
                           (normally a few microseconds).  0: 0.25 s.  Must lie in [0, 10].
                           A wait that runs out makes the step return HYDRO_ETIMEOUT; the
                           tile then finishes without the copied data (so that no block leaves
                           a barrier early and no copy is left in flight at exit), which
                           leaves the step's results invalid. */
  int32_t test_withhold_copies; /* fault injection for tests: 1 = tiles arm their copy barriers
                           but issue no TMA copy, so every such wait runs out and the step
                           (hydro_step, hydro_batch_step) returns HYDRO_ETIMEOUT (nothing is
                           in flight when the tiles exit).  0 in normal use; the adjoint
                           rejects 1, the allocation-free step issues no TMA copy. */
  int32_t test_check_tighten; /* test hook of the bounds-checked build: 1 = every checked bound
                           is halved, so that accesses to the upper half of each buffer are
                           recorded (and redirected into the lower half: no access leaves its
                           buffer) and the step returns HYDRO_ECHECK.  Must be 0 in the regular
                           build (HYDRO_EINVAL otherwise) and for the adjoint. */
} hydro_config;

typedef struct hydro_ctx hydro_ctx;

/* Diagnostics of a context (hydro_get_diag). */
typedef struct {
  double t;                     /* time of the current state [fm/c] */
  int64_t steps;                /* completed RK3 steps */
  double max_speed;             /* largest spectral radius |lambda| over cells and axes at the
                                   first stage of the last step (units of c) */
  int64_t floor_hits;           /* cells whose primitive recovery needed a floor, all stages */
  double dep_E;                 /* energy deposited by all jets, RK3-weighted, [GeV] */
  double dep_M[3];              /* momentum deposited by all jets, [GeV] */
  int32_t njet;
  int32_t jet_cell[HYDRO_MAX_JETS][3]; /* cell where each jet deposited at the last stage, as
                                          recorded by the device; -1 if it deposited nothing */
  int32_t status;               /* first error status raised on the device since creation */
  int32_t check_site;           /* bounds-checked build: the first failed check's site, 0 if none:
                                   1-3 a cell offset formed for the phase-3 operand copies, a
                                   staged cell or an updated cell; 4 a TMA load, 5 a TMA store;
                                   6-8 the adjoint's reverse sweeps (window, result, jet cell) */
  uint32_t check_index;         /* ... and the index it computed (for a TMA site: the coordinate) */
} hydro_diag;

/* Paper defaults (Sec. 1, Sec. 2, Fig. 3 caption) for an nx x ny x nz grid, FP64,
 * outflow, WENO7.  Never fails. */
void hydro_config_default(hydro_config* cfg, int32_t nx, int32_t ny, int32_t nz);

/* Bytes of device workspace a context with this configuration needs: three
 * state copies and one right-hand-side accumulator (5 fields each), in FP64 the
 * primitive cache of the sweeps (5 fields), in mixed precision the FP32
 * shadows of the three states (6 fields each), and a small diagnostics block.
 * HYDRO_EINVAL for an invalid configuration. */
hydro_status hydro_workspace_size(const hydro_config* cfg, size_t* bytes);

/* Validates cfg, sets up device memory and returns a new context in *out.
 * The context is the field store of the uniform Cartesian grid of Sec. 1: the
 * five conserved densities of Eq. 1 (energy, momentum, charge) as SoA arrays,
 * plus the RK3 stage states and the right-hand-side accumulator; the paper
 * names no API, so this call is library plumbing around that state.
 * HYDRO_EINVAL: invalid configuration (non-positive sizes or steps, unknown
 * enum values, workspace not aligned); HYDRO_ENOMEM: workspace too small or
 * cudaMalloc failed; HYDRO_ECUDA: other CUDA failure.  On failure *out = NULL. */
hydro_status hydro_create(const hydro_config* cfg, hydro_ctx** out);

/* Uploads the state at t0.  kind = HYDRO_PRIMITIVE takes (e, u^x, u^y, u^z, n)
 * and converts to conserved variables on the device (Eq. 1 with p = e/3);
 * kind = HYDRO_CONSERVED takes (E, M^x, M^y, M^z, R).  host5 holds 5*nx*ny*nz
 * doubles in host memory (pinned memory makes the copy asynchronous) or in
 * device memory of the context's device (unified addressing picks the copy's
 * direction; a state built on the GPU needs no host copy of its own).
 * Resets time to t0 and the step counter to 0; keeps the jets.
 * HYDRO_EINVAL: NULL pointer, unknown kind, or e < 0 / non-finite values. */
hydro_status hydro_set_initial(hydro_ctx* ctx, int32_t kind, const double* host5);

/* Adds a jet that starts at x0 [fm] at time t_start [fm/c] and flies at light
 * speed along dir (normalised inside: n = dir/|dir|).  It deposits energy at
 * the rate of Eq. 3 and momentum n times that (Eq. 2) into the cell that holds
 * it at each RK stage time.  *jet_id (may be NULL) receives its index.
 * HYDRO_EINVAL: zero or non-finite direction, or HYDRO_MAX_JETS reached. */
hydro_status hydro_add_jet(hydro_ctx* ctx, const double x0[3], const double dir[3], double t_start,
                           int32_t* jet_id);

/* Advances nsteps SSP-RK3 steps of length dt (Shu-Osher form, Sec. 1):
 *   U1 = U + dt L(U, t),  U2 = 3/4 U + 1/4 (U1 + dt L(U1, t+dt)),
 *   U  = 1/3 U + 2/3 (U2 + dt L(U2, t+dt/2)),
 * with L = -div F + S.  Synchronises the stream at the end and returns the
 * first error raised: HYDRO_EUNPHYSICAL (NaN/Inf), HYDRO_ECFL, HYDRO_ECUDA,
 * HYDRO_ETIMEOUT (a bounded wait ran out: the state is invalid until the
 * next hydro_set_initial; the CUDA context stays usable); HYDRO_ESTATE before
 * hydro_set_initial; HYDRO_EINVAL for nsteps < 0; in the bounds-checked build
 * also HYDRO_ECHECK. */
hydro_status hydro_step(hydro_ctx* ctx, int32_t nsteps);

/* Copies the current state to host5 as FP64 (FP32 storage is widened):
 * kind = HYDRO_CONSERVED gives (E, M^x, M^y, M^z, R), the conserved densities
 * of Eq. 1; kind = HYDRO_PRIMITIVE gives (e, u^x, u^y, u^z, n), Eq. 1 with
 * p = e/3 inverted on the device in FP64 with the same closed form the step
 * uses.  The paper names no read-back call; this is library plumbing (with
 * hydro_set_initial(HYDRO_CONSERVED) it also checkpoints and resumes a run).
 * host5 holds 5*nx*ny*nz doubles, in host or device memory as for
 * hydro_set_initial. */
hydro_status hydro_read_fields(hydro_ctx* ctx, int32_t kind, double* host5);

/* Fills *out with the context's diagnostics (synchronises the stream): the
 * energy and momentum the jets deposited (the time integral of the source
 * S^nu of Eq. 2 at the rate of Eq. 3, RK3-weighted), the cells they deposited
 * into, the maximum signal speed and floor counts of the step.  Diagnostic
 * plumbing: the paper has no counterpart. */
hydro_status hydro_get_diag(hydro_ctx* ctx, hydro_diag* out);

/* Per-kernel timing with CUDA events on the context's stream, for profiling.
 * hydro_profile_enable(ctx, 1) starts recording (and clears the counters);
 * hydro_profile_query returns, for kernel kind k (see HYDRO_KERNEL_*), the
 * summed device time in ms and the launch count of the launches recorded so
 * far (synchronises the stream).  HYDRO_EINVAL for an unknown kind. */
enum {
  HYDRO_KERNEL_SWEEP_X = 0,   /* x flux divergence into the RHS accumulator */
  HYDRO_KERNEL_SWEEP_Y = 1,   /* y flux divergence added to the RHS accumulator */
  HYDRO_KERNEL_SWEEP_Z = 2,   /* z flux divergence + jet source + RK3 stage combination */
  HYDRO_KERNEL_OTHER = 3,     /* initial-state conversion, field read-back */
  HYDRO_KERNEL_COUNT = 4
};
hydro_status hydro_profile_enable(hydro_ctx* ctx, int32_t on);
hydro_status hydro_profile_query(hydro_ctx* ctx, int32_t kind, double* total_ms, int64_t* launches);

/* ---------------------------------------------------------------------------
 * Batched ensembles: nevents grids of uneven sizes advanced together (the
 * ensemble form of the same step, for many events with their own profiles and
 * jet paths; the paper has no counterpart).  All
 * grids share the configuration (precision, boundary, dx, dt, t0, Eq. 3
 * constants, WENO7 only); nx/ny/nz of cfg are ignored, dims[3*e .. 3*e+2] give
 * grid e.  Each sweep of each RK3 stage is one launch over the tiles of all
 * grids (one block per tile, or persistent blocks walking the tile list; the
 * autotuner picks), and hydro_batch_step records up to 64 steps into one CUDA
 * graph that it replays.  Device work runs on a stream the batch creates; calls
 * synchronise cfg->cuda_stream first and their own stream before returning.
 * Results are identical to advancing each grid with hydro_step.
 * ------------------------------------------------------------------------- */
typedef struct hydro_batch hydro_batch;

/* Device bytes a batch needs (states, accumulator, diagnostics, tile and jet
 * tables).  HYDRO_EINVAL for a bad configuration, nevents < 1, a zero
 * dimension, or weno_order other than 7. */
hydro_status hydro_batch_workspace_size(const hydro_config* cfg, int32_t nevents, const int32_t* dims,
                                        size_t* bytes);

/* Creates a batch; the workspace comes from cfg->workspace (>= the size above,
 * 256-byte aligned, caller-owned) or from cudaMalloc.  Errors as hydro_create. */
hydro_status hydro_batch_create(const hydro_config* cfg, int32_t nevents, const int32_t* dims, hydro_batch** out);

/* Initial state of grid `event` (as hydro_set_initial, from host or device
 * memory); resets the batch's
 * step counter.  Every grid needs one before stepping (else HYDRO_ESTATE). */
hydro_status hydro_batch_set_initial(hydro_batch* b, int32_t event, int32_t kind, const double* host5);

/* Adds a jet to grid `event` (as hydro_add_jet, up to HYDRO_MAX_JETS per grid). */
hydro_status hydro_batch_add_jet(hydro_batch* b, int32_t event, const double x0[3], const double dir[3],
                                 double t_start, int32_t* jet_id);

/* Selects the tile shape of each sweep axis (0..2 per axis; see
 * hydro_batch_autotune).  HYDRO_EINVAL for an unknown shape. */
hydro_status hydro_batch_set_tiles(hydro_batch* b, const int32_t variant[3]);

/* Selects the launch form of each sweep axis: per_tile[d] = 1 launches one
 * block per tile of every grid (the hardware scheduler balances the uneven
 * grids; the default), 0 launches persistent blocks (blocks per SM x SMs) that
 * walk the tile list.  Results are identical.  HYDRO_EINVAL for other values. */
hydro_status hydro_batch_set_launch(hydro_batch* b, const int32_t per_tile[3]);

/* The current tile shape and launch form of each axis (either may be NULL). */
hydro_status hydro_batch_get_tuning(hydro_batch* b, int32_t variant[3], int32_t per_tile[3]);

/* Times every compiled tile shape of each sweep axis on this ensemble, each in
 * both launch forms (three first-stage launches each, writing only scratch),
 * and keeps the fastest shape and form.  variant_out (may be NULL) receives the
 * shape per axis, ms_out (may be NULL) the 9 times in ms, axis-major, each the
 * faster of its two launch forms (hydro_batch_get_tuning gives the forms).
 * Needs every grid initialised. */
hydro_status hydro_batch_autotune(hydro_batch* b, int32_t variant_out[3], double ms_out[9]);

/* Advances every grid by nsteps SSP-RK3 steps; statuses as hydro_step (the
 * first error over the grids). */
hydro_status hydro_batch_step(hydro_batch* b, int32_t nsteps);

/* Fields of grid `event` (as hydro_read_fields). */
hydro_status hydro_batch_read_fields(hydro_batch* b, int32_t event, int32_t kind, double* host5);

/* Diagnostics of grid `event` (as hydro_get_diag). */
hydro_status hydro_batch_get_diag(hydro_batch* b, int32_t event, hydro_diag* out);

/* Releases a batch; NULL is a no-op. */
void hydro_batch_destroy(hydro_batch* b);

/* ---------------------------------------------------------------------------
 * Adjoint: gradients of a final-time observable, the energy J = sum E dx^3 in a
 * cone (apex, axis, half angle, radius rmax) after nsteps RK3 steps, with
 * respect to k_rad and k_coll of Eq. 3 and the initial energy density field.
 * Reverse mode of the step written by hand (vector-Jacobian products of the
 * WENO7 fluxes, the LLF split, the primitive recovery and the jet source),
 * states checkpointed every `checkpoint_every` steps and recomputed segment by
 * segment in reverse.  Outflow, WENO7 only; precision HYDRO_FP64, or
 * HYDRO_MIXED (its vector-Jacobian products in FP32 flux arithmetic, adjoint
 * states and stage combinations in FP64).  The forward runs the step exactly
 * as hydro_step does for the same configuration, so J and its gradient belong
 * to the step of the context API.  The derivative
 * of the LLF alpha = max over the stencil is split equally among tying cells
 * (within 1e-12 relative in FP64, 1e-6 in mixed).
 * ------------------------------------------------------------------------- */
typedef struct hydro_adjoint hydro_adjoint;

/* Device bytes an adjoint run needs (checkpoints; two sets of segment step
 * states with, in FP64, the stage states and the primitive cache or, in mixed
 * precision, the FP32 shadows of the stage states; adjoint and scratch fields).
 * HYDRO_EINVAL as hydro_adjoint_create. */
hydro_status hydro_adjoint_workspace_size(const hydro_config* cfg, int32_t nsteps, int32_t checkpoint_every,
                                          size_t* bytes);

/* Sets up an adjoint run.  Its buffers come from cfg->workspace (>= the size
 * above, 256-byte aligned, caller-owned, kept alive until
 * hydro_adjoint_destroy; the Python binding passes a PyTorch tensor) or, with a
 * NULL workspace, from cudaMalloc.  HYDRO_EINVAL unless precision is HYDRO_FP64
 * or HYDRO_MIXED, boundary = HYDRO_OUTFLOW and weno_order = 7, for grids of
 * more than 4e8 cells (the kernels index with 32 bits), for non-positive sizes
 * or cone, or a misaligned workspace; HYDRO_ENOMEM: workspace too small or
 * cudaMalloc failed. */
hydro_status hydro_adjoint_create(const hydro_config* cfg, int32_t nsteps, int32_t checkpoint_every,
                                  const double apex[3], const double axis[3], double half_angle_deg, double rmax,
                                  hydro_adjoint** out);

/* Adds a jet (as hydro_add_jet). */
hydro_status hydro_adjoint_add_jet(hydro_adjoint* a, const double x0[3], const double dir[3], double t_start);

/* Changes k_rad and k_coll of Eq. 3 for the next forward run. */
hydro_status hydro_adjoint_set_params(hydro_adjoint* a, double k_rad, double k_coll);

/* Runs the forward steps from the primitive fields in device memory d_prim5
 * (5 x nx*ny*nz doubles: e, u^x, u^y, u^z, n), keeping checkpoints, and
 * returns the observable in *J (host).  Statuses as hydro_step (a NaN state,
 * HYDRO_EUNPHYSICAL; HYDRO_EINVAL for a bad initial state). */
hydro_status hydro_adjoint_forward(hydro_adjoint* a, const double* d_prim5, double* J);

/* Reverse sweep for an upstream derivative dJ (1 for the plain gradient):
 * writes dJ/dk_rad and dJ/dk_coll to the host doubles (may be NULL) and
 * dJ/de(x) at fixed u^i and n to d_grad_e (device, nx*ny*nz doubles).
 * HYDRO_ESTATE before hydro_adjoint_forward; a status the device raised while
 * recomputing the checkpointed segments (as hydro_step; in the bounds-checked
 * build also HYDRO_ECHECK from the reverse sweeps). */
hydro_status hydro_adjoint_backward(hydro_adjoint* a, double dJ, double* grad_k_rad, double* grad_k_coll,
                                    double* d_grad_e);

/* Releases an adjoint run; NULL is a no-op. */
void hydro_adjoint_destroy(hydro_adjoint* a);

/* Largest grid (nx*ny*nz cells) that hydro_step_noalloc accepts. */
#define HYDRO_NOALLOC_MAX_CELLS 65536

/* Allocation-free stepping, for callers that cannot allocate device memory
 * (code that runs inside a memory pool or arena it does not own, plugins
 * whose host forbids cudaMalloc after start-up, real-time loops where an
 * allocation's latency or failure is not acceptable).  The paper has no
 * counterpart: this is a library-side convenience around the same step.
 *
 * Advances the conserved state in d_state by nsteps SSP-RK3 steps exactly as
 * hydro_step does (same kernels, same arithmetic), starting at step index
 * step0 (time t0 + step0*dt).  d_state is caller-owned device memory holding
 * 5*nx*ny*nz values (E, M^x, M^y, M^z, R; x fastest) in the storage type of
 * cfg->precision (double for HYDRO_FP64 and HYDRO_MIXED, float for
 * HYDRO_FP32); it is read and overwritten in place.  jets (host memory, may be
 * NULL when njet = 0) holds njet rows of 7 doubles: x0[3], dir[3], t_start,
 * with dir normalised inside as in hydro_add_jet.  diag_out (may be NULL)
 * receives the diagnostics of this call only.  cfg->workspace is ignored; all
 * work runs on cfg->cuda_stream and the call synchronises it before returning.
 *
 * The two intermediate stages, the right-hand-side accumulator, the cached
 * primitives and the diagnostics live in one fixed device array inside the
 * library (about 10.5 MB), which every GPU that loads the library holds until the process
 * exits.  The first call on a device, made with that device current, looks up
 * the array's device address (cudaGetSymbolAddress).  Every call copies its
 * diagnostics to host memory and synchronises cfg->cuda_stream, so the call
 * cannot be made while that stream is being captured into a CUDA graph.
 * Every call uses the same array, so calls that may overlap on the GPU (other
 * streams or threads on the same device) race on it and must be serialised by
 * the caller.  The call clears what must start at zero; it calls no cudaMalloc
 * or cudaFree.  Its tiles load their cells with plain loads (no tensor maps),
 * which gives the same values as hydro_step's TMA staging.
 *
 * Returns HYDRO_ENOMEM when nx*ny*nz > HYDRO_NOALLOC_MAX_CELLS (the fixed
 * array is too small), HYDRO_EINVAL for an invalid configuration (the checks
 * of hydro_create, including ny, nz <= 65535), NULL or misaligned d_state, bad
 * jets, step0 < 0 or nsteps < 0, and otherwise the statuses of hydro_step
 * (HYDRO_EUNPHYSICAL, HYDRO_ECFL, HYDRO_ECUDA). */
hydro_status hydro_step_noalloc(const hydro_config* cfg, void* d_state, int64_t step0, int32_t nsteps,
                                const double* jets, int32_t njet, hydro_diag* diag_out);

/* ---------------------------------------------------------------------------
 * Checks of the device arithmetic (test support; the paper has no counterpart).
 * hydro_eval_math evaluates one of the routines the sweeps use, elementwise
 * on device memory, so that tests can hold it to its stated error bound
 * against IEEE arithmetic and the FP64 oracle:
 *   HYDRO_MATH_RCP          out[i] = 1/in[i] by the FP64 Newton-Raphson
 *                           reciprocal of the sweeps (normal in[i] with a
 *                           normal reciprocal); in: n, out: n doubles.
 *   HYDRO_MATH_SQRT_RSQRT   out[i] = sqrt(in[i]), out[n + i] = 1/sqrt(in[i]) by
 *                           the FP64 Newton-Raphson pair (in[i] > 0, normal);
 *                           in: n, out: 2n doubles.
 *   HYDRO_MATH_C2P_FP64, HYDRO_MATH_C2P_FP32, HYDRO_MATH_C2P_MIXED
 *                           the closed-form recovery of Eq. 1 with p = e/3
 *                           (the inverse of the conserved densities) as the
 *                           FP64, FP32 and mixed-precision sweeps run it: in =
 *                           (E, M^x, M^y, M^z) as 4 arrays of n doubles (FP32
 *                           rounds them first, as its storage does), out =
 *                           (e, v^x, v^y, v^z, floor hit 0/1) as 5 arrays of n
 *                           doubles; param = e_floor.
 *   HYDRO_MATH_D2F          out = the FP32 rounding of in[i] by the integer-pipe
 *                           conversion of the mixed-precision path (nearest,
 *                           ties to even; below the FP32 normal range signed
 *                           zero, above it infinity, NaN stays NaN); in: n
 *                           doubles, out: n FP32 values (the first 4n bytes).
 *   HYDRO_MATH_F2D          out[i] = the FP64 value of an FP32 input by the
 *                           integer-pipe widening of the mixed-precision path
 *                           (exact; FP32 subnormals give signed zero); in: n
 *                           FP32 values (4n bytes at d_in), out: n doubles.
 * Runs on cuda_stream and synchronises it.  HYDRO_EINVAL for an unknown fn,
 * n < 0 or NULL pointers; HYDRO_ECUDA on a launch failure. */
enum {
  HYDRO_MATH_RCP = 0,
  HYDRO_MATH_SQRT_RSQRT = 1,
  HYDRO_MATH_C2P_FP64 = 2,
  HYDRO_MATH_C2P_FP32 = 3,
  HYDRO_MATH_C2P_MIXED = 4,
  HYDRO_MATH_D2F = 5,
  HYDRO_MATH_F2D = 6
};
hydro_status hydro_eval_math(int32_t fn, int64_t n, const double* d_in, double* d_out, double param,
                             void* cuda_stream);

/* ---------------------------------------------------------------------------
 * Measurement support for the roofline (the paper has no counterpart).
 * hydro_alu_peak times a throughput kernel of independent fused multiply-add
 * chains filling every SM (HYDRO_PEAK_FFMA: FP32 FMA; HYDRO_PEAK_FFMA2: the
 * packed FP32x2 FMA; HYDRO_PEAK_DFMA: FP64 FMA), `iters` iterations of 8
 * chains per thread, with CUDA events on cuda_stream.  *flop receives the
 * floating-point operations performed (an FMA counts 2) and *ms the kernel
 * time.  Allocates nothing.  HYDRO_EINVAL for an unknown kind or iters < 1. */
enum { HYDRO_PEAK_FFMA = 0, HYDRO_PEAK_FFMA2 = 1, HYDRO_PEAK_DFMA = 2 };
hydro_status hydro_alu_peak(int32_t kind, int64_t iters, void* cuda_stream, double* flop, double* ms);

/* Releases the context and any memory the library allocated (library
 * plumbing; the paper has no counterpart).  NULL is a no-op. */
void hydro_destroy(hydro_ctx* ctx);

/* Static string naming a status code. */
const char* hydro_status_string(hydro_status s);

#ifdef __cplusplus
}
#endif

#endif /* HYDRO_H */
