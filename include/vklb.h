/*
 * vklb.h -- C ABI of the B300 (sm_103a) weighted-upwind vector kinetic lattice
 * Boltzmann (WU-VKLB) library, libvklb.so.
 *
 * The method is the one of Brown, Chaudhry and Shadid, "A Weighted Upwind Vector
 * Kinetic Lattice Boltzmann Method For Hyperbolic Conservation Laws":
 *   - the conservation law  dU/dt + sum_d dF^(d)(U)/dx_d = 0      (Sec. 2.1, Eq. 1)
 *   - vector distributions f_q in R^p on the D1Q3 / D2Q5 lattices (Sec. 2.2, Eq. 38)
 *   - weighted upwind equilibria                                   (Eqs. 22-24, 41)
 *     built from the sigmoid-weighted eigen split of F            (Eqs. 25-27)
 *   - collide  f* = f - omega (f - f^eq)                           (Eq. 42)
 *   - stream   f_q(x + v_q dt) = f*_q(x)                           (Eq. 43)
 *   - moments  U = sum_q f_q                                       (Eq. 3)
 *   - CFL lattice speed  xi = max_j |lambda_j| / nu                (Eq. 29)
 *     (or sqrt(3/2) max_j |lambda_j| / eta, the subcharacteristic rule, Sec. 2.3)
 *   - periodic (Eq. 37) and characteristic (Eqs. 33-36) boundaries.
 * One call to vklb_step advances the state by the flow chart of Fig. 5.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - All pointers are plain host or device pointers; sizes are element counts
 *    unless stated otherwise.  No call keeps a caller pointer after it returns.
 *  - Conserved-state arrays are double, laid out fields-first, x fastest:
 *        U[k * ny * nx + j * nx + i],  k = 0..p-1 (1D: ny = 1).
 *    Field order: advection (u); shallow water (h, hu[, hv]) (Eq. 52);
 *    Euler (rho, rho u[, rho v], E) (Eq. 54);
 *    MHD-GLM (rho, rho u, rho v, rho w, E, Bx, By, Bz, psi) (Eq. 58).
 *  - Every call returns a vklb_status.  Calls that enqueue GPU work are
 *    asynchronous on the simulation's CUDA stream; a device-side fault of the
 *    method (non-physical state, CFL violated with a fixed dt) is latched in a
 *    device error word and returned by the next synchronising call
 *    (vklb_sync, vklb_moments, vklb_conservation_totals, vklb_time,
 *    vklb_get_state).  No call aborts the process.
 *  - The library allocates its own device memory for the state (distributions,
 *    or moments in the moment form of vklb_set_form) and a few control words,
 *    as stream-ordered allocations on the simulation's stream (cudaMallocAsync);
 *    vklb_destroy waits for that stream alone and frees them on it, so it does
 *    not wait for work on other streams.  A batch's buffers live on the batch's
 *    own stream the same way.  vklb_conservation_totals_noalloc is the one call
 *    that allocates nothing.
 */
#ifndef VKLB_H
#define VKLB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  VKLB_OK = 0,
  VKLB_ERR_ARG = -1,          /* invalid argument (null pointer, bad size or parameter) */
  VKLB_ERR_NOMEM = -2,        /* device or host allocation failed */
  VKLB_ERR_CUDA = -3,         /* a CUDA runtime call failed (no device, launch error) */
  VKLB_ERR_NONPHYSICAL = -4,  /* NaN or non-positive h / rho / p produced on the device */
  VKLB_ERR_CFL = -5,          /* fixed lattice speed below max |lambda| (Eq. 28 violated) */
  VKLB_ERR_TIMEOUT = -6,      /* a bounded device wait gave up: a row stage of the bulk-copy
                                 step variant, or the row barrier of a tile march (2 s);
                                 see vklb_selftest_wait_timeout */
  VKLB_ERR_STATE = -7,        /* call out of order (e.g. stepping before vklb_set_state) */
  VKLB_ERR_UNSUPPORTED = -8,  /* combination not built (e.g. D1Q3 with MHD-GLM) */
  VKLB_ERR_LIMIT = -9         /* beyond the fixed scratch of vklb_conservation_totals_noalloc */
} vklb_status;

/* Hyperbolic system (Sec. 2.1).  gamma: ideal-gas index (Euler, MHD-GLM);
 * g: gravity (shallow water); ch_factor: c_h = ch_factor * max c_f for the GLM
 * cleaning speed (Sec. 5.3, the paper uses 6); adv_speed: (a_x, a_y) for
 * scalar advection. */
typedef enum { VKLB_ADVECT = 0, VKLB_SWE = 1, VKLB_EULER = 2, VKLB_MHD_GLM = 3 } vklb_system_kind;
typedef struct {
  int32_t kind;
  double gamma;
  double g;
  double ch_factor;
  double adv_speed[2];
} vklb_system;

/* Lattices: D1Q3 (Sec. 2.2, Fig. 1) and D2Q5 (Sec. 3.4, Eq. 38). */
typedef enum { VKLB_D1Q3 = 13, VKLB_D2Q5 = 25 } vklb_lattice;

/* Uniform grid: n cells per dimension on [lo, hi]; cell centres
 * x_i = lo + (i + 1/2) dx.  D2Q5 needs dx == dy (Sec. 3.4). */
typedef struct {
  int32_t dim;
  int64_t n[2];
  double lo[2];
  double hi[2];
} vklb_grid;

/* Boundary kinds per side: periodic (Eq. 37), characteristic /
 * non-reflecting (Eqs. 33-36), or transmissive (zero-order extrapolation, the
 * textbook outflow condition: a boundary node takes U_b^{n+1} = U^{n+1} of the
 * node one cell inwards along each non-periodic face it lies on, a 2D corner
 * its diagonal neighbour, and f^eq(U_b^{n+1}) with xi_{n+1} as its
 * distributions).  1D: both ends alike.  2D (D2Q5): per axis, lo[i] == hi[i],
 * and the non-periodic axes all of one kind (VKLB_ERR_ARG otherwise); a
 * characteristic axis applies the 1D construction of
 * Eqs. 33-35 along the normal of its two faces (the paper writes it for D1Q3
 * only): a boundary node takes U_b^{n+1} = U_b^n - (1/xi_n) P Lambda^out P^-1 D U^n
 * with the one-sided difference D towards the interior, a corner sums its two
 * faces, and its distributions become f^eq(U_b^{n+1}) with xi_{n+1} (Eq. 36).
 * Non-periodic 2D faces (either kind) are built for every system (MHD-GLM:
 * the nine waves of its Jacobian, c_h of step n; the paper itself runs MHD-GLM
 * on periodic grids only), with the plain step kernel in the distribution
 * form, outside batches; they need 3 or more cells across. */
typedef enum { VKLB_BC_PERIODIC = 0, VKLB_BC_CHARACTERISTIC = 1, VKLB_BC_TRANSMISSIVE = 2 } vklb_bc_kind;
typedef struct {
  int32_t lo[2];
  int32_t hi[2];
} vklb_bc;

/* Equilibrium set (Sec. 2.2 / 3.1): weighted upwind (Eqs. 22-27, parameters c and
 * k), centered flux (Eqs. 8-10, 39: c = 1/Q, F+- = F/2) or discontinuous upwind
 * (Eqs. 12-18: c = 0, Heaviside weights).  omega: relaxation in (0, 2]
 * (Sec. 2.3); cfl: nu of Eq. (29).  The paper uses c = 0.05, k = 2, nu = 0.9
 * (Sec. 5).  eta: 0 for the CFL rule; in (0, 1) the lattice speed follows the
 * centered set's subcharacteristic condition instead (Sec. 2.3),
 * xi = sqrt(3/2) max_j |lambda_j| / eta, as the paper runs the centered set
 * (eta = 0.9, Sec. 5); cfl is then not used.
 * alpha_norm: the normaliser max_j |lambda_j| of the sigmoid weight (Eq. 27),
 * which the paper does not place.  VKLB_ALPHA_GLOBAL (0, the default of a
 * zero-initialised struct) takes, for every cell of a step, the grid-wide
 * maximum over cells, directions and eigenvalues of the state being split (the
 * quantity Eq. 29 divides by nu; with +-c_h for MHD-GLM), independent of eta,
 * a fixed dt or the landing rule of vklb_step_to; it reproduces the paper's
 * omega = 2 vortex convergence (Sec. 5.2, N up to 1024) and its Table 1 dam
 * break at CFL 0.9 up to N = 4096 (Sec. 5.1).  VKLB_ALPHA_LOCAL (1) takes it
 * per cell and direction.  Only the weighted set uses it. */
typedef enum { VKLB_SET_WEIGHTED = 0, VKLB_SET_CENTERED = 1, VKLB_SET_DISCONTINUOUS = 2 } vklb_set;
typedef enum { VKLB_ALPHA_GLOBAL = 0, VKLB_ALPHA_LOCAL = 1 } vklb_alpha_norm;
typedef struct {
  int32_t set;
  double c;
  double k;
  double omega;
  double cfl;
  double eta;
  int32_t alpha_norm;
} vklb_weight;

/* Arithmetic: FP64 everywhere; FP32 distributions and arithmetic (conservation
 * totals still reduce in FP64); BF16 storage of the distributions with FP32
 * arithmetic (an explicit experiment: half the bytes, lower accuracy). */
typedef enum { VKLB_FP64 = 0, VKLB_FP32 = 1, VKLB_BF16_STORE = 2 } vklb_precision;

typedef struct vklb_sim vklb_sim;
typedef struct vklb_batch vklb_batch;

/* Static facts about a simulation (filled by vklb_info). */
typedef struct {
  int32_t p;                 /* conserved fields */
  int32_t q;                 /* lattice velocities (3 or 5) */
  int32_t precision;         /* vklb_precision */
  int32_t store_bytes;       /* bytes per stored distribution value */
  int64_t cells;             /* nx * ny */
  int64_t bytes_per_lup;     /* algorithmic bytes per cell update: 2 * q * p * store_bytes
                                (moment form: 2 * p * store_bytes) */
  int64_t state_bytes;       /* bytes of one state buffer (distributions, or moments) */
  double dx;
  int32_t tile_x, tile_y;    /* launch shape of the step kernel */
  int32_t kernels_per_step;  /* kernel launches one vklb_step(1) makes */
  int32_t variant;           /* step kernel: 0 plain loads, 1 bulk-copy (TMA) row pipeline */
  int64_t pitch;             /* cells per padded row of the device layout (>= nx; 2D: a multiple of 32) */
  int32_t blocks_per_sm;     /* 2D: resident blocks per SM of the step kernel at this launch shape
                                (CUDA occupancy calculator); 1D: 0 */
  int32_t sms;               /* SMs of the current device */
  int32_t form;              /* 0: distributions are the state; 1: moments (vklb_set_form) */
} vklb_info_t;

/* Create a simulation.  dt > 0 fixes xi = dx / dt for every step; dt <= 0
 * selects the adaptive CFL rule of Eq. (29).  cuda_stream is a cudaStream_t
 * (NULL: the legacy default stream) on which every kernel of this simulation
 * runs.  Parameter checks (returning VKLB_ERR_ARG): omega in (0, 2]
 * (Sec. 2.3); 0 < cfl <= 1 (Eq. 28); eta = 0 or 0 < eta < 1 (Sec. 2.3);
 * alpha_norm one of vklb_alpha_norm; dx == dy for D2Q5 (Sec. 3.4); lattice
 * matches grid->dim; boundary kinds as above (VKLB_ERR_UNSUPPORTED for the
 * combinations not built).  On success
 * *out owns two device distribution buffers of q * p * cells values each. */
int vklb_create(const vklb_system* sys, int32_t lattice, const vklb_grid* grid,
                const vklb_bc* bc, const vklb_weight* weight, double dt,
                int32_t precision, void* cuda_stream, vklb_sim** out);

/* Like vklb_create, but the two distribution buffers are the caller's: device
 * allocations (for example framework tensors) that the simulation borrows and
 * never frees, f_buf[0] and f_buf[1], each of buf_bytes >= vklb_buffer_bytes
 * bytes, 256-byte aligned, not overlapping, and alive until vklb_destroy
 * returns.  The simulation writes zeros into both when it is created and then
 * owns their contents (layout: vklb_device_state).  Everything else is
 * allocated and owned as by vklb_create.  VKLB_ERR_ARG for a null, misaligned,
 * overlapping or short buffer (checked before any device call);
 * vklb_set_form then returns VKLB_ERR_UNSUPPORTED (the moment form needs
 * buffers of another size). */
int vklb_create_borrowed(const vklb_system* sys, int32_t lattice, const vklb_grid* grid,
                         const vklb_bc* bc, const vklb_weight* weight, double dt,
                         int32_t precision, void* cuda_stream, void* const f_buf[2],
                         size_t buf_bytes, vklb_sim** out);

/* Bytes of one distribution buffer of a simulation of this system kind,
 * lattice, grid and precision: q * p values a cell of the padded grid
 * (rows padded to whole 32-cell bricks in 2D) times the store size. */
int vklb_buffer_bytes(int32_t system_kind, int32_t lattice, const vklb_grid* grid, int32_t precision,
                      size_t* bytes);

/* Set U(x, 0) (layout above; host pointer if on_device == 0, else device).
 * Initialises as Fig. 5: xi_0 from Eq. (29) over U (and c_h for MHD-GLM), then
 * f_q = f_q^eq(U) (Eq. 2b); t = 0, steps = 0.  Enqueued on the stream; the
 * host buffer may be reused when the call returns. */
int vklb_set_state(vklb_sim* sim, const double* U, int32_t on_device);

/* Launch shape of the step kernel (tile_x cells along x by tile_y rows per
 * block): tile_x a multiple of 32 in 32..256, tile_y in 1..256; 0 takes the
 * built-in default (128, then the wave-fit height; also the shape a new 2D
 * simulation starts with).  tile_y = -1 (2D only) picks the height that
 * makes the grid fill whole waves of resident blocks (SM count x blocks per SM
 * of the kernel this tile_x and variant launch, from the CUDA occupancy
 * calculator, on the current device), in as few waves as keep tile_y <= 256.
 * The resolved shape is reported by vklb_info.  ERR_ARG for a shape outside
 * these ranges or whose shared memory does not fit.  Used by the autotuner. */
int vklb_set_tiling(vklb_sim* sim, int32_t tile_x, int32_t tile_y);

/* Step-kernel variant for D2Q5: 0 = plain coalesced loads, rows exchanged
 * through shared memory with one block barrier per row; 1 = rows streamed into
 * shared memory by bulk asynchronous copies (TMA) with `stages` rows in flight
 * (2..8).  Both compute the same arithmetic.  Default: 0 (4 stages kept for
 * 1).  ERR_ARG for an unknown variant, a stage count outside 2..8 or a tiling
 * whose shared memory does not fit; ERR_UNSUPPORTED for variant 1 on a 1D
 * grid, in the moment form or with characteristic faces. */
int vklb_set_variant(vklb_sim* sim, int32_t variant, int32_t stages);

/* State form.  0 (default): the 5p distributions of Eq. (38)-(43) are the
 * state.  1 (D2Q5, omega == 1 only): the p moments U are the state.  At
 * omega = 1 the collision (Eq. 42) leaves f* = f^eq(U) (Eq. 41), so the step
 * is the finite-volume update of Thm 4.3, U^{n+1}(x) = sum_q f^eq_q(U^n(x - v_q)),
 * and storing U moves 2p instead of 10p values a cell.  Both forms run the same
 * march and the same arithmetic from U (form 0 relaxes to f^eq exactly at
 * omega = 1), so form 1's U after every step equals the sum
 * ((((f1 + f2) + f3) + f4) + f5) of form 0's stored distributions up to
 * rounding (the compiler may fuse multiply-adds differently in the two
 * kernels), not bit for bit.  The
 * initial U is that sum of f^eq(U_0).  Reallocates the device buffers (p components a cell for form
 * 1) and resets the launch shape to the default; the state must be set again
 * (VKLB_ERR_STATE until then).  Errors: VKLB_ERR_ARG for omega != 1 or an
 * unknown form; VKLB_ERR_UNSUPPORTED on a 1D grid or with the bulk-copy variant
 * (which form 1 does not use); VKLB_ERR_NOMEM. */
int vklb_set_form(vklb_sim* sim, int32_t form);

/* Enqueue n steps of Fig. 5 (no host synchronisation). */
int vklb_step(vklb_sim* sim, int64_t n);

/* Step until t == t_end: every step takes xi_eff = m dx / (t_end - t) with m
 * the number of CFL-limited steps left, so the last step ends on t_end.
 * Synchronises a few times to read t. */
int vklb_step_to(vklb_sim* sim, double t_end);

/* Wait for the stream and return the latched device error (VKLB_OK if none). */
int vklb_sync(vklb_sim* sim);

/* U = sum_q f_q (Eq. 3) in the layout above, as double, into a host (on_device
 * == 0) or device buffer of p * cells values.  Synchronises. */
int vklb_moments(vklb_sim* sim, double* U_out, int32_t on_device);

/* totals[k] = sum_x U_k(x) dx^D in FP64 with a fixed reduction order
 * (deterministic), host buffer of p values.  Conserved to rounding on periodic
 * grids (Thm 4.3).  Synchronises. */
int vklb_conservation_totals(vklb_sim* sim, double* totals);

/* Current time, steps taken and the lattice speed of the next step.  Synchronises. */
int vklb_time(vklb_sim* sim, double* t, int64_t* steps, double* xi);

int vklb_info(const vklb_sim* sim, vklb_info_t* info);

/* Device pointer of the current distribution buffer in the store type of the
 * precision, pitch from vklb_info.  D1Q3: component planes,
 * f[(q * p + k) * pitch + x].  D2Q5: 32-cell bricks, component j = q * p + k of
 * cell (x, y) at f[((y * (pitch / 32) + x / 32) * 5 * p + j) * 32 + x % 32] (a
 * row of bricks holds all components of 32 neighbouring cells contiguously).
 * In the moment form (vklb_set_form) the buffer holds U instead, field k of
 * cell (x, y) at f[((y * (pitch / 32) + x / 32) * p + k) * 32 + x % 32].
 * Borrowed and read-only (a step of MHD-GLM also keeps a copy of the tiles'
 * edge columns, which writes through this pointer would leave stale); valid
 * until the next vklb_step. */
int vklb_device_state(const vklb_sim* sim, void** f_dev);

/* Checking aid (no counterpart in the paper): fill the buffer that the next
 * step writes with all-ones bytes (NaN in every precision), enqueued on the
 * simulation's stream.  After that step every cell of the grid must hold a
 * finite state again: a cell the step failed to write stays NaN and shows in
 * vklb_moments.  Cells of the row padding (x >= nx) are never written or read. */
int vklb_poison_next(vklb_sim* sim);

/* Checkpoint / resume: the blob holds the device state (distributions, or U in
 * the moment form) and the control words (t, steps, xi, c_h).  A blob loads
 * only into a simulation of the same system, grid, precision and form.
 * vklb_state_bytes gives its size; get synchronises. */
int vklb_state_bytes(const vklb_sim* sim, size_t* bytes);
int vklb_get_state(vklb_sim* sim, void* blob, size_t bytes);
int vklb_put_state(vklb_sim* sim, const void* blob, size_t bytes);

int vklb_destroy(vklb_sim* sim);
const char* vklb_strerror(int status);

/* Batched form: n simulations with the same system kind, D2Q5 lattice,
 * periodic boundaries, weight and precision but any grid sizes advance together,
 * one kernel launch per step over a tile work-list spanning all of them (each
 * keeps its own xi and c_h).  The batch borrows the simulations (they must
 * outlive it); their per-simulation state is left as if each had been stepped
 * alone.  vklb_batch_step(n) enqueues n steps on the stream of the first
 * simulation; use_graph != 0 captures them in a CUDA graph and replays it.
 * VKLB_ERR_STATE if a member's state form, kernel variant or state changed
 * (vklb_set_form / vklb_set_variant) since the batch was created. */
int vklb_batch_create(int32_t n, vklb_sim* const* sims, vklb_batch** out);
/* Same ranges as vklb_set_tiling.  tile_y = -1: the members' grids differ, so
 * the height (1..64) maximises (fill of the last wave of the work-list) x
 * (tile_y / (tile_y + 2)), the share of a tile's rows that are not the
 * recomputed ring. */
int vklb_batch_set_tiling(vklb_batch* b, int32_t tile_x, int32_t tile_y);
int vklb_batch_step(vklb_batch* b, int64_t n, int32_t use_graph);
int vklb_batch_destroy(vklb_batch* b);

/* Conservation totals that allocate nothing (the paper has no counterpart: this
 * serves callers that cannot call cudaMalloc, e.g. code that only receives
 * device pointers from another runtime or runs where allocation is forbidden).
 * f_dev: a distribution buffer (form 0) in the layout of vklb_device_state, store type
 * of `precision`, q in {3, 5}, p <= 16 fields (else VKLB_ERR_LIMIT), nx x ny
 * cells with row pitch `pitch` >= nx (a multiple of 32 for q = 5).  totals[k] = cell_volume * sum_x sum_q f,
 * FP64, same reduction order as vklb_conservation_totals; `totals` is a host
 * pointer (the call synchronises the stream) or, with totals_on_device != 0, a
 * device pointer (the call returns after enqueueing).  The partial sums live in
 * one file-scope device array of 16 x 296 + 16 doubles (38 KB) that every GPU
 * loading the library keeps until the process exits; every slot a call reads is
 * written earlier in the same call, so nothing needs clearing, but calls that
 * overlap on the GPU (other streams, other host threads) race on that array.
 * The first call on a device resolves the array's address (cudaGetSymbolAddress)
 * and should come before any stream capture; that address is kept for the life
 * of the process, so a caller that tears the device's primary context down
 * (cudaDeviceReset) must not call this entry point on that device afterwards.
 * No cudaMalloc or cudaFree. */
int vklb_conservation_totals_noalloc(const void* f_dev, int32_t precision, int32_t q, int32_t p, int64_t nx,
                                     int64_t ny, int64_t pitch, double cell_volume, double* totals,
                                     int32_t totals_on_device, void* cuda_stream);

/* Number of kernel launches this process has enqueued through the library. */
int64_t vklb_launch_count(void);

/* Self-test of the device-side failure detection (no counterpart in the paper):
 * runs the bounded mbarrier wait of the bulk-copy step on a barrier that nothing
 * arrives at, with a limit of limit_ns nanoseconds (1 us .. 100 ms, else
 * VKLB_ERR_ARG), and returns what a step would: VKLB_ERR_TIMEOUT from the
 * device error word.  The wait is bounded, so the GPU and the context stay
 * usable afterwards.  Synchronises cuda_stream; allocates one control block. */
int vklb_selftest_wait_timeout(int64_t limit_ns, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* VKLB_H */
