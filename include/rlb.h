/*
 * rlb.h -- C ABI of librlb, the GB300 (sm_103a) implementation of the relativistic lattice
 * Boltzmann model with improved dissipation (Mendoza, Karlin, Succi, Herrmann, arXiv:1301.3423).
 *
 * The model (Sec. II):
 *   - one population f_i per discrete 4-momentum p_i^mu = p0_i (1, v_i / R), v_i integer with
 *     |v_i|^2 = R^2 (Eqs. (eq:dio), (eq:mrecon2)); third order: R^2 = 41, Q = 128 (Sec. II.C);
 *     second order: R^2 = 9, Q = 66 (App. A);
 *   - one time step of the time-dilated equation (Eq. (rlb:disc), delta x = delta t' = 1):
 *       f_i(x + v_i, t' + 1) = f_i(x, t') - (p_i^mu U_mu) / (tau' p0_i) (f_i - f_i^eq),
 *     with U^mu, eps, n from Landau matching T^{ab} U_b = eps U^a, n = U_mu N^mu, eps = 3 n T
 *     (Eq. (eigenproblem), Sec. II.D) and f_i^eq the projected Maxwell-Juttner equilibrium
 *     (Eq. (eq:disc1); explicit forms Eq. (eq:equi3rd), Eq. (eq:equi2nd)).
 *
 * Lattice and memory.  Cells are indexed (x, y, z) with x fastest: cell = (z * ny + y) * nx + x.
 * Field arrays passed to this ABI are double precision, structure of arrays: a scalar field is
 * double[cells], a vector field is double[components][cells].  Populations are
 * double[q][cells] at the boundary, whatever the storage precision inside.
 *
 * Conventions common to every call.
 *   - Every call returns an rlb_status and never aborts, traps or throws.
 *   - Work is enqueued on the context's CUDA stream; rlb_step returns before the GPU finishes.
 *     Kernel faults and per-cell failures (Landau matching without a timelike solution) are
 *     reported by the next synchronising call (rlb_sync, rlb_moments, rlb_get_populations).
 *   - The caller owns every buffer it passes; the library copies what it needs before returning
 *     (host buffers) or before the enqueued work completes (device buffers: keep them alive and
 *     unmodified until the next synchronising call).
 *   - A context is used by one host thread at a time.
 *   - rlb_last_error() describes the most recent failure of that context.
 */
#ifndef RLB_H
#define RLB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rlb_ctx rlb_ctx;

typedef enum {
  RLB_OK = 0,
  RLB_EINVAL = 1,   /* invalid argument or parameter (nothing was changed) */
  RLB_ENOMEM = 2,   /* device memory could not be allocated */
  RLB_ECUDA = 3,    /* a CUDA call failed; the context should be destroyed */
  RLB_ENONCONV = 4, /* Landau matching found no timelike eigenvector in some cell */
  RLB_ENAN = 5,     /* non-finite populations (found by rlb_moments) */
  RLB_ETIMEOUT = 6, /* a bounded device-side wait of the pipelined step kernel ran out; the state
                       that step produced is not valid (rlb_init or rlb_set_populations restores one) */
  RLB_ESTATE = 7    /* call not valid in the context's current state */
} rlb_status;

/* Boundary condition of one axis, applied at both ends.
 *   RLB_BC_PERIODIC  : the pull wraps around.
 *   RLB_BC_COPYOUT   : a population pulled from beyond an end is taken from the nearest edge cell.
 *   RLB_BC_BOUNCEBACK: solid walls just beyond both ends.  A population whose pull source lies
 *                      beyond a wall is the same cell's post-collision population of the reversed
 *                      momentum (same p0, -v): everything that would cross the wall comes back
 *                      reversed into the cell it left, so sum N^0 and sum T^00 are conserved and
 *                      the wall is no-slip.  The weights are equal under v -> -v for this purpose
 *                      (Sec. II.C); the paper states no rule for links longer than one cell. */
typedef enum { RLB_BC_PERIODIC = 0, RLB_BC_COPYOUT = 1, RLB_BC_BOUNCEBACK = 2 } rlb_bc;

/* Storage precision of the populations in device memory.
 *   RLB_F64   : double populations, double arithmetic.
 *   RLB_F32   : float populations, float arithmetic; Landau matching in double above gamma_thr.
 *   RLB_F16DEV: half-precision store of d_i = f_i / w_i - n_ref / 2 (the deviation from the
 *               weight-scaled rest equilibrium at density n_ref, temperature 1), float arithmetic. */
typedef enum { RLB_F64 = 0, RLB_F32 = 1, RLB_F16DEV = 2 } rlb_storage;

typedef struct {
  int order;          /* 3: third-order model, R^2 = 41, Q = 128 (Sec. II.C); 2: second order,
                         R^2 = 9, Q = 66 (App. A) */
  int nx, ny, nz;     /* lattice size in cells, each >= 1 */
  int bc[3];          /* per axis x, y, z: an rlb_bc value (periodic, copy-out or bounce-back) */
  double eta_over_s;  /* shear viscosity over entropy density; mapped to tau' by
                         tau' = 1/2 + 6 (eta/s) / (R kappa T), kappa = T_unit_GeV dx_fm / (hbar c)
                         (Sec. II.D, Sec. III), unless tau_prime > 1/2 */
  double tau_prime;   /* > 1/2: constant relaxation time in lattice units; otherwise mapped */
  int tau_local_T;    /* 1: T in the mapping is each cell's Landau temperature; 0: T_ref */
  double T_ref;       /* reference temperature in lattice units (default 1.0 = 400 MeV, Sec. III) */
  double dx_fm;       /* cell size in fm (default 0.008, Sec. III) */
  double T_unit_GeV;  /* lattice temperature unit in GeV (default 0.4, Sec. III) */
  int storage;        /* rlb_storage */
  int landau_fp64;    /* RLB_F32 / RLB_F16DEV only: 1 = solve Landau matching in double for every
                         cell (from the Eckart vector to 1e-12 U0); 0 = in float, in double for
                         cells above gamma_thr */
  double gamma_thr;   /* RLB_F32 / RLB_F16DEV only: cells whose Eckart Lorentz factor exceeds this
                         are solved in double (default 2.0) */
  double n_ref;       /* RLB_F16DEV only: reference density of the stored deviation (default 1.0) */
  int step_variant;   /* -1 = library default, or force a step-kernel variant (see rlb_autotune);
                         a variant that does not exist for the context falls back to the default */
  void* stream;       /* cudaStream_t to enqueue on; NULL = the default stream */
  int debug_flags;    /* testing only, 0 in normal use.  Bit 0: the pipelined step kernel's producer
                         warps do nothing, so its consumers' bounded waits (2 s) run out and the next
                         synchronising call reports RLB_ETIMEOUT; the context stays usable. */
  /* Optional quadrature (Sec. II.C, App. A).  When q > 0 these arrays are compared with the
   * quadrature compiled into the library for this order and must match exactly (RLB_EINVAL
   * otherwise); rlb_quadrature() returns the built-in one. */
  int q;
  const int* vel;     /* [q][3] integer velocities v_i */
  const int* level;   /* [q] energy level of each population */
  const double* p0;   /* [q] energy p0_i */
  const double* w;    /* [q] weight w_i */
} rlb_params;

/* Fill *p with the defaults above: order 3, 1x1x1 periodic, eta/s 0.1 mapped with the local
 * temperature, T_ref 1, dx 0.008 fm, T unit 0.4 GeV, RLB_F64 storage, gamma_thr 2, n_ref 1, default
 * stream, no quadrature check. */
void rlb_default_params(rlb_params* p);

/* Device bytes a context with these parameters allocates (two population buffers plus fields
 * and reduction scratch).  0 if the parameters are invalid. */
size_t rlb_bytes_required(const rlb_params* p);

/* Create a context: validate parameters, allocate two population buffers of q * cells elements
 * in the storage precision and the per-cell field and reduction buffers on the current device.
 * *out receives the handle (NULL on failure).  Errors: RLB_EINVAL, RLB_ENOMEM, RLB_ECUDA. */
rlb_status rlb_create(const rlb_params* p, rlb_ctx** out);

/* Set every population to the discrete equilibrium f_i^eq(n, T, U) (Eq. (eq:disc1)) of the given
 * fields, U = gamma (1, u): n, T double[cells], u double[3][cells] (u_x, u_y, u_z, |u| < 1).
 * on_device = 0: host pointers, read before return (page-locked arrays, e.g. from cudaHostAlloc
 * or cudaHostRegister, are read by the init kernel in place over the CPU-GPU link; pageable ones
 * are copied through a device staging buffer); 1: device pointers.  Resets the step counter to 0.  Errors: RLB_EINVAL (null pointer; invalid values are reported as RLB_EINVAL by
 * the next synchronising call), RLB_ECUDA. */
rlb_status rlb_init(rlb_ctx* ctx, const double* n, const double* T, const double* u, int on_device);

/* Enqueue nsteps >= 0 time steps of Eq. (rlb:disc): pull streaming by v_i, then Anderson-Witting
 * collision with Landau matching in every cell.  Asynchronous.  Errors: RLB_EINVAL, RLB_ECUDA. */
rlb_status rlb_step(rlb_ctx* ctx, long nsteps);

/* Landau-frame fields of the pre-collision populations of the current time level (the initial
 * populations before the first step; afterwards the populations the last step pulled): n, eps
 * double[cells], U double[4][cells] (U^0..U^3), and totals[5] = sum over cells of N^0, T^00,
 * T^0x, T^0y, T^0z (the conserved densities of Eqs. (eq:conser1), (eq:conser2)), summed in double
 * in a fixed order.  Any output pointer may be NULL.  on_device = 1: n, eps, U are device
 * pointers (totals is always host); 0: host pointers (when n, eps and U are all page-locked the
 * fields kernel writes them in place, otherwise they are copied out of a device buffer).
 * Synchronises the stream.  Errors, from this call or from
 * enqueued work since the last synchronising call: RLB_ENAN (cells whose populations are not
 * finite), RLB_ENONCONV (cells without a Landau frame, here or in a step; their fields are NaN),
 * RLB_EINVAL (invalid initial fields given to rlb_init), RLB_ETIMEOUT (a bounded device-side wait
 * of the pipelined step ran out), RLB_ECUDA. */
rlb_status rlb_moments(rlb_ctx* ctx, double* n, double* eps, double* U, double totals[5], int on_device);

/* Wait for enqueued work and report deferred errors: RLB_ENONCONV, RLB_EINVAL, RLB_ETIMEOUT,
 * RLB_ECUDA (as rlb_moments; RLB_ENAN only comes from rlb_moments, which looks at the moments). */
rlb_status rlb_sync(rlb_ctx* ctx);

/* Copy the stored (post-collision) populations out as double[q][cells].  Synchronises. */
rlb_status rlb_get_populations(rlb_ctx* ctx, double* f, int on_device);

/* Replace the stored populations by double[q][cells] values (converted to the storage precision)
 * and treat them as the initial state: the step counter is reset to 0 and rlb_moments reports
 * their own fields.  Errors: RLB_EINVAL, RLB_ECUDA. */
rlb_status rlb_set_populations(rlb_ctx* ctx, const double* f, int on_device);

/* Upper bound on the number of step-kernel variants. */
#define RLB_MAX_VARIANTS 24

/* Autotuner: time every step-kernel variant that exists for this context and keep the fastest for
 * later rlb_step calls.  Variants:
 *   0..3  one cell per thread with all populations in registers, two launches per step (rows whose
 *         y and z are interior, then the boundary rows); float and half storage only, except 0:
 *         bit 0 = scalar or mirror pairs in paired-FMA float2 arithmetic, bit 1 = 2 or 3 resident
 *         blocks per SM.  Double storage has variant 0, which reads its populations twice.
 *   4..11 the pipelined kernel, one launch per step: producer warps stage each tile's pulled
 *         populations in shared memory with bulk copies and consumer warps relax the cells from
 *         there; a tile is a 64- or 128-cell segment of a row, and the variants differ in tile
 *         width, consumer warps and producer warps per block.  Every storage; only for lattices
 *         whose nx is a multiple of 16 bytes' worth of populations (4 float, 8 half, 2 double).
 *   12..14 the pipelined kernel with row tiles: a tile is 128 / nx whole rows (one bulk copy per
 *         population and run of consecutive source rows, the periodic x wrapped in shared memory);
 *         only for lattices with a periodic x of at most 128 cells (and at least the stencil's
 *         x reach), nx again a multiple of 16 bytes' worth of populations.
 *   15..18 row segments (15, 17) and row tiles (16, 18) in three consumer groups of four warps
 *         per block, 4 (15, 16) or 2 (17, 18) producer warps; float storage relaxes each cell in
 *         one warp here instead of two.
 *   19    96-cell row tiles (rows of at most 96 cells; 96, 48 and 32 fill them), four consumer
 *         groups of three warps, one warp per float cell.
 * Each variant repeats one step from the current populations into the spare buffer `reps` times, so
 * the state does not change; this is allowed only before the first step after rlb_init /
 * rlb_set_populations (RLB_ESTATE otherwise).  *variant (may be NULL) receives the choice;
 * ms[RLB_MAX_VARIANTS] (may be NULL) the milliseconds per step of each variant (0 where a variant
 * does not exist for this context).  Synchronises the stream.
 * Errors: RLB_EINVAL (reps < 1), RLB_ESTATE, RLB_ECUDA, RLB_ETIMEOUT. */
rlb_status rlb_autotune(rlb_ctx* ctx, int reps, int* variant, double ms[RLB_MAX_VARIANTS]);

/* ---------------------------------------------------------------------------------------------
 * Batched stepping.  A batch steps many contexts of the same order and storage together: each
 * time step of Eq. (rlb:disc) is one launch of persistent kernels per kernel kind, advancing every
 * member with steps left over tiles shared by all members, so lattices of very different sizes
 * fill the GPU together.  With a register variant (0..3) every member goes through the register
 * kernels (two launches: the members' interior rows in 32-cell segments, four per tile, then their
 * boundary cells).  With a pipelined variant (4 and up) the members whose rows start on 16-byte
 * boundaries and fill enough of the tile lanes (7/8; 3/4 with one warp per float cell) go through
 * one launch of the batched pipelined kernel over their row segments.  With a row-tile variant
 * the members with a periodic x whose row tiles use at least 3/4 of the lanes go through a launch
 * of the row-tile kernel (with two warps per float cell only those whose rows do not fill segment
 * tiles), members that fill a 96-cell row tile better than a 128-cell one through a launch of the
 * 96-cell row-tile kernel with the same warps (variant 19 beside 16), and the other pipelined
 * members through the row-segment kernel of the same block layout.  The others (e.g. 1 x 1 x N
 * tubes) run through the register kernels with the variant a context of that storage runs when it
 * has no pipelined one (3 float, 2 half, 0 double; see rlb_batch_member_variant).  Members keep
 * their own buffers, parameters, status and step counters; a member's populations after a batched
 * run are bitwise those of the same steps taken alone with the same step-kernel variant.  Members
 * must use the batch's stream.
 * ------------------------------------------------------------------------------------------- */
typedef struct rlb_batch rlb_batch;

/* Create an empty batch for order 2/3 and storage RLB_F64/F32/F16DEV on the current device,
 * enqueuing on `stream` (NULL: default stream).  Errors: RLB_EINVAL, RLB_ENOMEM, RLB_ECUDA. */
rlb_status rlb_batch_create(int order, int storage, void* stream, rlb_batch** out);

/* Add ctx as a member that is to take `steps` more steps; *slot (may be NULL) receives its slot.
 * The batch does not own the context; keep it alive while it is a member.  Errors: RLB_EINVAL
 * (order / storage mismatch, already a member, steps < 0). */
rlb_status rlb_batch_add(rlb_batch* b, rlb_ctx* ctx, long steps, int* slot);

/* Remove the member in `slot`; its context keeps its state.  Errors: RLB_EINVAL. */
rlb_status rlb_batch_remove(rlb_batch* b, int slot);

/* Steps the member in `slot` still has to take (-1 for an empty slot). */
long rlb_batch_steps_left(const rlb_batch* b, int slot);

/* Enqueue up to nsteps steps: launch k advances every member with more than k steps left, so each
 * member stops at its own count.  use_graph = 1 captures the nsteps launches once as a CUDA graph
 * and replays it while the member set and nsteps are unchanged.  *active (may be NULL) receives the
 * number of members with steps left afterwards.  Asynchronous; member failures are reported by the
 * members' own synchronising calls.  Errors: RLB_EINVAL, RLB_ENOMEM, RLB_ECUDA. */
rlb_status rlb_batch_run(rlb_batch* b, long nsteps, int use_graph, int* active);

/* Autotuner for the batch: time every step-kernel variant of the batched kernel on the current
 * members (each repetition recomputes the members' next state into their spare buffers, so no
 * state changes; allowed only while no member has taken a step, RLB_ESTATE otherwise) and keep the
 * fastest.  *variant and ms[RLB_MAX_VARIANTS] as for rlb_autotune. */
rlb_status rlb_batch_autotune(rlb_batch* b, int reps, int* variant, double ms[RLB_MAX_VARIANTS]);

/* Force the batch's step variant (numbered as for rlb_autotune; see above for how members are
 * split between kernels).  Errors: RLB_EINVAL for a variant the batch's storage does not have. */
rlb_status rlb_batch_set_variant(rlb_batch* b, int variant);

/* The step-kernel variant the batch runs the member in `slot` with, under the batch's current
 * variant: the batch's own; the 96-cell row-tile variant for a member that runs in those beside a
 * 128-cell row-tile variant; for a row-tile variant and a member that runs in row segments, the
 * row-segment variant of the same block layout; for a pipelined variant and a member whose rows do
 * not suit the tiles, the register fallback (3 float, 2 half, 0 double).  Running that member
 * alone with this variant gives the same populations bitwise.  -1 for an empty slot or NULL. */
int rlb_batch_member_variant(const rlb_batch* b, int slot);

/* Kernel launches the batch has enqueued (-1 for NULL). */
long rlb_batch_kernel_launches(const rlb_batch* b);

/* Text of the batch's most recent error. */
const char* rlb_batch_last_error(const rlb_batch* b);

/* Release the batch (not its members' contexts).  Synchronises its stream.  NULL is accepted. */
rlb_status rlb_batch_destroy(rlb_batch* b);

/* The step-kernel variant rlb_step uses (see rlb_autotune; -1 for NULL): the one rlb_params asked
 * for if it exists for this context, else the library default, or the autotuner's choice. */
int rlb_step_variant(const rlb_ctx* ctx);

/* Number of time steps taken since rlb_init / rlb_set_populations (-1 for NULL). */
long rlb_steps_done(const rlb_ctx* ctx);

/* Kernel launches this context has enqueued since creation (-1 for NULL). */
long rlb_kernel_launches(const rlb_ctx* ctx);

/* Release the context's device memory.  NULL is accepted.  Synchronises the stream. */
rlb_status rlb_destroy(rlb_ctx* ctx);

/* Text of the context's most recent error ("" if none).  Valid until the next call on ctx.
 * With ctx == NULL: the most recent failure of a call without a context (rlb_create,
 * rlb_totals_noalloc) on the calling thread. */
const char* rlb_last_error(const rlb_ctx* ctx);

/* Largest lattice rlb_totals_noalloc accepts: 65536 blocks of 128 cells. */
#define RLB_NOALLOC_MAX_CELLS 8388608

/* Conserved totals of a caller-owned population buffer, computed without allocating anything.
 * The paper has no counterpart.  It exists for callers that cannot call the device allocator:
 * plug-ins whose host application owns every device allocation, processes whose memory pools
 * already hold the whole device, and code that runs under a hard memory budget in which an
 * allocation by a library would fail or break the budget.
 *
 * f is a device buffer of q * nx * ny * nz populations in the layout and precision of `storage`
 * (the layout of the context buffers: [q][cells], x fastest; RLB_F16DEV stores f_i / w_i - n_ref/2).
 * totals[5] (host) receives sum over cells of N^0, T^00, T^0x, T^0y, T^0z of these populations,
 * the same sums rlb_moments reports before the first step.  The call enqueues two kernels on
 * `stream` (NULL: default stream), copies the 5 sums to totals and synchronises the stream.
 *
 * Scratch: a fixed device array inside the library (RLB_NOALLOC_MAX_CELLS / 128 * 5 + 5 doubles,
 * about 2.6 MB) that every device loading the library holds until the process exits.  No
 * cudaMalloc, cudaFree or other allocating routine is called ("no allocation" means exactly
 * that; the call still copies the 5 sums to host memory and synchronises the stream).  The first
 * call on a device looks up that array's device address, with the device current; make that first
 * call before any stream capture.  Every call shares the array: calls whose work overlaps on the
 * GPU (other streams, other host threads) race and must be serialised by the caller.  Nothing in
 * it needs to start at zero: every slot a call reads, the same call has written.
 *
 * Errors: RLB_EINVAL (order, storage, null pointer, empty lattice, or more than
 * RLB_NOALLOC_MAX_CELLS cells; rlb_last_error(NULL) explains), RLB_ECUDA. */
rlb_status rlb_totals_noalloc(int order, int storage, int nx, int ny, int nz, double n_ref, const void* f,
                              double totals[5], void* stream);

/* The quadrature built into the library for order 2 or 3 (Sec. II.C, App. A): q populations with
 * velocities vel[q][3], energy levels, energies p0 and weights w.  The arrays are static and owned
 * by the library.  Host-only; needs no GPU.  Errors: RLB_EINVAL for other orders. */
rlb_status rlb_quadrature(int order, int* q, const int** vel, const int** level, const double** p0,
                          const double** w);

#ifdef __cplusplus
}
#endif

#endif /* RLB_H */
