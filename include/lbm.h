/*
 * lbm.h -- C-ABI of the GB300 lattice Boltzmann library implementing the
 * Galilean-invariant filtered collision of Chen, Zhang & Gopalakrishnan,
 * "Filtered lattice Boltzmann collision formulation enforcing isotropy and
 * Galilean invariance" (arXiv 2002.02503).
 *
 * The state is a set of particle distributions f_i(x, t) on a periodic
 * Cartesian lattice (Sec. 1, Eq. lbe).  One step applies the filtered collision
 * of Eq. lbe-reg with the truncated Galilean-invariant non-equilibrium part of
 * Eq. hermite-coll (closed forms Eq. filter-Pi, filter-1st, filter-2nd) and the
 * truncated equilibrium of Eq. hermite, then streams every f_i one link along
 * c_i (Eq. lbe).  The observables are rho and u of Eq. mme.
 *
 * Conventions shared by every call
 *   - dims = {nx, ny, nz}; D2Q9 requires nz == 1.  Cell index = x + nx*(y + ny*z).
 *   - Density fields are double[C]; velocity fields are double[D][C] (SoA).
 *   - Distributions exchanged as double are [Q][C] in the library's velocity
 *     order (lbm_lattice_info): index 0 is the rest velocity, then pairs
 *     (2p+1, 2p+2) with c_{2p+2} = -c_{2p+1}.
 *   - lbm_mem says whether a pointer is host memory (pageable or pinned) or
 *     device memory of the solver's device.
 *   - Every call returns an lbm_status; none throws, aborts or exits.  On an
 *     error, lbm_last_error() holds a message for the calling thread.
 *   - The calls that do host-visible work mark it with NVTX ranges named after the
 *     call (for timeline profilers; no cost beyond a branch without one).
 *   - The library makes no device-memory allocation: the caller owns the
 *     workspace, the pool arena and every buffer.  It creates CUDA streams,
 *     events and graphs for its own scheduling, pinned host memory for a pool's
 *     slot tables, and holds one fixed 128 KiB device array (see
 *     lbm_conservation_noalloc).
 *   - A solver is not thread-safe: calls on one solver must not overlap; distinct
 *     solvers are independent.  A pool serialises its own calls internally.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LBM_OK = 0,
    LBM_ERR_INVALID_ARG = 1,   /* a NULL pointer, a size out of range, tau <= 1/2 ... */
    LBM_ERR_UNSUPPORTED = 2,   /* truncation order outside [2, 2N-1] for the lattice, unknown storage */
    LBM_ERR_OUT_OF_MEMORY = 3, /* workspace or pool too small for the request */
    LBM_ERR_CUDA = 4,          /* a CUDA runtime call failed (message in lbm_last_error) */
    LBM_ERR_NONFINITE = 5,     /* a reduction met NaN or Inf: the run has gone unstable */
    LBM_ERR_TIMEOUT = 6,       /* a bounded device-side wait gave up */
    LBM_ERR_BUSY = 7,          /* no free slot or memory in a pool right now */
    LBM_ERR_NOT_FOUND = 8,     /* unknown request id */
    LBM_ERR_RANGE = 9,         /* a value left the range of the fixed-point storage (or was not
                                  finite); the stored state is no longer valid */
    LBM_ERR_BOUNDS = 10        /* only in the bounds-check build (lbm_bounds_checked() == 1): a
                                  kernel computed an index outside its buffer; the access was
                                  skipped, the stored state is not valid */
} lbm_status;

/* Velocity sets.  D2Q9, D3Q15, D3Q19: isotropy class 2N = 4, T0 = 1/3 (Sec. 2
 * after Eq. iso); D3Q39: 2N = 6, T0 = 2/3; D3Q27 (not in the paper): 2N = 4, T0 = 1/3. */
typedef enum { LBM_D2Q9 = 0, LBM_D3Q19 = 1, LBM_D3Q27 = 2, LBM_D3Q39 = 3, LBM_D3Q15 = 4 } lbm_lattice;

/* How distributions are stored in HBM.  The collision always computes in FP32
 * (FP64 for LBM_STORE_F64).  Every form stores the shifted, scaled value
 * h_i = (g_i - w_i rho0) / w_i, rounded to nearest (even) in the storage type.
 * LBM_STORE_Q16 is 16-bit fixed point: h = q * R / 2^15 with the integer q in
 * [-32768, 32767] (stored as q + 2^15) and the range R a power of two
 * (lbm_set_storage_range; default 1).
 * Its grid step is uniform, where FP16's grows with |h|, so for flows whose |h|
 * stays below R/2 it rounds 4-16 times finer than FP16 at the same two bytes.  A
 * value outside [-R, R) (or not finite) is not stored faithfully: the step records it
 * and the next synchronising call returns LBM_ERR_RANGE.  Q16 runs on the register
 * pull step (variant 0, every cells_per_thread, BGK and the energy-flux term) and in
 * pools (lbm_pool_set_storage_range); the staged variant and lbm_conservation_noalloc
 * reject it (LBM_ERR_UNSUPPORTED).
 * LBM_STORE_F16_REF and LBM_STORE_BF16_REF store, beside the Q distribution planes, D
 * planes of a per-cell reference velocity a = u / T0 (the cell's velocity after its
 * collision, rounded to the storage type), and in place of h_i the residual
 * h_i - r_i, r_i = s + s^2/2 with s = c_i . a, rounded to FP16 or BF16.  The reader adds
 * r_i of the cell that wrote the value back in FP32, so only the residual is rounded: its
 * size is that of (rho - rho0), rho |u|^2 / (2 T0), the higher orders and the
 * non-equilibrium part, not of c_i . u / T0, and the rounding error shrinks by the same
 * factor.  Per cell update they move
 * 2 (Q + D) x 2 bytes (D3Q19: 88 against 76 for FP16 and 152 for FP32).  They run on
 * the register-pull step (variant 0, every cells_per_thread, BGK and the energy-flux
 * term); the staged and flat-pair variants, pools and lbm_conservation_noalloc reject
 * them (LBM_ERR_UNSUPPORTED). */
typedef enum {
    LBM_STORE_F32 = 0,
    LBM_STORE_F16 = 1,
    LBM_STORE_BF16 = 2,
    LBM_STORE_F64 = 3,
    LBM_STORE_Q16 = 4,
    LBM_STORE_F16_REF = 5,
    LBM_STORE_BF16_REF = 6
} lbm_storage;

typedef enum { LBM_MEM_HOST = 0, LBM_MEM_DEVICE = 1 } lbm_mem;

typedef struct lbm_solver lbm_solver; /* opaque; owned by the library */

/* Velocity table of a lattice.  Any output pointer may be NULL.  c: int[Q*3]
 * (z component 0 for D2Q9), w: double[Q].  kmax = 2N - 1, the highest
 * truncation order the lattice supports (Sec. 2 truncation rule, Sec. 3). */
lbm_status lbm_lattice_info(lbm_lattice lattice, int *D, int *Q, int *c, double *w, double *T0, int *kmax);

/* Bytes of device workspace lbm_create needs: two distribution buffers of
 * Q*C values of the storage type (Q+D planes of C values for the forms with a
 * reference velocity; pull streaming ping-pongs between them) plus a small
 * reduction area.  Returns 0 for invalid arguments. */
size_t lbm_workspace_bytes(lbm_lattice lattice, const int64_t dims[3], lbm_storage storage);

/* Create a solver for a periodic lattice (Eq. lbe, Eq. lbe-reg).
 *   tau               relaxation time, > 1/2 (Eq. post-1); viscosity T0 (tau - 1/2)
 *   truncation_order  K, the highest Hermite order kept in BOTH Eq. hermite and
 *                     Eq. hermite-coll; 2 <= K <= 2N-1 of the lattice.  K = 2 is the
 *                     prior filtered form (Eq. filter-Pi), K = 3 Eq. filter-1st,
 *                     K = 4 Eq. filter-2nd, K = 5 the next term of Eq. hermite-coll.
 *   rho0              reference density of the storage shift (> 0)
 *   device_workspace  caller-owned device memory of at least lbm_workspace_bytes,
 *                     256-byte aligned; it must outlive the solver.
 *   cuda_stream       cudaStream_t for all device work (NULL = legacy default stream)
 * Validation happens before any device work.  The distributions are undefined
 * until lbm_set_fields or lbm_set_distributions. */
lbm_status lbm_create(lbm_lattice lattice, const int64_t dims[3], double tau, int truncation_order,
                      lbm_storage storage, double rho0, void *device_workspace, size_t workspace_bytes,
                      void *cuda_stream, lbm_solver **out);

/* Set f_i(x, 0) = f^eq_i(rho(x), u(x)) truncated at K (Eq. hermite) and t = 0.
 * rho: double[C], u: double[D][C].  Host inputs are staged through the idle
 * distribution buffer; the call returns once the data has been consumed. */
lbm_status lbm_set_fields(lbm_solver *s, const double *rho, const double *u, lbm_mem mem);

/* Advance n >= 0 steps of pull-streaming + collision (Eq. lbe-reg).  Asynchronous
 * on the solver's stream; no host synchronisation. */
lbm_status lbm_step(lbm_solver *s, int64_t n);

/* rho(x, t) and u(x, t) of the pre-collision distributions at the current t
 * (Eq. mme).  Either pointer may be NULL.  Synchronises the stream. */
lbm_status lbm_get_moments(lbm_solver *s, double *rho, double *u, lbm_mem mem);

/* The pre-collision distributions f_i(x, t) as double[Q][C] (library velocity
 * order).  Synchronises the stream. */
lbm_status lbm_get_f(lbm_solver *s, double *f, lbm_mem mem);

/* Global FP64 sums over the lattice: out = {sum rho, sum rho u_x, sum rho u_y,
 * sum rho u_z} (Eq. inv summed over x: constant in time up to rounding).
 * Host output; synchronises.  LBM_ERR_NONFINITE if any sum is NaN/Inf. */
lbm_status lbm_conservation(lbm_solver *s, double out[4]);

/* Fourier amplitude of one velocity component at integer wave vector k:
 * out = {Re, Im} of sum_x u_comp(x) exp(-2 pi i (kx x/nx + ky y/ny + kz z/nz)),
 * accumulated in FP64.  Host output; synchronises. */
lbm_status lbm_mode_amplitude(lbm_solver *s, const int64_t k[3], int component, double out[2]);

/* Checkpoint: the raw stored distributions (bytes = Q*C*sizeof(storage); (Q+D)*C*2
 * for the forms with a reference velocity, whose planes follow the Q distribution
 * planes) and the step counter.  get synchronises and, like the other synchronising calls, first
 * reports a pending status (LBM_ERR_RANGE, LBM_ERR_TIMEOUT) instead of saving a state known
 * to be invalid; set replaces the state and clears any pending status of the old one (so
 * does lbm_set_fields).  A fixed-point checkpoint restores under the range and reference shift
 * it was taken with (the stored codes carry neither). */
lbm_status lbm_get_distributions(lbm_solver *s, void *dst, size_t bytes, lbm_mem mem, int64_t *t);
lbm_status lbm_set_distributions(lbm_solver *s, const void *src, size_t bytes, lbm_mem mem, int64_t t);

/* Current step counter t. */
lbm_status lbm_time(const lbm_solver *s, int64_t *t);

/* Kernel configuration of the step.  variant: 0 = register pull (vector loads
 * plus warp shuffles for the x shift; cells_per_thread 1, 2, 4 or 8 x-neighbours, which
 * must divide nx), 1 = persistent shared-memory row staging through bulk asynchronous
 * copies (cells_per_thread 1), 2 = two consecutive cells of the flat index per thread with
 * direct loads (cells_per_thread 2, any nx: the paired collision for odd nx).  The
 * collision runs on the paired FP32 instructions whenever a thread holds two or more cells.
 * block_threads: 32..1024, a multiple of 32.  A negative variant and a zero
 * cells_per_thread or block_threads keep the current setting.  LBM_ERR_UNSUPPORTED if the
 * combination is not built (BGK and the energy-flux term run variant 0 with one cell). */
lbm_status lbm_set_kernel(lbm_solver *s, int variant, int cells_per_thread, int block_threads);
lbm_status lbm_get_kernel(const lbm_solver *s, int *variant, int *cells_per_thread, int *block_threads);

/* Collision operator of the step.  LBM_COLLISION_FILTERED_GI (the default) is
 * the paper's filtered collision, Eq. lbe-reg with the truncated Eq. hermite-coll.
 * LBM_COLLISION_BGK is Eq. BGK, C_i = -(f_i - f^eq_i)/tau, with the same truncated
 * f^eq: the unfiltered comparison baseline of Sec. 1 and Sec. 4 (it relaxes every
 * non-equilibrium moment, including those the lattice does not support).  The BGK
 * step runs one cell per thread; selecting it resets the kernel configuration. */
typedef enum { LBM_COLLISION_FILTERED_GI = 0, LBM_COLLISION_BGK = 1 } lbm_collision;
lbm_status lbm_set_collision(lbm_solver *s, lbm_collision model);

/* Energy-flux term (Sec. 4, Eq. pq): fhat^neq = fhat^{neq,p} + theta fhat^{neq,q}, with
 * fhat^{neq,q} the Hermite series of Eq. filter-Q (the relative-frame flux Qt of
 * Eq. Q_def) truncated at the solver's K, so theta needs K >= 3.  theta = 0 (the
 * default) is the paper's Sec. 3 collision.  Applies to the filtered collision;
 * runs one cell per thread.  LBM_ERR_UNSUPPORTED for K = 2. */
lbm_status lbm_set_energy_flux(lbm_solver *s, double theta);

/* Range R of the fixed-point storage (LBM_STORE_Q16): -R <= h_i < R, grid step d = R / 2^15.
 * A value is stored as its nearest grid point (ties to an even code); one whose nearest point
 * does not fit -- at or above R - d/2, or below -R - d/4 (where FP32 rounds at d/2) -- is
 * reported as out of range.
 * R must be a power of two in [2^-8, 2^8], or 0 for an automatic range: each later
 * lbm_set_fields first measures max |h| of the initial f^eq on the device and takes the
 * smallest power of two R >= 1.25 max |h| (read it back with lbm_get_storage_range); a later
 * exit from that range is reported as usual.  A nonzero R turns the automatic choice off.
 * The stored codes are not converted, so set R before lbm_set_fields or
 * lbm_set_distributions (a checkpoint restores with the range it was taken with).  |h_i| is about |c_i . u| / T0 plus the density excursion
 * rho - rho0 and the non-equilibrium part, so R = 1/4 holds flows with |c_i . u| up to
 * about 0.07 on the T0 = 1/3 lattices.  LBM_ERR_UNSUPPORTED for the floating forms. */
lbm_status lbm_set_storage_range(lbm_solver *s, double range);
lbm_status lbm_get_storage_range(const lbm_solver *s, double *range);

/* Reference shift of the fixed-point storage (LBM_STORE_Q16): the stored value of velocity i
 * becomes h_i - href_i, with href_i = rho0 (s_i + (s_i^2 - |U|^2/T0) / 2), s_i = c_i.U / T0,
 * the scaled equilibrium at the reference velocity U (Eq. hermite truncated at second order;
 * rounded to the grid, so decode adds back exactly what encode takes off).  The shift is a
 * storage device with no counterpart in the paper.  The shifted codec holds one constant per velocity, so
 * it runs its own kernels, used only while a shift is set; unshifted solvers keep the
 * kernels with one constant for every velocity.  For a flow near a uniform U -- a wave on a
 * background flow -- the stored values, and with them the automatic range and the rounding
 * step, shrink by the background's share.  U = {0, 0, 0} (the default) turns it off;
 * |U| <= 1/2; on D2Q9 U[2] is ignored.  Set it before lbm_set_fields; the range is
 * raised if needed so that every shift stays below 2^22 grid steps.  LBM_ERR_INVALID_ARG for
 * a NULL U, a non-finite component or |U| > 1/2; LBM_ERR_UNSUPPORTED for the floating forms;
 * the solver is unchanged on error. */
lbm_status lbm_set_storage_reference(lbm_solver *s, const double U[3]);

/* Autotuner: times every built kernel configuration for this solver on its own
 * buffers (reads the current state, writes only the idle buffer, so the state is
 * unchanged) over `iters` launches each and keeps the fastest.  best_us, if not
 * NULL, receives the average step time of the chosen configuration.  With the
 * environment variable LBM_AUTOTUNE_CACHE naming a file, a choice stored there for the
 * same device, lattice, K, storage (and reference shift on or off), dims and collision mode
 * is applied without timing
 * (best_us then reports the stored time), and a new choice is appended to the file. */
lbm_status lbm_autotune(lbm_solver *s, int iters, double *best_us);

/* Global FP64 sums {sum rho, sum rho u_x, sum rho u_y, sum rho u_z} of stored
 * distributions the caller passes in, for callers that cannot allocate device
 * memory: a plugin whose host framework owns all device memory through its own
 * pool, a process whose memory another allocator has fully reserved, or a
 * latency-critical loop where an allocation (which may synchronise the device)
 * is forbidden.  It needs no solver and no workspace, and it calls no
 * cudaMalloc, cudaFree or other allocating routine.  The paper has no
 * counterpart to this call: it is a deployment convenience.
 *   distributions  device pointer to Q*nx*ny*nz stored values in the layout
 *                  lbm_get_distributions produces (any solver's raw state)
 *   dims           the same limits as lbm_create (nz == 1 for D2Q9, each side
 *                  >= the largest velocity component), and nz <= 4096
 *   out            four doubles, host or device memory as out_mem says; a host
 *                  output makes the call synchronise the stream and return
 *                  LBM_ERR_NONFINITE when a sum is not finite; a device output
 *                  is left for the caller to read later, so that check is not
 *                  made (the same state can then return LBM_OK)
 * Scratch: a fixed device array inside the library (about 128 KiB per GPU,
 * held until the process exits) with room for nz <= 4096 z-planes; larger nz
 * is rejected with LBM_ERR_INVALID_ARG.  Under CUDA's lazy module loading (the
 * default) that array is committed on a device at the first call there, not
 * when the library is loaded: a caller whose device memory another allocator
 * will reserve should make one call early.  The first call on a device also
 * looks up the array's device address, so make it before any stream capture;
 * later calls outside capture look it up again, so a device reset between
 * calls does not leave a stale address.
 * All calls share the array: calls whose GPU work overlaps race on it and must
 * be serialised by the caller. */
lbm_status lbm_conservation_noalloc(lbm_lattice lattice, lbm_storage storage, const int64_t dims[3], double rho0,
                                   const void *distributions, double out[4], lbm_mem out_mem, void *cuda_stream);

/* 1 when this library is the bounds-check build (compiled with LBM_DEBUG_BOUNDS, a
 * separate file): every kernel then checks each load and store index against the buffer
 * or velocity plane it addresses, skips an access outside it and records the event, and
 * the next synchronising call returns LBM_ERR_BOUNDS.  0 in the normal build.  The paper
 * has no counterpart: it is a check of the library's own indexing. */
int lbm_bounds_checked(void);

/* Host walk of the register-pull step's index arithmetic (no device work, any build): for
 * every thread of one launch with cells_per_thread V (1, 2, 4, 8; V must divide nx) on
 * dims, the offsets its loads and stores compute inside a velocity plane (the x-shift
 * scheme of the plain storage forms: whole-chunk loads on D3Q39, warp shuffles with direct
 * loads at warp and row edges on the other lattices), each checked against a plane of P
 * elements with the same test the bounds-check build's kernels apply.
 * Returns how many accesses fall outside (0 for a consistent P = nx*ny*nz) and sets
 * *accesses (if not NULL) to the number checked; -1 for invalid arguments.  The paper has
 * no counterpart: it is a check of the library's own indexing. */
int64_t lbm_bounds_walk(lbm_lattice lattice, int cells_per_thread, const int64_t dims[3], int64_t P,
                        int64_t *accesses);

/* Release the solver (not the workspace).  Synchronises its stream. */
lbm_status lbm_destroy(lbm_solver *s);

/* ------------------------------------------------------------------------
 * Pool: many independent periodic lattices (uneven sizes, own tau and rho0,
 * own step budget) advanced together -- each launch of the persistent batch
 * kernel performs one step of Eq. lbe-reg on every resident lattice -- with
 * admission by device memory and continuous batching: requests join and leave
 * at chunk boundaries while the others keep running.  One pool serves one
 * (lattice, truncation order, storage) class.  The per-lattice arithmetic is the
 * single-lattice step's; results do not depend on what else is resident.
 * ------------------------------------------------------------------------ */
typedef struct lbm_pool lbm_pool;

/* Device bytes one request of these dims occupies in a pool's arena: its two
 * distribution buffers (Q planes of px*ny*nz values, px = nx rounded up to a multiple of
 * 4) and a 256-byte status word.  0 for invalid arguments, for dims whose padded plane
 * px*ny*nz exceeds 2^31-1 cells (lbm_pool_submit rejects those with LBM_ERR_INVALID_ARG),
 * and for the storage forms pools do not run (the reference-velocity forms). */
size_t lbm_pool_request_bytes(lbm_lattice lattice, const int64_t dims[3], lbm_storage storage);

/* arena: caller-owned device memory (256-byte aligned) that the pool carves
 * request buffers from; max_slots bounds the resident requests.  compute_stream
 * runs the batched steps, io_stream the uploads and result downloads (either may
 * be NULL; distinct non-NULL streams let transfers overlap the steps). */
lbm_status lbm_pool_create(lbm_lattice lattice, int truncation_order, lbm_storage storage, void *arena,
                           size_t arena_bytes, int max_slots, void *compute_stream, void *io_stream, lbm_pool **out);

/* Admit one solve: f = f^eq(rho, u) (Eq. hermite) on a periodic lattice of dims,
 * to be advanced `steps` steps.  rho: double[C], u: double[D][C], in memory `mem`.
 * The inputs are consumed before the call returns.  LBM_ERR_BUSY when the arena
 * or the slot count has no room now (retry after results are collected);
 * LBM_ERR_RANGE when f^eq does not fit a fixed-point pool's range (not admitted). */
lbm_status lbm_pool_submit(lbm_pool *p, const int64_t dims[3], double tau, double rho0, const double *rho,
                           const double *u, lbm_mem mem, int64_t steps, int64_t *id);

/* Launch the next chunk of up to chunk_steps steps for every resident, unfinished
 * request (asynchronous; at most two chunks are in flight).  active receives the
 * number of requests in the launched chunk (0: nothing to do). */
lbm_status lbm_pool_advance(lbm_pool *p, int64_t chunk_steps, int *active);

/* done = 1 once the request's last step has completed on the device. */
lbm_status lbm_pool_poll(lbm_pool *p, int64_t id, int *done, int64_t *steps_done);

/* For a done request: rho and u after its steps (Eq. mme, pre-collision state),
 * then the request's memory returns to the arena.  Synchronises the io stream.
 * LBM_ERR_RANGE (fixed-point pools): a value of this request left the storage range
 * during its steps; the outputs are not valid and the request is released all the same.
 * Other requests are unaffected. */
lbm_status lbm_pool_result(lbm_pool *p, int64_t id, double *rho, double *u, lbm_mem mem);

/* Withdraw a request, done or not (a client that has gone away, a solve that is no longer
 * wanted): no further steps are scheduled for it, and once the chunks in flight and its upload
 * have finished (the call waits for them) its memory returns to the arena.  The other requests
 * run on unaffected.  LBM_ERR_NOT_FOUND for an unknown (or already collected) id. */
lbm_status lbm_pool_cancel(lbm_pool *p, int64_t id);

/* Wait for every launched chunk. */
lbm_status lbm_pool_sync(lbm_pool *p);

/* Free arena bytes, resident requests, and requests done but not collected. */
lbm_status lbm_pool_stats(const lbm_pool *p, size_t *free_bytes, int *resident, int *done);

/* Range R of a fixed-point pool (LBM_STORE_Q16), as lbm_set_storage_range: a power of two
 * in [2^-8, 2^8], default 1, the same for every request; or 0: each request gets its own
 * range at admission, the smallest power of two >= 1.25 max |h| of its f^eq (measured on the
 * device; lbm_pool_request_range reads it; the get call then reports 0).  Only while no
 * request is resident (LBM_ERR_BUSY otherwise).  A request whose f^eq does not fit is refused
 * by lbm_pool_submit with LBM_ERR_RANGE.  LBM_ERR_UNSUPPORTED for the floating forms. */
lbm_status lbm_pool_set_storage_range(lbm_pool *p, double range);
lbm_status lbm_pool_get_storage_range(const lbm_pool *p, double *range);
lbm_status lbm_pool_request_range(const lbm_pool *p, int64_t id, double *range);

/* Kernel configuration of the batched step.  cells_per_thread: the x-neighbours a thread
 * updates, 1, 2 or 4 (the default).  A pool stores each request with its rows padded to a
 * multiple of 4 cells whose pad cells hold periodic images of the row's first cells, so
 * every request runs this setting whatever its nx, and a request's arithmetic depends on the
 * setting and its own dims only, never on the other residents.  Two and four cells per
 * thread run the collision on the paired FP32 instructions.  block_threads: 128 (the
 * default) or 256.  Zero keeps the current value.  Waits for the launched chunks.
 * LBM_ERR_UNSUPPORTED for other values. */
lbm_status lbm_pool_set_kernel(lbm_pool *p, int cells_per_thread, int block_threads);
lbm_status lbm_pool_get_kernel(const lbm_pool *p, int *cells_per_thread, int *block_threads);

/* Autotuner for the batch kernel: times each built configuration (cells per thread 1, 2 or
 * 4 x block 128 or 256) on the current resident set (state unchanged) and keeps the fastest.
 * best_us: time per step. */
lbm_status lbm_pool_autotune(lbm_pool *p, int iters, double *best_us);

/* Release the pool (not the arena).  Synchronises both streams. */
lbm_status lbm_pool_destroy(lbm_pool *p);

const char *lbm_status_string(lbm_status status);
const char *lbm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
