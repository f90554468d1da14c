/*
 * swapmd.h -- C-ABI of the GB300 (sm_103a) associative bond-swap MD library.
 *
 * The library evaluates, every time step, the two-body bonding potential of
 * reactive type pairs, Eq. 2b of Ciarella & Ellenbroek ("Associative bond
 * swaps in molecular dynamics"):
 *     v(r) = 4 eps [(sigma/r)^(2n) - (sigma/r)^n],  r < r_cut,
 * plus the three-body swap term of Eq. 3bp,
 *     v3_ijk = lambda eps vh(r_ij) vh(r_ik)   (centre i, unordered {j, k}),
 * with vh the normalised two-body term of Eq. pot (1 inside
 * r_min = sigma 2^(1/n), -v/eps beyond), and repulsive WCA between like
 * types (section "Effect of swaps").  It returns forces, the two- and
 * three-body energies, the virial of Eq. p3 and the bond count, over a Verlet
 * neighbour list built from a cell list, and advances the system with velocity
 * Verlet (NVE) or BAOAB Langevin (NVT, the paper's "canonical Langevin
 * dynamics", section "Self-assembly pitfalls").
 *
 * Conventions
 *  - Every call returns an int status: SWP_OK (0) or a negative SWP_ERR_*.
 *    No call throws.  swp_last_error() gives a message owned by the context,
 *    valid until the next call on it.
 *  - Calls that launch work are asynchronous on the stream given to
 *    swp_bind_workspace().  Errors raised on the device (neighbour-row
 *    overflow, a device wait past its time bound, non-finite forces) are
 *    latched and reported by the next swp_sync() or swp_read_*() call.
 *  - Particle arrays exchanged with the caller are in USER order: entry i
 *    belongs to the particle given as entry i to swp_set_state() (its tag).
 *    Internally particles are re-ordered by cell; nothing of that leaks out.
 *  - Positions are 3 doubles per particle (x, y, z), row-major [n][3].
 *  - `where` is SWP_HOST (pointer in host memory; pinned or pageable) or
 *    SWP_DEVICE (pointer in device memory of the bound device).
 *  - Ownership: the library allocates NO device memory.  The caller allocates
 *    the workspace and the neighbour-list buffer (sizes from
 *    swp_workspace_size() / swp_nlist_size()) and keeps them alive until
 *    swp_destroy() or until they are re-bound.  The context object itself is
 *    host memory owned by the library (swp_create / swp_destroy).
 */
#ifndef SWAPMD_H
#define SWAPMD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define SWP_API __attribute__((visibility("default")))
#else
#define SWP_API
#endif

#define SWP_ABI_VERSION 6

/* Status codes. */
#define SWP_OK 0
#define SWP_ERR_INVALID (-1)         /* bad argument; the context is unchanged */
#define SWP_ERR_CUDA (-2)            /* a CUDA runtime call failed (no device, launch error) */
#define SWP_ERR_NLIST_OVERFLOW (-3)  /* a neighbour row exceeded max_nn: grow it (see below) */
#define SWP_ERR_TIMEOUT (-4)         /* a device-side wait ran past its bound; state lost */
#define SWP_ERR_STATE (-5)           /* call out of order (nothing bound / no state set) */
#define SWP_ERR_NONFINITE (-6)       /* a non-finite force was produced */

/* Arithmetic precision of a context.  SWP_FP32: pair and three-body arithmetic
 * in FP32, per-thread energy/virial terms of at most one block sub-chunk in
 * FP32, block sums compensated (double-float, as accurate as FP64 sums of the
 * FP32 terms), sums over blocks in FP64, positions accumulated in 64-bit fixed
 * point; distances come from 32-bit fractions of the box edges (the minimum
 * image is the wrap-around difference), so their error does not grow with the
 * box. */
#define SWP_FP32 0
#define SWP_FP64 1 /* FP64 everywhere (parity and validation) */

/* Kinds of type pairs. */
#define SWP_PAIR_NONE 0 /* no interaction */
#define SWP_PAIR_WCA 1  /* Eq. 2b cut at r_min and shifted up by eps: purely repulsive */
#define SWP_PAIR_SWAP 2 /* Eq. 2b two-body term plus the Eq. 3bp three-body term */

#define SWP_HOST 0
#define SWP_DEVICE 1

typedef struct swp_ctx swp_ctx;

/* Thermodynamic record of the last force evaluation (one time step). */
typedef struct {
    double U2;        /* two-body energy (sum of Eq. 2b / WCA over interacting pairs) */
    double U3;        /* three-body energy (sum of Eq. 3bp over centres and partner pairs) */
    double K;         /* kinetic energy sum 1/2 m v^2 at the same time */
    double W[6];      /* virial sum over pairs r_ij (x) F_ij: xx, yy, zz, xy, xz, yz (Eq. p3 for
                         the three-body part; pressure = (2K/3 + tr W / 3) / V) */
    int64_t n_bonds;  /* reactive pairs closer than their bond radius */
    int64_t step;     /* completed time steps of the state */
    int64_t n_rebuilds;  /* neighbour-list builds since swp_set_state() */
    int64_t steps_done;  /* steps completed by the last step call */
    int32_t max_row;     /* longest neighbour row of the last build */
    int32_t state;       /* 0: forces current; 1: forces stale; 2: inside a step (after overflow) */
    int32_t resident_steps; /* steps of the last step call taken in the resident mode
                               (see swp_set_resident) */
    int32_t reserved;
} swp_thermo;

/* ABI version (SWP_ABI_VERSION); needs no device. */
SWP_API int swp_abi_version(void);

/* Create a context for n particles of n_types types (1..8) in a periodic
 * orthorhombic box box[3] (edges in [2^-8, 30000]).  precision is SWP_FP32 or SWP_FP64; seed
 * keys the Langevin noise.  In FP32 the box lengths are rounded to float32;
 * in both the box is then rounded to the 2^-48 fixed-point grid.  Uses the
 * current CUDA device.  n may be 0 (every call is then a no-op).  n < 2^27.
 * Errors: SWP_ERR_INVALID for bad sizes, SWP_ERR_CUDA if no device. */
SWP_API int swp_create(swp_ctx** out, int n, int n_types, const double box[3], int precision,
               uint64_t seed);

/* Set the coefficients of type pair (ti, tj) (symmetric), the per-type-pair
 * table of the paper's pair_coeff.set(types, types, sigma, n, epsilon,
 * lambda3) (section "The swap potential").  kind is SWP_PAIR_*; n_exp is the
 * exponent n of Eq. 2b (1..128); rcut is r_cut of Eq. 2b (SWAP only; WCA is
 * cut at r_min); lambda3 is lambda of Eq. 3bp (>= 0, SWAP only).  shift = 1
 * selects the shifted form v - v(r_cut), vh = (v(r_cut) - v)/(eps + v(r_cut))
 * (continuous at r_cut); 0 is the paper's literal form.  rbond is the bond
 * radius (a reactive pair closer than it counts as a bond); <= 0 selects the
 * distance where vh = 1/2.  All pairs default to SWP_PAIR_NONE.
 * Errors: SWP_ERR_INVALID.  Marks the forces and the neighbour list stale. */
SWP_API int swp_set_pair(swp_ctx* ctx, int ti, int tj, int kind, double eps, double sigma, int n_exp,
                 double rcut, double lambda3, int shift, double rbond);

/* Neighbour-list skin (>= 0; list radius of a pair = its cut-off + skin) and
 * mean row capacity max_nn (>= 1): the list holds max_nn entries per
 * particle on average over each block's particles (a single row may be
 * longer).  Call before swp_nlist_size / swp_bind_nlist.
 * The box must hold >= 3 cells of edge max(cut-off) + skin per dimension:
 * SWP_ERR_INVALID otherwise. */
SWP_API int swp_set_nlist(swp_ctx* ctx, double skin, int max_nn);

/* Bytes of device workspace this context needs (state, cell list, staging). */
SWP_API int swp_workspace_size(const swp_ctx* ctx, size_t* bytes);

/* Bytes of the neighbour-list buffer for the current max_nn. */
SWP_API int swp_nlist_size(const swp_ctx* ctx, size_t* bytes);

/* Bind caller-owned device memory (256-byte aligned, >= the size above) and
 * the CUDA stream (cudaStream_t, may be NULL) every later call enqueues on.
 * Binding a workspace discards any state (call swp_set_state after). */
SWP_API int swp_bind_workspace(swp_ctx* ctx, void* device_ptr, size_t bytes, void* cuda_stream);

/* Bind the neighbour-list buffer.  May be re-bound with a larger max_nn after
 * SWP_ERR_NLIST_OVERFLOW without losing the state; marks the list stale. */
SWP_API int swp_bind_nlist(swp_ctx* ctx, void* device_ptr, size_t bytes);

/* Set the state in user order: x [n][3] (any real numbers: wrapped into the
 * box, the wraps added to img), v [n][3] (NULL: zero), type [n] (NULL: all 0),
 * mass [n] (> 0; NULL: all 1), img [n][3] (NULL: zero).  All pointers are of
 * kind `where`.  Resets the step counter to 0.  Forces become stale. */
SWP_API int swp_set_state(swp_ctx* ctx, const double* x, const double* v, const int32_t* type,
                  const double* mass, const int32_t* img, int where);

/* Set the step counter (keys the Langevin noise: resuming a saved state with
 * its step gives the same trajectory). */
SWP_API int swp_set_step(swp_ctx* ctx, int64_t step);

/* Rebuild the cell list and the neighbour list now (normally automatic). */
SWP_API int swp_build_nlist(swp_ctx* ctx);

/* Bring forces, energies, virial and bond count up to date for the current
 * positions (no time advance, except that a step interrupted by an overflow
 * is completed first). */
SWP_API int swp_compute_forces(swp_ctx* ctx);

/* Advance nsteps time steps of velocity Verlet (NVE), dt > 0. */
SWP_API int swp_step_nve(swp_ctx* ctx, double dt, int nsteps);

/* Advance nsteps time steps of BAOAB Langevin dynamics at temperature kT with
 * friction gamma (> 0; gamma = 0 is velocity Verlet).  The noise of step s
 * for particle with tag t is Philox4x32-10 with counter (t, s lo, s hi, 1)
 * and key (seed lo, seed hi), Box-Muller normals.  The list is rebuilt on the
 * device whenever the accumulated displacement bound exceeds skin/2.
 * On SWP_ERR_NLIST_OVERFLOW (reported by the next sync), thermo.steps_done
 * steps were completed and thermo.max_row gives the row length needed:
 * re-bind a larger list and call again for the remaining steps. */
SWP_API int swp_step_nvt(swp_ctx* ctx, double dt, double kT, double gamma, int nsteps);

/* Batched dynamics: advance n_systems independent systems nsteps time steps
 * each in ONE cooperative launch (the per-system step of swp_step_nvt, with
 * dt[r], kT[r], gamma[r] for system r; gamma[r] = 0 is velocity Verlet).  The
 * systems may differ in size, box, coefficients and temperature.  They must
 * share precision, device and bound stream, each must have its workspace,
 * list buffer and state, and none may appear twice; empty systems are
 * skipped.
 *
 * Work split, with w the particle count of a system and a block's load the
 * particles it advances (a group member: w / group size).  split = 0 (the
 * balanced plan, the default): the smallest largest load C for which every
 * system with w > C gets ceil(w / C) blocks (its device-side barriers span
 * only those blocks; no member share below `threads` particles) and every
 * other system, heaviest first, goes onto the least-loaded block, group
 * members included, with no load above C; a block runs its group share
 * first, then its single-block systems one after the other.  split > 0 (the
 * threshold plan): with T the mean load, a system with w > split * T gets
 * max(1, round(w / T)) blocks that run nothing else, the others are packed
 * the same way onto the remaining blocks.  A group has at most
 * min(threads, 304) blocks.  swp_batch_plan returns either plan.
 *
 * Block shape: threads per block of the batched kernel, 1024 (0 selects it;
 * 64 registers per thread, one block per SM), or in FP32 512 (128 registers),
 * 384 or 256 (as many registers as the kernel uses: no spills), one block per
 * SM each: smaller blocks give each thread more registers and a small system
 * fewer idle threads, larger ones more warps per SM.  Tune it by timing with
 * the split.
 *
 * ws: device scratch of at least swp_batch_workspace_size(n_systems) bytes,
 * owned by the caller and used until the launch completes.  Enqueued on the
 * shared stream; errors of system r (timeout, list overflow) are latched in
 * system r and reported by swp_sync(ctx[r]): on SWP_ERR_NLIST_OVERFLOW that
 * system completed thermo.steps_done steps (the others are unaffected).
 * Errors: SWP_ERR_INVALID (bad arguments, mixed precision/device/stream, a
 * block shape the precision does not have, ws too small, more large systems
 * than blocks), SWP_ERR_STATE, SWP_ERR_CUDA. */
SWP_API size_t swp_batch_workspace_size(int n_systems);
SWP_API int swp_batch_step(swp_ctx* const* ctx, int n_systems, const double* dt, const double* kT,
                           const double* gamma, int nsteps, double split, int threads, void* ws,
                           size_t ws_bytes);

/* The work split of swp_batch_step (host only; no device work): the plan
 * for systems of w[r] >= 0 particles on n_blocks blocks.  swp_batch_step uses
 * n_blocks = SMs x blocks per SM of the block shape, max_group =
 * min(threads, 304) and min_part = threads.  Outputs: item_ofs[n_blocks + 1]
 * (block k runs items item_ofs[k] .. item_ofs[k + 1] - 1, in that order) and
 * items[4 * i ..] = (system, rank in its group, group size, 0), at most
 * n_systems + n_blocks items (the caller's capacity), their count in
 * *n_items.  Errors: SWP_ERR_INVALID (bad arguments, more large systems than
 * blocks in the threshold plan). */
SWP_API int swp_batch_plan(const long long* w, int n_systems, int n_blocks, double split, int max_group,
                           int min_part, int* item_ofs, int* items, int* n_items);

/* Wait for the stream and report latched device errors. */
SWP_API int swp_sync(swp_ctx* ctx);

/* Harmonic bonds of a fixed topology, u = k/2 (r - r0)^2 per bond (minimum
 * image, no cut-off), acting besides the pair terms, which still act between
 * bonded particles (no exclusion).  They build the chains of the vitrimer
 * network (the paper's section "Applications to vitrimers" names bonded
 * chains carrying the swapping groups without giving their form; the
 * harmonic form is this library's).  bonds: host [n_bonds][2] tags; at most
 * 4 bonds per particle.  n_bonds = 0 removes them.  The bond energy is
 * reported inside thermo.U2 and the bonds' virial inside thermo.W.  Marks
 * forces stale.  Errors: SWP_ERR_INVALID (tag out of range, self bond,
 * duplicate, more than 4 bonds on a particle, k < 0 or r0 < 0). */
SWP_API int swp_set_bonds(swp_ctx* ctx, int n_bonds, const int32_t* bonds, double k, double r0);

/* Derivatives of the energy and of the forces with respect to the
 * coefficients (lambda, eps, sigma) of the reactive type pair (ti, tj), at
 * the current positions (Eq. 2b, Eq. pot, Eq. 3bp; the two-body term is
 * linear in eps, vh depends on sigma only through sigma/r, r_min = sigma
 * 2^(1/n) moves with sigma, r_cut stays fixed).  Needs current forces
 * (swp_compute_forces), the unshifted form and a single reactive type pair.
 * dU [3] (host): dU/dlambda, dU/deps, dU/dsigma.  dF_dev (device pointer or
 * NULL): [3][n][3] doubles, dF_dev[(k n + i) 3 + c] = d F_ic / d theta_k in
 * user order.  Uses the workspace's staging arrays (not concurrently with
 * other reads of this context); synchronises the stream.  Errors:
 * SWP_ERR_INVALID (bad types, not a swap pair, shifted form, more than one
 * reactive type pair), SWP_ERR_STATE (forces not current). */
SWP_API int swp_param_grad(swp_ctx* ctx, int ti, int tj, double dU[3], double* dF_dev);

/* One evaluation of the differentiable energy, enqueued on the context's
 * stream with no host synchronisation (for a fit that evaluates many
 * snapshots in a row).  Inputs in device memory: theta_dev = (lambda, eps,
 * sigma) of the reactive pair (ti, tj) (3 doubles; the unshifted form, one
 * reactive type pair, as for swp_param_grad), x_dev [n][3] positions in user
 * order, type_dev [n] types (NULL: all 0).  It replaces the state (as
 * swp_set_state with zero velocities, unit masses and no images), writes
 * theta's coefficients into the device copy of the pair table (the host
 * coefficients of swp_set_pair stay as they were and serve the next other
 * run), rebuilds the list and evaluates: U_dev [1] = U2 + U3 (Eq. pot);
 * F_dev [n][3] the forces (NULL: not read); dU_dev [3] = dU/d(lambda, eps,
 * sigma) and dF_dev [3][n][3] as for swp_param_grad (NULL: not formed).
 * Nothing is read back: errors the device latches (a list row longer than
 * max_nn, a non-finite force, e.g. from theta out of range) are reported by
 * the next swp_sync, and the outputs of that evaluation are then invalid; size
 * max_nn for the densest snapshot.  Errors returned at once: SWP_ERR_INVALID
 * (null theta/x/U, bad types, not a single unshifted swap pair),
 * SWP_ERR_STATE (no workspace or list buffer bound). */
SWP_API int swp_eval_grad(swp_ctx* ctx, int ti, int tj, const double* theta_dev, const double* x_dev,
                          const int32_t* type_dev, double* U_dev, double* F_dev, double* dU_dev, double* dF_dev);

/* Synchronising reads.  swp_read_thermo fills *out with the record of the
 * last force evaluation.  swp_read_forces needs current forces (state 0):
 * f [n][3].  swp_read_state: x [n][3] wrapped into [0, L), v [n][3], img
 * [n][3]; any of them may be NULL.  Pointers of kind `where`. */
SWP_API int swp_read_thermo(swp_ctx* ctx, swp_thermo* out);

/* Thermo log: a record of the energies, virial, kinetic energy and bond count
 * (the quantities of swp_read_thermo) of every step whose number is a
 * multiple of `every`, written by the step kernel into a ring of `capacity`
 * records that the caller provides.  A step kernel sums these terms only on
 * the steps it logs and on the last step of each launch (the one
 * swp_read_thermo reports); every = 0 (the default) turns the log off.
 *
 * swp_thermo_log_bytes: bytes of the ring for `capacity` records (0 if the
 * capacity is not in [1, 2^31 - 1]).  swp_set_thermo_log: every >= 0; with
 * every > 0, ring is a device buffer of this context's device, 256-byte
 * aligned, of at least swp_thermo_log_bytes(ctx, capacity) bytes, which the
 * library uses (does not own) until the log is set again or the context is
 * destroyed.  It restarts the count of records, and so does swp_set_state.
 * Errors: SWP_ERR_INVALID.
 *
 * swp_thermo_log: the newest min(written, capacity, max_records) records,
 * oldest first, into rec_dev [max_records][10] doubles (U2, U3, K, W[6],
 * n_bonds, each summed over the blocks as in swp_read_thermo) and step_dev
 * [max_records] (the step numbers), both device pointers; *n_records (host)
 * gets the count.  Synchronises the stream to read the count; the sums are
 * formed by a kernel enqueued on it.  Errors: SWP_ERR_INVALID (no log set,
 * null pointers), the latched errors of swp_sync. */
SWP_API size_t swp_thermo_log_bytes(const swp_ctx* ctx, int64_t capacity);
SWP_API int swp_set_thermo_log(swp_ctx* ctx, int every, int64_t capacity, void* ring, size_t ring_bytes);
SWP_API int swp_thermo_log(swp_ctx* ctx, double* rec_dev, int64_t* step_dev, int64_t max_records,
                           int64_t* n_records);
SWP_API int swp_read_forces(swp_ctx* ctx, double* f, int where);
SWP_API int swp_read_state(swp_ctx* ctx, double* x, double* v, int32_t* img, int where);

/* Neighbour rows in user order (device pointers only): rows [n][width]
 * holds the tags of each particle's list (the first min(total, width)
 * entries), reactive partners first; counts [n][2] = (reactive, total).
 * Needs a current list (swp_build_nlist). */
SWP_API int swp_read_nlist(swp_ctx* ctx, int32_t* rows_dev, int32_t* counts_dev, int width);

/* Launch shape of the step kernel: resident blocks per SM (0: as many as
 * fit; the kernel uses 768-thread blocks and most of an SM's shared memory,
 * so one fits).  Changing it marks the list stale (its block partition
 * follows the grid). */
SWP_API int swp_set_launch(swp_ctx* ctx, int blocks_per_sm);

/* Upper bound on the step kernel's blocks (0, the default: the resident
 * blocks of every SM); requests below 10 run on 10 blocks (one per thermo
 * quantity reduced in parallel), or on every SM's if there are fewer.  A
 * smaller grid leaves SMs free for other work on the device; the time per
 * step of a small system hardly depends on it (each step's dependent phases,
 * not the grid barriers, set it).  Results do not depend on it beyond the
 * order of floating-point sums.  Negative: SWP_ERR_INVALID.  Changing it
 * marks the list stale (its block partition follows the grid). */
SWP_API int swp_set_grid(swp_ctx* ctx, int blocks);

/* Bound, in nanoseconds, on every device-side wait (default 2 s). */
SWP_API int swp_set_timeout(swp_ctx* ctx, int64_t ns);

/* Resident mode of the FP32 step (enable: 1, the default; 0: off).  When a
 * run has one system in FP32 without bonds and every block of the step kernel
 * owns at most one sub-chunk of particles (n up to blockDim x grid, 116,736
 * on a 152-SM part), each block keeps in shared memory, between list builds,
 * its own rows and the reactive rows of its halo (the partners of its particles
 * that other blocks own) with partners as local indices; a step then copies
 * the halo's new positions in once, forms S (Eq. 3bp via S_i) for its own
 * particles and the reactive halo itself, and the forces and the integrator
 * from shared memory, with one grid barrier per step instead of two.  Blocks
 * whose structures exceed the shared-memory capacity (3,072 local particles,
 * 16,384 local entries, rows of 255 entries) make the whole run fall back to
 * the two-barrier path until the next list build.  Forces and trajectories are
 * the same bit for bit either way (same operations, same summation orders);
 * the energy and virial sums are grouped differently (equal within their
 * rounding).  thermo.resident_steps reports how many steps ran resident.
 * enable not 0 or 1: SWP_ERR_INVALID. */
SWP_API int swp_set_resident(swp_ctx* ctx, int enable);

/* Failure-detection test hook (the paper has no counterpart).  With on = 1 the
 * next step-kernel launch of ctx withholds one block's arrival at its first
 * grid barrier, so that every other block's bounded wait runs out after the
 * timeout of swp_set_timeout: the launch ends early with every block returned,
 * and the next swp_sync / swp_read_* reports SWP_ERR_TIMEOUT (the state is then
 * lost: set it again).  In a batched launch (swp_batch_step) the same happens
 * to the group of blocks of ctx's system, whose blocks then go on with the
 * other systems the plan gave them; a system on one block has no grid
 * barrier, and there the request has no effect.  Nothing faults and no wait is unbounded; it exercises
 * the path a real stall (a block starved by other work, a lost arrival) takes.
 * The request is consumed by that one launch.  on not 0 or 1: SWP_ERR_INVALID. */
SWP_API int swp_set_withhold_arrival(swp_ctx* ctx, int on);

/* Forces without any device allocation.  The paper has no counterpart: this
 * serves callers that cannot allocate device memory when they need forces --
 * code running inside a host framework whose memory pool has reserved the
 * device and forbids side allocations, or a latency-bound loop that cannot
 * afford the device-wide synchronisation of cudaMalloc / cudaFree.  It neither
 * allocates nor frees anything and needs no bound workspace or list buffer.
 * The call synchronises cuda_stream and copies small parameter blocks from
 * pageable host memory, so it cannot be recorded into a CUDA graph by stream
 * capture; call it outside any capture.
 *
 * Uses the coefficients, skin, max_nn and launch shape of ctx.  Inputs: x_dev
 * [n][3] positions and type_dev [n] types (NULL: all 0), device pointers.
 * Outputs (device pointers): f_dev [n][3] forces; thermo_dev (may be NULL)
 * [9] = U2, U3, W xx yy zz xy xz yz, n_bonds.  Velocities are taken as zero
 * and masses as one; the context's own state is not touched.
 *
 * Scratch: a file-scope device array of SWP_STATIC_SCRATCH_BYTES (8 MiB)
 * that every GPU loading this library keeps until the process exits.  The
 * state copy, cell list and neighbour list of the system must fit in it
 * (about 10,000 particles at max_nn 64 and liquid densities); larger systems
 * are rejected with SWP_ERR_INVALID and a message giving the bytes needed.
 * Every call shares that one array and leaves its contents behind (each call
 * re-initialises what must start at zero), so calls that overlap on the GPU
 * -- from two streams, threads or contexts at once -- race and corrupt each
 * other: serialise them.  The first call on each device looks up the array's
 * device address (with that device current).  The current device must be the
 * one ctx was created on (else SWP_ERR_INVALID).  Enqueues on cuda_stream and
 * returns after synchronising it.  Errors: as swp_compute_forces (row
 * overflow: SWP_ERR_NLIST_OVERFLOW, grow max_nn with swp_set_nlist; the next
 * call starts clean). */
#define SWP_STATIC_SCRATCH_BYTES (8u << 20)
SWP_API int swp_compute_forces_static(swp_ctx* ctx, const double* x_dev, const int32_t* type_dev,
                                      double* f_dev, double* thermo_dev, void* cuda_stream);

SWP_API const char* swp_last_error(const swp_ctx* ctx);

/* Free the context (not the caller's device buffers). NULL is accepted. */
SWP_API int swp_destroy(swp_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* SWAPMD_H */
