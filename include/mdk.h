/*
 * mdk.h -- C ABI of the GB300-native short-range molecular-dynamics hot path
 * (MDcraft, arXiv 2511.22951): cell-list Verlet neighbour lists with a skin
 * and a displacement-triggered rebuild, Lennard-Jones and tabulated-EAM
 * forces, velocity-Verlet NVE integration, a rigid-piston / moving-window
 * hook for shock runs, and the Appendix per-bin profiles.
 *
 * Every step runs in hand-written sm_103a CUDA kernels of libmdk.so.  No
 * call allocates device memory: all device scratch lives in one workspace
 * that the caller allocates (mdk_workspace_size / mdk_set_workspace).
 *
 * Conventions shared by every call
 *  - Units: eV, Angstrom, fs, atomic mass unit u.  Accelerations use
 *    a = F/m * 9.648533212e-3 Angstrom/fs^2 per eV/(Angstrom u).
 *  - Return value: MDK_OK (0) or a negative MDK_ERR_* code.  No C++
 *    exception crosses this boundary.  mdk_status_string() names a code.
 *  - Arrays are C-contiguous.  Positions, velocities and forces are
 *    [N][3] doubles (x, y, z per atom) in the caller's atom order; the
 *    library's internal spatial ordering is never visible.
 *  - Ownership: the caller owns every pointer it passes.  Host arrays are
 *    copied before the call returns.  Device arrays (on_device = 1) are read
 *    or written only inside the call, on the context's stream.
 *  - Streams: all work is enqueued on the stream given to mdk_create (NULL =
 *    legacy default stream).  A call that returns host data synchronises
 *    that stream; a call that only writes device memory does not.
 *  - Threading: a context is used by one host thread at a time.
 *  - Boxes: periodic dimensions must be at least rc + skin long (smaller
 *    periodic boxes return MDK_ERR_BOX_TOO_SMALL).  Free (non-periodic)
 *    dimensions use the box only to lay out cells; atoms outside it are
 *    still simulated exactly (they share the end cells).
 */
#ifndef MDK_H
#define MDK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ----------------------------------------------------- */
#define MDK_OK 0
#define MDK_ERR_BAD_ARG (-1)        /* invalid argument or size            */
#define MDK_ERR_BOX_TOO_SMALL (-2)  /* periodic length < rc + skin         */
#define MDK_ERR_NEIGH_OVERFLOW (-3) /* a list outgrew its capacity; the
                                       capacity was raised: resize the
                                       workspace and repeat the call       */
#define MDK_ERR_ATOM_LOST (-4)      /* reserved: an atom moved more than one
                                       cell between list builds (the
                                       displacement trigger rebuilds first,
                                       so no kernel raises it)             */
#define MDK_ERR_NONFINITE (-5)      /* NaN or Inf in a position or force   */
#define MDK_ERR_TIMEOUT (-6)        /* a bounded device-side wait ran out  */
#define MDK_ERR_CUDA (-7)           /* a CUDA runtime call failed          */
#define MDK_ERR_WORKSPACE (-8)      /* no workspace, or it is too small    */
#define MDK_ERR_ORDER (-9)          /* call made before a required call    */
#define MDK_ERR_RHO_RANGE (-10)     /* an EAM density left the F table
                                       (F was extrapolated linearly)       */
#define MDK_ERR_TOO_LARGE (-11)     /* size above the fixed maximum of
                                       mdk_lj_compute_noalloc             */
#define MDK_ERR_CAPACITY (-12)      /* the moving window had more atoms to
                                       append than mdk_set_capacity left
                                       room for (as many as fit were)     */
#define MDK_ERR_BOUNDS (-13)        /* debug builds only (libmdk_debug.so,
                                       compiled with MDK_DEBUG): a kernel
                                       caught an index outside its array,
                                       skipped the access and went on; the
                                       results of the call are not valid  */

/* ---- precision modes ---------------------------------------------------- */
#define MDK_FP64 0  /* every operation in FP64                               */
#define MDK_MIXED 1 /* FP32 pair arithmetic from cell-relative FP32 offsets,
                       compensated FP32 sums per atom, FP64 positions,
                       velocities, integration and per-atom results        */

typedef struct mdk_ctx mdk_ctx; /* opaque, library-owned host object */

/* ---- lifetime ----------------------------------------------------------- */

/*
 * Create a context for one periodic/free box holding N atoms.
 * Follows the paper's statement of the MD problem: N atoms in a domain with
 * free or periodic boundaries (Sec. "Molecular dynamics").
 *   box_lo, box_hi : [3] box corners (host)
 *   periodic       : [3] 0 = free, 1 = periodic (host)
 *   N              : atom count, 0 <= N < 2^26
 *   masses         : [N] atomic masses in u (host); at most 16 distinct values
 *   precision      : MDK_FP64 or MDK_MIXED
 *   cuda_stream    : a cudaStream_t, or NULL
 * The context holds no device memory until mdk_set_workspace.
 */
int mdk_create(mdk_ctx **out, const double box_lo[3], const double box_hi[3],
               const int periodic[3], int64_t N, const double *masses,
               int precision, void *cuda_stream);

/*
 * Create one context for n_rep independent systems ("replicas"), each with
 * its own box, run together by the same kernels (one launch per phase for
 * all replicas).  Atoms of replica r are atoms [off_r, off_r + n_atoms[r])
 * of every [N][3] array, off_r = sum of the earlier n_atoms.
 *   box_lo, box_hi : [n_rep][3];  periodic : [n_rep][3];  n_atoms : [n_rep]
 *   masses         : [sum n_atoms]
 * Paper counterpart: the cold-curve and isotherm series (many small boxes).
 */
int mdk_create_batch(mdk_ctx **out, int n_rep, const double *box_lo,
                     const double *box_hi, const int *periodic,
                     const int64_t *n_atoms, const double *masses,
                     int precision, void *cuda_stream);

/* Destroy a context (the workspace stays the caller's). */
int mdk_destroy(mdk_ctx *ctx);

/* Reserve room for up to max_atoms atoms (moving window inserts atoms).
 * Default: the N given at creation.  Call before mdk_workspace_size. */
int mdk_set_capacity(mdk_ctx *ctx, int64_t max_atoms);

/* ---- potentials (Sec. "Potentials support") ------------------------------ */

/*
 * Lennard-Jones u(r) = 4 eps [(sigma/r)^12 - (sigma/r)^6] for r < rc.
 * shift_mode: 0 plain truncation, 1 energy shifted to 0 at rc,
 * 2 shifted force (value and slope 0 at rc).
 */
int mdk_set_potential_lj(mdk_ctx *ctx, double eps, double sigma, double rc,
                         int shift_mode);

/*
 * Single-element EAM from tabulated functions (the paper loads EAM from a
 * tabulated file; energy U = 1/2 sum_ij phi(r_ij) + sum_i F(rho_i),
 * rho_i = sum_j rho(r_ij)).
 *   phi, rho : [nr] knot values at r_k = k rc/(nr-1) (host); last knot at rc
 *   F        : [nrho] knot values at rho_k = k rho_max/(nrho-1) (host)
 * Between knots: cubic Hermite spline, knot slopes from 3-point differences
 * (one-sided at the ends).  r >= rc gives 0; rho > rho_max extrapolates F
 * linearly and makes mdk_compute/mdk_step return MDK_ERR_RHO_RANGE.
 * 3 <= nr <= 7168 (the FP64 phi and rho tables share 227 KB of shared
 * memory), 3 <= nrho <= 65536; otherwise MDK_ERR_BAD_ARG.  Same-size tables
 * replace the old ones in place (no new workspace needed).
 */
int mdk_set_potential_eam(mdk_ctx *ctx, int nr, double rc, const double *phi,
                          const double *rho, int nrho, double rho_max,
                          const double *F);

/*
 * Behler-Parrinello neural-network potential (Sec. "Molecular dynamics with
 * Behler-Parrinello neural networks"), single element: E = sum_i E_i, E_i
 * from atom i's network applied to its symmetry functions over the
 * neighbours closer than rc, cut off by f_c(R) = 1/2 [cos(pi R/rc) + 1]:
 *   rad_kind[m] 1: G1 = sum_j f_c(R_ij)                        (rad_par unused)
 *               2: G2 = sum_j exp(-eta (R_ij - R_s)^2) f_c(R_ij)  rad_par = (eta, R_s)
 *               3: G3 = sum_j cos(kappa R_ij) f_c(R_ij)          rad_par = (kappa, -)
 *   ang_kind[m] 4: G4 = 2^(1-zeta) sum_{j<k} (1 + lambda cos theta_ijk)^zeta
 *                   exp(-eta (R_ij^2 + R_ik^2 + R_jk^2)) f_c(R_ij) f_c(R_ik) f_c(R_jk)
 *               5: G5 = the same without the R_jk factors
 *               ang_par = (zeta, lambda, eta): zeta an integer in [1, 64],
 *               lambda = +1 or -1; sums over unordered pairs of distinct
 *               neighbours (each angle once).
 * Network input G = [radial functions, angular functions] in the order
 * given; h1 = tanh(b1 + G W01), h2 = tanh(b2 + h1 W12), E_i = b3 + h2 . w23.
 *   W01 [n_rad + n_ang][H1], b1 [H1], W12 [H1][H2], b2 [H2], w23 [H2] (host,
 *   row-major, copied).
 * Forces F_k = -dE/dR_k (Eq. force); the virial of E_i is kept by atom i.
 * Limits (else MDK_ERR_BAD_ARG): n_rad <= 8; n_ang <= 64 with at most 8
 * distinct (eta, kind) and at most 4 distinct zeta among the angular
 * functions, no function given twice; 1 <= H1, H2 <= 32; finite values.
 * Runs on full lists (a half list kind is reset to full).
 */
int mdk_set_potential_bpnn(mdk_ctx *ctx, double rc, int n_rad, const int *rad_kind,
                           const double *rad_par, int n_ang, const int *ang_kind,
                           const double *ang_par, int H1, int H2, const double *W01,
                           const double *b1, const double *W12, const double *b2,
                           const double *w23, double b3);

/* ---- device memory ---------------------------------------------------- */

/* Bytes of device workspace the context needs for its current capacity,
 * potential and neighbour parameters (call mdk_plan_neighbors first to
 * size for a given skin; default skin 0.3 Angstrom). */
int mdk_workspace_size(const mdk_ctx *ctx, size_t *bytes);

/*
 * Hand the context a device buffer of at least mdk_workspace_size bytes,
 * 256-byte aligned.  The caller keeps ownership and must keep it alive
 * until the context is destroyed or given another workspace.  Setting a
 * new workspace discards the device state: call mdk_set_state again.
 */
int mdk_set_workspace(mdk_ctx *ctx, void *dev_ptr, size_t bytes);

/* ---- state ---------------------------------------------------------------- */

/*
 * Copy positions x [N][3] and velocities v [N][3] (Angstrom, Angstrom/fs)
 * into the context.  on_device: 0 = host pointers, 1 = device pointers.
 * v may be NULL (zero velocities).  Invalidates the neighbour list, numbers
 * the atoms 0..N-1 and restarts the step counter that keys the Langevin
 * noise (use a checkpoint to carry those over).
 */
int mdk_set_state(mdk_ctx *ctx, const double *x, const double *v, int on_device);

/*
 * Copy the current positions and velocities out, in the caller's atom
 * order.  Periodic coordinates are those wrapped into the box at the last
 * list build (then moved by the integrator since).  Either pointer may be
 * NULL.  Host copies synchronise the stream.  While a step is pending after
 * a list overflow (mdk_step), the velocities are those of the half step.
 */
int mdk_get_state(mdk_ctx *ctx, double *x, double *v, int on_device);

/* Current number of atoms (changes with the moving window; synchronises
 * when a window is set). */
int mdk_get_natoms(mdk_ctx *ctx, int64_t *n);

/*
 * Checkpoints: the whole dynamic state of a context in one host buffer, so a
 * run can stop and resume bit for bit (Sec. "Moving window simulation": long
 * shock runs restart from saved states), and so the Python binding can carry
 * a run over to a new, larger workspace.  A checkpoint holds, per atom, the
 * positions, velocities and stored forces, the positions of the last list
 * build (and of the last full build with two-level lists), the permanent id
 * and the type/piston word; and the step counter that keys the Langevin
 * noise, the build counters, the moving window's id counter and counts, the
 * piston speed and whether a step is pending (see mdk_step).
 * Configuration is not in it: load into a context made and configured like
 * the saving one (potential, list plan and kind, outer skin, capacity,
 * thermostats, window, thermo sampling), with its workspace set.  Loading
 * rebuilds the lists by replaying the last list build(s) at the saved build
 * positions, so cells, atom order, lists and the displacement trigger's
 * references equal the saving run's, and the continued run is bitwise the
 * uninterrupted one (same launch shape).
 *   mdk_checkpoint_size : bytes of a checkpoint of the current state
 *                         (synchronises)
 *   mdk_save_checkpoint : write it into the host buffer buf (bytes at least
 *                         mdk_checkpoint_size); synchronises.  Works while a
 *                         call reports MDK_ERR_WORKSPACE or
 *                         MDK_ERR_NEIGH_OVERFLOW, as long as the current
 *                         workspace is still allocated.
 *   mdk_load_checkpoint : replace the context's state by the checkpoint in
 *                         buf; synchronises.
 * Errors: MDK_ERR_ORDER (no state to save), MDK_ERR_BAD_ARG (buffer too
 * small, not a checkpoint, other precision or replica count, more atoms than
 * the capacity), MDK_ERR_WORKSPACE (no workspace to load into),
 * MDK_ERR_NEIGH_OVERFLOW (the replayed lists do not fit this context's list
 * capacity: the capacity was raised; set a larger workspace and load again).
 */
int mdk_checkpoint_size(mdk_ctx *ctx, size_t *bytes);
int mdk_save_checkpoint(mdk_ctx *ctx, void *buf, size_t bytes);
int mdk_load_checkpoint(mdk_ctx *ctx, const void *buf, size_t bytes);

/* ---- neighbour lists (Sec. "Neighbor lists construction", Eq. rhrz) ------ */

/*
 * Set the list parameters without building: search radius r_ns = rc + skin
 * (the paper's (1 + beta) r_cut with beta = skin/rc), per-atom capacity
 * max_neighbors (0 = estimate from the density), and the rebuild policy
 * rebuild_every (0 = rebuild when an atom has moved more than skin/2 since
 * the last build; k > 0 = also every k steps).  Changes the workspace size.
 */
int mdk_plan_neighbors(mdk_ctx *ctx, double rc, double skin, int max_neighbors,
                       int rebuild_every);

/*
 * Build the Verlet lists now: wrap periodic coordinates into the box, bin
 * atoms into cells of size >= rc + skin by a counting sort, reorder the
 * atoms into cell order, and keep every (j, image) with
 * |(x_j - x_i) + n L|^2 < (rc + skin)^2, (j, n) != (i, 0).  rc must be at
 * least the potential's cutoff.  MDK_ERR_NEIGH_OVERFLOW: the capacity was
 * raised; resize the workspace, set the state and build again.
 */
int mdk_build_neighbors(mdk_ctx *ctx, double rc, double skin);

/* Total number of (i, j, image) entries in the current lists. */
int mdk_neighbor_count(mdk_ctx *ctx, int64_t *total);

/*
 * Export the lists in the caller's atom order (host arrays):
 *   offsets [N+1]: entries of atom i are [offsets[i], offsets[i+1])
 *   j       [total]: neighbour atom (caller's index)
 *   image   [total][3]: periodic image n of the neighbour (box lengths),
 *                       relative to the positions mdk_get_state returns
 * Order within a list is unspecified.
 */
int mdk_get_neighbors(mdk_ctx *ctx, int64_t *offsets, int32_t *j, int32_t *image);

/* ---- forces and stepping -------------------------------------------------- */

/*
 * Potential energy E [1] (or [n_rep] for a batch), forces F [N][3] and
 * virial [6] (or [n_rep][6]: xx yy zz xy xz yz, W = 1/2 sum_i sum_j
 * r_ij (x) f_ij with r_ij = r_i - r_j; pressure P = (sum m v v + W)/V) at the
 * current positions.  Any output may be NULL.  f_i = sum_j V'(r_ij) r_ji/r_ji
 * (Sec. "Potentials support").  Rebuilds the lists first if needed.
 * on_device: 0 = host outputs (synchronises), 1 = device outputs.
 */
int mdk_compute(mdk_ctx *ctx, double *E, double *F, double *virial, int on_device);

/*
 * Per-atom potential energy U_i [N] and per-atom virial W_i [N][6] (host),
 * from the last mdk_compute (U = sum U_i, W = sum W_i).  Either may be NULL.
 */
int mdk_get_per_atom(mdk_ctx *ctx, double *Ui, double *Wi);

/*
 * Advance nsteps velocity-Verlet NVE steps of dt fs (Sec. "Molecular
 * dynamics"): v += dt/2 a; x += dt v; rebuild lists when triggered;
 * a = f(x)/m; v += dt/2 a.  All control stays on the GPU; the call only
 * enqueues work (errors of the steps themselves are read afterwards with
 * mdk_last_device_status).
 * List overflow (Sec. "Neighbor lists construction": every pair within r_ns
 * must be in the list): when a build triggered during the steps finds more
 * neighbours than the list capacity, stepping stops there -- every later
 * kernel of the call does nothing -- and mdk_last_device_status reports
 * MDK_ERR_NEIGH_OVERFLOW (the capacity is raised; the workspace must grow).
 * The state is then that of the moment of the build: the steps before it
 * are complete (mdk_get_counters counts them), positions have drifted and
 * velocities are at the half step, and that step's force pass is pending.
 * To resume: save a checkpoint, set a larger workspace, load the
 * checkpoint, and call mdk_step with the steps not yet done; it starts with
 * the pending force pass, and the run is bitwise the one a large enough
 * capacity would have given.  The Python binding does this by itself.
 */
int mdk_step(mdk_ctx *ctx, double dt, int64_t nsteps);

/*
 * Sample kinetic energy, potential energy and virial every `every` steps
 * of mdk_step (0 = off) into a device ring of up to `capacity` samples.
 */
int mdk_set_thermo(mdk_ctx *ctx, int every, int capacity);

/*
 * Copy the samples taken since the last call (host, synchronises): out
 * [max_samples][4 + 6] = step, E_kin, E_pot, n_atoms, virial[6] per sample
 * and per replica (replica-major within a sample).  n_out = samples copied.
 */
int mdk_get_thermo(mdk_ctx *ctx, double *out, int max_samples, int *n_out);

/* Number of list builds and of steps done so far (host, synchronises); after
 * a stepping overflow, the steps completed before it. */
int mdk_get_counters(mdk_ctx *ctx, int64_t *n_builds, int64_t *n_steps);

/*
 * Two-level lists (no paper counterpart: a way of building the same Verlet
 * list faster).  skin_outer > 0 keeps an outer list of every pair within
 * rc + skin_outer (full kind, built from cells of that size); at a rebuild
 * that the displacement trigger asks for, the Verlet list (rc + skin, full or
 * half) is filtered from the outer list instead of rebuilt from the cells,
 * as long as no atom has moved more than (skin_outer - skin) / 2 since the
 * outer list's build (measured at every build) -- then every pair within
 * rc + skin is in the outer list, and the Verlet list equals the
 * definition (the same FP32 pre-filter and exact FP64 test as a build from
 * cells).  Otherwise, and for explicit builds, window builds and the
 * list-free cell kernel, the build is a full one (re-bin, re-sort, outer
 * list, Verlet list).  skin_outer must exceed the planned skin; 0 turns the
 * outer list off (the default).  Call after mdk_plan_neighbors (or after a
 * potential setter, which plans with its cutoff and skin 0.3 when no plan
 * exists; MDK_ERR_ORDER with no plan at all); a later plan keeps the outer
 * skin while it exceeds the new skin.  The cells grow to rc + skin_outer
 * (periodic boxes must be at least that long: MDK_ERR_BOX_TOO_SMALL, and the
 * previous setting stays), the workspace grows by the outer list and the
 * positions of the last full build (mdk_workspace_size), and the next call
 * that needs the list rebuilds it.  Other errors: MDK_ERR_BAD_ARG for a
 * negative or non-finite value, one not above the skin, or one above
 * 10 (rc + skin) (the FP32 pre-filter's error bound, proportional to the
 * cell size, stays far inside its band below that).
 */
int mdk_set_outer_skin(mdk_ctx *ctx, double skin_outer);

/* Builds so far and, of them, full builds (with the outer list off every
 * build is full) (host, synchronises). */
int mdk_get_build_counts(mdk_ctx *ctx, int64_t *n_builds, int64_t *n_full);

/* ---- shock hook (Sec. "Moving window simulation") -------------------------- */

/*
 * Rigid piston: atoms with is_piston[i] != 0 (host, [N], caller's order)
 * move at v = (u_p, 0, 0) and ignore forces.  u_p in Angstrom/fs.
 * is_piston = NULL clears the piston.
 */
int mdk_set_piston(mdk_ctx *ctx, double u_p, const uint8_t *is_piston);

/*
 * Moving window along x for a piston-driven shock (Sec. "Moving window
 * simulation": atoms are inserted ahead of the shock from a prepared fresh
 * sample and deleted behind it).  Applied at every list build after this
 * call, on the device, in this order:
 *   the front: the box along x is cut into bins of width front_bin from
 *   box_lo[0] (atoms outside go to the end bins); a bin is shocked when the
 *   mean v_x of its atoms exceeds u_p/2 (decided exactly on velocities
 *   rounded to multiples of 2^-40 Angstrom/fs); x_front = upper edge of the
 *   last shocked bin (none: nothing happens);
 *   atoms with x < x_front - L_behind are deleted;
 *   while the leading edge x_max < x_front + L_ahead, copies of the fresh
 *   slab are appended: k = ceil((x_front + L_ahead - x_max)/slab_lx) copies,
 *   at most floor(((box_hi[0] - x_max) - slab_gap)/slab_lx) of them (none
 *   starts past the box), copy c shifted by ((x_max + slab_gap) + c slab_lx,
 *   0, 0), velocities slab_v, mass slab_mass, new ids counting up from N;
 *   atoms with x < x_min + piston_depth (x_min of the atoms left) join the
 *   piston.
 *   slab_x, slab_v : host [n_slab][3] positions (x in [0, slab_lx)) and
 *                    velocities of one fresh slab; copied.
 * The atom count changes: reserve room with mdk_set_capacity (appends that
 * do not fit are dropped and raise MDK_ERR_CAPACITY).  Once a window is
 * set, per-atom outputs come in ascending atom-id order (mdk_get_ids).
 * fixed_front: NaN to locate the front as above; a finite value fixes the
 * front at that x instead (the paper's stationary-shock window: outflow
 * deletion at fixed_front - L_behind, inflow layers -- give slab_v the
 * inflow velocity -- up to fixed_front + L_ahead; combine with
 * mdk_set_langevin for the inflow and outflow thermostats).
 * Single-system contexts with a free (non-periodic) x only; front_bin > 0
 * with at most 2^24 bins over the box.  Takes effect at the next list build.
 */
int mdk_set_window(mdk_ctx *ctx, double L_behind, double L_ahead, const double *slab_x,
                   const double *slab_v, int64_t n_slab, double slab_lx, double slab_gap,
                   double slab_mass, double piston_depth, double front_bin,
                   double fixed_front);

/* Ids of the atoms present, ascending (the order of every per-atom output). */
int mdk_get_ids(mdk_ctx *ctx, int64_t *ids);

/*
 * Langevin thermostat regions (Sec. "Molecular dynamics": a Langevin force
 * added to the right-hand side of Eq. MD-system gives the NVT ensemble;
 * Sec. "Moving window simulation": thermostats with a target temperature, a
 * target mean velocity and a stiffness beta in the inflow and outflow
 * regions).  At every force evaluation of mdk_step, an atom whose x lies in
 * region r (the first with x_lo[r] <= x < x_hi[r], piston atoms excluded)
 * gets, per component,
 *   F += -beta m (v - u_r) / A + sqrt(24 beta m k_B T_r / (dt A)) (xi - 1/2)
 * with v its half-step velocity, A = 9.648533212331e-3 (Angstrom/fs^2 per
 * eV/(Angstrom u)), k_B = 8.617333262e-5 eV/K, and xi uniform on [0, 1):
 * component d of Philox4x64-10 (Salmon et al., SC 2011) with counter
 * (permanent atom id, step index, 0, 0) and key (seed, 0), as (out >> 11)
 * 2^-53.  The step index counts the force evaluations of mdk_step since
 * mdk_set_state.  mdk_compute returns conservative forces only.
 *   n_regions   : 0 (off) to 8
 *   x_lo, x_hi  : host [n_regions], Angstrom
 *   T           : host [n_regions], K, >= 0
 *   u           : host [n_regions][3], Angstrom/fs
 *   beta        : host [n_regions], 1/fs, >= 0
 * Errors: MDK_ERR_BAD_ARG.  Takes effect at the next mdk_step.
 */
int mdk_set_langevin(mdk_ctx *ctx, int n_regions, const double *x_lo, const double *x_hi,
                     const double *T, const double *u, const double *beta, uint64_t seed);

/*
 * Per-replica Langevin thermostats for batched contexts (the isotherm runs of
 * Sec. "Argon shock Hugoniot": each replica of a volume-temperature grid
 * relaxed by a Langevin thermostat of stiffness beta at its own T).  Every
 * atom of replica r gets the force of mdk_set_langevin with T = T[r],
 * beta = beta[r] and target mean velocity 0, whatever its position (region
 * thermostats are then ignored).
 *   T, beta : host [n_replicas] (K, 1/fs), >= 0; T = NULL turns them off
 * Errors: MDK_ERR_BAD_ARG.
 */
int mdk_set_langevin_replicas(mdk_ctx *ctx, const double *T, const double *beta,
                              uint64_t seed);

/* Atoms appended and deleted by the moving window so far (synchronises). */
int mdk_window_counts(mdk_ctx *ctx, int64_t *inserted, int64_t *deleted);

/*
 * Per-bin statistics of the paper's Appendix along `axis` (0..2), for bins
 * [origin + l bin_w, origin + (l+1) bin_w), l < nbins, of volume
 * V_l = bin_w * cross_area; atoms outside every bin are ignored.
 * out [nbins][17] = N_l, M_l (u), u_l[3] (COM velocity, Angstrom/fs),
 * T_l[3] (K, per degree of freedom, about u_l), E_pot,l (sum of U_i, eV),
 * P_l[6] (eV/Angstrom^3; xx yy zz xy xz yz; kinetic + virial), E_kin,l
 * (peculiar, eV), V_l.  Per-atom energies and virials are taken at the
 * current positions (one force evaluation if the last one was not an
 * mdk_compute at these positions).  nbins * 41 <= 9 * capacity.
 * on_device: 0 = host out (synchronises), 1 = device out.
 */
int mdk_profiles(mdk_ctx *ctx, int axis, double origin, double bin_w, int nbins,
                 double cross_area, double *out, int on_device);

/* ---- adjoint of the EAM tables ------------------------------------------------ */

/*
 * Gradient of the loss L = sum_r gE[r] E_r + sum_i gF_i . F_i with respect to
 * the knot values of the EAM tables (EAM as in mdk_set_potential_eam and the
 * embedded-atom form of Sec. "Comparison of aluminum shock Hugoniot ...";
 * forces f_i = sum_j V'(r_ij) r_ji / r_ji of Sec. "Potentials support"), at
 * the current positions.  No counterpart in the paper, which evaluates the
 * tables only; this is the vector-Jacobian product of mdk_compute's E and F.
 *
 *   gE     : [n_replicas] weight of each replica's potential energy, or NULL (0)
 *   gF     : [N][3] weights of the forces, caller's atom order, or NULL (0)
 *   dtheta : [2 nr + nrho] output: dL/dphi_k (k < nr), dL/drho_k (nr knots),
 *            dL/dF_k (nrho knots), in the order of mdk_set_potential_eam
 *   on_device : 0 = host arrays (the call synchronises and returns the
 *            device status, as mdk_compute); 1 = device arrays (returns
 *            after enqueueing).
 * Pair distances are recomputed from the positions and the Verlet list (none
 * are stored).  Pair arithmetic is in the context's precision (FP32 in
 * MDK_MIXED); per-atom terms and all gradient sums are FP64.  Gradients are
 * summed with FP64 atomics, so two calls agree to rounding, not bit for bit.
 * The kernels need 32 * nr bytes of shared memory (nr <= 7168).
 * Errors: MDK_ERR_ORDER when the potential is not EAM, the state is not set
 * or the moving window is on; MDK_ERR_WORKSPACE as mdk_compute.
 */
int mdk_eam_vjp(mdk_ctx *ctx, const double *gE, const double *gF, double *dtheta, int on_device);

/* ---- allocation-free variant ------------------------------------------------ */

/* Fixed maximum sizes of mdk_lj_compute_noalloc. */
#define MDK_NOALLOC_MAX_ATOMS 32768
#define MDK_NOALLOC_MAX_CELLS 32768

/*
 * Lennard-Jones energy and forces of one small system, for callers that
 * cannot allocate device memory: code whose device memory is owned by
 * another allocator (a framework's caching pool or a fixed arena reserved at
 * start-up, where an extra cudaMalloc would fail or fragment it), or a host
 * loop that must not pay for an allocation or the device-wide
 * synchronisation cudaFree implies.  This entry point allocates nothing and
 * needs no context or workspace.  (No counterpart in the paper; it is a
 * variant of the force kernel behind mdk_compute.)
 *
 * Its scratch (cell histogram and starts, atoms sorted by cell, wrapped
 * positions, per-atom energies: about 1.9 MB) is one file-scope __device__
 * array in libmdk.so, which every GPU that loads the library holds until the
 * process exits.  The first call on a device looks that array's address up
 * (with the device current) and keeps it; make the first call on each device
 * before any stream capture.  The kept address belongs to the device's
 * context of that moment: after cudaDeviceReset on a device, do not call
 * this entry point on that device again in the same process.  All calls
 * share the array and each call clears what it needs, so two calls whose
 * work overlaps on one GPU (for example, calls on two streams) race:
 * serialise them.
 *
 *   x        : device [N][3] positions (Angstrom), read only
 *   N        : 0 <= N <= MDK_NOALLOC_MAX_ATOMS, else MDK_ERR_TOO_LARGE
 *   box_lo/hi, periodic : host [3]; periodic lengths must be >= rc; the
 *              grid of cells of size >= rc must have at most
 *              MDK_NOALLOC_MAX_CELLS cells (else MDK_ERR_TOO_LARGE)
 *   eps, sigma, rc, shift_mode : as mdk_set_potential_lj
 *   F        : device [N][3] forces (eV/Angstrom), written
 *   E        : device [1] potential energy (eV), written
 *   cuda_stream : stream to run on (NULL = legacy default stream)
 * Same definitions, pair vectors and FP64 arithmetic as mdk_compute in
 * MDK_FP64 mode (the cell search replaces the Verlet list; pairs with
 * r < rc only).  Returns without synchronising, so device-side problems
 * show in the results: an atom with a NaN or Inf coordinate takes part in
 * no pair, and its row of F and E are NaN (the other atoms' forces are
 * those of the system without it).
 */
int mdk_lj_compute_noalloc(const double *x, int64_t N, const double box_lo[3],
                           const double box_hi[3], const int periodic[3], double eps,
                           double sigma, double rc, int shift_mode, double *F, double *E,
                           void *cuda_stream);

/* ---- launch shape ---------------------------------------------------------- */

/*
 * Autotuner: time every launch shape of the force kernels -- threads per atom
 * in {1, 2, 4, 8, 32} (32: a warp per atom) x threads per block in {128, 256,
 * 512} (LJ: <= 256) -- on this context's system (reps force passes each, CUDA
 * events on the context's stream) and keep the fastest for later calls.  With
 * LJ and EAM it also times half lists (one thread per atom; 128 and 256
 * threads per block), with LJ the list-free cell kernel (128 and 256 threads
 * per block), and keeps the fastest list kind (mdk_get_list_kind reports it; a
 * switch rebuilds the list).  The BPNN kernel has one shape (a warp per atom).
 * Outputs may be NULL.  Small systems (few atoms per SM)
 * and long lists favour several threads per atom.  The state must be set;
 * the lists are built if needed.  (No paper counterpart: the paper chunks
 * arrays over a thread pool.)
 */
int mdk_autotune(mdk_ctx *ctx, int reps, int *tpa, int *block, double *ms);

/* Set the launch shape directly: tpa (list-walking lanes per atom) in {1, 2, 4, 8, 32}
 * (32: a warp per atom), block in {128, 256, 512}. */
int mdk_set_launch(mdk_ctx *ctx, int tpa, int block);

/*
 * Verlet-list kind (Sec. "Neighbor lists" keeps every pair within r_ns; how
 * a pair is stored is the implementation's choice):
 *   MDK_LIST_FULL (default): every atom lists all its neighbours, each pair
 *     is evaluated twice, once for each atom, and the per-atom force sums
 *     need no atomics (fused with the velocity-Verlet update).
 *   MDK_LIST_HALF: each unordered pair (i, j, image) appears in one of the
 *     two lists; the force pass adds f_ij to i and -f_ij to j (Newton's
 *     third law) with reduction atomics into per-atom accumulators and a
 *     per-atom pass finishes the step (EAM: the density pass adds rho(r)
 *     to both atoms, a per-atom pass evaluates F and F', then the force
 *     pass).  Mixed precision accumulates in 64-bit fixed point (unit 2^-40
 *     eV/A): bitwise reproducible, the forces sum to exactly zero, a pair
 *     term at or above 2^22 eV/A reports MDK_ERR_NONFINITE.  FP64
 *     accumulates with FP64 atomics (reproducible to rounding, not
 *     bitwise).  LJ and EAM: MDK_ERR_ORDER before a potential is set,
 *     MDK_ERR_BAD_ARG with the BPNN potential (setting one returns the
 *     context to full lists).  mdk_eam_vjp walks full lists and switches a
 *     half-list context back to full lists (the next call rebuilds).
 *   MDK_LIST_CELLS (LJ only): no Verlet list.  A build sorts the atoms into
 *     cells of size >= rc + skin as usual and skips the list; the force pass
 *     takes one warp per cell, stages 32 neighbour records at a time from
 *     the 27 template cells in shared memory and tests all of them against
 *     the cell's atoms (pairs closer than rc at the current positions are in
 *     adjacent build cells while no atom has moved more than skin/2).  Same
 *     definitions and bars as the list kernels; mdk_get_neighbors and
 *     mdk_neighbor_count return MDK_ERR_ORDER.  Setting an EAM potential
 *     returns the context to full lists.
 * A change of kind makes the next call rebuild the list; mdk_get_neighbors
 * returns the list of the current kind.
 */
#define MDK_LIST_FULL 0
#define MDK_LIST_HALF 1
#define MDK_LIST_CELLS 2
int mdk_set_list_kind(mdk_ctx *ctx, int kind);
int mdk_get_list_kind(const mdk_ctx *ctx, int *kind);

/*
 * enable != 0 (the default): mdk_step runs pairs of plain steps (neither a
 * thermo step nor the last step of the call) as one CUDA graph -- force pass
 * and rebuild chain twice -- captured on first use and re-captured whenever a
 * parameter it baked in changes (workspace, potential, launch shape, dt,
 * window...).  Steps taken while mdk_profile records run without graphs.
 */
int mdk_set_graphs(mdk_ctx *ctx, int enable);

/* ---- measurement ----------------------------------------------------------- */

/*
 * FMA throughput of the current device in TFLOP/s (one FMA = 2 FLOP):
 * precision MDK_FP64 times FP64 FMAs, MDK_MIXED FP32 FMAs; 8 independent
 * chains per thread, 8 blocks of 256 threads per SM, one warm-up launch,
 * CUDA events around the timed launch (~20-70 ms).  The denominator of the
 * ALU rooflines (FP64 force loops, FP32 BPNN kernel).  Synchronous; uses
 * the legacy default stream and a small temporary allocation.
 */
int mdk_fma_peak(int precision, double *tflops);

/*
 * enable != 0: from now on bracket every force pass and every list-rebuild
 * chain enqueued by mdk_step / mdk_compute with CUDA events on the context's
 * stream, and count the kernels launched.  enable = 0 stops recording.
 * Either call clears the counters.  (Measurement aid; no paper counterpart.)
 */
int mdk_profile(mdk_ctx *ctx, int enable);

/*
 * Read the counters (host, synchronises the stream).  out [8]:
 *   [0] total ms of force passes   [1] number of force passes
 *   [2] total ms of rebuild chains [3] number of rebuild chains
 *   [4] kernels launched           [5] list builds done (device count)
 *   [6] ms of the first-kick/drift kernels  [7] number of them
 */
int mdk_get_profile(mdk_ctx *ctx, double *out);

/* ---- errors ------------------------------------------------------------- */

/* Static string naming a status code. */
const char *mdk_status_string(int status);

/* Device-side status bits raised since the last call (synchronises). */
int mdk_last_device_status(mdk_ctx *ctx, int *bits);

#ifdef __cplusplus
}
#endif

#endif /* MDK_H */
