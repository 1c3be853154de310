/*
 * libmpm: the explicit material point method (MPM) time step of JAX-MPM
 * (Du & He, "JAX-MPM: A Learning-Augmented Differentiable Meshfree Framework
 * for GPU-Accelerated Lagrangian Simulation and Geophysical Inverse Modeling",
 * arXiv 2507.04192), on hand-written CUDA kernels for sm_103a.
 *
 * One step (Sec. 2.2, restated as the map S^{t+1} = Phi(S^t; alpha) of Eq.
 * mapping in Sec. 3.1) is: particle-to-grid transfer of mass, APIC momentum
 * (Appendix B) and stress force (Eq. update_m, Eq. semi); the explicit grid
 * update with gravity (Eq. semi_eq) and Coulomb wall friction (Eq.
 * coulomb_friction, Sec. 5.3); and the grid-to-particle transfer with the
 * velocity gradient (Eq. update_v_gradient), deformation gradient, density
 * and stress update (Sec. 2.3, Appendix A), updated stress last.  Particles
 * are re-sorted by grid cell every few steps so that the transfers work on
 * shared-memory tiles of the grid.
 *
 * Conventions for every call:
 *  - Every function returns an mpm_status (MPM_OK = 0 or a negative code);
 *    mpm_last_error() gives a one-line message for the last failure.
 *  - Host buffers are owned by the caller; the library copies from them
 *    before the call returns and keeps no pointer to them.
 *  - Particle arrays are indexed in load order (the order of
 *    mpm_load_particles), whatever the internal sorted order.
 *  - Per-particle tensors are row-major: x and v are n x dim, C and F are
 *    n x dim x dim, sigma is n x 3 x 3 (plane strain in 2D).
 *  - Device work is queued on the context's CUDA stream and runs
 *    asynchronously; device-side faults (a non-finite particle state) are
 *    recorded in a device status word and reported by the next call that
 *    synchronises (mpm_synchronize, mpm_get_particles), never by a trap.
 *  - A context is not thread-safe: use one context per host thread/stream.
 */
#ifndef LIBMPM_MPM_H
#define LIBMPM_MPM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mpm_ctx mpm_ctx;

typedef enum {
    MPM_OK = 0,
    MPM_EINVAL = -1,     /* invalid argument or unsupported configuration */
    MPM_ENOMEM = -2,     /* device or host allocation failed */
    MPM_ECUDA = -3,      /* a CUDA runtime call failed */
    MPM_ENAN = -4,       /* a particle state became non-finite */
    MPM_EDOMAIN = -5,    /* a particle index left the grid (never expected: positions are clamped) */
    MPM_ETIMEOUT = -6,   /* a bounded device wait ran out */
    MPM_ECORRUPT = -7,   /* a state blob failed its checksum */
    MPM_ESTATE = -8      /* call not valid in the context's current state */
} mpm_status;

enum { MPM_FP32 = 0, MPM_FP64 = 1 };
enum { MPM_FLUID = 0, MPM_DRUCKER_PRAGER = 1 };

/* Particle fields for mpm_get_particles / mpm_set_particle_field.
 * Widths per particle: X, V: dim; C, F: dim*dim; RHO, EPS: 1; SIGMA: 9. */
enum {
    MPM_FIELD_X = 0,      /* position x_p */
    MPM_FIELD_V = 1,      /* velocity v_p */
    MPM_FIELD_C = 2,      /* APIC affine matrix C_p = B_p D_p^{-1} (Appendix B) */
    MPM_FIELD_F = 3,      /* deformation gradient F_p */
    MPM_FIELD_RHO = 4,    /* density rho_p */
    MPM_FIELD_SIGMA = 5,  /* Cauchy stress sigma_p (fluid: -p I from the equation of state) */
    MPM_FIELD_EPS = 6     /* equivalent plastic strain (Drucker-Prager) */
};

/*
 * Grid and time step.  The domain is [0, n_cells[a] * dx] per axis a < dim;
 * walls sit on its faces (Sec. 2.2, ghost cells: one node beyond each face).
 *   dim        2 or 3
 *   n_cells    cells per axis (entries >= dim are ignored), each in [1, 4096]
 *   dx, dt     grid spacing and fixed time step (> 0)
 *   gravity    body force per unit mass b (Eq. semi)
 *   precision  MPM_FP32 (all particle and grid arithmetic in float) or MPM_FP64
 *   sort_every re-sort particles by cell every this many steps (>= 1); a
 *              particle that has moved more than one cell since the last sort
 *              stays correct through a slower path
 *   batch      number of independent simulations sharing the grid shape (>= 1);
 *              particles carry a simulation id (mpm_load_particles)
 *   transfer   G2P transfer (Sec. 2.2 G2P transfer, Appendix B): MPM_TRANSFER_APIC
 *              (affine matrix C_p = B_p D_p^-1 carried to the next P2G), _TPIC (the
 *              particle velocity gradient instead), _PIC (no particle matrix),
 *              _FLIP (v_p += sum phi (v_i^{n+1} - v_i^n), blended with PIC:
 *              v_p = v_PIC + flip_alpha (v_p - sum phi v_i^n); no particle matrix;
 *              positions advance with the PIC velocity)
 *   flip_alpha FLIP share of the blend, in [0, 1] (used by _FLIP only)
 */
enum { MPM_TRANSFER_APIC = 0, MPM_TRANSFER_TPIC = 1, MPM_TRANSFER_PIC = 2, MPM_TRANSFER_FLIP = 3 };
typedef struct {
    int dim;
    int n_cells[3];
    double dx;
    double dt;
    double gravity[3];
    int precision;
    int sort_every;
    int batch;
    int transfer;
    double flip_alpha;
} mpm_grid_desc;

/*
 * Material (Sec. 2.3).
 *   kind = MPM_FLUID: weakly compressible fluid, Tait equation of state
 *       p = (bulk_K / gamma) ((rho / rho0)^gamma - 1); gamma = 1 is the paper's
 *       linear EOS c^2 (rho - rho0) with c^2 = bulk_K / rho0 (Eq. eos).
 *       viscosity must be 0 (the paper's inviscid cases; MPM_EINVAL otherwise).
 *   kind = MPM_DRUCKER_PRAGER: Drucker-Prager with tension cutoff and the
 *       Jaumann rate (Eq. dp_stress, Appendix A); Young's modulus E, Poisson
 *       ratio nu, friction and dilation angles in degrees, cohesion, tensile
 *       strength sigma_t (capped at the cone apex k_phi / q_phi).
 *       dp_literal = 1 applies Appendix A exactly as printed; 0 (default) adds
 *       the corner return when a return lands past the tension cutoff.
 *   rho0: reference density (fluid) or initial density (sand); particle mass
 *       is rho0 * particle_volume.
 * mpm_create rejects (MPM_EINVAL) non-finite or non-positive rho0, bulk_K, gamma
 * and E; nu outside (-1, 0.5); angles outside [0, 90) degrees; a negative or
 * non-finite cohesion or sigma_t.
 */
typedef struct {
    int kind;
    double rho0, bulk_K, gamma, viscosity;
    double E, nu, phi_deg, psi_deg, cohesion, sigma_t;
    int dp_literal;
} mpm_material;

/*
 * Create a context for one grid shape and material.  cuda_stream is a
 * cudaStream_t (NULL: the library creates its own non-blocking stream).
 * The context owns all its device memory.  Returns MPM_EINVAL for an invalid
 * descriptor, MPM_ENOMEM/MPM_ECUDA on device failures; *out is set only on
 * success.
 */
int mpm_create(const mpm_grid_desc *grid, const mpm_material *material, void *cuda_stream,
               mpm_ctx **out);

/* Free the context and all its device memory (NULL is accepted). */
void mpm_destroy(mpm_ctx *ctx);

/*
 * Load n particles (the initial state S^0 of Sec. 3.1): positions x (n x dim,
 * host, inside the domain), optional velocities v (n x dim, NULL = at rest),
 * the common initial volume V_p^0, and optional simulation ids (n, each in
 * [0, batch), NULL = all 0).  The rest of the state starts at C = 0, F = I,
 * rho = rho0, sigma = 0, eps = 0.  Replaces any previous particles.
 */
int mpm_load_particles(mpm_ctx *ctx, int64_t n, const double *x, const double *v,
                       double particle_volume, const int32_t *sim_id);

/*
 * mpm_load_particles from device memory: x_dev (n x dim doubles), v_dev (n x dim
 * doubles or NULL) and sim_id_dev (n int32 or NULL) are device pointers the
 * caller owns (e.g. the data_ptr() of CUDA tensors); they are read on the
 * context's stream, so work the caller queued on that stream before the call
 * is ordered before the read, and the call returns after the copy (they may be
 * freed then).  The same checks as mpm_load_particles, made on the device, with
 * the same statuses.
 */
int mpm_load_particles_dev(mpm_ctx *ctx, int64_t n, const double *x_dev, const double *v_dev,
                           double particle_volume, const int32_t *sim_id_dev);

/*
 * Overwrite one particle field from a host array in load order, with
 * mpm_field_width() values per particle (the caller keeps ownership; it is
 * copied before the call returns).  Returns MPM_EINVAL for a NULL array, an
 * unknown field, sigma or eps of a fluid (its stress follows from the density),
 * or positions outside the domain or not finite; MPM_ESTATE before any
 * particles are loaded.  Non-finite values of the other fields are accepted:
 * those that feed the dynamics (v, C, rho, sigma) surface as MPM_ENAN at the
 * synchronisation after the next step; F and eps do not feed back and are not
 * checked.
 */
int mpm_set_particle_field(mpm_ctx *ctx, int field, const double *values);

/*
 * Friction field of one wall (Eq. coulomb_friction).  Walls are numbered
 * 2*axis + side (side 0 = low face, 1 = high face); the floor is the low face
 * of the last axis (wall 2 in 2D, 4 in 3D).  The wall is cut into
 * n_seg[0] x n_seg[1] equal segments along its tangential axes in increasing
 * axis order (n_seg[1] = 1 in 2D); mu holds batch * n_seg[1] * n_seg[0]
 * coefficients >= 0, row-major [sim][s1][s0].  A node at tangential coordinate
 * x_t belongs to segment floor(x_t / L_t * n_seg) clamped to [0, n_seg - 1].
 * Walls without a friction field are slip walls (mu = 0).  MPM_EINVAL for a
 * wall out of range, a segment count outside 1..65536, or a negative or
 * non-finite coefficient.
 */
int mpm_set_friction_field(mpm_ctx *ctx, int wall, const int n_seg[2], const double *mu);

/*
 * Stationary rigid obstacles with frictionless contact (Sec. 4.1, 3D dam break:
 * the predicted grid velocity loses its normal component at the obstacle,
 * v_i = v~_i - (v~_i . n_i) n_i).  boxes holds n_obstacles axis-aligned boxes,
 * each dim low-corner coordinates then dim high-corner coordinates (metres,
 * host, copied); at most MPM_MAX_OBSTACLES; n_obstacles = 0 removes them.  A
 * grid node whose coordinate lies in a closed box (box extents rounded to the
 * nodes ceil(lo / dx - 1e-9) .. floor(hi / dx + 1e-9)) takes the outward normal
 * of the nearest box face that lies strictly inside the domain (ties: the first
 * of x-, x+, y-, y+, z-, z+) and, when it moves into the box (v . n < 0), loses
 * its normal velocity.  Obstacles act before the walls; they apply to every
 * simulation of a batch and are differentiated by mpm_step_adjoint.
 * MPM_EINVAL for a count out of range, a box with lo > hi on some axis, or a
 * box with no face inside the domain.
 */
#define MPM_MAX_OBSTACLES 8
int mpm_set_obstacles(mpm_ctx *ctx, int n_obstacles, const double *boxes);

/* Queue n_steps explicit MPM steps on the context's stream (asynchronous).
 * MPM_EINVAL for n_steps < 0, MPM_ESTATE before any particles are loaded,
 * MPM_ECUDA when a launch fails; a non-finite state or a bounded device wait
 * that ran out is reported by the next synchronising call. */
int mpm_step(mpm_ctx *ctx, int n_steps);

/*
 * Sort the particles by cell at the start of the next step, whatever the sort
 * interval says (the interval restarts there).  The sort is an internal
 * reordering (not part of the paper's method, which scatters unsorted
 * particles, Sec. 3.3.1): results depend on it only through the rounding of
 * the summation order.  MPM_EINVAL for a NULL context.
 */
int mpm_request_sort(mpm_ctx *ctx);

/*
 * Conservation sums of the particle-to-grid transfer (Sec. 2.2: the grid mass
 * m_i of Eq. update_m and the momentum q_i + dt f_i of Eq. semi before the grid
 * update).  With enable != 0, every later step also sums, on the device and in
 * double precision, the grid values the transfer produced and the particle
 * state it read; mpm_get_diagnostics copies the sums of the last such step
 * (synchronises) into out[0 .. n) (n <= MPM_DIAG_COUNT):
 *   out[0]     sum_i m_i over every grid node (all simulations of a batch)
 *   out[1..3]  sum_i (q_i + dt f_i), components beyond dim are 0
 *   out[4]     sum_p m_p of the particles
 *   out[5..7]  sum_p m_p v_p
 *   out[8]     grid nodes with a non-finite mass or momentum value
 *   out[9]     particles with a non-finite position or velocity
 *   out[10]    sum_i of |q_i + dt f_i| summed over its components (the scale
 *              of the rounding of out[1..3])
 * The B-spline weights form a partition of unity with linear reproduction and
 * sum_i grad w_ip = 0 (Sec. 2.1), so out[0] = out[4] and out[1..3] = out[5..7]
 * up to rounding.  Enabling costs one extra kernel per step and a reduction in
 * the grid update.  MPM_EINVAL for bad arguments, MPM_ENOMEM when the 88-byte
 * device buffer cannot be allocated, MPM_ESTATE when no step has run with the
 * sums enabled.
 */
#define MPM_DIAG_COUNT 11
int mpm_set_diagnostics(mpm_ctx *ctx, int enable);
int mpm_get_diagnostics(mpm_ctx *ctx, double *out, int n);

/*
 * Test hook of the error paths (not part of the method): flags =
 * MPM_DEBUG_WITHHOLD_WINDOW_COPY makes the grid-to-particle kernel arm no copy
 * for its shared-memory grid window, so that its bounded device wait (about one
 * second) runs out with no copy in flight; the next synchronising call then
 * returns MPM_ETIMEOUT and the particle state is left partly updated.  0 turns
 * the hook off.  MPM_EINVAL for an unknown flag.
 */
#define MPM_DEBUG_WITHHOLD_WINDOW_COPY 1
int mpm_set_debug(mpm_ctx *ctx, int flags);

/* Wait for queued work; returns MPM_ENAN if any particle state became non-finite. */
int mpm_synchronize(mpm_ctx *ctx);

/* Copy one particle field to host memory (load order, doubles, the field's
 * width per particle); synchronises.  MPM_EINVAL for a NULL buffer or an
 * unknown field, MPM_ESTATE before any particles are loaded, and any status the
 * queued steps recorded (MPM_ENAN, MPM_ETIMEOUT). */
int mpm_get_particles(mpm_ctx *ctx, int field, double *out);

/* mpm_get_particles into device memory: out_dev (n x the field's width doubles,
 * load order) is a device pointer the caller owns; the copy is queued on the
 * context's stream and the call returns without waiting (later work on that
 * stream sees the values).  MPM_EINVAL for a NULL pointer or an unknown field,
 * MPM_ESTATE before any particles are loaded; statuses the queued steps record
 * are reported by the next synchronising call. */
int mpm_get_particles_dev(mpm_ctx *ctx, int field, double *out_dev);

/* Number of doubles per particle of a field (or a negative status). */
int mpm_field_width(const mpm_ctx *ctx, int field);

/* Number of loaded particles (0 before mpm_load_particles). */
int64_t mpm_num_particles(const mpm_ctx *ctx);

/* Copy the last error message (NUL-terminated, truncated to len). */
int mpm_last_error(const mpm_ctx *ctx, char *buf, int len);

/*
 * Observations for the inverse loss of Eq. inverse_loss (Sec. 3.2), Lagrangian
 * form (tracked particles, Q_l(z) = [z]_l): n_track load-order particle ids
 * (distinct), n_obs observation steps (>= 1, increasing, counted from the state
 * at the start of mpm_step_adjoint) and the observed positions z_obs
 * (n_obs x n_track x dim, host).  The loss is
 *     L = sum_obs sum_l |x_{id_l}^{step} - z_obs|^2.
 * n_track = 0 clears them (the other arguments are then ignored).  MPM_EINVAL
 * for an id out of range or repeated, or steps that are not >= 1 and
 * increasing; MPM_ESTATE before any particles are loaded.
 */
int mpm_set_observations(mpm_ctx *ctx, int n_track, const int64_t *ids, int n_obs, const int *steps,
                         const double *z_obs);

/*
 * Eulerian observations of Eq. inverse_loss (Sec. 5.2, Case 3): velocity
 * monitors.  n_mon (<= 64) closed boxes (boxes: per monitor dim low-corner then
 * dim high-corner coordinates, metres), n_obs observation steps (>= 1,
 * increasing) and the observed mean velocities v_obs (n_obs x n_mon x dim, host,
 * copied).  At an observation step the monitor's quantity is the mean velocity
 * Q_l = (1 / |P_l|) sum_{p in P_l} v_p of the particles P_l whose position lies
 * in the box; the loss adds sum_obs sum_l |Q_l - v_obs|^2 over the monitors
 * holding particles (an empty monitor adds nothing).  In the adjoint the
 * membership P_l is held at its forward value.  n_mon = 0 clears the monitors.
 */
#define MPM_MAX_MONITORS 64
int mpm_set_velocity_monitors(mpm_ctx *ctx, int n_mon, const double *boxes, int n_obs, const int *steps,
                              const double *v_obs);

/*
 * The monitors' quantities on the current state (boxes as in
 * mpm_set_velocity_monitors, batch 1): per monitor the mean velocity (dim
 * values, 0 when empty) and the particle count, out = n_mon x (dim + 1) doubles
 * (host); synchronises.  Used to record Eulerian observations of a run.
 * MPM_EINVAL for n_mon outside 1..MPM_MAX_MONITORS, a box with lo > hi or a
 * non-finite bound, or batch != 1; MPM_ESTATE before any particles are loaded.
 */
int mpm_monitor_means(mpm_ctx *ctx, int n_mon, const double *boxes, double *out);

/*
 * Loss and its gradient with respect to one wall's friction field (the
 * reverse-mode recursion of Eq. dzda, Sec. 3.1; loss gradient of Sec. 3.2).
 * Runs n_steps explicit steps from the current state, saving the particle
 * state every checkpoint_every steps (Sec. 3.3.2); then walks the segments
 * backwards, recomputing each segment's states from its checkpoint and
 * applying the adjoint of each step.  Writes the loss (tracked particles and
 * velocity monitors together) and dL/dmu (the wall's n_seg[0] x n_seg[1]
 * coefficients, set by mpm_set_friction_field; wall = -1 asks for no friction
 * gradient and dL_dmu_out may then be NULL) to host memory and leaves the
 * context at the state after n_steps steps; the adjoint of the initial state
 * is then available through mpm_get_initial_adjoint.  Both
 * materials (the adjoint state is (x, v, C, rho) for the fluid and (x, v, C,
 * rho, sigma) for Drucker-Prager; the zone and contact branches of the forward
 * step are held fixed), batch 1.  Device memory: checkpoints of
 * (2 dim + dim^2 + 1) reals per particle each (+ 6 for Drucker-Prager), plus
 * two banks of checkpoint_every states with their grids (more segments with
 * mpm_set_adjoint_memory), plus in 3D single precision 21 reals per particle of
 * scatter coefficients and the sort tables of each sort generation the kept
 * states span.  With the default memory setting and more than one segment, the
 * reverse steps of a segment run on a second stream the library owns while the
 * segment before it is recomputed on the context's stream; the call returns
 * with all of that work ordered before later work on the context's stream.
 * MPM_EINVAL for n_steps or checkpoint_every < 1, a NULL loss_out (or a NULL
 * dL_dmu_out with wall >= 0), a batch other than 1, a transfer other than APIC,
 * a wall without a friction field, or an observation beyond n_steps;
 * MPM_ESTATE before any particles or observations are set; MPM_ENOMEM when the
 * checkpoints do not fit; and any status the steps recorded.
 */
int mpm_step_adjoint(mpm_ctx *ctx, int n_steps, int checkpoint_every, int wall, double *loss_out,
                     double *dL_dmu_out);

/*
 * One step and its vector-Jacobian product (Eq. dzda for a single step, Sec.
 * 3.1): from the current state S^t, runs the step to S^{t+1} (the context is
 * left there) and, given lam_next = dL/dS^{t+1}, writes lam_prev = dL/dS^t and,
 * for wall >= 0, this step's d<lam_next, S^{t+1}>/dmu of the wall's friction
 * field (n_seg[0] x n_seg[1] doubles; wall = -1: none, dL_dmu_out may be NULL).
 * A caller chains it backwards over stored states (mpm_save_state before each
 * forward step, mpm_restore_state before each call), adding the gradient of
 * its loss at each observed state to lam between calls: the per-step form of
 * mpm_step_adjoint, for an autograd function of one step.  Adjoint layout (host
 * memory, load order, doubles): per particle mpm_adjoint_width() values, the
 * adjoints of x (dim), v (dim), C (dim^2, row-major), rho (1) and, for
 * Drucker-Prager, sigma (6: xx yy zz xy xz yz); the zone and contact branches
 * of the step are held fixed, as in mpm_step_adjoint.  APIC transfer, batch 1.
 * MPM_EINVAL for a NULL array (or NULL dL_dmu_out with wall >= 0), a batch
 * other than 1, a transfer other than APIC, a wall without a friction field;
 * MPM_ESTATE before any particles are loaded; MPM_ENOMEM; and any status the
 * step recorded.  Synchronises.
 */
int mpm_step_adjoint_1(mpm_ctx *ctx, int wall, const double *lam_next, double *lam_prev, double *dL_dmu_out);

/* Adjoint values per particle of mpm_step_adjoint_1 (2 dim + dim^2 + 1, + 6 for
 * Drucker-Prager), or a negative status. */
int mpm_adjoint_width(const mpm_ctx *ctx);

/*
 * Device memory (bytes) mpm_step_adjoint may use, beyond what one segment of
 * checkpoint_every states needs, to keep more segments of the first forward
 * pass: the last 1 + bytes / (one segment's size) segments are then reversed
 * without recomputation (Sec. 3.3.2 trades memory for recomputation; a GPU with
 * memory to spare can keep the whole horizon).  Default 0: only the last
 * segment is kept and every other one is recomputed from its checkpoint (into
 * the other of two banks, while the segment after it is reversed).  A
 * segment of K states takes K x ((2 dim + dim^2 + 1 [+ 6]) reals per particle
 * + two grids of 4 reals per node + 4 bytes per particle) plus the sort tables
 * of its sort generations.  The result does not depend on the setting.
 */
int mpm_set_adjoint_memory(mpm_ctx *ctx, int64_t bytes);

/*
 * dL/d(field of the initial state) of the last mpm_step_adjoint (the adjoint
 * state lambda^0 of Eq. dzda): MPM_FIELD_X, MPM_FIELD_V, MPM_FIELD_C (the APIC
 * affine matrix) or MPM_FIELD_RHO, written to host memory in load order with
 * the field's width per particle (synchronises).  With it the loss gradient
 * with respect to any parametrisation of the initial state (Sec. 5.2: an initial
 * velocity constant or a network field v0(x)) follows by the chain rule.
 * MPM_ESTATE before any adjoint; MPM_EINVAL for other fields.
 */
int mpm_get_initial_adjoint(mpm_ctx *ctx, int field, double *out);

/*
 * Device state slots (0..15): copy of the whole particle state (all fields, in
 * the current internal order).  mpm_restore_state puts it back; used to rerun
 * a trajectory from the same start (inversion loops).  Slots are freed with
 * the particles.  MPM_EINVAL for a slot out of range; MPM_ESTATE to save before
 * any particles are loaded or to restore an empty slot (or one saved for
 * another particle count).
 */
int mpm_save_state(mpm_ctx *ctx, int slot);
int mpm_restore_state(mpm_ctx *ctx, int slot);

/*
 * Host blob of the particle state for checkpoint/resume across processes.
 * mpm_state_blob_size gives the bytes needed; mpm_export_state writes the blob
 * (header, all fields, ids, simulation ids, FNV-1a checksum of the payload);
 * mpm_import_state verifies it before anything reaches the device
 * (MPM_ECORRUPT on a bad magic, a payload size other than the loaded particles'
 * state, truncation, a checksum mismatch, particle ids that are not a
 * permutation of 0..n-1 or simulation ids outside the batch; MPM_EINVAL if its
 * header does not match the loaded particles).  The caller owns the blob.
 */
int64_t mpm_state_blob_size(const mpm_ctx *ctx);
int mpm_export_state(mpm_ctx *ctx, void *blob, int64_t size);
int mpm_import_state(mpm_ctx *ctx, const void *blob, int64_t size);

/*
 * Kernel timing.  When enabled, every kernel launch is bracketed by CUDA
 * events on the context's stream; mpm_get_timing returns, for one kernel
 * class, the summed device time in milliseconds and the launch count since
 * the last reset (synchronises).  Kernel classes: see MPM_KERNEL_*.
 */
enum {
    MPM_KERNEL_SORT = 0,        /* keys, radix passes, permutation, tile lists */
    MPM_KERNEL_P2G = 1,
    MPM_KERNEL_GRID = 2,
    MPM_KERNEL_G2P = 3,
    MPM_KERNEL_REVERSE = 4,     /* one reverse step of mpm_step_adjoint (all its kernels) */
    MPM_KERNEL_COUNT = 5
};
int mpm_set_timing(mpm_ctx *ctx, int enable);
int mpm_get_timing(mpm_ctx *ctx, int kernel, double *total_ms, int64_t *launches);
int mpm_reset_timing(mpm_ctx *ctx);

/*
 * Counters (synchronises).  out[0] active tiles, out[1] work units (tiles) after the
 * last sort, out[2] particles that took the out-of-tile path since creation,
 * out[3] sorts, out[4] steps, out[5] kernel launches since creation.
 */
int mpm_get_stats(mpm_ctx *ctx, int64_t *out, int n);

/*
 * One explicit step that allocates no memory (the paper has no counterpart:
 * this is a deployment entry point of this library).
 *
 * For callers that cannot call cudaMalloc: plugins inside an application that
 * owns all device memory, and real-time loops that must not enter the
 * allocator (cudaMalloc may synchronise the device and take unbounded time).  The
 * particle state comes in and goes out through caller-owned device buffers
 * (layouts as for mpm_get_particles, doubles, n particles); the only scratch,
 * the background grid, lives in a static device array of this library holding
 * at most 131072 grid nodes (4 MiB, kept by every GPU that loads the library
 * until the process exits).  Supports dim 2 or 3, MPM_FP64, batch 1, the APIC
 * transfer, slip walls
 * (no friction fields, no obstacles), no sorting; gravity, Tait fluid and
 * Drucker-Prager as in mpm_step.  `out` may alias `in` particle by particle.
 *
 * Rules: the call queues its kernels on cuda_stream (NULL = the legacy default
 * stream) and returns without waiting.  The first call on each device resolves
 * the device address of the static scratch (cudaGetSymbolAddress) and loads
 * the four kernels (cudaFuncGetAttributes, so that lazy module loading takes no
 * memory at a later launch).  The address is kept per device ordinal for the
 * life of the process: it is valid in the device's primary context (the
 * runtime's) only, and not after a cudaDeviceReset.  Every call on a device
 * shares the scratch and clears it before use, so calls whose work overlaps on the GPU
 * race: serialise them.  A grid of more than 131072 nodes ((N_x + 3)(N_y + 3)
 * [(N_z + 3)]) is rejected with MPM_EINVAL, and so are the parameters that
 * mpm_create rejects; both checks come before any device use.  On failure a
 * one-line message is written to err (when err_len > 0).
 */
typedef struct {
    double *x, *v, *C, *F, *rho, *sigma, *eps;   /* device pointers; sigma/eps for Drucker-Prager only */
} mpm_state_ptrs;

int mpm_step_noalloc(const mpm_grid_desc *grid, const mpm_material *material, void *cuda_stream, int64_t n,
                     double particle_volume, mpm_state_ptrs in, mpm_state_ptrs out, char *err, int err_len);

/*
 * BF16 GEMM on the tcgen05 tensor cores: C = A B^T with A (M x K) and B (N x K)
 * bf16 row-major device matrices (leading dimensions lda, ldb >= K, multiples
 * of 8; 16-byte aligned pointers) and C (M x N) fp32 device, ldc >= N.  Accumulates
 * in fp32 (TMEM).  Queued on cuda_stream; a tensor-core wait that runs out sets
 * bit 2 of *status_dev (a device int32 the caller owns).  MPM_EINVAL on bad
 * shapes or alignment.  The building block of the MLP below.
 */
int mpm_gemm_bf16(int M, int N, int K, const void *A, int lda, const void *B, int ldb, float *C, int ldc,
                  int32_t *status_dev, void *cuda_stream);

/*
 * A fully connected network on the tensor cores: the learned warm start of the
 * basal-friction inversion (a map from tracked-particle displacements to the
 * per-segment friction field) and the paper's coordinate network of Eq.
 * nn_apprx (Sec. 3.2, 5.2).  widths[0..n_layers] (multiples of 8); by default
 * hidden layers use GELU (exact erf form) and the output is y = out_lo +
 * (out_hi - out_lo) sigmoid(z) (see mpm_mlp_set_activations).  Weights and Adam state in fp32 with bf16
 * copies as GEMM operands; activations enter GEMMs as bf16; fp32 accumulation.
 * Parameter vectors (host, fp32) list, per layer, W (out x in, row-major) then b.
 */
typedef struct mpm_mlp mpm_mlp;
int mpm_mlp_create(int n_layers, const int *widths, int max_batch, double out_lo, double out_hi, void *cuda_stream,
                   mpm_mlp **out);
void mpm_mlp_destroy(mpm_mlp *mlp);
int64_t mpm_mlp_num_params(const mpm_mlp *mlp);
/* Set the parameters (and reset the Adam state). */
int mpm_mlp_set_params(mpm_mlp *mlp, const float *params);
/* Copy the parameters (which = 0) or the gradients of the last train step (which = 1). */
int mpm_mlp_get_params(mpm_mlp *mlp, float *params, int which);
/* y (batch x widths[L]) = network(x (batch x widths[0])); host or device pointers. */
int mpm_mlp_infer(mpm_mlp *mlp, int batch, const float *x, float *y, int device_ptrs);
/*
 * One training step on the mean squared error to target (batch x widths[L]):
 * forward, backward, and (update != 0) one Adam step (beta 0.9 / 0.999, eps
 * 1e-8, bias-corrected) with rate lr.  batch must be a multiple of 8.  Writes
 * the loss before the update.  Synchronises.
 */
int mpm_mlp_train_step(mpm_mlp *mlp, int batch, const float *x, const float *target, double lr, int update,
                       double *loss_out, int device_ptrs);
/*
 * The same training step (update on) with device pointers only and no
 * synchronisation: queued on the network's stream; the loss before the update
 * goes to loss_dev (a device double, or NULL).  A bounded tensor-core wait that
 * ran out is reported by the next synchronising call.  MPM_EINVAL as above.
 */
int mpm_mlp_train_step_async(mpm_mlp *mlp, int batch, const float *x_dev, const float *target_dev, double lr,
                             double *loss_dev);
/*
 * Activations (default GELU hidden layers and the scaled sigmoid output): hidden
 * = MPM_ACT_GELU or MPM_ACT_RELU (max(z, 0), derivative 0 at z = 0); output =
 * MPM_OUT_SIGMOID (out_lo + (out_hi - out_lo) sigmoid(z)) or MPM_OUT_LINEAR
 * (y = z: the coordinate network v(x) of Eq. nn_apprx, Sec. 3.2 and 5.2).
 * MPM_EINVAL for another value.
 */
enum { MPM_ACT_GELU = 0, MPM_ACT_RELU = 1 };
enum { MPM_OUT_SIGMOID = 0, MPM_OUT_LINEAR = 1 };
int mpm_mlp_set_activations(mpm_mlp *mlp, int hidden, int output);
/*
 * Back-propagation of a given output gradient dy = dL/dy (batch x widths[L]) for
 * a loss L computed outside the network (the chain rule of Sec. 3.2: dL/dtheta =
 * dL/dy dy/dtheta, with dL/dy from mpm_get_initial_adjoint for a network that
 * parameterises the initial velocity field): forward at x, backward, and
 * (update != 0) one Adam step with rate lr.  The parameter gradients are then
 * readable with mpm_mlp_get_params(which = 1).  batch a multiple of 8;
 * synchronises.
 */
int mpm_mlp_backward(mpm_mlp *mlp, int batch, const float *x, const float *dy, double lr, int update,
                     int device_ptrs);
int mpm_mlp_last_error(const mpm_mlp *mlp, char *buf, int len);

#ifdef __cplusplus
}
#endif

#endif /* LIBMPM_MPM_H */
