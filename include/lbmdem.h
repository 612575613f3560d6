/*
 * lbmdem.h -- C ABI of the GB300 four-way coupled lattice Boltzmann / discrete
 * element library (Rettinger & Ruede, "An efficient four-way coupled lattice
 * Boltzmann - discrete element method for fully resolved simulations of
 * particle-laden flows", arXiv 2003.01490).
 *
 * One context advances one simulation box of D3Q19 fluid with spherical
 * particles on one CUDA device. lbm_step() runs Algorithm 1 of Sec. 4.2 per
 * time step: moving no-slip boundary conditions (Eq. (14)) and the momentum
 * exchange force/torque (Eqs. (15)-(17)) fused into the pull-stream + TRT+aB
 * collision (Eqs. (1)-(2), (5), (12), Sec. 2.3.2), two-step force averaging
 * (Sec. 4.2), n_sub DEM subcycles with lubrication (Eqs. (25)-(33)), linear
 * spring-dashpot contact (Eqs. (39)-(52)) and Velocity Verlet (Eqs. (37)-(38)),
 * then the particle mapping update and PDF refill (Sec. 2.2, Eq. (18)).
 * Particles may instead be held fixed or moved by prescribed velocities
 * (lbm_dem.fixed_particles, lbm_set_motion, lbm_set_particle_velocity).
 *
 * Units are lattice units (dx = dt = rho0 = 1, c_s^2 = 1/3, Sec. 2.1). Cell
 * (i, j, k) has its centre at (i + 1/2, j + 1/2, k + 1/2); walls lie on the
 * domain faces. Host arrays are x-fastest: cell index = i + nx (j + ny k).
 *
 * Conventions for every call:
 *   - All pointer arguments are HOST memory owned by the caller; a call reads
 *     or fills them before it returns (getters synchronise the context stream).
 *   - The context owns its device memory (lbm_create) or carves it from a
 *     caller-owned device arena (lbm_create_in_arena); either way the caller
 *     never frees pieces of it.
 *   - Every call returns an lbm_status; none aborts the process. Errors raised
 *     asynchronously on the device (capacity overflow, unstable density) are
 *     sticky and are reported by the next lbm_sync() or getter.
 *   - A context is used by one host thread at a time; distinct contexts are
 *     independent.
 */
#ifndef LBMDEM_H
#define LBMDEM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;

typedef enum {
    LBM_OK = 0,
    LBM_ERR_INVALID = -1,   /* bad argument: size, parameter range, overlap, ... */
    LBM_ERR_OOM = -2,       /* device allocation failed or arena too small       */
    LBM_ERR_CUDA = -3,      /* a CUDA runtime call failed                        */
    LBM_ERR_UNSTABLE = -4,  /* NaN or |rho - 1| > 0.5 on the device, or a particle
                               faster than 0.5 cells per step                    */
    LBM_ERR_CAPACITY = -5,  /* a fixed-capacity device list overflowed           */
    LBM_ERR_TIMEOUT = -6,   /* a bounded wait inside a kernel ran out (1 s)      */
    LBM_ERR_STATE = -7      /* call not allowed in the current state             */
} lbm_status;

/* PDF storage format. Every format stores the shifted value f_q - w_q; the
 * collision and the DEM's pair and wall laws run in float64 for
 * LBM_STORE_F64 and in float32 otherwise (particle state, integration and
 * sphere overlaps stay float64). */
typedef enum {
    LBM_STORE_F64 = 0,
    LBM_STORE_F32 = 1,
    LBM_STORE_F16 = 2,
    LBM_STORE_BF16 = 3
} lbm_storage;

/* Flag bits returned by lbm_get_fields(). */
#define LBM_FLAG_SOLID 0x01u     /* cell centre inside a particle (Sec. 2.2)              */
#define LBM_FLAG_SHELL 0x02u     /* fluid cell inside the TRT+aB shell (Sec. 2.3.2)       */
#define LBM_FLAG_NEAR 0x04u      /* fluid cell that may have a particle link              */
#define LBM_FLAG_MISS 0x08u      /* solid cell that may own a missing link (Sec. 2.2)     */
#define LBM_FLAG_NEWFLUID 0x10u  /* solid before the last mapping update, fluid after     */
#define LBM_FLAG_MULTI 0x20u     /* solid cell inside more than one sphere (owner: lowest) */

/* Box: every axis is either periodic or closed by a no-slip wall on both of
 * its faces (halfway bounce-back, Eq. (14) with delta = 1/2). */
typedef struct {
    int nx, ny, nz;
    int periodic[3];                 /* 1 = periodic axis, 0 = walls on both faces */
    double wall_vel_lo[3][3];        /* [axis][component] velocity of the low face  */
    double wall_vel_hi[3][3];        /* [axis][component] velocity of the high face */
} lbm_grid;

/* Relaxation parameters of the TRT+aB collision (Secs. 2.1.1-2.1.3, 2.3.2). */
typedef struct {
    double tau;            /* 1/s_nu, > 0.5; viscosity nu = (tau - 1/2)/3, Eq. (7)   */
    double magic;          /* Lambda of Eq. (11); paper value 3/16                    */
    double lambda_b_shell; /* Lambda_b of Eq. (13) inside the shell; paper value 100  */
    double lambda_b_bulk;  /* Lambda_b elsewhere; 1 gives TRT+aB, != 1 gives TRT+B    */
    double shell_width;    /* delta_aB of Sec. 2.3.2; paper value 2                   */
} lbm_relax;

/* Particle parameters (Secs. 3.1, 4.1, 4.2). */
typedef struct {
    double e_dry;          /* dry coefficient of restitution, Eq. (42)                    */
    double Tc;             /* collision time; <= 0 selects T_c = 2.31 D / c_s, Eq. (55)   */
    double nu_p;           /* Poisson's ratio, Eq. (52)                                   */
    double mu_p;           /* Coulomb friction coefficient, Eq. (47)                      */
    int n_sub;             /* DEM subcycles per LBM step (Algorithm 1), >= 1              */
    double lub_cut_n;      /* normal lubrication cut-off, Eq. (34): 2/3                   */
    double lub_cut_tt;     /* tangential translation cut-off, Eq. (34): 1/2               */
    double lub_cut_tr;     /* tangential rotation cut-off, Eq. (34): 1/2                  */
    double lub_min_a;      /* delta_min = (a + b R) R, Eq. (56): a = 0.001                */
    double lub_min_b;      /*                                   b = 0.00007               */
    double gravity[3];     /* g; particles feel V (rho_p - rho_f) g (Sec. 4.1.1)          */
    int lubrication;       /* 1 = apply Eqs. (25)-(33)                                    */
    int tangential_lubrication; /* 1 = include Eqs. (30)-(33)                             */
    int force_averaging;   /* 1 = average F^fp, T^fp over two steps (Sec. 4.2)            */
    int fluid_counterforce;/* 1 = fluid body force -sum V (rho_p - 1) g / N_fluid         */
    int fixed_particles;   /* 0 = DEM (Algorithm 1); 1 = particles keep position and
                              velocity (no DEM); 2 = prescribed motion: each step moves
                              every particle by its velocity, x += u (Eq. (37) with no
                              force, one time step), with the velocities the caller set
                              (lbm_add_spheres, lbm_set_particle_velocity); no DEM
                              forces; mapping and refill as in Algorithm 1             */
    int missing_links;     /* 1 = missing-link correction F_q = 2 w_q c_q (Sec. 2.2)       */
} lbm_dem;

/* Fill *relax and *dem with the paper's values (tau is set to 0.6). */
lbm_status lbm_default_params(lbm_relax *relax, lbm_dem *dem);

/* Device bytes that lbm_create_in_arena() needs for this box, storage format
 * and particle capacity. Host arithmetic only (no CUDA call).
 * Errors: LBM_ERR_INVALID (NULL grid or bytes_out, an axis of fewer than 3
 * cells, max_particles < 0, an unknown storage format). */
lbm_status lbm_required_bytes(const lbm_grid *grid, lbm_storage storage, int max_particles,
                              size_t *bytes_out);

/* Create a context on the current CUDA device. body_force is the fluid body
 * force per unit volume (3 doubles, may be NULL for zero). cuda_stream is a
 * cudaStream_t (NULL = legacy default stream); all work of the context is
 * queued on it. The fluid starts at rest with rho = 1 and no particles.
 * Device memory is allocated by the library and released by lbm_destroy().
 * Errors: LBM_ERR_INVALID (bad sizes, a box of more than 2^31 - 2^24 cells,
 * tau <= 1/2, max_particles outside [0, 4,000,000], an unknown storage
 * format, n_sub < 1, e_dry outside (0, 1], nu_p outside [0, 1), mu_p < 0, a
 * lubrication cut-off <= 0, fixed_particles outside {0, 1, 2}; all checked
 * before any CUDA call), LBM_ERR_OOM, LBM_ERR_CUDA. */
lbm_status lbm_create(const lbm_grid *grid, const lbm_relax *relax, const double *body_force,
                      const lbm_dem *dem, lbm_storage storage, int max_particles,
                      void *cuda_stream, lbm_ctx **out);

/* As lbm_create(), but every device buffer is carved from the caller-owned
 * device allocation [arena, arena + arena_bytes), which must stay valid and
 * untouched until lbm_destroy(). arena must be 256-byte aligned. */
lbm_status lbm_create_in_arena(const lbm_grid *grid, const lbm_relax *relax,
                               const double *body_force, const lbm_dem *dem,
                               lbm_storage storage, int max_particles, void *cuda_stream,
                               void *arena, size_t arena_bytes, lbm_ctx **out);

/* Add n spheres (Sec. 2.2 mapping is applied at once). pos, vel, omega: n x 3
 * doubles; radius, density: n doubles, density = rho_p / rho_f. Allowed only
 * before the first lbm_step(). Errors: LBM_ERR_INVALID if a centre lies
 * outside the box, a radius is outside [1, 100] cells, a density is <= 0, two spheres
 * overlap (centre distance < R_i + R_j), a sphere crosses a wall or a
 * periodic side is not longer than 2 R + 4 cells (a sphere and its own
 * periodic image would share boundary cells);
 * LBM_ERR_CAPACITY if the total exceeds max_particles; LBM_ERR_STATE after the
 * first step. *first_id_out (may be NULL) receives the index of the first new
 * sphere; spheres are numbered in insertion order. */
lbm_status lbm_add_spheres(lbm_ctx *ctx, int n, const double *pos, const double *vel,
                           const double *omega, const double *radius, const double *density,
                           int *first_id_out);

/* Advance n_steps time steps of Algorithm 1 (asynchronous on the stream). */
lbm_status lbm_step(lbm_ctx *ctx, int n_steps);

/* Copy particle state to host buffers of n_cap entries (x 3 doubles each where
 * vector valued); any pointer may be NULL. force_hyd / torque_hyd receive the
 * momentum-exchange force and torque F^fp, T^fp of Eqs. (16)-(17) of the last
 * step, including the missing-link term, before averaging. *n_out (may be
 * NULL) receives the particle count. Synchronises the stream. */
lbm_status lbm_get_particle_state(lbm_ctx *ctx, int n_cap, double *pos, double *vel,
                                  double *omega, double *force_hyd, double *torque_hyd,
                                  int *n_out);

/* The same read-out without waiting: queues a device snapshot of the state
 * after every step queued so far (on the context's stream) and its copy into
 * the host buffers (on a read-out stream of the context, so the copy overlaps
 * the steps queued after it), and returns. The values are in the buffers once
 * lbm_sync() returns; the buffers must stay valid until then, and must be
 * page-locked for the copies to run asynchronously. A later call's snapshot
 * waits for the previous call's copies. Reading in this way after every step
 * of a loop costs no host wait per step. The first call allocates the
 * snapshot (15 doubles per particle of max_particles). Device errors of the
 * steps are reported by lbm_sync().
 * Errors: LBM_ERR_INVALID (NULL ctx, n_cap too small), LBM_ERR_CUDA. */
lbm_status lbm_get_particle_state_async(lbm_ctx *ctx, int n_cap, double *pos, double *vel,
                                        double *omega, double *force_hyd, double *torque_hyd,
                                        int *n_out);

/* Switch how particles move from the next step on (mode as lbm_dem.fixed_particles:
 * 0 DEM, 1 fixed, 2 prescribed motion), e.g. to release a sphere whose
 * approach velocity was prescribed (Sec. 4.4 turns the prescribed settling
 * velocity off once the gap to the wall is below one diameter). Switching to
 * the DEM after the first step evaluates the force of the first
 * Velocity-Verlet position update at the current state, including the
 * current averaged fluid force. Errors: LBM_ERR_INVALID for another mode.
 * Synchronises the stream. */
lbm_status lbm_set_motion(lbm_ctx *ctx, int mode);

/* Replace the translational and angular velocities of particles 0 .. n-1
 * (vel, omega: n x 3 doubles each, either may be NULL), e.g. to prescribe a
 * particle's motion step by step (Sec. 2.3.3 prescribes the settling velocity
 * of a sphere this way). The new velocities enter the next step's boundary
 * condition, position update and refill. Errors: LBM_ERR_INVALID if n is
 * negative or above the particle count. Synchronises the stream. */
lbm_status lbm_set_particle_velocity(lbm_ctx *ctx, int n, const double *vel, const double *omega);

/* Copy rho (cells doubles), u (3 x cells doubles, component-major: u_x block,
 * then u_y, then u_z) and flags (cells bytes, LBM_FLAG_* bits) to host
 * buffers; any pointer may be NULL. rho = sum_q f_q and u = (sum_q f_q c_q -
 * a/2)/rho0 of the stored post-collision PDFs, with a the fluid body force of
 * the last step; both are 0 in solid cells. Synchronises the stream. */
lbm_status lbm_get_fields(lbm_ctx *ctx, double *rho, double *u, unsigned char *flags);

/* Density at n points (pos: n x 3 doubles, lattice units; rho: n doubles):
 * trilinear interpolation of the cell-centred density (cell i centred at
 * i + 1/2), wrapping periodic axes and clamping at walls; solid cells count
 * with the reference density 1 (a probe like the one of Sec. 2.3.3). n at
 * most min(cells, 4 Mi). Synchronises the stream. */
lbm_status lbm_sample_density(lbm_ctx *ctx, int n, const double *pos, double *rho);

/* Copy the owning particle index of every cell (int32; -1 for fluid cells).
 * Synchronises the stream. */
lbm_status lbm_get_owner(lbm_ctx *ctx, int *owner);

/* Copy / replace the post-collision PDFs f_q (unshifted values), 19 x cells
 * doubles, direction-major (q = 0..18 in the order fixed by App. A). Solid
 * cells read as NaN: every PDF slot of a solid cell holds a NaN marker (with
 * the owning particle in its payload for f32 and f64 storage), by which the
 * dense kernel finds particle links; values given for solid cells are
 * replaced by that marker. Synchronises the stream. */
lbm_status lbm_get_pdfs(lbm_ctx *ctx, double *f);
lbm_status lbm_set_pdfs(lbm_ctx *ctx, const double *f);

/* Checkpoints: the whole simulation state (device memory of the context and
 * the host-side step state) in one host buffer of lbm_checkpoint_bytes()
 * bytes. lbm_save copies it out (synchronises the stream; LBM_ERR_INVALID if
 * the buffer is smaller); lbm_restore puts it back into a context created
 * with the same grid, storage format and max_particles (LBM_ERR_INVALID
 * otherwise, or for a buffer that is not a checkpoint, is truncated or
 * carries a particle count, buffer parity or motion mode out of range; the
 * context is left unchanged then). Stepping a restored
 * context continues exactly where the saved one stood (bit for bit in the
 * float32 and 16-bit formats, whose particle sums are exact integers). */
lbm_status lbm_checkpoint_bytes(const lbm_ctx *ctx, size_t *bytes);
lbm_status lbm_save(lbm_ctx *ctx, void *buf, size_t bytes);
lbm_status lbm_restore(lbm_ctx *ctx, const void *buf, size_t bytes);

/* Wait for all queued work and report device-side errors (sticky). */
lbm_status lbm_sync(lbm_ctx *ctx);

/* Queue the context's later work on another stream of the same device
 * (NULL: the legacy default stream). Waits for the work queued so far on the
 * old stream first. Contexts that share a stream run one after another; a
 * batch (lbm_batch_create) orders its steps after the streams its contexts
 * had when it was created, so move contexts before creating their batch.
 * Errors: LBM_ERR_INVALID (NULL ctx), LBM_ERR_STATE (phase timing on),
 * LBM_ERR_CUDA, and device errors of the finished work (as lbm_sync). */
lbm_status lbm_set_stream(lbm_ctx *ctx, void *cuda_stream);

/* Device timing of lbm_step() by phase, with CUDA events recorded on the
 * context stream between the launches of each step. Phases: 0 the boundary
 * kernel (particle links, Eqs. (14)-(17), and missing links), 1 the dense
 * stream + collide kernel (Eqs. (2), (5) with wall bounce-back), 2 the force
 * finalisation and averaging (Sec. 4.2), 3 the DEM subcycles (neighbour
 * lists, lubrication, contact, Velocity Verlet), 4 the mapping update
 * (Sec. 2.2), 5 the refill (Eq. (18)). lbm_profile(ctx, 1) clears the totals
 * and starts recording; lbm_profile(ctx, 0) stops. lbm_profile_read()
 * synchronises the stream and returns the summed milliseconds of the 6 phases
 * (phase_ms must hold 6 doubles) and the number of timed steps. Recording
 * costs a few event records per step; it is off by default. */
lbm_status lbm_profile(lbm_ctx *ctx, int enable);
lbm_status lbm_profile_read(lbm_ctx *ctx, double *phase_ms, long long *steps);

/* Sphere-to-cell mapping that allocates no device memory. The paper has no
 * counterpart of this call; it serves callers that cannot call cudaMalloc,
 * for instance a host framework that owns all device memory through its own
 * pool and forbids other allocations, or a loop that cannot afford the device
 * synchronisation an allocation may cause.
 *
 * Unlike the other calls, every array argument is DEVICE memory owned by the
 * caller: d_pos (n x 3 doubles) and d_radius (n doubles) are read; d_flags
 * (nx*ny*nz bytes, LBM_FLAG_SOLID/SHELL/NEAR/MISS bits) and d_owner (nx*ny*nz
 * int32, the lowest sphere index whose sphere holds the cell centre, -1 for
 * fluid) are cleared and written, x fastest, exactly as lbm_add_spheres() maps
 * the same spheres into a new context (solid cells, and the shell of width
 * shell_width around each sphere). grid->wall_vel_* are ignored. All four
 * buffers must be memory of the current device (LBM_ERR_INVALID otherwise).
 *
 * The temporary tile lists live in one file-scope device array of about 29 MB
 * that every GPU which loads the library holds until the process exits.
 * Limits: at most 98,304 mapping tiles of 32 x 4 x 4 cells (for example
 * 256 x 256 x 512 cells) and 65,536 spheres; larger inputs return
 * LBM_ERR_INVALID before any work. The first call on a device looks up the
 * device address of that array with the device current; make that first call
 * before any stream capture. All calls on a device share the array; a host
 * lock per device, held from the first queued copy to the final stream
 * synchronise, serialises them, so calls from several host threads are safe
 * (and never overlap on the GPU). The call queues its work on cuda_stream (a
 * cudaStream_t, NULL = legacy default stream) and synchronises that stream
 * before returning, on errors too once work is queued. Errors: LBM_ERR_INVALID,
 * LBM_ERR_CAPACITY (more than 64 spheres reach one tile), LBM_ERR_CUDA; the
 * message is returned by lbm_last_error(NULL). */
lbm_status lbm_map_spheres_noalloc(const lbm_grid *grid, double shell_width, int n,
                                   const double *d_pos, const double *d_radius,
                                   unsigned char *d_flags, int *d_owner, void *cuda_stream);

/* Measured float64 FMA throughput of the current device in TFLOP/s (2 FLOP
 * per FMA): a kernel of eight independent FMA chains per thread, 8 blocks of
 * 256 threads per multiprocessor, iters FMAs per chain, best of three timed
 * launches (CUDA events on a private stream). The paper has no counterpart;
 * it is the peak of the float64 roofline that bench.py reports for the
 * float64 storage form. Allocates and frees one small device buffer.
 * Errors: LBM_ERR_INVALID (iters < 1, tflops_out NULL), LBM_ERR_CUDA; the
 * message is returned by lbm_last_error(NULL). */
lbm_status lbm_fp64_fma_rate(int iters, double *tflops_out);

/* ------------------------------------------------------------------ batches
 * A batch advances many independent contexts (instances: boxes of any size,
 * their own relaxation and particle parameters) in lock step, one CUDA graph
 * per step: each instance's boundary, finalisation and mapping kernels stay
 * per instance (on parallel branches of the graph); the DEM steps of all
 * instances with at most 32 particles run as one launch (a block each), and the
 * dense kernels of all active instances run as ONE persistent launch over a
 * table of work items (instance, tile, chunk of z planes), whose tile width and
 * chunk depth are set per instance (lbm_batch_set_launch; tune.py picks them
 * by timing). Every instance computes exactly what lbm_step() computes for it
 * alone (same arithmetic per cell; the per-particle sums of the 4- and 2-byte
 * formats are exact integer sums, so the results are bit-identical with the
 * same tile and chunk). The method of the paper has no batches; this is the
 * library's way of running many of its simulations at once (Algorithm 1 per
 * instance and step).
 *
 * lbm_batch_create(ctxs, n, cuda_stream, out): n >= 1 distinct contexts of
 *   one storage format. The batch queues its graph launches on cuda_stream (a
 *   cudaStream_t; NULL = the first context's stream); when that differs from a
 *   context's stream, each lbm_batch_step() call is ordered after the work
 *   already queued on the contexts' streams and before work queued on them
 *   later (events), so several batches over disjoint contexts can run
 *   concurrently on their own streams. The batch borrows the contexts:
 *   destroy the batch before them.
 *   Errors: LBM_ERR_INVALID, LBM_ERR_CUDA (message by lbm_batch_last_error(NULL)).
 * lbm_batch_set_launch(b, instance, tile_bx, zchunk, blocks_per_sm): launch
 *   shape of the batched dense kernel for one instance (instance = -1: all):
 *   tile width tile_bx in x (0 automatic: the narrowest of 32, 64, 128 that
 *   covers the box width, else 32, 64 or 128; 256 / tile_bx rows),
 *   zchunk z planes per work item (0 automatic = 16), and blocks_per_sm
 *   resident blocks per multiprocessor for the whole launch (0 automatic:
 *   4, 2 for float64). Synchronises the stream and drops the captured graphs.
 * lbm_batch_set_active(b, instance, active): whether the instance takes part
 *   in the following lbm_batch_step() calls (finished instances are
 *   deactivated; an inactive instance's state is not touched).
 * lbm_batch_step(b, n_steps): queue n_steps steps of every active instance on
 *   the stream (asynchronous). Each active instance must have stepped at least
 *   once with lbm_step() (the first step sets up the DEM state), must not have
 *   a pending motion switch and must not be under phase timing
 *   (LBM_ERR_STATE). A graph is captured the first time each combination of
 *   active set, launch shape and buffer parities occurs and replayed after.
 * lbm_batch_sync(b): wait for the stream; returns the first device error of
 *   an instance (as lbm_sync()).
 * lbm_batch_launch_count(b): launches of the batched kernels so far (the
 *   persistent dense kernel and the one launch per step that runs the DEM of
 *   every instance with at most 32 particles; the other kernels are counted by
 *   each instance's lbm_launch_count()).
 * lbm_batch_capture_stats(b, captures, capture_ms): graphs captured so far and
 *   the host time spent capturing and instantiating them (either pointer may
 *   be NULL).
 * lbm_batch_destroy(b): releases the batch (not its contexts). NULL is a no-op.
 */
typedef struct lbm_batch lbm_batch;
lbm_status lbm_batch_create(lbm_ctx *const *ctxs, int n, void *cuda_stream, lbm_batch **out);
lbm_status lbm_batch_set_launch(lbm_batch *b, int instance, int tile_bx, int zchunk, int blocks_per_sm);
lbm_status lbm_batch_set_active(lbm_batch *b, int instance, int active);
lbm_status lbm_batch_step(lbm_batch *b, int n_steps);
lbm_status lbm_batch_sync(lbm_batch *b);
long long lbm_batch_launch_count(const lbm_batch *b);
lbm_status lbm_batch_capture_stats(const lbm_batch *b, int *captures, double *capture_ms);
const char *lbm_batch_last_error(const lbm_batch *b);
void lbm_batch_destroy(lbm_batch *b);

/* Number of kernel launches this context has issued so far. */
long long lbm_launch_count(const lbm_ctx *ctx);

/* Human-readable text of the last error of ctx (never NULL; ctx may be NULL). */
const char *lbm_last_error(const lbm_ctx *ctx);

/* Release the context and, for lbm_create(), its device memory. NULL is a no-op. */
void lbm_destroy(lbm_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* LBMDEM_H */
