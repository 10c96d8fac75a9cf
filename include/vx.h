/*
 * vx.h - C ABI of the GB300 voxel lattice soft-body simulator.
 *
 * The simulator is the heterogeneous voxel lattice of Hiller & Lipson,
 * "Dynamic Simulation of Soft Heterogeneous Objects" (arXiv 1212.2845):
 * adjacent voxels are joined by Euler-Bernoulli beam bonds with composite
 * material properties (Sec 2.1.1-2.1.2); each step computes every bond force
 * and then updates every voxel synchronously with "double Euler" integration
 * (Sec 2.1.3), with bond and ground damping (Sec 2.1.5), gravity, floor
 * contact with Coulomb friction (Sec 2.2.1), surface-voxel collisions behind a
 * collision horizon (Sec 2.2.2) and volumetric (thermal) actuation (Sec 2.3).
 * The object model follows the paper's App. B (CVX_Object / CVX_Environment /
 * CVX_Sim); here one opaque vx_sim plays all three roles.
 *
 * Conventions for every entry point:
 *   - Return value: VX_OK (0) on success, a negative VX_ERR_* code otherwise;
 *     vx_last_error() then gives a message (thread-local, valid until the
 *     next failing call on the same thread).  No C++ exception crosses the ABI.
 *   - All voxel arrays are in CANONICAL ORDER: bodies in order, then occupied
 *     sites x-fastest, then y, then z (index x + nx*(y + ny*z), empty sites
 *     skipped).  Vectors are interleaved: [N][3] or [N][4].
 *   - The caller owns every pointer it passes; the library copies what it
 *     needs before returning and keeps no caller pointer.  The library owns
 *     its device memory (allocated in vx_create, released in vx_destroy).
 *   - Host pointers are plain (pageable or pinned) host memory unless an
 *     argument says "device".  Streams are cudaStream_t passed as void*
 *     (NULL = legacy default stream).
 *   - Units: SI (m, kg, s, Pa, N, K).
 *   - A vx_sim must not be used from two host threads at once.
 */
#ifndef VX_H
#define VX_H

#include <stdint.h>

#if defined(__GNUC__)
#define VX_API __attribute__((visibility("default")))
#else
#define VX_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define VX_OK 0
#define VX_ERR_ARG (-1)       /* invalid argument (paper: SetMat returns false)   */
#define VX_ERR_CUDA (-2)      /* a CUDA runtime call failed                        */
#define VX_ERR_OOM (-3)       /* device or host allocation failed                  */
#define VX_ERR_UNSTABLE (-4)  /* non-finite state (paper: TimeStep returns false)  */
#define VX_ERR_TIMEOUT (-5)   /* a bounded device wait ran out                     */
#define VX_ERR_STATE (-6)     /* call not valid in the current state               */
#define VX_ERR_CAPACITY (-7)  /* a fixed-size buffer (collision pairs) overflowed  */
#define VX_ERR_BOUNDS (-8)    /* bounds-checked debug builds only: an index read from a device
                                 table was out of range (the access was skipped) */

typedef struct vx_sim vx_sim;

/* Material of a palette entry (paper App. B, CVX_Object::AddMat: elastic
 * modulus and Poisson ratio; density, thermal expansion and friction are the
 * "other physical properties"). E > 0, -1 < nu < 0.5, rho > 0, mu >= 0. */
typedef struct {
  float E;    /* elastic modulus [Pa]                          */
  float nu;   /* Poisson ratio                                 */
  float rho;  /* density [kg/m^3]                              */
  float cte;  /* coefficient of thermal expansion [1/K] (Sec 2.3) */
  float mu_s; /* static friction coefficient with the floor (Sec 2.2.1) */
  float mu_k; /* dynamic friction coefficient with the floor        */
} vx_material;

/* Lattice description (paper App. B, CVX_Object::InitializeMatter + SetMat).
 * Each body is its own workspace nx*ny*nz of cubic voxels of edge voxel_size;
 * grid holds one byte per site, bodies concatenated, x fastest:
 * 0 = empty, k > 0 = palette[k-1].  Bodies never interact (independent
 * worlds stepped together). origin: [n_bodies][3] position of each
 * workspace's corner, or NULL for zeros.
 * Limits: 1 <= nx, ny <= 2048, 1 <= nz <= 1024 per body, n_materials <= 255,
 * total voxels < 2^31. */
typedef struct {
  int32_t n_bodies;
  const int32_t* dims;
  const uint8_t* grid;
  float voxel_size;
  const vx_material* palette;
  int32_t n_materials;
  const float* origin;
} vx_desc;

/* State of every voxel in canonical order.  Positions are stored as FP32
 * offsets from each voxel's lattice anchor (its rest centre,
 * origin + (i+1/2, j+1/2, k+1/2) l), so that small strains keep full FP32
 * precision; vx_get_anchors gives the anchors.  Any field may be NULL
 * (skipped).  flags: bit 0 = fixed (immobile), bit 1 = static friction. */
typedef struct {
  float* offset;   /* [N][3] position minus anchor [m]          */
  float* quat;     /* [N][4] orientation (w, x, y, z), unit     */
  float* vel;      /* [N][3] linear velocity [m/s]              */
  float* angvel;   /* [N][3] angular velocity, world frame [rad/s] */
  uint8_t* flags;  /* [N]                                       */
} vx_state_view;

#define VX_FLAG_FIXED 1u
#define VX_FLAG_STATIC 2u

/* ---- version / errors --------------------------------------------------- */
VX_API const char* vx_version(void);
/* Message of the last failing call on this thread ("" if none). */
VX_API const char* vx_last_error(void);

/* ---- host-only planning (no GPU needed) --------------------------------- */
/* Counts of the lattice a description would create: occupied voxels, bonds
 * (adjacent occupied sites of one body, Sec 2.1.2) and surface voxels (fewer
 * than 6 occupied face neighbours, Sec 2.2.2).  Any output may be NULL. */
VX_API int vx_plan_counts(const vx_desc* desc, int64_t* n_voxels, int64_t* n_bonds, int64_t* n_surface);

/* Stable timestep of every body (Sec 2.1.4): dt = dt_factor / (2 pi w_max),
 * w_max the largest sqrt(k/m) over the body's bonds (k = E_c l, m the smaller
 * mass) and over its voxels' own contact springs (k = E l).  log_E: per-voxel
 * natural-log modulus overriding the palette, or NULL.  dt_out: [n_bodies]. */
VX_API int vx_plan_dt(const vx_desc* desc, const float* log_E, float dt_factor, double* dt_out);

/* Voxels of `body` touching a region given as fractions of its workspace
 * (paper App. B, AddFixedRegion/AddForcedRegion: "all voxels touching this
 * region"): the closed voxel cube [i/nx,(i+1)/nx] x ... intersects the closed
 * box [loc, loc+size].  mask: [N] canonical order (set to 1 or 0);
 * n_out: number selected. */
VX_API int vx_region_mask(const vx_desc* desc, int32_t body, const float loc[3], const float size[3],
                   uint8_t* mask, int64_t* n_out);

/* Tiles of the fused step kernel for a description: voxels are ordered in
 * 4x4x4-site bricks along a Morton curve and cut into runs of at most
 * tile_max voxels (128, 256 or 512); each tile also stages its halo (face
 * neighbours outside it).  Outputs (nullable): number of tiles, halo entries
 * over all tiles, bonds over all tiles (bonds on a tile border counted in both
 * tiles), the largest owned + halo set of one tile, and the longest list of
 * bonds entering one tile from its halo (both at most 2 tile_max: tiles are
 * shortened until they fit the kernels' staging). */
VX_API int vx_plan_tiles(const vx_desc* desc, int32_t tile_max, int64_t* n_tiles, int64_t* n_halo,
                         int64_t* n_tile_bonds, int32_t* max_local, int32_t* max_halo_bonds);

/* ---- lifetime ------------------------------------------------------------ */
/* Build the lattice (Sec 2.1: voxelised geometry, composite bonds,
 * precomputed surface list) on the current CUDA device and reset the state
 * to rest.  Defaults: zeta_bond 1, zeta_ground 0, zeta_collision 1, no
 * gravity, floor or collisions, no actuation, dt_factor 0.9.  Errors:
 * VX_ERR_ARG for an invalid description, VX_ERR_OOM when device memory runs
 * out (for tests, the environment variable VX_DEVICE_ALLOC_CAP=<bytes> makes
 * every larger device allocation of the library fail this way),
 * VX_ERR_CUDA without a usable device. */
VX_API int vx_create(const vx_desc* desc, vx_sim** out);
VX_API void vx_destroy(vx_sim* sim);
VX_API int vx_get_counts(vx_sim* sim, int64_t* n_voxels, int64_t* n_bonds, int64_t* n_surface);
/* Lattice anchors (rest centres) [N][3] in double precision, host memory. */
VX_API int vx_get_anchors(vx_sim* sim, double* anchors);

/* Kernel form of the step.  VX_FORM_FUSED: one kernel per step,
 * one CTA per tile, bond forces kept in shared memory.  VX_FORM_TWO_PASS: a
 * bond kernel writes every bond's forces to device memory and a voxel kernel
 * gathers them.  VX_FORM_PIPELINED (default): the fused step with persistent
 * CTAs that stream the next tile into shared memory (cp.async) while
 * computing the current one.  All forms compute the same arithmetic and give
 * bitwise-identical states.  tile_max (fused forms): 128, 256 or 512 voxels
 * per tile (any form), 0 keeps the current size (256 at create).
 * The state is kept. */
#define VX_FORM_FUSED 0
#define VX_FORM_TWO_PASS 1
#define VX_FORM_PIPELINED 2
VX_API int vx_set_step_form(vx_sim* sim, int32_t form, int32_t tile_max);
/* Batched form for many independent bodies (thousands of bodies of uneven
 * size, as in the design automation the paper motivates).  group_voxels > 0: consecutive
 * bodies are grouped to about that many voxels and spread over persistent
 * CTAs (largest first onto the least loaded); vx_step / vx_step_async then
 * run all n steps in ONE launch, each CTA stepping one group at a time with
 * a barrier between steps so the group's state stays in L2.  Same arithmetic
 * and bits as the per-step forms.  Ignored while self-collision is on.
 * 0 turns it off.  Needs a fused form with tiles of 128 or 256.
 *
 * group_voxels = VX_GROUPS_RESIDENT: the shared-memory-resident form.
 * Consecutive whole bodies are grouped so that a group fits the shared memory
 * of one cluster of up to 16 CTAs (about 1,000 voxels per CTA; the cluster
 * size is the smallest power of two that holds the largest body, widened to
 * up to 8 CTAs when there are few groups).  vx_step / vx_step_async run all n
 * steps in ONE launch: each cluster loads a group's state into shared memory
 * once, steps it n times with cluster barriers between the bond and voxel
 * phases (partners in another CTA of the cluster are read through
 * distributed shared memory) and writes it back once.  Same arithmetic and
 * bits as the per-step forms.  VX_ERR_STATE if a body does not fit 16 CTAs;
 * ignored while self-collision is on. */
#define VX_GROUPS_RESIDENT (-1)
/* The same form with its bond phase split one way: one thread per bond
 * (shortest phases: the automatic choice when every group has a cluster of
 * its own) or one thread per voxel evaluating its +x, +y, +z bonds with one
 * rotation matrix (the automatic choice when clusters take several groups
 * each).  Both give the same bits. */
#define VX_GROUPS_RESIDENT_BOND (-2)
#define VX_GROUPS_RESIDENT_VOXEL (-3)
VX_API int vx_set_batching(vx_sim* sim, int64_t group_voxels);
/* Multi-step launches (on by default): in the pipelined form without
 * batching or collisions, on lattices of at most 4 tiles per persistent CTA
 * (about 300,000 voxels), vx_step / vx_step_async with n_steps > 1 run all
 * steps in ONE cooperative launch of co-resident persistent CTAs that meet
 * at a grid barrier between steps, so the lattice stays in L2 and no launch
 * separates the steps.  Lattices of at most 8,192 voxels without collisions
 * take the resident form instead (see vx_set_batching: the lattice stays in
 * the shared memory of one cluster of CTAs).  Same arithmetic and bits as
 * one launch per step.  The barrier waits are bounded (about a second); if
 * one gives up, the launch ends and vx_get_status / vx_step report
 * VX_ERR_TIMEOUT.  If the device cannot hold the grid at once the call falls
 * back to one launch per step.  on = 0 always launches once per step; on = 2
 * uses the cooperative grid launch on small lattices too. */
VX_API int vx_set_multistep(vx_sim* sim, int32_t on);
/* Fault-injection aid for tests of the bounded waits: the budget of one grid
 * barrier wait in units of 128 SM clock cycles (0 restores the default of
 * 2^24, about one second) and a number of phantom CTAs the barrier also waits for (0 in
 * normal use; any other value makes every barrier run out, after which the
 * launch ends with VX_ERR_TIMEOUT and the state is that of a partial step
 * sequence: reset or write it before stepping on).  Host-side only; no GPU
 * fault is involved. */
VX_API int vx_set_barrier_limits(vx_sim* sim, int64_t max_spins, int32_t phantom_ctas);
/* Current tiling: tile size, tile count, largest staged set, dynamic shared
 * memory of the fused kernel in bytes.  Any output may be NULL. */
VX_API int vx_get_tiling(vx_sim* sim, int32_t* tile_max, int64_t* n_tiles, int32_t* max_local, int64_t* smem_bytes);

/* ---- configuration (host inputs, copied) -------------------------------- */
/* Replace the palette (same count); recomputes bonds' composites and dt. */
VX_API int vx_set_materials(vx_sim* sim, const vx_material* palette, int32_t n_materials);
/* Per-voxel natural-log elastic modulus (overrides the palette's E) and
 * actuation phase [rad]; NULL leaves that field unchanged.  log_E recomputes dt. */
VX_API int vx_set_voxel_params(vx_sim* sim, const float* log_E, const float* phase);
/* Per-voxel fixed flags (1 = immobile). */
VX_API int vx_set_fixed_mask(vx_sim* sim, const uint8_t* mask);
/* Paper App. B AddFixedRegion: fix every voxel of `body` touching the region.
 * n_out (nullable): voxels selected. */
VX_API int vx_add_fixed_region(vx_sim* sim, int32_t body, const float loc[3], const float size[3], int64_t* n_out);
/* Paper App. B AddForcedRegion: F [N] split equally among the voxels of
 * `body` touching the region (added to any force already there). */
VX_API int vx_add_forced_region(vx_sim* sim, int32_t body, const float loc[3], const float size[3],
                         const float F[3], int64_t* n_out);
/* Per-voxel external force [N][3] (replaces all forces), or NULL to clear. */
VX_API int vx_set_forces(vx_sim* sim, const float* F);
/* Damping ratios (paper App. B SetBondDampZ, SetSlowDampZ, SetCollisionDampZ);
 * each in [0, 1]; larger values may be unstable (the paper says the same). */
VX_API int vx_set_damping(vx_sim* sim, float zeta_bond, float zeta_ground, float zeta_collision);
/* Gravity along z [m/s^2] (e.g. -9.81), floor plane z = 0 on/off, and
 * voxel-voxel collisions (Sec 2.2.2): 0 off; 1 within each body (bodies are
 * separate worlds); 2 one shared world, in which voxels of different bodies
 * collide too (never excluded by lattice distance), one horizon accumulator
 * covers all bodies and every body runs on the smallest body timestep.
 * Other values return VX_ERR_ARG. */
VX_API int vx_set_environment(vx_sim* sim, float gravity_z, int32_t floor_on, int32_t collide_on);
/* Volumetric actuation (Sec 2.3): the temperature offset of voxel v at step n
 * is offset + amplitude * sin(2 pi n / period + phase_v) (period 0: offset
 * only).  Bond rest length l (1 + (cte1 dT1 + cte2 dT2) / 2). */
VX_API int vx_set_actuation(vx_sim* sim, float amplitude_K, int64_t period_steps, float offset_K);
/* Independent temperature signals per material (Sec 2.3: several separately
 * controlled temperatures may drive different materials).  Material m then
 * follows offset[m] + amplitude[m] * sin(2 pi n / period + phase_v + phase[m]),
 * on the common period of vx_set_actuation (period 0: offset[m] only).  Each
 * array is host memory of n_materials floats, copied; NULL amplitude or
 * offset means the global value from vx_set_actuation, NULL phase means 0.
 * All three NULL restores the single global signal.  Non-finite values return
 * VX_ERR_ARG.  Invalidates a recorded rollout and a captured graph. */
VX_API int vx_set_material_actuation(vx_sim* sim, const float* amplitude_K, const float* offset_K,
                                     const float* phase_rad);
/* Stable-timestep safety factor f in (0, 1]; recomputes dt. */
VX_API int vx_set_dt_factor(vx_sim* sim, float f);
/* dt of every body [n_bodies] (double on the host; the device steps in FP32).
 * A simulator computes it (at creation and whenever the materials, the
 * per-voxel moduli, dt_factor or the shared-world mode change) from an FP32
 * warp and block max-reduction of w^2 = k / m over the device lattice, with
 * the definition of vx_plan_dt; the result is within 2e-7 of vx_plan_dt's
 * FP64 value (3.5e-7 with per-voxel moduli). */
VX_API int vx_get_dt(vx_sim* sim, double* dt_per_body);
/* Override dt of every body (frozen until the next recompute). */
VX_API int vx_set_dt(vx_sim* sim, const double* dt_per_body);

/* ---- state -------------------------------------------------------------- */
/* Rest state: zero offsets, identity orientations, velocity v0 (if NULL,
 * the one set by vx_set_initial_velocity, zero by default) for non-fixed
 * voxels, zero angular velocity, static flags clear, step counter 0,
 * collision candidates rebuilt.  Synchronous. */
VX_API int vx_reset(vx_sim* sim, const float v0[3]);
/* Initial velocity (App. B: the environment's initial velocity) [m/s]: sets
 * the linear velocity of every non-fixed voxel to v now (positions,
 * orientations and angular velocities unchanged) and makes v the velocity of
 * later vx_reset(sim, NULL) calls.  v: 3 host floats; non-finite values or
 * NULL return VX_ERR_ARG.  Synchronous. */
VX_API int vx_set_initial_velocity(vx_sim* sim, const float v[3]);
/* Copy the state to caller buffers (dst_on_device = 1: device pointers, else
 * host).  Synchronous with respect to work already queued on `stream`. */
VX_API int vx_read_state(vx_sim* sim, const vx_state_view* out, int32_t dst_on_device, void* stream);
/* Overwrite the state from caller buffers (NULL fields unchanged).  With
 * collisions on, the write counts as motion for the collision horizon: each
 * body's accumulator grows by twice the largest distance the write moves one
 * of its voxels, and the candidate lists of the bodies that reach the
 * threshold (every body after a rebuild that timed out or overflowed) are
 * rebuilt from the written state; lists kept hold every pair that can touch
 * before the next rebuild, so a write that moves nothing (velocities, flags,
 * or the state just read) costs no rebuild and changes no result.
 * Together with vx_read_state and the step counter (vx_get_step /
 * vx_set_step) this is a bit-exact checkpoint and resume. */
VX_API int vx_write_state(vx_sim* sim, const vx_state_view* in, int32_t src_on_device, void* stream);
/* Same, without waiting: the copies and the unpacking are enqueued on
 * `stream` and the call returns at once; the caller keeps the source buffers
 * unchanged (and alive) until that work is done (a later synchronising call
 * on the stream, e.g. vx_read_state, or a stream synchronisation). */
VX_API int vx_write_state_async(vx_sim* sim, const vx_state_view* in, int32_t src_on_device, void* stream);
/* Step counter n (number of steps taken since the last reset). */
VX_API int vx_get_step(vx_sim* sim, int64_t* step);
VX_API int vx_set_step(vx_sim* sim, int64_t step);

/* ---- stepping ----------------------------------------------------------- */
/* Advance n_steps explicit steps (paper App. B CVX_Sim::TimeStep, repeated),
 * enqueued on `stream`; then waits for them and returns VX_ERR_UNSTABLE if any
 * voxel state became non-finite (the first bad step/voxel is kept, see
 * vx_get_status).  */
VX_API int vx_step(vx_sim* sim, int64_t n_steps, void* stream);
/* Same, without waiting: the status is checked by a later vx_get_status. */
VX_API int vx_step_async(vx_sim* sim, int64_t n_steps, void* stream);
/* Wait for `stream`, then report: status (VX_OK / VX_ERR_UNSTABLE /
 * VX_ERR_CAPACITY), first bad step and voxel (canonical index) or -1. */
VX_API int vx_get_status(vx_sim* sim, void* stream, int32_t* status, int64_t* bad_step, int64_t* bad_voxel);
/* Relaxation to a static state (the use of App. A: a fixed and loaded,
 * damped structure stepped until it stops moving): steps in chunks of
 * check_every steps until the largest voxel speed is at most v_tol [m/s]
 * after at least one chunk, or max_steps steps are done.  Outputs (any may
 * be NULL): steps taken, the last largest speed [m/s], converged (1) or not
 * (0).  Not converging is not an error; VX_ERR_UNSTABLE as vx_step.
 * Synchronous (one device-to-host read per chunk). */
VX_API int vx_relax(vx_sim* sim, int64_t max_steps, double v_tol, int32_t check_every, int64_t* steps_taken,
                    double* max_speed, int32_t* converged, void* stream);

/* ---- collisions (Sec 2.2.2) ---------------------------------------------- */
/* Rebuild the surface-voxel candidate list from the current positions now.
 * Synchronous.  VX_ERR_CAPACITY when a voxel has more than 48 candidates;
 * VX_ERR_TIMEOUT when a grid barrier of the rebuild gave up waiting (the
 * candidate lists are then unspecified until the next rebuild: vx_reset, a
 * vx_write_state, which then rebuilds every body, or this call). */
VX_API int vx_rebuild_collisions(vx_sim* sim, void* stream);
/* Collision scheme (the paper compares these, Sec 3 "Speedup of self
 * collision schemes"): all_voxels = 1 searches every voxel instead of the
 * precomputed surface voxels; every_step = 1 rebuilds the candidates every
 * step instead of when the horizon accumulator says so.  Defaults 0, 0
 * (surface + horizon).  Rebuilds the candidates now if collisions are on. */
VX_API int vx_set_collision_scheme(vx_sim* sim, int32_t all_voxels, int32_t every_step);
/* Current candidate pairs (i < j, canonical indices, sorted by i then j) into
 * host memory pairs [cap][2]; n_out = total count (may exceed cap). */
VX_API int vx_get_collision_pairs(vx_sim* sim, int32_t* pairs, int64_t cap, int64_t* n_out);
/* Number of candidate-list rebuilds since create, and the horizon
 * accumulator of body 0 [m]. */
VX_API int vx_collision_stats(vx_sim* sim, int64_t* n_rebuilds, double* accumulator);

/* ---- FP64 audit (the only FP64 arithmetic on the GPU) -------------------
 * Deterministic FP64 reductions over the current state: out[0..2] total
 * linear momentum sum m v; out[3..5] angular momentum about the world origin
 * sum (D x m v + I w) with D the absolute centre (anchor + offset, formed in
 * FP64) and I = m l^2 / 6; out[6] translational and out[7] rotational
 * kinetic energy; out[8] elastic energy of the bonds, 1/2 u^T [K] u of each
 * bond's reduced beam (Sec 2.1.2) in its co-rotational frame, stretch taken
 * beyond the thermal rest length (Sec 2.3); out[9] gravitational energy
 * -sum m g z.  Units SI.  Synchronous (waits for `stream`).  */
VX_API int vx_audit(vx_sim* sim, double* out, void* stream);

/* ---- captured launches and autotuning of the batched form ---------------
 * The paper steps one body per call; these serve populations of independent
 * bodies (design automation, which the paper names as a use).
 *
 * vx_graph_capture: capture n_steps of the batched form (vx_set_batching
 * must be on, collisions off) as one CUDA graph holding one persistent
 * launch.  The captured kernel reads its first step number and state buffer
 * from a device counter, so each replay continues from the current step.
 * Any later change of the model or the step form (vx_set_* calls other than
 * state writes) makes the graph stale; vx_graph_launch then returns
 * VX_ERR_STATE until the next capture.
 * vx_graph_launch: replay on `stream` (asynchronous; the status word is read
 * by vx_get_status as after vx_step_async).
 *
 * vx_autotune_batching: time tile sizes {128, 256} x group sizes {per-step
 * launches, 1024, 4096, 16384, 65536 voxels} and the resident form (where
 * the lattice fits it) on sample_steps steps from the current state
 * (restored afterwards), keep the fastest for the lattice's size class (log2
 * voxels, log2 mean body size, per-voxel arrays in use) in a process-wide
 * cache, and apply it.  A cached class is applied without timing.  Outputs
 * (any may be NULL): tile size, group size (0 = per-step launches,
 * VX_GROUPS_RESIDENT = the resident form) and the sampled voxel-steps/s.
 * Synchronous. */
VX_API int vx_graph_capture(vx_sim* sim, int64_t n_steps, void* stream);
VX_API int vx_graph_launch(vx_sim* sim, void* stream);
VX_API int vx_autotune_batching(vx_sim* sim, int32_t sample_steps, int32_t* tile_max, int64_t* group_voxels,
                                double* voxel_steps_per_s, void* stream);

/* ---- adjoint form: design gradients over a rollout ----------------------
 * The loss of body b is the x travel of its centre of mass over a rollout,
 *   L_b = sum_v m_v (x_v(n) - x_v(0)) / sum_v m_v,
 * and the gradients are dL/d(log E_v) (voxel stiffness, Sec 2.1.4 mixes it
 * into every bond) and dL/d(phase_v) (actuation, Sec 2.3), obtained by the
 * reverse of the step of Sec 2.1-2.2: co-rotational beam bonds, damping,
 * floor contact and friction (its stick/slip decisions held as taken in the
 * forward run), integration.  The timestep is held fixed (no derivative
 * through the stability limit).  The paper has no gradients; they serve
 * design optimisation of the kind its examples show.
 *
 * vx_rollout_forward: run n_steps steps from the current state with the
 * current step form, keeping a copy of the state and flags every
 * checkpoint_every steps on the device (ceil(n_steps / K) copies of 53 bytes
 * per voxel).  loss_body: host array [n_bodies] receiving L_b, or NULL.
 * Returns VX_ERR_STATE if voxel-voxel collisions are on (no adjoint for
 * them), VX_ERR_UNSTABLE if the state became non-finite.  Synchronous.
 *
 * vx_rollout_backward: gradients of sum_b w_b L_b for the last forward
 * rollout.  w_body: host array [n_bodies] or NULL for all ones.  grad_logE,
 * grad_phase: DEVICE arrays [n_voxels] (canonical order) overwritten with
 * the gradients; either may be NULL.  The state is recomputed segment by
 * segment from the checkpoints into a device buffer of (K + 1) states; the
 * simulator's own state (the end of the rollout) is not touched.  Returns
 * VX_ERR_STATE if no rollout was recorded or the simulator was stepped,
 * reset, written or reconfigured since.  Synchronous.  */
VX_API int vx_rollout_forward(vx_sim* sim, int64_t n_steps, int32_t checkpoint_every, float* loss_body,
                              void* stream);
VX_API int vx_rollout_backward(vx_sim* sim, const float* w_body, float* grad_logE, float* grad_phase,
                               void* stream);

/* ---- collision candidates with no device allocation ----------------------
 * The paper has no counterpart to this entry point: it exists for callers
 * that cannot allocate device memory where they need collision candidates
 * (code inside a memory pool or arena that owns the device heap, a plug-in
 * handed only pre-sized buffers, a real-time loop that must not hit
 * cudaMalloc's implicit synchronisation).  It computes the same candidate
 * lists as a vx_sim's collision rebuild, for surface voxels the caller
 * describes, and calls no cudaMalloc, cudaFree or allocating library routine.
 *
 * Inputs (device memory): lat[n_surface] packed lattice coordinates
 * i | j << 11 | k << 22 within each voxel's body; offset_planes[3][n_surface]
 * offsets from the lattice anchors (all x, then all y, then all z) [m];
 * body[n_surface] body of each voxel (may be NULL when n_bodies == 1).
 * Outputs (device memory, caller-owned): cand_count[n_surface] and
 * cand[n_surface][48]: for each surface voxel, its candidates as indices into
 * the same input arrays, ascending.  Candidates: same body, lattice
 * Manhattan distance > 3, quantised centre distance below 2 voxel_size.
 *
 * Limits: n_surface <= VX_STATIC_MAX_SURFACE, n_bodies <= VX_STATIC_MAX_BODIES
 * (larger inputs return VX_ERR_ARG); a body id outside [0, n_bodies) (read on
 * the device before the search) returns VX_ERR_ARG naming the first such
 * voxel; more than 48 candidates for a voxel returns VX_ERR_CAPACITY; a grid
 * barrier of the search that waits longer than about a second returns
 * VX_ERR_TIMEOUT.  On any error the outputs are unspecified.  Scratch comes from one fixed device array of
 * about 8.3 MiB that every GPU loading the library holds until exit.  The first
 * call on a device (with that device current) looks up the array's address;
 * make it before any stream capture.  Calls share the array: calls whose GPU
 * work overlaps race and must be serialised by the caller.  Work is enqueued
 * on `stream`; the call waits for it before returning. */
#define VX_STATIC_MAX_SURFACE 65536
#define VX_STATIC_MAX_BODIES 4096
VX_API int vx_collision_candidates_static(const uint32_t* lat, const float* offset_planes, const int32_t* body,
                                          int32_t n_surface, int32_t n_bodies, float voxel_size,
                                          int32_t* cand_count, int32_t* cand, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* VX_H */
