/*
 * dem.h -- C ABI of the GB300 library for soft-sphere DEM with rigid
 * aggregates of bonded spheres and softened self-gravity, after Marohnic et
 * al., "An efficient numerical approach to modeling the effects of particle
 * shape on rubble-pile dynamics" (arXiv 2311.11322).
 *
 * One library call advances any number of independent rubble piles ("piles")
 * on one GPU.  A pile is a set of aggregates; an aggregate is a rigid set of
 * touching spheres.  Each step does, for every pile (paper Sec. 2):
 *   kick-drift of aggregate COMs and spins (Sec. 2.1 leapfrog, Sec. 2.2.1
 *   Euler equations), sphere positions and predicted velocities (Sec. 2.2.2,
 *   Eq. pred-vel), a uniform-cell contact search that skips pairs inside one
 *   aggregate, spring-dashpot normal / tangential / rolling / twisting contact
 *   forces at the contact point (Sec. 2.1, 2.2.4, Eq. lever_arm), softened
 *   direct-sum self-gravity (Sec. 2.2.3, Eq. particle_gravity), reduction of
 *   sphere forces and torques onto each aggregate (Eq. agg_gravity,
 *   Eq. gravity_torque, Eq. agg_contact_accel and the contact torque of
 *   Sec. 2.2.4), and the closing kick.  Optional per-pile external terms: a
 *   point-mass planet (Sec. 4.2) and a constant spin increment (Sec. 4.1).
 *
 * Conventions for every entry point:
 *   - SI units, double precision at the boundary, row-major [n][3] vectors.
 *   - Host arrays are owned by the caller and only read (inputs) or written
 *     (outputs) during the call; the library copies what it keeps.
 *   - Device memory is owned by the world; it is obtained at add time (never
 *     inside dem_step) through the allocator set by dem_set_allocator, or
 *     cudaMalloc by default.
 *   - All GPU work is issued on the CUDA stream given to dem_create.
 *   - Every call returns a dem_status; dem_last_error() then holds a one-line
 *     message.  No C++ exception crosses the ABI and no kernel traps.
 *   - A world is not thread-safe: one host thread at a time.
 */
#ifndef DEM_H
#define DEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dem_world dem_world;

typedef enum {
    DEM_OK = 0,
    DEM_ERR_ARG = 1,       /* invalid argument (NULL, size, non-finite input, unknown id) */
    DEM_ERR_OOM = 2,       /* device allocation failed or the HBM budget would be exceeded */
    DEM_ERR_CUDA = 3,      /* a CUDA runtime call failed (message has the CUDA error string) */
    DEM_ERR_OVERLAP = 4,   /* reserved: overlaps above 10% of a radius are reported as flags */
    DEM_ERR_SLOTS = 5,     /* a sphere had more contacts than max_contacts history slots */
    DEM_ERR_NONFINITE = 6, /* a pile's state became NaN or infinite, or its gravity sum left
                              the range of its accumulators (DEM_FLAG_GRAV_RANGE); that pile
                              is frozen */
    DEM_ERR_TIMEOUT = 7,   /* reserved for bounded device waits */
    DEM_ERR_STATE = 8      /* call not valid in the current state (e.g. pile removed) */
} dem_status;

enum { DEM_FP64 = 0, DEM_MIXED = 1 };

/* Per-pile parameters (paper Sec. 2.1; the force-law constants are user inputs). */
typedef struct {
    double G;            /* gravitational constant (m^3 kg^-1 s^-2); 0 disables self-gravity */
    double dt;           /* fixed step h (s) */
    double kn, kt;       /* normal / tangential spring constants (N/m) */
    double cn, ct;       /* normal / tangential dashpot constants (N s/m) */
    double mu_s;         /* sliding (static = dynamic) friction coefficient */
    double mu_r, mu_t;   /* rolling / twisting friction coefficients */
    double w0;           /* rolling/twisting regularisation rate (rad/s), > 0 */
    double eps_soft;     /* Plummer softening length (m) */
    int32_t precision;   /* DEM_FP64 or DEM_MIXED; all piles of a world must agree */
    int32_t max_contacts;/* K history slots per sphere, 1..64 */
    double cell_size;    /* contact cell edge (m); 0 = automatic (>= 2 x largest radius) */
    double ext_mass;     /* point-mass planet (kg); 0 = none (Sec. 4.2) */
    double ext_pos[3];   /* planet position at t = 0 (m) */
    double ext_vel[3];   /* planet velocity at t = 0 (m/s) */
    double spin_inc[3];  /* spin increment per step (rad/s, space frame); 0 = none (Sec. 4.1) */
    double rot_tol;      /* torque-free rotation over each step: 0 = one classical RK4 step;
                            > 0 = the paper's time-adaptive fifth-order Runge-Kutta (embedded
                            Cash-Karp RK5(4) substeps, error in q absolute and in w relative
                            to |w| at most rot_tol; Sec. 2.2.1), in FP64 in both precisions */
} dem_params;

/* Fields for dem_read_state.  A = aggregates of the pile, N = spheres, K = max_contacts. */
enum dem_field {
    DEM_FIELD_COM = 0,         /* A x 3  aggregate COM position r_A (Eq. agg_position) */
    DEM_FIELD_VEL = 1,         /* A x 3  COM velocity */
    DEM_FIELD_QUAT = 2,        /* A x 4  orientation (w, x, y, z), body frame = space frame at add time */
    DEM_FIELD_OMEGA = 3,       /* A x 3  spin, space frame */
    DEM_FIELD_SPHERE_POS = 4,  /* N x 3  sphere centres r_A + R(q) b_i */
    DEM_FIELD_FORCE = 5,       /* A x 3  total force of the last step */
    DEM_FIELD_TORQUE = 6,      /* A x 3  total torque about the COM of the last step */
    DEM_FIELD_CONTACTS = 7,    /* N x (1 + 4K): count, then K x (partner, Sx, Sy, Sz); S of a
                                  pair as seen from its lower-index sphere, so both rows agree */
    DEM_FIELD_FORCE_CONTACT = 8,   /* A x 3 */
    DEM_FIELD_TORQUE_CONTACT = 9,  /* A x 3 */
    DEM_FIELD_FORCE_GRAV = 10,     /* A x 3 */
    DEM_FIELD_TORQUE_GRAV = 11,    /* A x 3 */
    DEM_FIELD_FORCE_EXT = 12,      /* A x 3 */
    DEM_FIELD_TORQUE_EXT = 13,     /* A x 3 */
    DEM_FIELD_SPHERE_FC = 14,      /* N x 3  contact force on each sphere */
    DEM_FIELD_SPHERE_TC = 15,      /* N x 3  contact torque on each sphere about its centre */
    DEM_FIELD_SPHERE_FG = 16,      /* N x 3  gravity on each sphere from other aggregates */
    DEM_FIELD_ACC = 17,            /* A x 3  stored a_A */
    DEM_FIELD_PLANET = 18,         /* 9      planet position, velocity, acceleration */
    DEM_FIELD_MASS = 19,           /* A      aggregate mass (Eq. agg_mass) */
    DEM_FIELD_BODY_OFFSETS = 20,   /* N x 3  body-frame offsets b_i (never rewritten) */
    DEM_FIELD_OMEGA_BODY = 21,     /* A x 3  spin, body frame */
    DEM_FIELD_INFO = 22,           /* 20     n_agg, n_sph, steps, flags, nx, ny, nz, cell, K,
                                              precision, frame origin[3], failed, parity,
                                              M_total, rebuilds, skin, rebuild next step, 0 */
    DEM_FIELD_FRAME = 23,          /* 6      origin and velocity of the pile frame */
    DEM_FIELD_TORQUE_STORED = 24   /* A x 3  stored N_A used by the next step's first half kick */
};

/* Pile flag bits (dem_pile_flags). */
/* DEM_FLAG_TREE: tree gravity ran out of traversal stack for some group of
 * spheres and took a cell as far that it would have opened (less accurate,
 * not fatal). */
/* DEM_FLAG_GRAV_RANGE (mixed precision, direct sum): a tile's gravity sum on
 * some sphere exceeded the range of the pile's fixed-point gravity
 * accumulators.  The range is set when the pile is added, from its total mass
 * and min(0.385 / eps_soft^2, 4 / s_min^2) (s_min = smallest radius): it holds
 * for any configuration when eps_soft >= 0.31 s_min, else for any in which
 * spheres of different aggregates stay more than s_min / 2 apart.  Fatal: the
 * pile is frozen. */
enum { DEM_FLAG_SLOTS = 1, DEM_FLAG_NONFINITE = 2, DEM_FLAG_OVERLAP = 4, DEM_FLAG_TREE = 8,
       DEM_FLAG_GRAV_RANGE = 16 };

/* Kernels that dem_step_profiled can time. */
enum dem_kernel {
    DEM_K_AGG_BEGIN = 0, DEM_K_PILE_BEGIN = 1, DEM_K_KEYS = 2, DEM_K_SCAN = 3, DEM_K_SCATTER = 4,
    DEM_K_CELL_ORDER = 5, DEM_K_GATHER = 6, DEM_K_CONTACT = 7, DEM_K_GRAVITY = 8,
    DEM_K_AGG_END = 9, DEM_K_PILE_END = 10, DEM_K_COUNT = 11
};

/*
 * Device allocator hook.  alloc returns a device pointer (NULL on failure) of
 * at least `bytes`, usable on `stream`; free releases it.  ctx is passed back.
 */
typedef void *(*dem_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*dem_free_fn)(void *ptr, void *ctx);

/*
 * Create an empty world on the current CUDA device.  cuda_stream: a
 * cudaStream_t other than the legacy default stream, on which every later
 * call issues its work (the per-step CUDA graph cannot be captured on the
 * legacy stream); NULL = the world creates and owns a non-blocking stream.  hbm_budget_bytes: the most device memory the world may
 * hold (0 = no limit).  *out receives the world.
 * Errors: DEM_ERR_ARG (out NULL), DEM_ERR_CUDA.
 */
dem_status dem_create(void *cuda_stream, size_t hbm_budget_bytes, dem_world **out);

/* Replace the device allocator (call before the first dem_add_aggregates). */
dem_status dem_set_allocator(dem_world *w, dem_alloc_fn alloc, dem_free_fn free_fn, void *ctx);

/*
 * Add one pile of n_agg aggregates (paper Sec. 2.2.1).
 *   spheres_per_agg [n_agg]: sphere count of each aggregate (>= 1);
 *   sphere_pos [N][3], sphere_radius [N], sphere_density [N]: the spheres in
 *     aggregate order, N = sum(spheres_per_agg), space frame at t = 0;
 *   agg_vel, agg_omega [n_agg][3]: COM velocity and spin (space frame), NULL = 0.
 * The library computes in FP64 on the host each aggregate's mass M = sum m_i
 * (Eq. agg_mass, m_i = rho 4/3 pi s^3), COM (Eq. agg_position), inertia tensor
 * about the COM (sphere moments 2/5 m s^2 plus parallel-axis terms) and its
 * inverse, and the body offsets b_i = r_i - r_A (body frame = space frame at
 * t = 0, q = identity); b_i are never rewritten.  The stored acceleration and
 * torque start at zero.  *out_pile_id receives the pile id.
 * Errors: DEM_ERR_ARG (sizes, non-positive radius/density, non-finite input,
 * singular inertia, precision differing from earlier piles, max_contacts out
 * of 1..64), DEM_ERR_OOM (budget or allocation), DEM_ERR_CUDA.
 */
dem_status dem_add_aggregates(dem_world *w, const dem_params *p, int64_t n_agg,
                              const int32_t *spheres_per_agg, const double *sphere_pos,
                              const double *sphere_radius, const double *sphere_density,
                              const double *agg_vel, const double *agg_omega,
                              int32_t *out_pile_id);

/*
 * Advance piles by n_steps fixed steps (one captured CUDA graph per step).
 * pile_ids [n_piles] lists the piles to advance; NULL = every live pile.
 * Asynchronous on the world's stream.  Returns the status of the previous
 * dem_step call (it waits for that batch's 4-byte flag word per pile): a pile
 * whose state became non-finite or whose history slots overflowed is frozen
 * and reported as DEM_ERR_NONFINITE / DEM_ERR_SLOTS once.
 * Errors: DEM_ERR_ARG (unknown pile id, n_steps < 0), DEM_ERR_CUDA, the above.
 */
dem_status dem_step(dem_world *w, const int32_t *pile_ids, int32_t n_piles, int64_t n_steps);

/* Wait for all issued work; returns the status of the last dem_step. */
dem_status dem_sync(dem_world *w);

/*
 * Like dem_step with NULL pile_ids, but launches the kernels one by one
 * (no graph) and records CUDA events on the world's stream around every
 * launch of kernel `which` (enum dem_kernel).  ms_out [n_steps] receives that
 * kernel's duration in each step.  Synchronises before returning.
 */
dem_status dem_step_profiled(dem_world *w, int64_t n_steps, int32_t which, float *ms_out);

/*
 * Put CUDA event records around kernel `which` (enum dem_kernel; -1 = none)
 * inside the captured step graph.  Recaptures the graph on the next step.
 */
dem_status dem_set_timed_kernel(dem_world *w, int32_t which);

/*
 * One step of every live pile as one graph launch, bracketed by CUDA events
 * on the world's stream; synchronises.  step_ms receives the launch's device
 * time; kernel_ms (may be NULL) the time of the kernel chosen with
 * dem_set_timed_kernel inside that launch (0 if none was chosen).
 */
dem_status dem_step_timed(dem_world *w, float *step_ms, float *kernel_ms);

/* Number of kernel nodes in the captured step graph (captures it if needed). */
dem_status dem_graph_kernel_count(dem_world *w, int32_t *n_out);

/*
 * Copy one field of a pile to host_out (n_out doubles, see enum dem_field for
 * the layout); synchronises the stream first.
 * Errors: DEM_ERR_ARG (unknown pile/field, n_out too small), DEM_ERR_CUDA.
 */
dem_status dem_read_state(dem_world *w, int32_t pile_id, int32_t field, double *host_out,
                          int64_t n_out);

/*
 * Asynchronous read of one per-aggregate state field (DEM_FIELD_COM, VEL,
 * QUAT, OMEGA_BODY, ACC, TORQUE_STORED or MASS; layouts as dem_read_state):
 * enqueues the copy to host_out on the world's stream and returns without
 * waiting, so that the host can issue the next dem_step and work on an
 * earlier result while the device steps.  The copy sees the state after the
 * steps issued before the call.  host_out (n_out doubles, owned by the
 * caller; pinned memory lets the copy run asynchronously) must stay valid
 * and untouched until dem_read_wait returns, and holds the world's internal
 * slot format until then.  At most DEM_MAX_ASYNC_READS reads may be pending.
 * Errors: DEM_ERR_ARG (unknown pile, a field other than those above, NULL or
 * too small host_out, too many pending reads), DEM_ERR_CUDA.
 */
#define DEM_MAX_ASYNC_READS 8
dem_status dem_read_state_async(dem_world *w, int32_t pile_id, int32_t field, double *host_out,
                                int64_t n_out);

/*
 * Wait for every pending dem_read_state_async copy (and only for those: steps
 * issued after them keep running) and convert the values to FP64 in place.
 * Errors: DEM_ERR_CUDA.
 */
dem_status dem_read_wait(dem_world *w);

/*
 * Overwrite one field of a pile from host memory (checkpoint restore, or
 * re-synchronising with another integrator).  Writable fields, same layouts
 * as dem_read_state: COM, VEL, QUAT (renormalised is the caller's duty),
 * OMEGA_BODY, ACC, TORQUE_STORED, CONTACTS (only the first count entries of
 * each sphere are read; partners must be pile-local indices < N), PLANET
 * (position, velocity, acceleration) and FRAME.  Synchronises the stream
 * first; the next dem_step starts from the written state.
 * Errors: DEM_ERR_ARG (unknown pile or field, n_in too small, non-finite
 * value, bad contact count or partner), DEM_ERR_CUDA.
 */
dem_status dem_write_state(dem_world *w, int32_t pile_id, int32_t field, const double *host_in,
                           int64_t n_in);

/* Flag bits (DEM_FLAG_*) raised so far for a pile; synchronises. */
dem_status dem_pile_flags(dem_world *w, int32_t pile_id, int32_t *flags_out);

/* Remove a pile and release its share of device memory (compacts the rest). */
dem_status dem_remove_pile(dem_world *w, int32_t pile_id);

/*
 * Tuning knobs (normally chosen by dem_autotune).  key: "grav_block"
 * (threads per gravity block: 64, 128 or 256), "grav_ib" (i-spheres per
 * thread: 1, 2 or 4), "grav_item" (target pair interactions per gravity work
 * item, >= 1024; sets the j-range split), "grav_jchunk" (fixed j-range length
 * per work item, 0 = use grav_item), "grav_pack" (1 = packed f32x2 pair terms
 * when grav_ib is even, 0 = scalar FP32), "grav_sym" (1 = symmetric
 * tile-pair form, each pair evaluated once and applied to both spheres, the
 * default in both precisions; 0 = one-sided form shaped by the keys above),
 * "grav_tile" (spheres per tile of the symmetric form in the mixed path:
 * 512, or 128 or 256 for worlds whose piles all have at most 8,192 spheres,
 * or 64 when they have at most 2,048 -- more, smaller work items when the
 * 512-sphere tile pairs would not fill the GPU; 0 = choose automatically
 * (when the 512-sphere tile pairs of all piles fill less than one wave of
 * the persistent grid: 64 up to 2,048 spheres, else 128), the default;
 * larger piles always use 512),
 * "grav_theta" (mixed path: > 0 replaces the direct sum by tree gravity with
 * this opening angle, in [0, 1): cells of an octree rebuilt every step with
 * multipoles up to the hexadecapole (Sec. 2.1), leaves of ~4 spheres summed
 * directly; 0 = direct sum, the default), "grav_order" (highest multipole
 * rank of the tree's accepted cells: 4, the default, or 2 -- monopole and
 * quadrupole only, cheaper per cell and less accurate),
 * "contact_mode" (0, the default: one thread per sphere evaluates every pair
 * of its candidate list; 1: tiles of 128 consecutive sorted spheres evaluate
 * each pair inside the tile once and pass both halves through a
 * shared-memory inbox; the two give bitwise the same results),
 * "contact_inbox" (mode 1: list entries a tile evaluates together through
 * its inbox, 1..1280, default 1280 (the FP64 path uses at most 640); tiles
 * with more entries are split into sphere ranges that fit, and pairs across
 * ranges are evaluated from both sides: results are bitwise the same for
 * every value, only the speed changes),
 * "cell_factor" (cell edge / (2 x
 * largest radius), >= 1), "skin" (neighbour-list skin as a fraction of the
 * pile's largest radius, in [0, 4], default 0.1; 0 = search contacts afresh
 * every step).  With a skin the cell list and the per-sphere candidate lists
 * are rebuilt only when some aggregate may have moved more than half the skin
 * relative to the pile frame since the last rebuild (and after any state
 * write or layout change).  Neither knob changes results: contacts are summed
 * in partner order, so trajectories are bitwise the same for every cell size
 * and skin.  Changing cell_factor or skin re-grids every pile.  Invalidates
 * the captured graph.
 */
dem_status dem_set_tuning(dem_world *w, const char *key, double value);

/* Current value of a tuning knob (the keys of dem_set_tuning).
 * Errors: DEM_ERR_ARG (NULL argument, unknown key). */
dem_status dem_get_tuning(dem_world *w, const char *key, double *value_out);

/*
 * Autotuner: time the candidate gravity shapes (the symmetric form, with
 * 512-sphere tiles and, in the mixed path, 64-, 128- and 256-sphere tiles;
 * the one-sided form with block 64/128/256, 1/2/4 i-spheres per thread,
 * scalar or packed, three work-item sizes), then cell factors 1, 1.25,
 * 1.5, 2, then both forms of the contact pass (contact_mode 0 and 1) on the
 * current piles, one warm and `trial_steps` timed step graph launches per
 * candidate, and keep the fastest (no candidate changes the contact results;
 * the gravity shapes reorder FP32 sums only).  The trials step the live
 * piles, so the tuner first copies every field that carries state from step
 * to step (positions, velocities, orientations, spins, stored accelerations
 * and torques, contact history, step counters, flags, planet) into a
 * temporary device buffer (one allocation through the world's allocator, the
 * size of that state) and copies it back at the end, on success and on every
 * error path: the piles leave the tuner in the state they entered it, and the
 * next step recomputes the cell and candidate lists.  On an error the
 * original tuning is restored.  best_ms_out (may be NULL) receives the
 * fastest step time.  Synchronises the stream.
 * Errors: DEM_ERR_ARG (trial_steps < 1), DEM_ERR_OOM (no room for the
 * snapshot), DEM_ERR_CUDA.
 */
dem_status dem_autotune(dem_world *w, int32_t trial_steps, double *best_ms_out);

/*
 * Bulk shape and spin of a pile: the quantities behind the critical spin
 * ratio (Sec. 4.1) and the disruption ratio (Sec. 4.2).  Computed on the
 * device from the aggregate state after the last step, in FP64:
 *   M, COM r_c, v_c: sums over the aggregates;
 *   I: inertia tensor about r_c, sum of M_A (|x_A|^2 1 - x_A x_A^T) +
 *      R_A I_A R_A^T with x_A = r_A - r_c (the spheres' own moments enter
 *      through I_A);
 *   L: angular momentum about r_c, sum of M_A x_A x (v_A - v_c) + R_A I_A w_A;
 *   principal moments I1 <= I2 <= I3 of I (cyclic Jacobi);
 *   semi-axes a >= b >= c of the uniform ellipsoid with the same mass and
 *      principal moments: a^2 = 5 (I2 + I3 - I1) / (2 M), b^2 = 5 (I1 + I3 - I2)
 *      / (2 M), c^2 = 5 (I1 + I2 - I3) / (2 M);
 *   bulk radius R_b = (a b c)^(1/3) and bulk density rho_b = 3 M / (4 pi a b c);
 *   spin w = I^-1 L (the rigid rotation carrying L), period 2 pi / |w|
 *      (infinity at rest);
 *   nominal critical period P_crit = sqrt(3 pi / (G rho_b)) (Sec. 4.1;
 *      infinity when G = 0);
 *   distance from r_c to the point-mass planet (0 when there is none).
 * out [DEM_BULK_LEN] receives the record laid out as enum dem_bulk.
 * Synchronises the stream.
 * Errors: DEM_ERR_ARG (unknown pile, n_out < DEM_BULK_LEN), DEM_ERR_CUDA.
 */
enum dem_bulk {
    DEM_BULK_MASS = 0, DEM_BULK_COM = 1, DEM_BULK_VCOM = 4, DEM_BULK_AXES = 7,
    DEM_BULK_RADIUS = 10, DEM_BULK_DENSITY = 11, DEM_BULK_SPIN = 12, DEM_BULK_PERIOD = 15,
    DEM_BULK_PCRIT = 16, DEM_BULK_PLANET_DIST = 17, DEM_BULK_L = 18, DEM_BULK_MOMENTS = 21,
    DEM_BULK_LEN = 24
};
dem_status dem_pile_bulk(dem_world *w, int32_t pile_id, double *out, int64_t n_out);

/*
 * Radius-growth watch (the stopping rule of Sec. 4.1 and 4.2): evaluate the
 * bulk record of a pile on the device inside the step graph, every `every`
 * steps (counted from the pile's step counter), and latch the first record
 * whose bulk radius reaches (1 + growth) R_b0, R_b0 being the bulk radius
 * when the watch is armed.  growth > 0 arms (taking R_b0 and the record at
 * that moment, and clearing an earlier latch); growth = 0 disarms.  The host
 * polls with dem_watch_result; nothing is copied back while stepping.
 * Arming or disarming recaptures the step graph on the next step.
 * Errors: DEM_ERR_ARG (unknown pile, growth < 0 or not finite, every < 1),
 * DEM_ERR_CUDA.
 */
dem_status dem_watch(dem_world *w, int32_t pile_id, double growth, int64_t every);

/*
 * State of a pile's watch, out [DEM_WATCH_LEN]: [0] step count at the latch
 * (-1 while not reached), [1] growth, [2] every, [3] armed (1/0), [4..27] the
 * bulk record when armed (enum dem_bulk), [28..51] the latched bulk record
 * (zeros while not reached).  Synchronises the stream.
 * Errors: DEM_ERR_ARG (unknown pile, n_out < DEM_WATCH_LEN), DEM_ERR_CUDA.
 */
enum { DEM_WATCH_LEN = 52 };
dem_status dem_watch_result(dem_world *w, int32_t pile_id, double *out, int64_t n_out);

/*
 * Softened direct-sum gravity of one set of spheres that allocates nothing.
 * The paper has no counterpart: this entry point serves callers that cannot
 * allocate device memory -- code running inside another program's memory
 * pool or arena, real-time loops that forbid allocation after start-up, or
 * plugins whose host owns every allocation -- and so cannot create a world.
 * It computes, for i < n,
 *   F_i = G m_i sum_{j : agg_id[j] != agg_id[i]} m_j (r_j - r_i) / (|r_j - r_i|^2 + eps^2)^{3/2}
 * with FP32 pair terms and FP64 sums: the world's gravity formula, agreeing
 * with the world's gravity pass within the mixed-precision tolerance (not
 * bitwise: the summation order differs).  With eps_soft = 0, two coincident
 * spheres of different aggregates contribute nothing to each other.
 *   pos_mass  device, float4 [n] (16-byte aligned): x, y, z in m about any
 *             common origin, mass in kg (used in the pair terms);
 *   mass      device, double [n] (8-byte aligned): masses in kg (the final
 *             G m_i factor);
 *   agg_id    device, int32 [n] (4-byte aligned): aggregate of each sphere (pairs with equal
 *             ids are skipped, and so is i = j);
 *   force_out device, double [n][4] (32-byte aligned): Fx, Fy, Fz, 0 in N.
 * The caller owns all four buffers.  Work is queued on cuda_stream (NULL =
 * legacy stream) and the call returns without waiting.  Scratch for the
 * partial sums is a fixed 16 MiB device array inside the library, present on
 * every GPU that loads it until the process exits; hence n <= 131072, and a
 * larger n is refused with DEM_ERR_ARG.  The first call on each device looks
 * up that array's device address (with the device current); make that first
 * call before any stream capture.  All calls share the array: two calls whose
 * kernels overlap on the GPU (different streams, or different host threads)
 * race on it and must be serialised by the caller.  No value from an earlier
 * call is read, so nothing needs clearing.  msg (may be NULL) receives a
 * one-line error text of at most msg_len bytes.
 * Errors: DEM_ERR_ARG (NULL pointer, n out of range, G or eps_soft negative
 * or not finite, a buffer below its stated alignment: pos_mass 16, force_out
 * 32, mass 8, agg_id 4 bytes), DEM_ERR_CUDA (no device, symbol lookup or
 * launch failure).
 */
dem_status dem_gravity_noalloc(const void *pos_mass, const double *mass, const int32_t *agg_id,
                               int32_t n, double G, double eps_soft, double *force_out,
                               void *cuda_stream, char *msg, size_t msg_len);

/*
 * Throughput probe: the peak rates that bound the step's kernels on this GPU,
 * measured the way the step uses the hardware (the paper has no counterpart;
 * these are the denominators of the roofline fractions the benchmark reports).
 *   kind DEM_PROBE_FMA32:   FP32 FMA rate of the CUDA cores (the gravity pair
 *                           terms), flop/s, 2 flop per FMA;
 *        DEM_PROBE_FMA32X2: the same with packed f32x2 FMAs, 4 flop each;
 *        DEM_PROBE_FMA64:   FP64 FMA rate (the all-FP64 path), flop/s;
 *        DEM_PROBE_COPY:    HBM copy, bytes read + written per second.
 *   size: FMA kinds: rounds per thread (each round 32 FMAs per thread, on a
 *         grid of 4 x 256 threads per SM); copy: bytes per buffer (multiple
 *         of 16).
 *   reps: launches, each timed alone with CUDA events on cuda_stream (NULL =
 *         legacy stream); the fastest is reported.
 *   src, dst: device buffers owned by the caller.  Copy: `size` bytes each,
 *         16-byte aligned, not overlapping.  FMA kinds: src unused, dst an
 *         8-byte aligned device word the kernel could write (it never does
 *         in practice).
 *   rate_out: the rate; ms_out (may be NULL): the fastest launch's time;
 *   sm_count_out (may be NULL): the device's SM count.
 * Synchronises cuda_stream.  msg (may be NULL) receives a one-line error text.
 * Errors: DEM_ERR_ARG (unknown kind, size or reps < 1, NULL or misaligned
 * buffer), DEM_ERR_CUDA.
 */
enum { DEM_PROBE_FMA32 = 0, DEM_PROBE_FMA32X2 = 1, DEM_PROBE_FMA64 = 2, DEM_PROBE_COPY = 3 };
dem_status dem_probe_peak(int32_t kind, int64_t size, int32_t reps, const void *src, void *dst,
                          void *cuda_stream, double *rate_out, double *ms_out, int32_t *sm_count_out,
                          char *msg, size_t msg_len);

/* Device bytes one pile of this size needs with direct-sum gravity (state, sorted
 * copies, cells, history, gravity partial sums).  Tree gravity (grav_theta > 0)
 * needs instead about 1.1 KB per sphere plus 280 B per tree cell. */
size_t dem_footprint_bytes(int64_t n_spheres, int64_t n_agg, int32_t max_contacts,
                           int32_t precision);

/* Device bytes the world holds now. */
size_t dem_world_bytes(const dem_world *w);

/* Message of the last failed call on this world (never NULL). */
const char *dem_last_error(const dem_world *w);

/* Release everything (waits for the stream). NULL is allowed. */
void dem_destroy(dem_world *w);

#ifdef __cplusplus
}
#endif

#endif /* DEM_H */
